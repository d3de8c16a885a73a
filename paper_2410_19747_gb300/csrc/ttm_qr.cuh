// ttm_qr.cuh -- Householder QR for the gauge moves (QR decompositions after every
// Contract, the paragraph after Eq. eps), float64 on the GPU.
//
// A carriage C reshaped to the m x n matrix [(l, s), r] (column-major copy in a
// workspace) is factored as C = Q R with k = min(m, n): Q (m x k) has orthonormal
// columns and becomes the left-orthonormal carriage; R (k x n) is merged into the
// right neighbour by a GEMM. Reflectors follow the usual construction
// H = I - tau v v^T with v_j = 1 and beta = -sign(alpha) ||x|| (Golub & Van Loan,
// Alg. 5.1.1); a zero sub-column gives tau = 0.
//
// One cooperative launch per QR (batched over products). Column j's reflector is
// built by the warp that applied reflector j-1 to that column, so each column costs
// a single grid-wide barrier; the explicit Q is then accumulated backwards
// (Q = H_0 ... H_{k-1} I[:, :k]) with one barrier per reflector.
#pragma once
#include <cooperative_groups.h>
#include "ttm_common.cuh"

namespace cg = cooperative_groups;

namespace ttm {

struct QRArgs {
  Tables t;
  int ba, btau, br, bq;  // A (m x n col-major, overwritten), tau[k], R (k x n row-major), Q (m x k col-major)
  Dim m, n;
  int ik;                // bond id that receives k = min(m, n)
  int n_ub, k_ub;
};

// Reflector for column j of A (rows j..m-1), computed by one warp.
__device__ __forceinline__ void make_reflector(double* A, double* tau, int m, int j, int lane) {
  double* col = A + (long)j * m;
  double sig = 0.0;
  for (int i = j + 1 + lane; i < m; i += 32) sig = fma(col[i], col[i], sig);
  sig = warp_sum(sig);
  const double alpha = col[j];
  double t = 0.0;
  if (sig > 0.0) {
    const double mu = sqrt(fma(alpha, alpha, sig));
    const double beta = (alpha <= 0.0) ? mu : -mu;
    t = (beta - alpha) / beta;
    const double scale = 1.0 / (alpha - beta);
    for (int i = j + 1 + lane; i < m; i += 32) col[i] *= scale;
    __syncwarp();
    if (lane == 0) col[j] = beta;
  }
  if (lane == 0) tau[j] = t;
  __syncwarp();
}

// Apply H_j (stored in column j of V, implicit 1 at row j) to column c of X.
__device__ __forceinline__ void apply_reflector(const double* V, double tj, double* X, int m, int j,
                                                int c, int lane) {
  if (tj == 0.0) return;
  const double* v = V + (long)j * m;
  double* x = X + (long)c * m;
  double w = 0.0;
  for (int i = j + 1 + lane; i < m; i += 32) w = fma(v[i], x[i], w);
  w = warp_sum(w) + x[j];
  const double f = tj * w;
  __syncwarp();
  for (int i = j + 1 + lane; i < m; i += 32) x[i] = fma(-f, v[i], x[i]);
  if (lane == 0) x[j] -= f;
  __syncwarp();
}

__global__ void __launch_bounds__(256) householder_kernel(QRArgs a) {
  cg::grid_group grid = cg::this_grid();
  const int lane = threadIdx.x & 31;
  const long gthread = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long nthreads = (long)gridDim.x * blockDim.x;
  // consecutive work items on different SMs (see the Jacobi kernel)
  const long gwarp = (long)(threadIdx.x >> 5) * gridDim.x + blockIdx.x, nwarps = nthreads >> 5;
  const int nz = a.t.nz;

  for (long z = gwarp; z < nz; z += nwarps) {
    const int m = a.m.eval(a.t, (int)z), n = a.n.eval(a.t, (int)z);
    const int k = min(m, n);
    if (lane == 0) a.t.bond[z * a.t.nbd + a.ik] = k;
    if (k >= 1) make_reflector(bufp(a.t, (int)z, a.ba), bufp(a.t, (int)z, a.btau), m, 0, lane);
  }
  grid.sync();

  for (int j = 0; j < a.k_ub; ++j) {
    const int cols = a.n_ub - j - 1;
    if (cols > 0) {
      const long items = (long)nz * cols;
      for (long it = gwarp; it < items; it += nwarps) {
        const int z = (int)(it / cols), c = j + 1 + (int)(it % cols);
        const int m = a.m.eval(a.t, z), n = a.n.eval(a.t, z);
        const int k = min(m, n);
        if (j >= k || c >= n) continue;
        double* A = bufp(a.t, z, a.ba);
        double* tau = bufp(a.t, z, a.btau);
        apply_reflector(A, tau[j], A, m, j, c, lane);
        if (c == j + 1 && c < k) make_reflector(A, tau, m, c, lane);
      }
    }
    grid.sync();
  }

  // R (k x n, row-major, zero below the diagonal) and Q = I[:, :k]
  for (int z = 0; z < nz; ++z) {
    const int m = a.m.eval(a.t, z), n = a.n.eval(a.t, z);
    const int k = min(m, n);
    const double* A = bufp(a.t, z, a.ba);
    double* R = bufp(a.t, z, a.br);
    double* Q = bufp(a.t, z, a.bq);
    for (long e = gthread; e < (long)k * n; e += nthreads) {
      const int i = (int)(e / n), c = (int)(e % n);
      R[e] = (i <= c) ? A[i + (long)c * m] : 0.0;
    }
    for (long e = gthread; e < (long)m * k; e += nthreads) {
      const int i = (int)(e % m), c = (int)(e / m);
      Q[e] = (i == c) ? 1.0 : 0.0;
    }
  }
  grid.sync();

  for (int j = a.k_ub - 1; j >= 0; --j) {
    const int cols = a.k_ub - j;
    const long items = (long)nz * cols;
    for (long it = gwarp; it < items; it += nwarps) {
      const int z = (int)(it / cols), c = j + (int)(it % cols);
      const int m = a.m.eval(a.t, z), n = a.n.eval(a.t, z);
      const int k = min(m, n);
      if (j >= k || c >= k) continue;
      const double* A = bufp(a.t, z, a.ba);
      const double* tau = bufp(a.t, z, a.btau);
      apply_reflector(A, tau[j], bufp(a.t, z, a.bq), m, j, c, lane);
    }
    grid.sync();
  }
}

}  // namespace ttm
