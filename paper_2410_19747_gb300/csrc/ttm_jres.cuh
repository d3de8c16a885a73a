// ttm_jres.cuh -- one-sided Jacobi with shared-memory-resident column blocks, for the Swap SVD
// (Fig. 1C, Eq. eps): float32 for the preconditioning passes, float64 for the fallback polish.
//
// The scalar kernel (ttm_svd.cuh) pairs single columns and ends every round of n/2 pairs at a
// grid-wide barrier, reading and writing both columns and both V columns through L2 each
// time: n - 1 barriers and L2 round trips per sweep. Here the columns are grouped into blocks
// of B and a round-robin tournament (Brent & Luk 1985) runs over the blocks. A CTA takes one
// block pair per block round, keeps its 2B columns of W in shared memory, and visits
//   - at the first block round of a sweep, the pairs inside each of its two blocks
//     (B - 1 inner rounds of B/2 + B/2 disjoint pairs), and
//   - at every block round, the B^2 pairs across its two blocks (B inner rounds of B
//     disjoint pairs: column i of the first block with column (i + s) mod B of the second),
// with a CTA barrier between inner rounds. Every column pair is visited once per sweep, as in
// the scalar kernel, with the same rotation, tests and skip rule. One warp takes one pair of an
// inner round; the column of the first block stays in its registers for the cross rounds.
// The rotations of a block round are accumulated into a 2B x 2B orthogonal factor Q, and the
// 2B columns of V are multiplied by Q once at the end of the block round (V stays in global
// memory). Grid barriers per sweep: ceil(n / B) - 1 (rounded up to an even count) instead of
// n - 1. The float64 instantiation starts from a given V and takes part only for the products
// whose predicate slot is set (the fallback of the Newton steps).
#pragma once
#include <cooperative_groups.h>
#include "ttm_common.cuh"

namespace cg = cooperative_groups;

namespace ttm {

constexpr int kJrB = 8;         // columns per block; one warp per pair of an inner round
constexpr int kJrMaxRows = 1024;  // rows held per column (32 lanes x 32)

struct JResArgs {
  Tables t;
  int bw, bv;        // W: m x n column-major (in/out); V: n x n column-major (in/out)
  Dim m, n;
  int nblk_pad_ub;   // even host upper bound of ceil(n / B)
  int max_sweeps;
  int* counters;     // [nz][max_sweeps] rotations per sweep, zeroed before launch
  double tol;        // rotate when |w_p . w_q| > tol |w_p| |w_q| ...
  double delta;      // ... and |w_p . w_q| > delta max(|w_p|, |w_q|) ||W||_F
  double* fro2;      // [nz] ||W||_F^2, zeroed before launch
  int flop_slot;     // stat slot that accumulates the algorithmic flops (as the scalar kernel)
  int bmark;         // workspace of n ints: last sweep in which each column was rotated
  int count_nonconv; // 1: a product that hits max_sweeps counts in IS_NONCONV
  int sweep_slot;    // -1, or stat slot accumulating the sweeps run per product
  int* svd_log;      // nullptr, or this SVD's record of product 0 (stride svd_stride per product)
  int svd_stride, svd_field;
  int init_v;        // 1: V starts at I; 0: V holds a starting rotation
  int islot_pred;    // -1, or istat slot: only products whose slot is non-zero take part
};

// Pair `i` of round `r` of the round-robin tournament on `k` (even) players.
__device__ __forceinline__ void jr_pair(int k, int r, int i, int& p, int& q) {
  if (i == 0) {
    p = k - 1;
    q = r;
  } else {
    p = (r + i) % (k - 1);
    q = (r - i + k - 1) % (k - 1);
  }
}

template <typename T>
__device__ __forceinline__ T jr_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Shared state of one CTA for the block pair it holds.
template <typename T, int B>
struct JrShared {
  T q[2 * B][2 * B + 1];      // accumulated rotations of the block round (row-major Q[r][c])
  int mark[2 * B];            // last sweep in which each local column was rotated
  int col[2 * B];             // global column index, or -1 for a column beyond n
  int dirty[2 * B];
  int nrot;
};

// Test and rotate the local pair (p, q) held in x (column p) and y (column q), rows
// lane + 32 k. Returns true when the pair was rotated (x and y then hold the new columns).
template <typename T, int B, int R>
__device__ __forceinline__ bool jr_visit(JrShared<T, B>& S, const JResArgs& a, int p, int q, int m, int n,
                                         int sweep, double fro, T (&x)[R], T (&y)[R], double& flops) {
  const int lane = threadIdx.x & 31;
  if (S.col[p] < 0 || S.col[q] < 0) return false;
  if (sweep >= 1 && S.mark[p] < sweep - 1 && S.mark[q] < sweep - 1) return false;
  T al = 0, be = 0, ga = 0;
#pragma unroll
  for (int k = 0; k < R; ++k) {
    al = fma(x[k], x[k], al);
    be = fma(y[k], y[k], be);
    ga = fma(x[k], y[k], ga);
  }
  al = jr_sum(al);
  be = jr_sum(be);
  ga = jr_sum(ga);
  flops += 6.0 * m;
  const double aga = fabs((double)ga);
  const double big = sqrt((double)(al > be ? al : be));
  if (!(ga != T(0) && aga > a.tol * sqrt((double)al) * sqrt((double)be) && aga > a.delta * big * fro)) return false;
  // zeta = (beta - alpha) / (2 gamma); t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2))
  const T zeta = (be - al) / (T(2) * ga);
  const T tt = copysign(T(1), zeta) / (fabs(zeta) + hypot(T(1), zeta));
  const T c = T(1) / sqrt(fma(tt, tt, T(1)));
  const T s = c * tt;
#pragma unroll
  for (int k = 0; k < R; ++k) {
    const T xp = x[k], yq = y[k];
    x[k] = c * xp - s * yq;
    y[k] = fma(s, xp, c * yq);
  }
  if (lane < 2 * B) {  // Q <- Q J on columns p, q (rows of Q are the lanes)
    const T qp = S.q[lane][p], qq = S.q[lane][q];
    S.q[lane][p] = c * qp - s * qq;
    S.q[lane][q] = fma(s, qp, c * qq);
  }
  if (lane == 0) {
    S.mark[p] = sweep;
    S.mark[q] = sweep;
    S.dirty[p] = 1;
    S.dirty[q] = 1;
    atomicAdd(&S.nrot, 1);
  }
  flops += 6.0 * m + 6.0 * n;
  return true;
}

// R: rows per lane (m <= 32 R). One CTA of B warps per block pair; dynamic shared memory
// holds the 2B columns (2B x 32R elements).
template <typename T, int B, int R>
__global__ void __launch_bounds__(B * 32) jacobi_res_kernel(JResArgs a) {
  extern __shared__ __align__(16) unsigned char jr_raw[];
  T* jr_cols = reinterpret_cast<T*>(jr_raw);  // [2B][32R]
  __shared__ JrShared<T, B> S;
  constexpr int MR = 32 * R;
  cg::grid_group grid = cg::this_grid();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const long gthread = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long nthreads = (long)gridDim.x * blockDim.x;
  const int nz = a.t.nz;
  auto active = [&](int z) { return a.islot_pred < 0 || a.t.istat[z * a.t.nis + a.islot_pred] != 0; };
  {  // every CTA reads the same flags, so all leave together before the first barrier
    bool any = false;
    for (int z = 0; z < nz; ++z) any = any || active(z);
    if (!any) return;
  }

  for (int z = 0; z < nz; ++z) {
    if (!active(z)) continue;
    const int n = a.n.eval(a.t, z), m = a.m.eval(a.t, z);
    T* V = reinterpret_cast<T*>(bufp(a.t, z, a.bv));
    if (a.init_v)
      for (long e = gthread; e < (long)n * n; e += nthreads) V[e] = (e % n == e / n) ? T(1) : T(0);
    int* mark = reinterpret_cast<int*>(bufp(a.t, z, a.bmark));
    for (long e = gthread; e < n; e += nthreads) mark[e] = -2;
    const T* W = reinterpret_cast<const T*>(bufp(a.t, z, a.bw));
    double f = 0.0;
    for (long e = gthread; e < (long)m * n; e += nthreads) f = fma((double)W[e], (double)W[e], f);
    f = warp_sum(f);
    if (lane == 0 && f != 0.0) atomicAdd(&a.fro2[z], f);
  }
  grid.sync();

  const int half = a.nblk_pad_ub / 2;
  const long items = (long)nz * half;
  double flops = 0.0;
  int sweeps_done = 0;
  for (int sweep = 0; sweep < a.max_sweeps; ++sweep) {
    for (int r = 0; r < a.nblk_pad_ub - 1; ++r) {
      for (long it = blockIdx.x; it < items; it += gridDim.x) {
        const int z = (int)(it / half), i = (int)(it % half);
        if (!active(z)) continue;
        const int n = a.n.eval(a.t, z);
        const int nb = (n + B - 1) / B;
        const int nbp = nb + (nb & 1);
        if (i >= nbp / 2 || r >= nbp - 1) continue;
        if (sweep > 0 && __ldcg(&a.counters[z * a.max_sweeps + sweep - 1]) == 0) continue;
        int P, Q;
        jr_pair(nbp, r, i, P, Q);
        const int m = a.m.eval(a.t, z);
        T* W = reinterpret_cast<T*>(bufp(a.t, z, a.bw));
        T* V = reinterpret_cast<T*>(bufp(a.t, z, a.bv));
        int* mark = reinterpret_cast<int*>(bufp(a.t, z, a.bmark));
        const double fro = sqrt(__ldcg(&a.fro2[z]));
        // stage the block pair: local columns 0..B-1 from block P, B..2B-1 from block Q
        if (threadIdx.x < 2 * B) {
          const int c = threadIdx.x;
          const int g = (c < B ? P * B + c : Q * B + c - B);
          const bool ok = (c < B ? P : Q) < nb && g < n;
          S.col[c] = ok ? g : -1;
          S.mark[c] = ok ? __ldcg(&mark[g]) : -2;
          S.dirty[c] = 0;
        }
        for (int e = threadIdx.x; e < 2 * B * (2 * B + 1); e += blockDim.x) {
          const int rr = e / (2 * B + 1), cc = e % (2 * B + 1);
          S.q[rr][cc] = (rr == cc) ? T(1) : T(0);
        }
        if (threadIdx.x == 0) S.nrot = 0;
        for (int e = threadIdx.x; e < 2 * B * MR; e += blockDim.x) {
          const int c = e / MR, row = e % MR;
          const int g = (c < B ? P * B + c : Q * B + c - B);
          const bool ok = (c < B ? P : Q) < nb && g < n && row < m;
          jr_cols[e] = ok ? __ldcg(W + (long)g * m + row) : T(0);
        }
        __syncthreads();
        T x[R], y[R];
        // pairs inside each block, once per sweep
        if (r == 0) {
          for (int s = 0; s < B - 1; ++s) {
            const int h = wid < B / 2 ? 0 : B, iw = wid % (B / 2);
            int p, q;
            jr_pair(B, s, iw, p, q);
            p += h;
            q += h;
            T* cp = jr_cols + p * MR;
            T* cq = jr_cols + q * MR;
#pragma unroll
            for (int k = 0; k < R; ++k) {
              x[k] = cp[lane + 32 * k];
              y[k] = cq[lane + 32 * k];
            }
            if (jr_visit<T, B, R>(S, a, p, q, m, n, sweep, fro, x, y, flops)) {
#pragma unroll
              for (int k = 0; k < R; ++k) {
                cp[lane + 32 * k] = x[k];
                cq[lane + 32 * k] = y[k];
              }
            }
            __syncthreads();
          }
        }
        // pairs across the two blocks: warp w keeps local column w in registers
        {
          const int p = wid;
          T* cp = jr_cols + p * MR;
#pragma unroll
          for (int k = 0; k < R; ++k) x[k] = cp[lane + 32 * k];
          bool px = false;
          for (int s = 0; s < B; ++s) {
            const int q = B + (wid + s) % B;
            T* cq = jr_cols + q * MR;
#pragma unroll
            for (int k = 0; k < R; ++k) y[k] = cq[lane + 32 * k];
            if (jr_visit<T, B, R>(S, a, p, q, m, n, sweep, fro, x, y, flops)) {
              px = true;
#pragma unroll
              for (int k = 0; k < R; ++k) cq[lane + 32 * k] = y[k];
            }
            __syncthreads();
          }
          if (px) {
#pragma unroll
            for (int k = 0; k < R; ++k) cp[lane + 32 * k] = x[k];
          }
        }
        __syncthreads();
        // write back the rotated columns, the marks and V <- V Q
        if (S.nrot > 0) {
          for (int e = threadIdx.x; e < 2 * B * MR; e += blockDim.x) {
            const int c = e / MR, row = e % MR;
            if (S.dirty[c] && row < m) W[(long)S.col[c] * m + row] = jr_cols[e];
          }
          if (threadIdx.x < 2 * B && S.col[threadIdx.x] >= 0) mark[S.col[threadIdx.x]] = S.mark[threadIdx.x];
          for (int row = threadIdx.x; row < n; row += blockDim.x) {
            T v[2 * B], o[2 * B];
#pragma unroll
            for (int c = 0; c < 2 * B; ++c) {
              v[c] = S.col[c] >= 0 ? __ldcg(V + (long)S.col[c] * n + row) : T(0);
              o[c] = T(0);
            }
#pragma unroll
            for (int c = 0; c < 2 * B; ++c)
#pragma unroll
              for (int j = 0; j < 2 * B; ++j) o[j] = fma(v[c], S.q[c][j], o[j]);
#pragma unroll
            for (int c = 0; c < 2 * B; ++c)
              if (S.dirty[c]) V[(long)S.col[c] * n + row] = o[c];
          }
          if (threadIdx.x == 0) atomicAdd(&a.counters[z * a.max_sweeps + sweep], S.nrot);
        }
        __syncthreads();  // the shared state is reused by the CTA's next item
      }
      grid.sync();
    }
    sweeps_done = sweep + 1;
    bool all = true;
    for (int z = 0; z < nz; ++z)
      if (__ldcg(&a.counters[z * a.max_sweeps + sweep]) != 0) all = false;
    if (all) break;
  }
  // every lane of a warp counted the same visits
  if (lane == 0 && flops > 0.0) atomicAdd(&a.t.stat[a.flop_slot], flops);
  if (gthread == 0) {
    for (int z = 0; z < nz; ++z) {
      if (!active(z)) continue;
      int used = 0;
      bool conv = false;
      for (int s = 0; s < sweeps_done; ++s) {
        used = s + 1;
        if (__ldcg(&a.counters[z * a.max_sweeps + s]) == 0) {
          conv = true;
          break;
        }
      }
      int* is = a.t.istat + z * a.t.nis;
      if (used > is[IS_SWEEPS_MAX]) is[IS_SWEEPS_MAX] = used;
      if (a.count_nonconv && !conv && a.n.eval(a.t, z) > 1) is[IS_NONCONV] += 1;
      if (a.sweep_slot >= 0) a.t.stat[z * a.t.ns + a.sweep_slot] += used;
      if (a.svd_log) a.svd_log[(long)z * a.svd_stride + a.svd_field] = used;
    }
  }
}

}  // namespace ttm
