// ttm_newton.cuh -- float64 refinement of the Swap SVD (Fig. 1C, Eq. eps) by Newton steps.
//
// After the float32 Jacobi passes the Swap holds W = Theta V (float64, m x n) whose columns
// are orthogonal to float32 accuracy, and V (n x n) orthonormal to float32 accuracy. A Newton
// step makes both exact to second order with one right factor X = I + Y applied to W and V:
//     V' = V X with V'^T V' = I      and      W' = W X with W'^T W' diagonal.
// With M = V^T V = I + E, G = W^T W and d_i = G_ii, the first-order conditions give
//     sym(Y) = -E / 2,
//     skew(Y) = S,  S_ij = (E_ij (d_i + d_j) / 2 - G_ij) / (d_i - d_j)        (i != j),
// the generalisation of a Jacobi rotation angle t_ij = G_ij / (d_j - d_i) to all pairs at
// once, together with the first step of the polar factor of V. Residual couplings and the
// orthogonality defect fall quadratically. W' = Theta V' keeps holding because both factors
// take the same X. All work is GEMM-shaped except the elementwise formation of X below.
//
// Which pairs a step rotates (S_ij = 0 for the others):
//   - only pairs that can matter for the truncation: the larger of d_i, d_j at least
//     kNewtonRelevance times the squared singular value at the provisional cut (the Eq. eps
//     rank and cap applied to the column norms before the first step). Pairs far below the
//     cut are dropped together whatever their coupling, and their columns still carry
//     couplings at float32 level inherited from the float32 passes, which a first-order
//     step cannot resolve;
//   - couplings above the float64 noise floor kNewtonFloor sqrt(max(d_i, d_j) trace G), the
//     floor of the float64 Jacobi (a coupling g left below it leaks at most g / |w_big| of a
//     kept column into a dropped one, so the floor bounds what an exact product loses);
//   - |S_ij| <= kNewtonMaxS: a pair nearly degenerate relative to its coupling is left
//     alone (counted as frozen).
// The steps need the float32 passes to have resolved every relevant pair to float32
// accuracy, including the small columns: the float64 apply W <- W V32 of a pass leaks a
// float32-size part of the large columns into the small ones, and the last float32 pass
// (whose rotations are tiny) is what removes that leakage before the Newton steps.
// A step in E-only mode applies the polar correction alone (S = 0). A product whose last
// step leaves max(|S_ij|, |E_ij| / 2) above kNewtonConverged takes the fallback path of the
// Swap (float64 one-sided Jacobi from the state before the Newton steps).
#pragma once
#include "ttm_common.cuh"

namespace ttm {

constexpr double kNewtonMaxS = 0.25;
constexpr double kNewtonRelevance = 1e-6;
constexpr double kNewtonFloor = 64 * 1.11e-16;

struct NewtonArgs {
  Tables t;
  int bg, bm, bx;    // G = W^T W and M = V^T V (n x n column-major, upper triangle valid); X out
  Dim n;
  int bsort, ikprov; // sorted squared column norms and the provisional rank (relevance cut)
  int slot_trace;    // stat slot holding trace G = ||W||_F^2 (from the provisional truncation)
  int eonly;         // 1: S = 0 (polar correction of V only)
  int slot_smax;     // stat slot receiving max(|S_ij|, |E_ij| / 2) over the product (-1: none)
  int islot_frozen;  // istat slot counting the pairs left unrotated (-1: none)
  int islot_pred;    // -1, or istat slot: products whose slot is 0 get X = I
};

__device__ __forceinline__ void atomic_max_pos(double* p, double v) {
  // non-negative doubles order like their bit patterns
  atomicMax(reinterpret_cast<unsigned long long*>(p), (unsigned long long)__double_as_longlong(v));
}

// One thread per element X_ij (column-major, i = row).
__global__ void newton_x_kernel(NewtonArgs a) {
  const int z = blockIdx.z;
  const int n = a.n.eval(a.t, z);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const bool off = a.islot_pred >= 0 && a.t.istat[z * a.t.nis + a.islot_pred] == 0;
  double smax = 0.0;
  int frozen = 0;
  if (i < n && j < n) {
    double x;
    if (off) {
      x = (i == j) ? 1.0 : 0.0;
    } else {
      const double* G = bufp(a.t, z, a.bg);
      const double* M = bufp(a.t, z, a.bm);
      const int lo = min(i, j), hi = max(i, j);
      const double e = M[lo + (long)hi * n] - (i == j ? 1.0 : 0.0);
      if (i == j) {
        x = 1.0 - 0.5 * e;
        smax = 0.5 * fabs(e);
      } else {
        double s = 0.0;
        if (!a.eonly) {
          const double g = G[lo + (long)hi * n];
          const double di = G[i + (long)i * n], dj = G[j + (long)j * n];
          const double dmax = fmax(di, dj);
          const int kp = bondv(a.t, z, a.ikprov);
          const double dcut = bufp(a.t, z, a.bsort)[max(0, min(kp, n) - 1)];
          const double tr = a.t.stat[z * a.t.ns + a.slot_trace];
          const double num = 0.5 * e * (di + dj) - g, den = di - dj;
          const bool relevant = dmax >= kNewtonRelevance * dcut &&
                                fabs(num) > kNewtonFloor * sqrt(dmax * tr);
          if (relevant) {
            if (fabs(num) <= kNewtonMaxS * fabs(den))
              s = num / den;
            else
              frozen = (i < j) ? 1 : 0;
          }
        }
        smax = fmax(fabs(s), 0.5 * fabs(e));
        x = s - 0.5 * e;
      }
    }
    bufp(a.t, z, a.bx)[i + (long)j * n] = x;
  }
  // block-level reduction of the diagnostics
  __shared__ double s_max[32];
  __shared__ int s_frz[32];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, lane = tid & 31, w = tid >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o));
    frozen += __shfl_xor_sync(0xffffffffu, frozen, o);
  }
  if (lane == 0) {
    s_max[w] = smax;
    s_frz[w] = frozen;
  }
  __syncthreads();
  if (tid == 0) {
    const int nw = (blockDim.x * blockDim.y + 31) >> 5;
    double m = 0.0;
    int f = 0;
    for (int q = 0; q < nw; ++q) {
      m = fmax(m, s_max[q]);
      f += s_frz[q];
    }
    if (a.slot_smax >= 0 && !(m <= 0.0)) atomic_max_pos(&a.t.stat[z * a.t.ns + a.slot_smax], m == m ? m : 1e300);
    if (a.islot_frozen >= 0 && f > 0) atomicAdd(&a.t.istat[z * a.t.nis + a.islot_frozen], f);
  }
}

// Before an extra Newton step: IS_NEWTON_MORE = 1 for a product whose last correction is still
// above kNewtonConverged (its ST_NEWTON_CUR is reset to record the extra step); the others keep
// their residual and skip the step.
__global__ void newton_more_kernel(Tables t) {
  const int z = blockIdx.x * blockDim.x + threadIdx.x;
  if (z >= t.nz) return;
  double* st = t.stat + z * t.ns;
  const bool more = !(st[ST_NEWTON_CUR] <= kNewtonConverged);
  t.istat[z * t.nis + IS_NEWTON_MORE] = more ? 1 : 0;
  if (more) st[ST_NEWTON_CUR] = 0.0;
}

// After the last Newton step: IS_FALLBACK = 1 for a product whose residual stayed above
// kNewtonConverged (it is counted in IS_NEWTON_BAD and its Swap finishes on the fallback
// path), the largest residual of the product is kept in ST_NEWTON_RES, and ST_NEWTON_CUR is
// reset for the next Swap.
__global__ void newton_check_kernel(Tables t) {
  const int z = blockIdx.x * blockDim.x + threadIdx.x;
  if (z >= t.nz) return;
  double* st = t.stat + z * t.ns;
  int* is = t.istat + z * t.nis;
  const double res = st[ST_NEWTON_CUR];
  st[ST_NEWTON_CUR] = 0.0;
  const bool bad = !(res <= kNewtonConverged);
  is[IS_FALLBACK] = bad ? 1 : 0;
  if (bad) is[IS_NEWTON_BAD] += 1;
  else if (res > st[ST_NEWTON_RES]) st[ST_NEWTON_RES] = res;
}

// Elementwise copy of a rows x cols buffer for the products whose istat slot equals `want`
// (islot < 0: every product).
struct PredCopyArgs {
  Tables t;
  int bsrc, bdst;
  Dim rows, cols;
  int islot, want;
};
__global__ void pred_copy_kernel(PredCopyArgs a) {
  const int z = blockIdx.y;
  if (a.islot >= 0 && a.t.istat[z * a.t.nis + a.islot] != a.want) return;
  const long n = (long)a.rows.eval(a.t, z) * a.cols.eval(a.t, z);
  const double* s = bufp(a.t, z, a.bsrc);
  double* d = bufp(a.t, z, a.bdst);
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) d[e] = s[e];
}

// A GEMM of the functor F for the products whose istat slot equals `want`; the others see an
// empty problem and their launch blocks exit at once.
template <class F>
struct PredFn {
  F f;
  int islot, want;
  Tables t;
  __device__ GemmDesc operator()(int z, int b) const {
    GemmDesc g = f(z, b);
    if (f.t.istat[z * f.t.nis + islot] != want) g.M = 0;
    return g;
  }
};

}  // namespace ttm
