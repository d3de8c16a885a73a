// ttm_svd.cuh -- truncated SVD of the Swap (Fig. 1C, Eq. eps) on the GPU in float64.
//
// Method: one-sided Jacobi (Hestenes 1958; the column-pair ordering is the
// round-robin tournament of Brent & Luk 1985). The m x n matrix W (initially Theta,
// column-major) is multiplied from the right by plane rotations until its columns
// are mutually orthogonal; the same rotations accumulate into V (n x n, starting at
// I). Then W = Theta V exactly up to rounding, the column norms of W are the
// singular values, and
//     new left carriage  = W[:, top k]   (= U Lambda: the singular values travel
//                                          with the mover, the gauge centre follows)
//     new right carriage = V[:, top k]^T (right-orthonormal to float64 rounding).
// No Gram matrix is formed, so small singular values keep relative accuracy and the
// untruncated product stays exact. The rank k follows Eq. eps on the sorted norms.
//
// All kernels are batched over the products of a launch; the Jacobi sweep is one
// cooperative launch with a grid-wide barrier after every round of n/2 disjoint
// column pairs.
#pragma once
#include <cooperative_groups.h>
#include "ttm_common.cuh"

namespace cg = cooperative_groups;

namespace ttm {

struct HestArgs {
  Tables t;
  int bw, bv;        // W: m x n column-major (in/out), V: n x n column-major (in/out)
  Dim m, n;
  int npad_ub;       // even host upper bound of n
  int max_sweeps;
  int* counters;     // [nz][max_sweeps] rotations per sweep, zeroed before launch
  double tol;        // rotate when |w_p . w_q| > tol * |w_p| |w_q| ...
  double delta;      // ... and |w_p . w_q| > delta * max(|w_p|, |w_q|) * ||W||_F
  double* fro2;      // [nz] ||W||_F^2, zeroed before launch
  int init_v;        // 1: start from V = I; 0: V holds a starting rotation
  int flop_slot;     // stat slot that accumulates the executed flops
  int bmark;         // workspace of n ints: last sweep in which each column was rotated
  int count_nonconv; // 1: a product that hits max_sweeps counts in IS_NONCONV
  int islot_pred;    // -1, or istat slot: only products whose slot is non-zero take part
  int sweep_slot;    // -1, or stat slot accumulating the sweeps run per product
  int* svd_log;      // nullptr, or this SVD's record of product 0 (stride svd_stride per product)
  int svd_stride, svd_field;
};

template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ int ldcg_int(const int* p) { return __ldcg(p); }

// Rows per lane per chunk: float covers 1024 rows per warp pass, double 512 (register budget).
template <typename T> struct ChunkOf { static constexpr int value = 32; };
template <> struct ChunkOf<double> { static constexpr int value = 16; };

// Partial sums of |x|^2, |y|^2, x.y over rows [base, base + 1024) of two columns, the
// chunk kept in registers (kChunk independent loads in flight per lane).
template <typename T, int kChunk = ChunkOf<T>::value>
__device__ __forceinline__ void load_chunk(const T* xp, const T* yp, int base, int rows, int lane,
                                           T (&x)[kChunk], T (&y)[kChunk]) {
#pragma unroll
  for (int k = 0; k < kChunk; ++k) {
    const int r = base + lane + 32 * k;
    x[k] = r < rows ? __ldcg(xp + r) : T(0);
    y[k] = r < rows ? __ldcg(yp + r) : T(0);
  }
}
template <typename T, int kChunk = ChunkOf<T>::value>
__device__ __forceinline__ void store_rotated(T* xp, T* yp, int base, int rows, int lane,
                                              const T (&x)[kChunk], const T (&y)[kChunk], T c, T s) {
#pragma unroll
  for (int k = 0; k < kChunk; ++k) {
    const int r = base + lane + 32 * k;
    if (r < rows) {
      xp[r] = c * x[k] - s * y[k];
      yp[r] = fma(s, x[k], c * y[k]);
    }
  }
}
template <typename T>
__device__ __forceinline__ void rotate_columns(T* xp, T* yp, int rows, int lane, T c, T s) {
  constexpr int kChunk = ChunkOf<T>::value;
  T x[kChunk], y[kChunk];
  for (int base = 0; base < rows; base += 32 * kChunk) {
    load_chunk(xp, yp, base, rows, lane, x, y);
    store_rotated(xp, yp, base, rows, lane, x, y, c, s);
  }
}

// One-sided Jacobi in precision T (float: the fast preconditioning pass; double: the
// polish). One warp handles one column pair, its rows in registers in chunks of 1024.
// Convergence test: a pair is rotated while its coupling is above both the relative
// test of one-sided Jacobi and an absolute floor tied to the larger of the two
// columns. A residual coupling gamma below delta |w_big| ||W||_F moves at most
// delta^2 ||W||_F^2 of weight across the truncation boundary, so it cannot change a
// truncation; and columns near rounding level carry absolute noise of order
// u ||W||_F that a purely relative test would keep chasing. The excess truncation
// error left by a relative coupling c is of order c^2 times the column weights, so
// the polish tolerance needs only c << 1, not c ~ u.
// A pair whose two columns were both left untouched since it last passed the test is
// skipped (its coupling cannot have changed).
template <typename T>
__global__ void __launch_bounds__(256) hestenes_kernel(HestArgs a) {
  cg::grid_group grid = cg::this_grid();
  const int lane = threadIdx.x & 31;
  const long gthread = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long nthreads = (long)gridDim.x * blockDim.x;
  // Work item i goes to warp (i mod gridDim.x) of CTA ..., i.e. consecutive items land on
  // different SMs, so a round with fewer items than warps still uses every SM.
  const long gwarp = (long)(threadIdx.x >> 5) * gridDim.x + blockIdx.x, nwarps = nthreads >> 5;
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
    const long tot = (long)n * n;
    int* mark = reinterpret_cast<int*>(bufp(a.t, z, a.bmark));
    for (long e = gthread; e < n; e += nthreads) mark[e] = -2;
    if (a.init_v)
      for (long e = gthread; e < tot; e += nthreads) V[e] = (e % n == e / n) ? T(1) : T(0);
    const T* W = reinterpret_cast<const T*>(bufp(a.t, z, a.bw));
    double f = 0.0;
    for (long e = gthread; e < (long)m * n; e += nthreads) f = fma((double)W[e], (double)W[e], f);
    f = warp_sum(f);
    if (lane == 0 && f != 0.0) atomicAdd(&a.fro2[z], f);
  }
  grid.sync();

  constexpr int kChunk = ChunkOf<T>::value;
  const int half = a.npad_ub / 2;
  const long items = (long)nz * half;
  double flops = 0.0;
  int sweeps_done = 0;
  for (int sweep = 0; sweep < a.max_sweeps; ++sweep) {
    for (int r = 0; r < a.npad_ub - 1; ++r) {
      for (long it = gwarp; it < items; it += nwarps) {
        const int z = (int)(it / half), i = (int)(it % half);
        if (!active(z)) continue;
        const int n = a.n.eval(a.t, z);
        const int npad = n + (n & 1);
        if (i >= npad / 2 || r >= npad - 1) continue;
        int p, q;
        if (i == 0) {
          p = npad - 1; q = r;
        } else {
          p = (r + i) % (npad - 1);
          q = (r - i + npad - 1) % (npad - 1);
        }
        if (p >= n || q >= n) continue;
        const int m = a.m.eval(a.t, z);
        int* mark = reinterpret_cast<int*>(bufp(a.t, z, a.bmark));
        T* W = reinterpret_cast<T*>(bufp(a.t, z, a.bw));
        T* wp = W + (long)p * m;
        T* wq = W + (long)q * m;
        // Every load of the pair is issued before any of them is tested: the product's
        // convergence counter, both marks, ||W||_F^2 and the first chunk of both columns
        // travel together, so a round costs one memory round trip instead of several.
        const int prev = sweep > 0 ? ldcg_int(&a.counters[z * a.max_sweeps + sweep - 1]) : 1;
        const int mp = sweep >= 1 ? ldcg_int(&mark[p]) : 0;
        const int mq = sweep >= 1 ? ldcg_int(&mark[q]) : 0;
        const double fro2 = __ldcg(&a.fro2[z]);
        T x[kChunk], y[kChunk];
        load_chunk(wp, wq, 0, m, lane, x, y);
        // float32: the two columns of V ride along when they fit one chunk (the rotation
        // of V needs only c and s), which removes the last dependent round trip.
        T* V = reinterpret_cast<T*>(bufp(a.t, z, a.bv));
        T* vp = V + (long)p * n;
        T* vq = V + (long)q * n;
        constexpr bool kPrefetchV = sizeof(T) == 4;
        T vx[kPrefetchV ? kChunk : 1], vy[kPrefetchV ? kChunk : 1];
        const bool vpre = kPrefetchV && n <= 32 * kChunk;
        if constexpr (kPrefetchV) {
          if (vpre) load_chunk(vp, vq, 0, n, lane, vx, vy);
        }
        if (prev == 0) continue;
        if (sweep >= 1 && mp < sweep - 1 && mq < sweep - 1) continue;
        T al = 0, be = 0, ga = 0;
        for (int base = 0; base < m; base += 32 * kChunk) {
          if (base > 0) load_chunk(wp, wq, base, m, lane, x, y);
#pragma unroll
          for (int k = 0; k < kChunk; ++k) {
            if (base + 32 * k < m) {  // warp-uniform: skips the zero padding of a short column
              al = fma(x[k], x[k], al);
              be = fma(y[k], y[k], be);
              ga = fma(x[k], y[k], ga);
            }
          }
        }
        al = warp_sum_t(al);
        be = warp_sum_t(be);
        ga = warp_sum_t(ga);
        flops += 6.0 * m;
        const double fro = sqrt(fro2);
        const double aga = fabs((double)ga);
        const double big = sqrt((double)(al > be ? al : be));
        if (ga != T(0) && aga > a.tol * sqrt((double)al) * sqrt((double)be) && aga > a.delta * big * fro) {
          // zeta = (beta - alpha) / (2 gamma); t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2))
          const T zeta = (be - al) / (T(2) * ga);
          const T tt = copysign(T(1), zeta) / (fabs(zeta) + hypot(T(1), zeta));
          const T c = T(1) / sqrt(fma(tt, tt, T(1)));
          const T s = c * tt;
          if (m <= 32 * kChunk)
            store_rotated(wp, wq, 0, m, lane, x, y, c, s);
          else
            rotate_columns(wp, wq, m, lane, c, s);
          if constexpr (kPrefetchV) {
            if (vpre)
              store_rotated(vp, vq, 0, n, lane, vx, vy, c, s);
            else
              rotate_columns(vp, vq, n, lane, c, s);
          } else {
            rotate_columns(vp, vq, n, lane, c, s);
          }
          flops += 6.0 * m + 6.0 * n;
          if (lane == 0) {
            atomicAdd(&a.counters[z * a.max_sweeps + sweep], 1);
            mark[p] = sweep;
            mark[q] = sweep;
          }
        }
      }
      grid.sync();
    }
    sweeps_done = sweep + 1;
    bool all = true;
    for (int z = 0; z < nz; ++z)
      if (ldcg_int(&a.counters[z * a.max_sweeps + sweep]) != 0) all = false;
    if (all) break;
  }
  if (lane == 0 && flops > 0.0) atomicAdd(&a.t.stat[a.flop_slot], flops);
  if (gthread == 0) {
    for (int z = 0; z < nz; ++z) {
      if (!active(z)) continue;
      int used = 0;
      bool conv = false;
      for (int s = 0; s < sweeps_done; ++s) {
        used = s + 1;
        if (ldcg_int(&a.counters[z * a.max_sweeps + s]) == 0) { conv = true; break; }
      }
      int* is = a.t.istat + z * a.t.nis;
      if (used > is[IS_SWEEPS_MAX]) is[IS_SWEEPS_MAX] = used;
      if (a.count_nonconv && !conv && a.n.eval(a.t, z) > 1) is[IS_NONCONV] += 1;
      if (a.sweep_slot >= 0) a.t.stat[z * a.t.ns + a.sweep_slot] += used;
      if (a.svd_log) a.svd_log[(long)z * a.svd_stride + a.svd_field] = used;
    }
  }
}

// Elementwise precision change between workspaces (n elements of m*n etc.).
struct CastArgs {
  Tables t;
  int bsrc, bdst;
  Dim rows, cols;
  int to_float;   // 1: double -> float, 0: float -> double, 2: double identity (rows x rows)
};
constexpr int kCastExpBias = 4096;
__global__ void cast_kernel(CastArgs a) {
  const int z = blockIdx.y;
  const int rows = a.rows.eval(a.t, z);
  const long n = (long)rows * a.cols.eval(a.t, z);
  // double -> float copies are scaled by 2^-e (e: binary exponent of max |W|, set by
  // absmax_exp_kernel), so that the float copy of a matrix of small norm keeps its small
  // entries out of the float32 subnormal range (the Jacobi rotations are scale-invariant)
  const int eb = a.t.istat[z * a.t.nis + IS_CAST_EXP];
  const int sh = eb > 0 ? -(eb - kCastExpBias) : 0;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    if (a.to_float == 2)
      bufp(a.t, z, a.bdst)[e] = (e % rows == e / rows) ? 1.0 : 0.0;
    else if (a.to_float)
      reinterpret_cast<float*>(bufp(a.t, z, a.bdst))[e] = (float)ldexp(bufp(a.t, z, a.bsrc)[e], sh);
    else
      bufp(a.t, z, a.bdst)[e] = (double)reinterpret_cast<const float*>(bufp(a.t, z, a.bsrc))[e];
  }
}

// Binary exponent of max |X| of a rows x cols matrix, biased by kCastExpBias, into
// IS_CAST_EXP (reset to 0 by the first block row of reset_cast_exp_kernel before).
__global__ void reset_cast_exp_kernel(Tables t) {
  const int z = threadIdx.x + blockIdx.x * blockDim.x;
  if (z < t.nz) t.istat[z * t.nis + IS_CAST_EXP] = 0;
}
__global__ void absmax_exp_kernel(CastArgs a) {
  const int z = blockIdx.y;
  const long n = (long)a.rows.eval(a.t, z) * a.cols.eval(a.t, z);
  const double* x = bufp(a.t, z, a.bsrc);
  double m = 0.0;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
    m = fmax(m, fabs(x[e]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.0 && m == m) {
    int e;
    frexp(m, &e);
    atomicMax(&a.t.istat[z * a.t.nis + IS_CAST_EXP], e + kCastExpBias);
  }
}

// Squared column norms of W (warp per column).
struct NormArgs {
  Tables t;
  int bw, bnrm;
  Dim m, n;
};
__global__ void colnorm_kernel(NormArgs a) {
  const int z = blockIdx.y;
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  const int n = a.n.eval(a.t, z);
  if (j >= n) return;
  const int m = a.m.eval(a.t, z);
  const double* w = bufp(a.t, z, a.bw) + (long)j * m;
  double s = 0.0;
  for (int r = lane; r < m; r += 32) s = fma(w[r], w[r], s);
  s = warp_sum(s);
  if (lane == 0) bufp(a.t, z, a.bnrm)[j] = s;
}

// Descending order of the squared norms: rank by counting (ties by index), so the
// permutation is deterministic. perm is stored as int in a double buffer.
struct RankArgs {
  Tables t;
  int bnrm, bsorted, bperm;
  Dim n;
};
__global__ void rank_kernel(RankArgs a) {
  const int z = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = a.n.eval(a.t, z);
  if (j >= n) return;
  const double* nr = bufp(a.t, z, a.bnrm);
  // squared norms are >= 0; a NaN sorts last, so that perm stays a permutation
  auto key = [](double x) { return x == x ? x : -1.0; };
  const double v = key(nr[j]);
  int rank = 0;
  for (int i = 0; i < n; ++i) {
    const double u = key(nr[i]);
    rank += (u > v) || (u == v && i < j);
  }
  bufp(a.t, z, a.bsorted)[rank] = v;
  reinterpret_cast<int*>(bufp(a.t, z, a.bperm))[rank] = j;
}

// Eq. eps (strict), then the cap, then 1 <= k <= min(m, n). One block per product.
// The discarded tail sum_{j>=k} lambda_j^2 is summed from the small end.
struct TruncArgs {
  Tables t;
  int bsorted;
  Dim m, n;
  int inew;       // bond id that receives k
  double eps;
  int cap;        // 0 = none
  int wslot;      // stat slot for this truncation's discarded weight (-1: none)
  int record;     // 1: final decision (statistics); 0: provisional (bond value only)
  int ikeep;      // -1, or (final rounding) the bond id of the current bond: when the
                  // product's rounding gate IS_ROUND is 0 no output bond exceeds chi_out,
                  // and the SVD keeps that many values (an exact refactorisation)
  int tslot;      // -1, or stat slot receiving the total sum_j lambda_j^2
  int* svd_log;   // nullptr, or this SVD's record of product 0 (stride svd_stride per product)
  int svd_stride;
};
__global__ void __launch_bounds__(1024) truncate_kernel(TruncArgs a) {
  const int z = blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int n = a.n.eval(a.t, z), m = a.m.eval(a.t, z);
  const double* s = bufp(a.t, z, a.bsorted);
  __shared__ double part[1024];
  __shared__ int kbest;
  const int per = (n + nt - 1) / nt;
  const int lo = min(n, tid * per), hi = min(n, lo + per);
  double loc = 0.0;
  for (int j = hi - 1; j >= lo; --j) loc += s[j];
  part[tid] = loc;
  if (tid == 0) kbest = n;
  __syncthreads();
  // inclusive suffix scan over the chunk sums (Hillis-Steele from the right)
  for (int off = 1; off < nt; off <<= 1) {
    const double add = (tid + off < nt) ? part[tid + off] : 0.0;
    __syncthreads();
    part[tid] += add;
    __syncthreads();
  }
  const double total = part[0];
  const double right = (tid + 1 < nt) ? part[tid + 1] : 0.0;
  // tail(kk) = sum_{j >= kk} s[j]; candidates kk in [max(lo,1), hi]
  double tail = right;
  for (int kk = hi; kk >= lo; --kk) {
    if (kk < hi) tail += s[kk];
    if (kk >= 1 && a.eps > 0.0 && tail < a.eps * total) atomicMin(&kbest, kk);
  }
  __syncthreads();
  if (tid == 0) {
    int k = kbest;
    if (!(total == total) || total > 1.79e308) atomicExch(&a.t.istat[z * a.t.nis + IS_STATUS], (int)TTM_ERR_NONFINITE);
    if (!(total > 0.0)) k = 1;
    if (a.cap > 0 && k > a.cap) k = a.cap;
    if (a.ikeep >= 0 && a.t.istat[z * a.t.nis + IS_ROUND] == 0) k = bondv(a.t, z, a.ikeep);
    const int kmax = max(1, min(m, n));
    k = max(1, min(k, kmax));
    double w = 0.0;
    for (int j = n - 1; j >= k; --j) w += s[j];
    a.t.bond[z * a.t.nbd + a.inew] = k;
    if (a.tslot >= 0) a.t.stat[z * a.t.ns + a.tslot] = total;
    if (!a.record) return;
    double* st = a.t.stat + z * a.t.ns;
    st[ST_WSUM] += w;
    st[ST_WSQRT] += sqrt(w);
    if (a.wslot >= 0) st[a.wslot] = w;
    int* is = a.t.istat + z * a.t.nis;
    if (k > is[IS_MAX_BOND]) is[IS_MAX_BOND] = k;
    if (a.svd_log) {
      int* rec = a.svd_log + (long)z * a.svd_stride;
      rec[SR_M] = m;
      rec[SR_N] = n;
      rec[SR_K] = k;
      rec[SR_FALLBACK] = is[IS_FALLBACK];
    }
  }
}

// Gate of the final rounding (reading A4): IS_ROUND of a product becomes 1 when one of the
// listed bonds (the output's internal bonds before the rounding) exceeds the cap.
struct RoundGateArgs {
  Tables t;
  int n;          // ids used (<= 32)
  int ids[32];
  int cap;
};
__global__ void round_gate_kernel(RoundGateArgs a) {
  const int z = blockIdx.x;
  const int i = threadIdx.x;
  if (i < a.n && bondv(a.t, z, a.ids[i]) > a.cap) atomicOr(&a.t.istat[z * a.t.nis + IS_ROUND], 1);
}

// New carriages after a Swap: left[(l, t), j] = W[(l, t), perm[j]] (row-major
// [Dl][d][k]) and right[j, (s, r)] = V[(s, r), perm[j]] (row-major [k][d][Dr]).
struct GatherArgs {
  Tables t;
  int bw, bv, bperm, bleft, bright;
  int il, ir, ik;
  int d;
};
__global__ void swap_gather_kernel(GatherArgs a) {
  const int z = blockIdx.z;
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  const int Dl = bondv(a.t, z, a.il), Dr = bondv(a.t, z, a.ir), k = bondv(a.t, z, a.ik);
  if (j >= k) return;
  const int m = Dl * a.d, n = a.d * Dr;
  const int pj = reinterpret_cast<const int*>(bufp(a.t, z, a.bperm))[j];
  if (pj < 0 || pj >= n) return;  // cannot happen for a permutation; never read outside W
  if (row < m) bufp(a.t, z, a.bleft)[(long)row * k + j] = bufp(a.t, z, a.bw)[row + (long)pj * m];
  if (row < n) bufp(a.t, z, a.bright)[(long)j * n + row] = bufp(a.t, z, a.bv)[row + (long)pj * n];
}

}  // namespace ttm
