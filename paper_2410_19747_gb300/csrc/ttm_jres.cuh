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

// 16-byte vectors of T for the shared-memory traffic of a column: lane l holds rows
// 32 VW k + VW l + u (k < R / VW, u < VW), so a warp moves a column with R / VW 16-byte
// accesses per lane. VW = 1 (plain rows lane + 32 k) when R is not a multiple of the width.
template <typename T, int R> struct JrVec {
  static constexpr int W16 = 16 / (int)sizeof(T);
  static constexpr int VW = (R % W16 == 0) ? W16 : 1;
};
template <typename T, int VW> struct JrVecT { using type = T; };
template <> struct JrVecT<float, 4> { using type = float4; };
template <> struct JrVecT<double, 2> { using type = double2; };

template <typename T, int R>
__device__ __forceinline__ void jr_load(const T* col, int lane, T (&x)[R]) {
  constexpr int VW = JrVec<T, R>::VW;
  using V = typename JrVecT<T, VW>::type;
  const V* c = reinterpret_cast<const V*>(col);
#pragma unroll
  for (int k = 0; k < R / VW; ++k) {
    const V v = c[32 * k + lane];
    const T* e = reinterpret_cast<const T*>(&v);
#pragma unroll
    for (int u = 0; u < VW; ++u) x[VW * k + u] = e[u];
  }
}
template <typename T, int R>
__device__ __forceinline__ void jr_store(T* col, int lane, const T (&x)[R]) {
  constexpr int VW = JrVec<T, R>::VW;
  using V = typename JrVecT<T, VW>::type;
  V* c = reinterpret_cast<V*>(col);
#pragma unroll
  for (int k = 0; k < R / VW; ++k) {
    V v;
    T* e = reinterpret_cast<T*>(&v);
#pragma unroll
    for (int u = 0; u < VW; ++u) e[u] = x[VW * k + u];
    c[32 * k + lane] = v;
  }
}

// Rotation that zeroes the coupling g of two columns with squared norms a, b (one-sided
// Jacobi): t = sign(d) 2 g / (|d| + sqrt(d^2 + 4 g^2)), d = b - a (the usual
// t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), zeta = d / (2 g), multiplied through by 2|g|),
// c = 1 / sqrt(1 + t^2), s = c t. The float version scales d and g by their larger magnitude
// and uses the fast reciprocal square root and division (the rotation needs c^2 + s^2 = 1 to a
// few float ulps, which c = rsqrt(1 + t^2), s = c t gives); it declines (returns false) a pair
// whose d and g are below the normal float range.
template <typename T>
__device__ __forceinline__ bool jr_rot(T a, T b, T g, T& c, T& s) {
  const T zeta = (b - a) / (T(2) * g);
  const T tt = copysign(T(1), zeta) / (fabs(zeta) + hypot(T(1), zeta));
  c = T(1) / sqrt(fma(tt, tt, T(1)));
  s = c * tt;
  return true;
}
template <>
__device__ __forceinline__ bool jr_rot<float>(float a, float b, float g, float& c, float& s) {
  const float d = b - a;
  const float sc = fmaxf(fabsf(d), 2.f * fabsf(g));
  if (!(sc > 1e-36f)) return false;
  const float r = __fdividef(1.f, sc);
  const float dn = d * r, gn = g * r;                       // max(|dn|, 2|gn|) = 1
  const float q = fmaf(dn, dn, 4.f * gn * gn);              // in [1, 2]
  const float den = fabsf(dn) + q * rsqrtf(q);              // in [1, 1 + sqrt 2]
  float t = __fdividef(2.f * gn, den);
  if (dn < 0.f) t = -t;
  c = rsqrtf(fmaf(t, t, 1.f));
  s = c * t;
  return true;
}

// Shared state of one CTA for the block pair it holds. Rows of Q are padded to a multiple
// of 16 bytes (vector reads in the V update) that spreads the per-lane column updates over
// the banks.
template <typename T, int B>
struct JrShared {
  static constexpr int QS = 2 * B + 16 / (int)sizeof(T);
  alignas(16) T q[2 * B][QS];  // accumulated rotations of the block round (row-major Q[r][c])
  int mark[2 * B];             // last sweep in which each local column was rotated
  int col[2 * B];              // global column index, or -1 for a column beyond n
  int dirty[2 * B];
  int nrot;
};

// Visits and rotations of a thread, for the flop count (lane 0 of each warp counts).
struct JrCount {
  unsigned long long visit_rows = 0, rot_rows = 0;  // sum of m per visit; of m + n per rotation
};

// Test and rotate the local pair (p, q) held in x (column p) and y (column q). Returns true
// when the pair was rotated (x and y then hold the new columns). The tests run in T: the
// float copies are scaled to max |W| ~ 1, so tol, delta and the column norms stay in the
// normal float range, and the float64 pipe (1/64 of the float32 rate) is not touched in the
// float32 kernel. Four partial sums per dot product shorten the dependent FMA chains.
template <typename T, int B, int R>
__device__ __forceinline__ bool jr_visit(JrShared<T, B>& S, T tol, T delta, int p, int q, int m, int n,
                                         int sweep, T fro, T (&x)[R], T (&y)[R], JrCount& cnt) {
  const int lane = threadIdx.x & 31;
  if (S.col[p] < 0 || S.col[q] < 0) return false;
  if (sweep >= 1 && S.mark[p] < sweep - 1 && S.mark[q] < sweep - 1) return false;
  constexpr int NA = R >= 4 ? 4 : R;
  T al[NA], be[NA], ga[NA];
#pragma unroll
  for (int u = 0; u < NA; ++u) al[u] = be[u] = ga[u] = T(0);
#pragma unroll
  for (int k = 0; k < R; ++k) {
    al[k % NA] = fma(x[k], x[k], al[k % NA]);
    be[k % NA] = fma(y[k], y[k], be[k % NA]);
    ga[k % NA] = fma(x[k], y[k], ga[k % NA]);
  }
#pragma unroll
  for (int u = 1; u < NA; ++u) {
    al[0] += al[u];
    be[0] += be[u];
    ga[0] += ga[u];
  }
  const T a2 = jr_sum(al[0]), b2 = jr_sum(be[0]), g2 = jr_sum(ga[0]);
  if (lane == 0) cnt.visit_rows += m;
  const T aga = fabs(g2);
  // rotate when |g| > tol |w_p| |w_q| and |g| > delta max(|w_p|, |w_q|) ||W||_F
  bool rot;
  if constexpr (sizeof(T) == 4) {
    const float ra = rsqrtf(a2), rb = rsqrtf(b2);
    rot = g2 != 0.f && a2 > 0.f && b2 > 0.f && aga * ra * rb > tol && aga * fminf(ra, rb) > delta * fro;
  } else {
    const T big = sqrt(a2 > b2 ? a2 : b2);
    rot = g2 != T(0) && aga > tol * sqrt(a2) * sqrt(b2) && aga > delta * big * fro;
  }
  T c, s;
  if (!rot || !jr_rot<T>(a2, b2, g2, c, s)) return false;
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
    cnt.rot_rows += m + n;
  }
  return true;
}

// R: rows per lane (m <= 32 R). One CTA of B warps per block pair; dynamic shared memory
// holds the 2B columns (2B x 32R elements).
template <typename T, int B, int R>
__global__ void __launch_bounds__(B * 32, 1) jacobi_res_kernel(JResArgs a) {
  extern __shared__ __align__(16) unsigned char jr_raw[];
  T* jr_cols = reinterpret_cast<T*>(jr_raw);  // [2B][32R]
  __shared__ JrShared<T, B> S;
  constexpr int MR = 32 * R;
  constexpr int NT = B * 32;                  // threads
  constexpr int W16 = 16 / (int)sizeof(T);    // elements per 16-byte vector
  using V16 = typename JrVecT<T, W16>::type;
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
  JrCount cnt;
  const T tolT = (T)a.tol, deltaT = (T)a.delta;
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
        int P, Q;
        jr_pair(nbp, r, i, P, Q);
        const int m = a.m.eval(a.t, z);
        T* W = reinterpret_cast<T*>(bufp(a.t, z, a.bw));
        T* Vm = reinterpret_cast<T*>(bufp(a.t, z, a.bv));
        int* mark = reinterpret_cast<int*>(bufp(a.t, z, a.bmark));
        // the product's convergence flag, ||W||_F^2 and the marks travel together (one L2
        // round trip)
        const int prev = sweep > 0 ? __ldcg(&a.counters[z * a.max_sweeps + sweep - 1]) : 1;
        const double fro2 = __ldcg(&a.fro2[z]);
        int gmark = -2, gcol = -1;
        if (threadIdx.x < 2 * B) {
          const int c = threadIdx.x;
          const int g = (c < B ? P * B + c : Q * B + c - B);
          if ((c < B ? P : Q) < nb && g < n) {
            gcol = g;
            gmark = __ldcg(&mark[g]);
          }
        }
        if (prev == 0) continue;  // uniform: the product converged in the previous sweep
        const T fro = (T)sqrt(fro2);
        if (threadIdx.x < 2 * B) {
          S.col[threadIdx.x] = gcol;
          S.mark[threadIdx.x] = gmark;
          S.dirty[threadIdx.x] = 0;
        }
        __syncthreads();
        // A pair is skipped when neither column was rotated since the previous sweep began;
        // when that holds for every column of the block pair, nothing needs staging.
        if (sweep >= 1) {
          bool live = false;
#pragma unroll
          for (int c = 0; c < 2 * B; ++c) live = live || (S.col[c] >= 0 && S.mark[c] >= sweep - 1);
          if (!live) {
            __syncthreads();  // the shared state is reused by the CTA's next item
            continue;
          }
        }
        for (int e = threadIdx.x; e < 2 * B * JrShared<T, B>::QS; e += NT) {
          const int rr = e / JrShared<T, B>::QS, cc = e % JrShared<T, B>::QS;
          S.q[rr][cc] = (rr == cc) ? T(1) : T(0);
        }
        if (threadIdx.x == 0) S.nrot = 0;
        // stage the 2B columns (local 0..B-1 from block P, B..2B-1 from block Q); every
        // thread issues all its loads before the first shared store
        // 16-byte aligned columns in global memory, and whole vectors per thread
        constexpr bool kVecOK = (2 * R) % W16 == 0;
        const bool vec = kVecOK && (m % W16) == 0;
        if constexpr (kVecOK) {
          if (vec) {
          constexpr int PER = 2 * R / W16;   // vectors per thread (2B MR / W16 over NT threads)
#pragma unroll
          for (int b0 = 0; b0 < PER; b0 += 16) {
            constexpr int BT = PER < 16 ? PER : 16;
            V16 v[BT];
#pragma unroll
            for (int u = 0; u < BT; ++u) {
              const int e = (threadIdx.x + (b0 + u) * NT) * W16;   // element index in [2B][MR]
              const int c = e / MR, row = e % MR;
              const int g = S.col[c];
              if (g >= 0 && row < m) {
                v[u] = __ldcg(reinterpret_cast<const V16*>(W + (long)g * m + row));
              } else {
                T* z0 = reinterpret_cast<T*>(&v[u]);
#pragma unroll
                for (int w = 0; w < W16; ++w) z0[w] = T(0);
              }
            }
#pragma unroll
            for (int u = 0; u < BT; ++u)
              reinterpret_cast<V16*>(jr_cols)[threadIdx.x + (b0 + u) * NT] = v[u];
          }
          }
        }
        if (!vec) {
          constexpr int PER = 2 * R;  // elements per thread
          constexpr int BATCH = (sizeof(T) == 4 ? 64 : 32) < PER ? (sizeof(T) == 4 ? 64 : 32) : PER;
#pragma unroll
          for (int b0 = 0; b0 < PER; b0 += BATCH) {
            T v[BATCH];
#pragma unroll
            for (int u = 0; u < BATCH; ++u) {
              const int e = threadIdx.x + (b0 + u) * NT;
              const int c = e / MR, row = e % MR;
              const int g = S.col[c];
              v[u] = (g >= 0 && row < m) ? __ldcg(W + (long)g * m + row) : T(0);
            }
#pragma unroll
            for (int u = 0; u < BATCH; ++u) jr_cols[threadIdx.x + (b0 + u) * NT] = v[u];
          }
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
            jr_load<T, R>(cp, lane, x);
            jr_load<T, R>(cq, lane, y);
            if (jr_visit<T, B, R>(S, tolT, deltaT, p, q, m, n, sweep, fro, x, y, cnt)) {
              jr_store<T, R>(cp, lane, x);
              jr_store<T, R>(cq, lane, y);
            }
            __syncthreads();
          }
        }
        // pairs across the two blocks: warp w keeps local column w in registers
        {
          const int p = wid;
          T* cp = jr_cols + p * MR;
          jr_load<T, R>(cp, lane, x);
          bool px = false;
          for (int s = 0; s < B; ++s) {
            const int q = B + (wid + s) % B;
            T* cq = jr_cols + q * MR;
            jr_load<T, R>(cq, lane, y);
            if (jr_visit<T, B, R>(S, tolT, deltaT, p, q, m, n, sweep, fro, x, y, cnt)) {
              px = true;
              jr_store<T, R>(cq, lane, y);
            }
            __syncthreads();
          }
          if (px) jr_store<T, R>(cp, lane, x);
        }
        __syncthreads();
        // write back the rotated columns, the marks and V <- V Q
        if (S.nrot > 0) {
          if (vec) {
            for (int e4 = threadIdx.x; e4 < 2 * B * MR / W16; e4 += NT) {
              const int e = e4 * W16, c = e / MR, row = e % MR;
              if (S.dirty[c] && row < m)
                *reinterpret_cast<V16*>(W + (long)S.col[c] * m + row) = reinterpret_cast<const V16*>(jr_cols)[e4];
            }
          } else {
            for (int e = threadIdx.x; e < 2 * B * MR; e += NT) {
              const int c = e / MR, row = e % MR;
              if (S.dirty[c] && row < m) W[(long)S.col[c] * m + row] = jr_cols[e];
            }
          }
          if (threadIdx.x < 2 * B && S.col[threadIdx.x] >= 0) mark[S.col[threadIdx.x]] = S.mark[threadIdx.x];
          // two rows per thread and iteration (4B loads in flight); Q read by 16-byte rows
          for (int row0 = threadIdx.x; row0 < n; row0 += 2 * NT) {
            const int row1 = row0 + NT;
            T v0[2 * B], v1[2 * B], o0[2 * B], o1[2 * B];
#pragma unroll
            for (int c = 0; c < 2 * B; ++c) {
              v0[c] = S.col[c] >= 0 ? __ldcg(Vm + (long)S.col[c] * n + row0) : T(0);
              v1[c] = (S.col[c] >= 0 && row1 < n) ? __ldcg(Vm + (long)S.col[c] * n + row1) : T(0);
            }
#pragma unroll
            for (int c = 0; c < 2 * B; ++c) {
              o0[c] = T(0);
              o1[c] = T(0);
            }
#pragma unroll
            for (int c = 0; c < 2 * B; ++c) {
              T qr[2 * B];
#pragma unroll
              for (int j4 = 0; j4 < 2 * B / W16; ++j4) {
                const V16 qv = *reinterpret_cast<const V16*>(&S.q[c][W16 * j4]);
                const T* qe = reinterpret_cast<const T*>(&qv);
#pragma unroll
                for (int w = 0; w < W16; ++w) qr[W16 * j4 + w] = qe[w];
              }
#pragma unroll
              for (int j = 0; j < 2 * B; ++j) {
                o0[j] = fma(v0[c], qr[j], o0[j]);
                o1[j] = fma(v1[c], qr[j], o1[j]);
              }
            }
#pragma unroll
            for (int j = 0; j < 2 * B; ++j) {
              if (!S.dirty[j]) continue;
              Vm[(long)S.col[j] * n + row0] = o0[j];
              if (row1 < n) Vm[(long)S.col[j] * n + row1] = o1[j];
            }
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
  // 6 m flops per pair test, 6 (m + n) per rotation (as the scalar kernel counts them)
  if (lane == 0 && cnt.visit_rows + cnt.rot_rows > 0)
    atomicAdd(&a.t.stat[a.flop_slot], 6.0 * (double)cnt.visit_rows + 6.0 * (double)cnt.rot_rows);
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
