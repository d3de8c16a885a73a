// ttm_gemm.cuh -- float64 GEMM for the contractions of the sweep.
//
// C = alpha * A * B + beta * C for every (product z, batch index b) of a launch.
// Each operand is a strided view (element (i, j) at p[i*rs + j*cs]), so the leg
// permutations of the Swap (Fig. 1C) and the "same physical index" selection of
// the Contract (Eq. contract) are expressed purely by strides: no permuted copy
// is ever materialised. A functor F maps (z, b) to the problem, reading the bond
// table, so sizes are the realised ones.
//
// Tile: 64 x 64 outputs per CTA, K panels of 16, 256 threads with a 4 x 4 register
// micro-tile each. On this part float64 runs on a narrow pipe (about 1.1 TFLOP/s
// for the whole GPU), so the kernel is bound by DFMA issue, not by memory.
#pragma once
#include "ttm_common.cuh"

namespace ttm {

struct MatRef {
  const double* p;
  long rs, cs;
};
struct OutRef {
  double* p;
  long rs, cs;
};
struct GemmDesc {
  int M, N, K;
  MatRef A, B;
  OutRef C;
  double alpha, beta;
  int upper;  // 1: only the output tiles that meet the upper triangle (symmetric results)
};

constexpr int GT = 64, GK = 16;

// Realised flops of one problem (2 M N K; M (M + 1) K for a symmetric Gram whose upper
// triangle is formed), added by one thread of the problem's first tile when fl is set: a
// predicated-off problem (M = 0) adds nothing.
__device__ __forceinline__ void gemm_count_flops(double* fl, int fl_stride, int z, const GemmDesc& g) {
  if (fl == nullptr) return;
  const double f = g.upper ? (double)g.M * (g.N + 1) * g.K : 2.0 * g.M * g.N * g.K;
  atomicAdd(fl + (long)z * fl_stride, f);
}

// Realised shape of a launch's GEMMs (per product and batch index), for the flop count.
struct GemmShape {
  Dim M, N, K;
  int nbatch;
  int sym;  // 1: symmetric result, only the upper triangle is counted
};

template <class F>
__global__ void __launch_bounds__(256) dgemm_kernel(F f, int nbatch, double* fl = nullptr, int fl_stride = 0) {
  const int z = blockIdx.z / nbatch, bi = blockIdx.z % nbatch;
  const GemmDesc g = f(z, bi);
  const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
  if (g.M <= 0 || g.N <= 0 || m0 >= g.M || n0 >= g.N) return;
  if (m0 == 0 && n0 == 0 && threadIdx.x == 0) gemm_count_flops(fl, fl_stride, z, g);
  if (g.upper && m0 > n0) return;
  __shared__ double As[GK][GT + 1];
  __shared__ double Bs[GK][GT + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  // Load mapping: pick the loop order so that consecutive threads follow the
  // unit stride of the operand when it has one.
  const bool a_kfast = (g.A.cs == 1);
  const bool b_nfast = (g.B.cs == 1);
  for (int k0 = 0; k0 < g.K; k0 += GK) {
#pragma unroll
    for (int e = tid; e < GT * GK; e += 256) {
      int mm, kk;
      if (a_kfast) { kk = e % GK; mm = e / GK; } else { mm = e % GT; kk = e / GT; }
      const int gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < g.M && gk < g.K) ? g.A.p[(long)gm * g.A.rs + (long)gk * g.A.cs] : 0.0;
    }
#pragma unroll
    for (int e = tid; e < GT * GK; e += 256) {
      int nn, kk;
      if (b_nfast) { nn = e % GT; kk = e / GT; } else { kk = e % GK; nn = e / GK; }
      const int gn = n0 + nn, gk = k0 + kk;
      Bs[kk][nn] = (gn < g.N && gk < g.K) ? g.B.p[(long)gk * g.B.rs + (long)gn * g.B.cs] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty + 16 * i;
    if (gm >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx + 16 * j;
      if (gn >= g.N) continue;
      double* c = g.C.p + (long)gm * g.C.rs + (long)gn * g.C.cs;
      double v = g.alpha * acc[i][j];
      if (g.beta != 0.0) v = fma(g.beta, *c, v);
      *c = v;
    }
  }
}

// ---------------------------------------------------------------------------
// Problem functors. All cores are row-major [Dl][d][Dr].

// Swap, two-site contraction with the physical legs permuted (Fig. 1C):
//   Theta[(l,t),(s,r)] = sum_m X[l,s,m] Y[m,t,r],
// stored column-major with m_rows = Dl*d rows (row = l*d + t, col = s*Dr + r),
// which is the layout the one-sided Jacobi SVD works on. Batch b = s*d + t.
// keep_legs = 1 forms the plain two-site tensor Theta[(l,s),(t,r)] instead (the SVD
// sweep of the final rounding, where the legs stay in place).
struct ThetaFn {
  Tables t;
  int bx, by, bth;  // buffers: X, Y, Theta workspace
  int il, im, ir;   // bond ids: left of X, shared, right of Y
  int d;
  int keep_legs;    // 0: permuted legs (Swap); 1: legs in place
  __device__ GemmDesc operator()(int z, int b) const {
    const int s = b / d, tt = b % d;
    const int Dl = bondv(t, z, il), Dm = bondv(t, z, im), Dr = bondv(t, z, ir);
    const double* X = bufp(t, z, bx);
    const double* Y = bufp(t, z, by);
    double* T = bufp(t, z, bth);
    const long mrows = (long)Dl * d;
    const int row_leg = keep_legs ? s : tt, col_leg = keep_legs ? tt : s;
    GemmDesc g;
    g.M = Dl; g.N = Dr; g.K = Dm;
    g.A = MatRef{X + (long)s * Dm, (long)d * Dm, 1};
    g.B = MatRef{Y + (long)tt * Dr, (long)d * Dr, 1};
    g.C = OutRef{T + row_leg + (long)col_leg * Dr * mrows, d, mrows};
    g.alpha = 1.0; g.beta = 0.0; g.upper = 0;
    return g;
  }
};

// Contract (Eq. contract): Pi[l, e, r] = sum_a K[l, e, a] M[a, e, r]; batch b = e.
// The COPY tensor makes sigma = omega = eta, so only the d diagonal products are formed.
struct ContractFn {
  Tables t;
  int bk, bm, bo;
  int il, ia, ir;
  int d;
  __device__ GemmDesc operator()(int z, int e) const {
    const int Dl = bondv(t, z, il), Da = bondv(t, z, ia), Dr = bondv(t, z, ir);
    GemmDesc g;
    g.M = Dl; g.N = Dr; g.K = Da;
    g.A = MatRef{bufp(t, z, bk) + (long)e * Da, (long)d * Da, 1};
    g.B = MatRef{bufp(t, z, bm) + (long)e * Dr, (long)d * Dr, 1};
    g.C = OutRef{bufp(t, z, bo) + (long)e * Dr, (long)d * Dr, 1};
    g.alpha = 1.0; g.beta = 0.0; g.upper = 0;
    return g;
  }
};

// Gauge move, second half: Next'[k, (s, r)] = sum_c R[k, c] Next[c, (s, r)].
// R is row-major k x n (n = bond between the two carriages before the move).
struct RMergeFn {
  Tables t;
  int br, bn, bo;
  int ik, in, irr;
  int d;
  __device__ GemmDesc operator()(int z, int) const {
    const int k = bondv(t, z, ik), n = bondv(t, z, in), Drr = bondv(t, z, irr);
    GemmDesc g;
    g.M = k; g.N = d * Drr; g.K = n;
    g.A = MatRef{bufp(t, z, br), n, 1};
    g.B = MatRef{bufp(t, z, bn), (long)d * Drr, 1};
    g.C = OutRef{bufp(t, z, bo), (long)d * Drr, 1};
    g.alpha = 1.0; g.beta = 0.0; g.upper = 0;
    return g;
  }
};

// W = Theta V0 with both column-major (Theta m x n, V0 n x n, W m x n).
struct ThetaVFn {
  Tables t;
  int bth, bv, bw;
  Dim m, n;
  __device__ GemmDesc operator()(int z, int) const {
    const int M = m.eval(t, z), N = n.eval(t, z);
    GemmDesc g;
    g.M = M; g.N = N; g.K = N;
    g.A = MatRef{bufp(t, z, bth), 1, M};
    g.B = MatRef{bufp(t, z, bv), 1, N};
    g.C = OutRef{bufp(t, z, bw), 1, M};
    g.alpha = 1.0; g.beta = 0.0; g.upper = 0;
    return g;
  }
};

// Gram matrix G = W^T W of a column-major m x n matrix (n x n column-major; the tiles of
// the upper triangle only: G is symmetric and its readers take G[min(i,j) + max(i,j) n]).
struct GramFn {
  Tables t;
  int bw, bg;
  Dim m, n;
  __device__ GemmDesc operator()(int z, int) const {
    const int M = m.eval(t, z), N = n.eval(t, z);
    const double* W = bufp(t, z, bw);
    GemmDesc g;
    g.M = N; g.N = N; g.K = M;
    g.A = MatRef{W, M, 1};
    g.B = MatRef{W, 1, M};
    g.C = OutRef{bufp(t, z, bg), 1, N};
    g.alpha = 1.0; g.beta = 0.0; g.upper = 1;
    return g;
  }
};

// Right-to-left rounding: Prev'[(l, s), j] = sum_c Prev[(l, s), c] Wk[c, j],
// Wk column-major (rows = c, ld = wrows), j < k.
struct LMergeFn {
  Tables t;
  int bp, bw, bo;
  int il, ic, ik;
  Dim wrows;
  int d;
  __device__ GemmDesc operator()(int z, int) const {
    const int Dl = bondv(t, z, il), c = bondv(t, z, ic), k = bondv(t, z, ik);
    const long ld = wrows.eval(t, z);
    GemmDesc g;
    g.M = Dl * d; g.N = k; g.K = c;
    g.A = MatRef{bufp(t, z, bp), c, 1};
    g.B = MatRef{bufp(t, z, bw), 1, ld};
    g.C = OutRef{bufp(t, z, bo), k, 1};
    g.alpha = 1.0; g.beta = 0.0; g.upper = 0;
    return g;
  }
};

}  // namespace ttm
