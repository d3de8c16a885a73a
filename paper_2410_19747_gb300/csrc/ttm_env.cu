// ttm_env.cu -- environments of products of tensor trains and the adjoint (gradient)
// contractions behind ttm_inner (two layers), ttm_inner3 (three layers, <W, A o B>)
// and ttm_backward (<W, A o B> and ||A o B - C||^2 w.r.t. every core of A and B).
//
// All layers of an environment are joined on the same physical index s (the COPY tensor
// of Eq. contract applied to several trains), which is a batch index of the strided GEMMs
// below: no permuted copy of a core is formed. Each core is read through a view with
// strides (l, s, r); a right environment is the left recursion on the transposed views
// (l and r exchanged). Gradients for B are the gradients for A of the problem with A and
// B exchanged, since <W, A o B> and <A o B, A o B> are symmetric in A and B.
//
// Layouts (row-major): two-layer E[x][y]; three-layer E[w][a][b]; four-layer
// E[a][x][b][y] for <A o B, A o B> with layers (A, A, B, B).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "ttm.h"
#include "ttm_gemm.cuh"
#include "ttm_host.hpp"

namespace ttm {

// ---------------------------------------------------------------- batched strided GEMM

struct Op {
  const double* p;
  long rs, cs, s1, s2;
};
struct OutOp {
  double* p;
  long rs, cs, s1, s2;
};
// Problem b of a launch: b + boff = b1 * nb2 + b2.
struct GenFn {
  int M, N, K, nb2, boff;
  Op A, B;
  OutOp C;
  double alpha, beta;
  __device__ GemmDesc operator()(int, int b) const {
    const int bb = b + boff;
    const long b1 = bb / nb2, b2 = bb % nb2;
    GemmDesc g;
    g.M = M; g.N = N; g.K = K;
    g.A = MatRef{A.p + b1 * A.s1 + b2 * A.s2, A.rs, A.cs};
    g.B = MatRef{B.p + b1 * B.s1 + b2 * B.s2, B.rs, B.cs};
    g.C = OutRef{C.p + b1 * C.s1 + b2 * C.s2, C.rs, C.cs};
    g.alpha = alpha; g.beta = beta; g.upper = 0;
    return g;
  }
};

static inline Op op(const double* p, long rs, long cs, long s1 = 0, long s2 = 0) { return Op{p, rs, cs, s1, s2}; }
static inline OutOp out(double* p, long rs, long cs, long s1 = 0, long s2 = 0) { return OutOp{p, rs, cs, s1, s2}; }

struct EnvRunner {
  HandleState& hs;
  long launches = 0;
  explicit EnvRunner(HandleState& h) : hs(h) {}
  void gemm(int M, int N, int K, int nb1, int nb2, Op A, Op B, OutOp C, double alpha = 1.0, double beta = 0.0) {
    if (M <= 0 || N <= 0 || nb1 <= 0 || nb2 <= 0) return;
    const long nb = (long)nb1 * nb2;
    for (long b0 = 0; b0 < nb; b0 += 65535) {
      const int cnt = (int)std::min<long>(65535, nb - b0);
      GenFn f{M, N, K, nb2, (int)b0, A, B, C, alpha, beta};
      dim3 grid((N + GT - 1) / GT, (M + GT - 1) / GT, cnt);
      dgemm_kernel<GenFn><<<grid, 256, 0, hs.stream>>>(f, cnt);
      TTM_CUDA(cudaGetLastError());
      ++launches;
    }
  }
};

// ---------------------------------------------------------------- core views

struct View {
  const double* p;
  int Dl, Dr;
  long cl, cs, cr;  // element [l, s, r] at p[l*cl + s*cs + r*cr]
};
struct TTv {
  int L, d;
  std::vector<int> D;
  std::vector<const double*> c;
  View at(int k) const { return View{c[k], D[k], D[k + 1], (long)d * D[k + 1], (long)D[k + 1], 1}; }
  View at_t(int k) const { return View{c[k], D[k + 1], D[k], 1, (long)D[k + 1], (long)d * D[k + 1]}; }  // l <-> r
};

// ---------------------------------------------------------------- two layers

// E'[x', y'] = sum_{x, y, s} E[x, y] X[x, s, x'] Y[y, s, y'].  T: Dx * d * Dy'.
static void env2_step(EnvRunner& r, int d, const double* E, View X, View Y, double* T, double* En) {
  // T[s][x][y'] = sum_y E[x, y] Y[y, s, y']              (batch s)
  r.gemm(X.Dl, Y.Dr, Y.Dl, 1, d, op(E, Y.Dl, 1), op(Y.p, Y.cl, Y.cr, 0, Y.cs),
         out(T, Y.Dr, 1, 0, (long)X.Dl * Y.Dr));
  // E'[x', y'] = sum_s sum_x X[x, s, x'] T[s][x][y']
  for (int s = 0; s < d; ++s)
    r.gemm(X.Dr, Y.Dr, X.Dl, 1, 1, op(X.p + s * X.cs, X.cr, X.cl), op(T + (long)s * X.Dl * Y.Dr, Y.Dr, 1),
           out(En, Y.Dr, 1), 1.0, s == 0 ? 0.0 : 1.0);
}

// ---------------------------------------------------------------- three layers (W, A, B)

// E'[w', a', b'] = sum E[w, a, b] W[w, s, w'] A[a, s, a'] B[b, s, b'].
// T1: d*Dw*Da*Db', T2: d*Dw*Da'*Db'.
static void env3_step(EnvRunner& r, int d, const double* E, View W, View A, View B, double* T1, double* T2,
                      double* En) {
  // T1[s][(w, a)][b'] = sum_b E[(w, a), b] B[b, s, b']    (batch s)
  r.gemm(W.Dl * A.Dl, B.Dr, B.Dl, 1, d, op(E, B.Dl, 1), op(B.p, B.cl, B.cr, 0, B.cs),
         out(T1, B.Dr, 1, 0, (long)W.Dl * A.Dl * B.Dr));
  // T2[s][w][a'][b'] = sum_a A[a, s, a'] T1[s][w][a][b']  (batch (s, w))
  r.gemm(A.Dr, B.Dr, A.Dl, d, W.Dl, op(A.p, A.cr, A.cl, A.cs, 0),
         op(T1, B.Dr, 1, (long)W.Dl * A.Dl * B.Dr, (long)A.Dl * B.Dr),
         out(T2, B.Dr, 1, (long)W.Dl * A.Dr * B.Dr, (long)A.Dr * B.Dr));
  // E'[w'][(a', b')] = sum_s sum_w W[w, s, w'] T2[s][w][(a', b')]
  for (int s = 0; s < d; ++s)
    r.gemm(W.Dr, A.Dr * B.Dr, W.Dl, 1, 1, op(W.p + s * W.cs, W.cr, W.cl),
           op(T2 + (long)s * W.Dl * A.Dr * B.Dr, (long)A.Dr * B.Dr, 1), out(En, (long)A.Dr * B.Dr, 1), 1.0,
           s == 0 ? 0.0 : 1.0);
}

// G[a, s, a'] (+)= alpha * sum E[w, a, b] W[w, s, w'] B[b, s, b'] R[w', a', b'] for the core A_k
// (G in the layout of A_k). P: d*Da*Dw*Db', Q: d*Da'*Dw*Db'.
static void adjoint3(EnvRunner& r, int d, const double* E, const double* R, View W, View A, View B, double* P,
                     double* Q, double* G, double alpha, double beta) {
  const long kk = (long)W.Dl * B.Dr;
  // P[s][a][w][b'] = sum_b E[w, a, b] B[b, s, b']          (batch (s, w))
  r.gemm(A.Dl, B.Dr, B.Dl, d, W.Dl, op(E, B.Dl, 1, 0, (long)A.Dl * B.Dl), op(B.p, B.cl, B.cr, B.cs, 0),
         out(P, kk, 1, (long)A.Dl * kk, B.Dr));
  // Q[s][a'][w][b'] = sum_w' W[w, s, w'] R[w', a', b']      (batch (s, a'))
  r.gemm(W.Dl, B.Dr, W.Dr, d, A.Dr, op(W.p, W.cl, W.cr, W.cs, 0), op(R, (long)A.Dr * B.Dr, 1, 0, B.Dr),
         out(Q, B.Dr, 1, (long)A.Dr * kk, kk));
  // G[a, s, a'] = sum_{(w, b')} P[s][a][(w, b')] Q[s][a'][(w, b')]   (batch s)
  r.gemm(A.Dl, A.Dr, (int)kk, 1, d, op(P, kk, 1, 0, (long)A.Dl * kk), op(Q, 1, kk, 0, (long)A.Dr * kk),
         out(G, (long)d * A.Dr, 1, 0, A.Dr), alpha, beta);
}

// ---------------------------------------------------------------- four layers (A, A, B, B)

// E'[a', x', b', y'] = sum E[a, x, b, y] A[a, s, a'] A[x, s, x'] B[b, s, b'] B[y, s, y'].
// T1, T2: d * Da^2 * Db * Db' and d * Da * Da' * Db'^2 at most (see sizes in env4_sizes).
static void env4_step(EnvRunner& r, int d, const double* E, View A, View B, double* T1, double* T2, double* En) {
  const int Da = A.Dl, Dap = A.Dr, Db = B.Dl, Dbp = B.Dr;
  const long ab = (long)Da * Da;
  // S1[s][(a, x, b)][y'] = sum_y E[(a, x, b), y] B[y, s, y']          (batch s)
  r.gemm((int)(ab * Db), Dbp, Db, 1, d, op(E, Db, 1), op(B.p, B.cl, B.cr, 0, B.cs),
         out(T1, Dbp, 1, 0, ab * Db * Dbp));
  // S2[s][(a, x)][b'][y'] = sum_b B[b, s, b'] S1[s][(a, x)][b][y']    (batch (s, (a, x)))
  r.gemm(Dbp, Dbp, Db, d, (int)ab, op(B.p, B.cr, B.cl, B.cs, 0), op(T1, Dbp, 1, ab * Db * Dbp, (long)Db * Dbp),
         out(T2, Dbp, 1, ab * Dbp * Dbp, (long)Dbp * Dbp));
  // S3[s][a][x'][(b', y')] = sum_x A[x, s, x'] S2[s][a][x][(b', y')] (batch (s, a))
  const long q = (long)Dbp * Dbp;
  r.gemm(Dap, (int)q, Da, d, Da, op(A.p, A.cr, A.cl, A.cs, 0), op(T2, q, 1, ab * q, (long)Da * q),
         out(T1, q, 1, (long)Da * Dap * q, (long)Dap * q));
  // E'[a'][(x', b', y')] = sum_s sum_a A[a, s, a'] S3[s][a][(x', b', y')]
  for (int s = 0; s < d; ++s)
    r.gemm(Dap, (int)(Dap * q), Da, 1, 1, op(A.p + s * A.cs, A.cr, A.cl),
           op(T1 + (long)s * Da * Dap * q, (long)Dap * q, 1), out(En, (long)Dap * q, 1), 1.0, s == 0 ? 0.0 : 1.0);
}

// G[x, s, x'] (+)= alpha * sum E[a, x, b, y] A[a, s, a'] B[b, s, b'] B[y, s, y'] R[a', x', b', y']:
// the adjoint for the second A layer (layout of A_k).
static void adjoint4(EnvRunner& r, int d, const double* E, const double* R, View A, View B, double* T1, double* T2,
                     double* G, double alpha, double beta) {
  const int Da = A.Dl, Dap = A.Dr, Db = B.Dl, Dbp = B.Dr;
  const long ab = (long)Da * Da, q = (long)Dbp * Dbp;
  // S1, S2 as in env4_step
  r.gemm((int)(ab * Db), Dbp, Db, 1, d, op(E, Db, 1), op(B.p, B.cl, B.cr, 0, B.cs),
         out(T1, Dbp, 1, 0, ab * Db * Dbp));
  r.gemm(Dbp, Dbp, Db, d, (int)ab, op(B.p, B.cr, B.cl, B.cs, 0), op(T1, Dbp, 1, ab * Db * Dbp, (long)Db * Dbp),
         out(T2, Dbp, 1, ab * q, q));
  // S3[s][x][a'][(b', y')] = sum_a A[a, s, a'] S2[s][a][x][(b', y')]  (batch (s, x))
  r.gemm(Dap, (int)q, Da, d, Da, op(A.p, A.cr, A.cl, A.cs, 0), op(T2, (long)Da * q, 1, ab * q, q),
         out(T1, q, 1, (long)Da * Dap * q, (long)Dap * q));
  // G[x, s, x'] = sum_a' sum_(b', y') S3[s][x][a'][(b', y')] R[a'][x'][(b', y')]   (batch s)
  for (int a = 0; a < Dap; ++a)
    r.gemm(Da, Dap, (int)q, 1, d, op(T1 + (long)a * q, (long)Dap * q, 1, 0, (long)Da * Dap * q),
           op(R + (long)a * Dap * q, 1, q), out(G, (long)d * Dap, 1, 0, Dap), alpha, a == 0 ? beta : 1.0);
}

// ---------------------------------------------------------------- drivers

static TTv make_view(const ttm_tt& t) {
  TTv v;
  v.L = t.L;
  v.d = t.d;
  v.D.resize(t.L + 1);
  v.c.resize(t.L);
  for (int i = 0; i <= t.L; ++i) v.D[i] = (int)t.bonds[i];
  for (int k = 0; k < t.L; ++k) v.c[k] = t.cores[k];
  return v;
}

static double* carve(char*& cur, size_t n) {
  double* p = (double*)cur;
  cur += ((n * sizeof(double) + 255) & ~(size_t)255);
  return p;
}

static double read_scalar(HandleState& hs, const double* p) {
  double v = 0.0;
  TTM_CUDA(cudaMemcpyAsync(&v, p, sizeof(double), cudaMemcpyDeviceToHost, hs.stream));
  TTM_CUDA(cudaStreamSynchronize(hs.stream));
  return v;
}

static void put_one(HandleState& hs, double* p) {
  static const double one = 1.0;
  TTM_CUDA(cudaMemcpyAsync(p, &one, sizeof(double), cudaMemcpyHostToDevice, hs.stream));
}

double env_inner(HandleState& hs, DeviceArena& ar, const ttm_tt& X_, const ttm_tt& Y_) {
  const TTv X = make_view(X_), Y = make_view(Y_);
  const int L = X.L, d = X.d;
  size_t e = 1, t = 1;
  for (int k = 0; k <= L; ++k) e = std::max(e, (size_t)X.D[k] * Y.D[k]);
  for (int k = 0; k < L; ++k) t = std::max(t, (size_t)d * X.D[k] * Y.D[k + 1]);
  ar.ensure((2 * e + t) * 8 + 4096);
  char* cur = (char*)ar.ptr;
  double *E0 = carve(cur, e), *E1 = carve(cur, e), *T = carve(cur, t);
  EnvRunner r(hs);
  put_one(hs, E0);
  for (int k = 0; k < L; ++k) {
    env2_step(r, d, E0, X.at(k), Y.at(k), T, E1);
    std::swap(E0, E1);
  }
  return read_scalar(hs, E0);
}

static void env3_sizes(const TTv& W, const TTv& A, const TTv& B, size_t& e, size_t& t1, size_t& t2, size_t& p, size_t& q) {
  const int L = W.L, d = W.d;
  e = t1 = t2 = p = q = 1;
  for (int k = 0; k <= L; ++k) e = std::max(e, (size_t)W.D[k] * A.D[k] * B.D[k]);
  for (int k = 0; k < L; ++k) {
    // left and right (transposed) steps
    t1 = std::max(t1, (size_t)d * W.D[k] * A.D[k] * B.D[k + 1]);
    t1 = std::max(t1, (size_t)d * W.D[k + 1] * A.D[k + 1] * B.D[k]);
    t2 = std::max(t2, (size_t)d * W.D[k] * A.D[k + 1] * B.D[k + 1]);
    t2 = std::max(t2, (size_t)d * W.D[k + 1] * A.D[k] * B.D[k]);
    p = std::max(p, (size_t)d * A.D[k] * W.D[k] * B.D[k + 1]);
    q = std::max(q, (size_t)d * A.D[k + 1] * W.D[k] * B.D[k + 1]);
  }
}

double env_inner3(HandleState& hs, DeviceArena& ar, const ttm_tt& W_, const ttm_tt& A_, const ttm_tt& B_) {
  const TTv W = make_view(W_), A = make_view(A_), B = make_view(B_);
  size_t e, t1, t2, p, q;
  env3_sizes(W, A, B, e, t1, t2, p, q);
  ar.ensure((2 * e + t1 + t2) * 8 + 4096);
  char* cur = (char*)ar.ptr;
  double *E0 = carve(cur, e), *E1 = carve(cur, e), *T1 = carve(cur, t1), *T2 = carve(cur, t2);
  EnvRunner r(hs);
  put_one(hs, E0);
  for (int k = 0; k < W.L; ++k) {
    env3_step(r, W.d, E0, W.at(k), A.at(k), B.at(k), T1, T2, E1);
    std::swap(E0, E1);
  }
  return read_scalar(hs, E0);
}

// Left environments L_0 .. L_L for a backward sweep. When all of them fit the budget they
// are stored; otherwise only every s-th one is kept (s = ceil(sqrt(L)), checkpoints), and
// the sweep recomputes a segment of s - 1 environments from its checkpoint when it reaches
// it: about 2 sqrt(L) environments held at a time for one extra forward sweep of work.
struct LeftEnvs {
  int L = 0, s = 1, cur = -1;
  std::vector<double*> ck, seg;
  // step(k, E_k, E_{k+1}) computes environment k + 1 from environment k
  template <class Step>
  double* get(int k, Step&& step) {
    if (s == 1) return ck[k];
    const int c = k / s;
    if (k % s == 0) return ck[c];
    if (cur != c) {
      const int hi = std::min(c * s + s - 1, L);
      const double* prev = ck[c];
      for (int j = c * s; j < hi; ++j) {
        step(j, prev, seg[j - c * s]);
        prev = seg[j - c * s];
      }
      cur = c;
    }
    return seg[k % s - 1];
  }
};

static size_t env_budget(const HandleState& hs) {
  return hs.opt.env_budget_bytes > 0 ? (size_t)hs.opt.env_budget_bytes : ((size_t)4 << 30);
}

// Carves the left environments of sizes esz[0..L] (elements) from cur: all of them when they
// fit the budget, else checkpoints and one segment buffer of the largest size emax.
static size_t left_bytes(const std::vector<size_t>& esz, size_t emax, size_t budget, int* s_out) {
  const int L = (int)esz.size() - 1;
  size_t all = 0;
  for (size_t e : esz) all += (e * 8 + 255) & ~(size_t)255;
  if (all <= budget || L < 4) {
    *s_out = 1;
    return all;
  }
  int s = 1;
  while (s * s < L) ++s;
  size_t b = 0;
  for (int k = 0; k <= L; k += s) b += (esz[k] * 8 + 255) & ~(size_t)255;
  b += (size_t)(s - 1) * ((emax * 8 + 255) & ~(size_t)255);
  *s_out = s;
  return b;
}

// Gradient of <W, A o B> w.r.t. every core of A: left environments stored, right ones
// built on the way back. G may be NULL (value only). Returns the value.
static double grad3(HandleState& hs, DeviceArena& ar, const TTv& W, const TTv& A, const TTv& B,
                    const std::vector<double*>* G, double alpha, double beta) {
  const int L = W.L, d = W.d;
  size_t e, t1, t2, p, q;
  env3_sizes(W, A, B, e, t1, t2, p, q);
  std::vector<size_t> esz(L + 1);
  for (int k = 0; k <= L; ++k) esz[k] = (size_t)W.D[k] * A.D[k] * B.D[k];
  int sck = 1;
  const size_t lb = G ? left_bytes(esz, e, env_budget(hs), &sck) : 0;
  ar.ensure(lb + (4 * e + t1 + t2 + p + q) * 8 + 8192);
  char* cur = (char*)ar.ptr;
  double *R0 = carve(cur, e), *R1 = carve(cur, e), *T1 = carve(cur, t1), *T2 = carve(cur, t2);
  double *P = carve(cur, p), *Q = carve(cur, q), *F0 = carve(cur, e), *F1 = carve(cur, e);
  LeftEnvs lv;
  lv.L = L;
  lv.s = sck;
  if (G) {
    for (int k = 0; k <= L; k += sck) lv.ck.push_back(carve(cur, esz[k]));
    for (int j = 0; j + 1 < sck; ++j) lv.seg.push_back(carve(cur, e));
  }
  EnvRunner r(hs);
  auto step = [&](int k, const double* Ein, double* Eout) {
    env3_step(r, d, Ein, W.at(k), A.at(k), B.at(k), T1, T2, Eout);
  };
  // forward sweep: the value, and the stored environments (or checkpoints)
  put_one(hs, F0);
  if (G) TTM_CUDA(cudaMemcpyAsync(lv.ck[0], F0, 8, cudaMemcpyDeviceToDevice, hs.stream));
  for (int k = 0; k < L; ++k) {
    step(k, F0, F1);
    std::swap(F0, F1);
    if (G && (k + 1) % sck == 0)
      TTM_CUDA(cudaMemcpyAsync(lv.ck[(k + 1) / sck], F0, esz[k + 1] * 8, cudaMemcpyDeviceToDevice, hs.stream));
  }
  const double val = read_scalar(hs, F0);
  if (!G) return val;
  put_one(hs, R0);
  for (int k = L - 1; k >= 0; --k) {
    adjoint3(r, d, lv.get(k, step), R0, W.at(k), A.at(k), B.at(k), P, Q, (*G)[k], alpha, beta);
    if (k > 0) {
      env3_step(r, d, R0, W.at_t(k), A.at_t(k), B.at_t(k), T1, T2, R1);
      std::swap(R0, R1);
    }
  }
  return val;
}

// Gradient of <A o B, A o B> w.r.t. every core of A (the derivative of both A layers:
// 2 x the adjoint of one layer). G may be NULL. Returns the value.
static double grad4(HandleState& hs, DeviceArena& ar, const TTv& A, const TTv& B, const std::vector<double*>* G,
                    double alpha, double beta) {
  const int L = A.L, d = A.d;
  std::vector<size_t> esz(L + 1);
  size_t e = 1, t1 = 1, t2 = 1;
  for (int k = 0; k <= L; ++k) {
    esz[k] = (size_t)A.D[k] * A.D[k] * B.D[k] * B.D[k];
    e = std::max(e, esz[k]);
  }
  for (int k = 0; k < L; ++k)
    for (int dir = 0; dir < 2; ++dir) {
      const size_t Da = dir ? A.D[k + 1] : A.D[k], Dap = dir ? A.D[k] : A.D[k + 1];
      const size_t Db = dir ? B.D[k + 1] : B.D[k], Dbp = dir ? B.D[k] : B.D[k + 1];
      t1 = std::max({t1, d * Da * Da * Db * Dbp, d * Da * Dap * Dbp * Dbp});
      t2 = std::max(t2, d * Da * Da * Dbp * Dbp);
    }
  int sck = 1;
  const size_t lb = G ? left_bytes(esz, e, env_budget(hs), &sck) : 0;
  ar.ensure(lb + (4 * e + t1 + t2) * 8 + 8192);
  char* cur = (char*)ar.ptr;
  double *R0 = carve(cur, e), *R1 = carve(cur, e), *T1 = carve(cur, t1), *T2 = carve(cur, t2);
  double *F0 = carve(cur, e), *F1 = carve(cur, e);
  LeftEnvs lv;
  lv.L = L;
  lv.s = sck;
  if (G) {
    for (int k = 0; k <= L; k += sck) lv.ck.push_back(carve(cur, esz[k]));
    for (int j = 0; j + 1 < sck; ++j) lv.seg.push_back(carve(cur, e));
  }
  EnvRunner r(hs);
  auto step = [&](int k, const double* Ein, double* Eout) { env4_step(r, d, Ein, A.at(k), B.at(k), T1, T2, Eout); };
  put_one(hs, F0);
  if (G) TTM_CUDA(cudaMemcpyAsync(lv.ck[0], F0, 8, cudaMemcpyDeviceToDevice, hs.stream));
  for (int k = 0; k < L; ++k) {
    step(k, F0, F1);
    std::swap(F0, F1);
    if (G && (k + 1) % sck == 0)
      TTM_CUDA(cudaMemcpyAsync(lv.ck[(k + 1) / sck], F0, esz[k + 1] * 8, cudaMemcpyDeviceToDevice, hs.stream));
  }
  const double val = read_scalar(hs, F0);
  if (!G) return val;
  put_one(hs, R0);
  for (int k = L - 1; k >= 0; --k) {
    adjoint4(r, d, lv.get(k, step), R0, A.at(k), B.at(k), T1, T2, (*G)[k], 2.0 * alpha, beta);
    if (k > 0) {
      env4_step(r, d, R0, A.at_t(k), B.at_t(k), T1, T2, R1);
      std::swap(R0, R1);
    }
  }
  return val;
}

// ttm_backward: value and gradients. kind 0: <W, A o B>; kind 1: ||A o B - C||^2.
double env_backward(HandleState& hs, DeviceArena& ar, int kind, const ttm_tt& A_, const ttm_tt& B_,
                    const ttm_tt& WC_, const ttm_tt* gA, const ttm_tt* gB) {
  const TTv A = make_view(A_), B = make_view(B_), W = make_view(WC_);
  std::vector<double*> GA, GB;
  if (gA) for (int k = 0; k < A.L; ++k) GA.push_back(gA->cores[k]);
  if (gB) for (int k = 0; k < B.L; ++k) GB.push_back(gB->cores[k]);
  if (kind == 0) {
    double v = grad3(hs, ar, W, A, B, gA ? &GA : nullptr, 1.0, 0.0);
    if (gB) grad3(hs, ar, W, B, A, &GB, 1.0, 0.0);
    return v;
  }
  // ||A o B - C||^2 = <A o B, A o B> - 2 <C, A o B> + <C, C>
  const double ab = grad4(hs, ar, A, B, gA ? &GA : nullptr, 1.0, 0.0);
  const double cab = grad3(hs, ar, W, A, B, gA ? &GA : nullptr, -2.0, 1.0);
  if (gB) {
    grad4(hs, ar, B, A, &GB, 1.0, 0.0);
    grad3(hs, ar, W, B, A, &GB, -2.0, 1.0);
  }
  const double cc = env_inner(hs, ar, WC_, WC_);
  return ab - 2.0 * cab + cc;
}

}  // namespace ttm
