// ttm_bjac.cuh -- block one-sided Jacobi for the float32 preconditioning passes of the
// Swap SVD (Fig. 1C, Eq. eps).
//
// The scalar kernel (ttm_svd.cuh) visits the n/2 column pairs of a round and then waits at
// a grid-wide barrier: n - 1 barriers per sweep. This kernel groups the columns into blocks
// of B and runs the round-robin tournament (Brent & Luk 1985) over blocks: n/B - 1 barriers
// per sweep. One CTA takes one block pair (K = 2B columns):
//   1. G = W_b^T W_b, the K x K Gram matrix of the pair, accumulated in float32 from row
//      chunks staged in shared memory;
//   2. one cyclic Jacobi sweep on G with the rotation and tests of the one-sided method
//      (G <- J^T G J for every rotation, J accumulated);
//   3. W_b <- W_b J and V_b <- V_b J (every row independently).
// A rotation of a big column p against a small one q changes G_qq by at most u G_pq^2 / G_pp
// <= u G_qq, so the couplings of small columns keep relative accuracy within a sweep, and
// every outer round recomputes G from the rotated columns.
#pragma once
#include <cooperative_groups.h>
#include "ttm_common.cuh"

namespace cg = cooperative_groups;

namespace ttm {

constexpr int kBjRows = 256;  // rows of a block pair staged in shared memory per chunk

struct BJacArgs {
  Tables t;
  int bw, bv;        // W: m x n float column-major (in/out); V: n x n float column-major (out, starts at I)
  Dim m, n;
  int nblk_pad_ub;   // even host upper bound of ceil(n / B)
  int max_sweeps;
  int* counters;     // [nz][max_sweeps] rotations per sweep, zeroed before launch
  double tol;        // rotate when |G_pq| > tol * sqrt(G_pp G_qq) ...
  double delta;      // ... and |G_pq| > delta * sqrt(max(G_pp, G_qq)) * ||W||_F
  double* fro2;      // [nz] ||W||_F^2, zeroed before launch
  int flop_slot;     // stat slot that accumulates the executed flops
  int count_nonconv; // 1: a product that hits max_sweeps counts in IS_NONCONV
};

__device__ __forceinline__ int bj_ldcg(const int* p) { return __ldcg(p); }

// Slot pair `i` of inner round `r` of the round-robin tournament on `k` (even) slots.
__device__ __forceinline__ void rr_pair(int k, int r, int i, int& p, int& q) {
  if (i == 0) {
    p = k - 1;
    q = r;
  } else {
    p = (r + i) % (k - 1);
    q = (r - i + k - 1) % (k - 1);
  }
}

template <int B>
__global__ void __launch_bounds__(256) block_jacobi_kernel(BJacArgs a) {
  constexpr int K = 2 * B;
  constexpr int NG = K * (K + 1) / 2;       // upper-triangle entries of G
  constexpr int GPER = (NG + 255) / 256;    // entries per thread
  __shared__ float Ws[kBjRows][K + 1];
  __shared__ float G[K][K + 1];
  __shared__ float J[K][K + 1];
  __shared__ float sc[B], ss[B];
  __shared__ int sp[B], sq[B];
  __shared__ int s_rot;
  __shared__ int s_col[K];

  cg::grid_group grid = cg::this_grid();
  const int tid = threadIdx.x;
  const long gthread = (long)blockIdx.x * blockDim.x + tid;
  const long nthreads = (long)gridDim.x * blockDim.x;
  const int nz = a.t.nz;

  for (int z = 0; z < nz; ++z) {
    const int n = a.n.eval(a.t, z), m = a.m.eval(a.t, z);
    float* V = reinterpret_cast<float*>(bufp(a.t, z, a.bv));
    for (long e = gthread; e < (long)n * n; e += nthreads) V[e] = (e % n == e / n) ? 1.f : 0.f;
    const float* W = reinterpret_cast<const float*>(bufp(a.t, z, a.bw));
    double f = 0.0;
    for (long e = gthread; e < (long)m * n; e += nthreads) f = fma((double)W[e], (double)W[e], f);
    f = warp_sum(f);
    if ((tid & 31) == 0 && f != 0.0) atomicAdd(&a.fro2[z], f);
  }
  grid.sync();

  const int half = a.nblk_pad_ub / 2;
  const long items = (long)nz * half;
  double flops = 0.0;
  int sweeps_done = 0;
  for (int sweep = 0; sweep < a.max_sweeps; ++sweep) {
    for (int r = 0; r < a.nblk_pad_ub - 1; ++r) {
      for (long it = blockIdx.x; it < items; it += gridDim.x) {  // CTA-uniform item
        const int z = (int)(it / half), i = (int)(it % half);
        if (sweep > 0 && bj_ldcg(&a.counters[z * a.max_sweeps + sweep - 1]) == 0) continue;
        const int n = a.n.eval(a.t, z), m = a.m.eval(a.t, z);
        const int nblk = (n + B - 1) / B;
        const int npad = nblk + (nblk & 1);
        if (i >= npad / 2 || r >= npad - 1) continue;
        int P, Q;
        rr_pair(npad, r, i, P, Q);
        if (P >= nblk || Q >= nblk) continue;
        float* W = reinterpret_cast<float*>(bufp(a.t, z, a.bw));
        float* V = reinterpret_cast<float*>(bufp(a.t, z, a.bv));
        const double fro = sqrt(__ldcg(&a.fro2[z]));
        if (tid < K) {
          const int j = (tid < B) ? P * B + tid : Q * B + (tid - B);
          s_col[tid] = (j < n) ? j : -1;  // -1: padding column of a short last block
        }
        if (tid == 0) s_rot = 0;
        __syncthreads();

        // 1. Gram matrix of the block pair (upper triangle; entry e -> (gi, gj), gi <= gj)
        float g[GPER];
        int gi[GPER], gj[GPER];
#pragma unroll
        for (int u = 0; u < GPER; ++u) {
          g[u] = 0.f;
          int e = tid + 256 * u, row = 0;
          while (e >= K - row && row < K) {  // row-wise enumeration of the upper triangle
            e -= K - row;
            ++row;
          }
          gi[u] = row;
          gj[u] = row + e;
        }
        for (int r0 = 0; r0 < m; r0 += kBjRows) {
          const int rows = min(kBjRows, m - r0);
          for (int e = tid; e < kBjRows * K; e += 256) {
            const int c = e / kBjRows, rr = e % kBjRows;  // consecutive threads: consecutive rows
            const int col = s_col[c];
            Ws[rr][c] = (col >= 0 && rr < rows) ? __ldcg(W + (long)col * m + r0 + rr) : 0.f;
          }
          __syncthreads();
#pragma unroll
          for (int u = 0; u < GPER; ++u) {
            if (tid + 256 * u < NG) {
              // four interleaved partial sums keep the rounding of a chunk near 64 terms
              float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
              const int x = gi[u], y = gj[u];
              int rr = 0;
              for (; rr + 3 < rows; rr += 4) {
                s0 = fmaf(Ws[rr][x], Ws[rr][y], s0);
                s1 = fmaf(Ws[rr + 1][x], Ws[rr + 1][y], s1);
                s2 = fmaf(Ws[rr + 2][x], Ws[rr + 2][y], s2);
                s3 = fmaf(Ws[rr + 3][x], Ws[rr + 3][y], s3);
              }
              for (; rr < rows; ++rr) s0 = fmaf(Ws[rr][x], Ws[rr][y], s0);
              g[u] += (s0 + s1) + (s2 + s3);
            }
          }
          __syncthreads();
        }
#pragma unroll
        for (int u = 0; u < GPER; ++u) {
          if (tid + 256 * u < NG) {
            G[gi[u]][gj[u]] = g[u];
            G[gj[u]][gi[u]] = g[u];
          }
        }
        for (int e = tid; e < K * K; e += 256) J[e / K][e % K] = (e / K == e % K) ? 1.f : 0.f;
        __syncthreads();
        flops += (double)m * K * (K + 1);

        // 2. one cyclic Jacobi sweep on G: K - 1 inner rounds of B disjoint slot pairs
        for (int ir = 0; ir < K - 1; ++ir) {
          if (tid < B) {
            int p, q;
            rr_pair(K, ir, tid, p, q);
            const float al = G[p][p], be = G[q][q], ga = G[p][q];
            float c = 1.f, s = 0.f;
            const double aga = fabs((double)ga);
            const double big = sqrt((double)fmaxf(al, be));
            if (s_col[p] >= 0 && s_col[q] >= 0 && ga != 0.f &&
                aga > a.tol * sqrt((double)fmaxf(al, 0.f)) * sqrt((double)fmaxf(be, 0.f)) &&
                aga > a.delta * big * fro) {
              // zeta = (beta - alpha) / (2 gamma); t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2))
              const float zeta = (be - al) / (2.f * ga);
              const float tt = copysignf(1.f, zeta) / (fabsf(zeta) + hypotf(1.f, zeta));
              c = 1.f / sqrtf(fmaf(tt, tt, 1.f));
              s = c * tt;
              atomicAdd(&s_rot, 1);
            }
            sc[tid] = c;
            ss[tid] = s;
            sp[tid] = p;
            sq[tid] = q;
          }
          __syncthreads();
          // columns p, q of G and J (G <- G J)
          for (int e = tid; e < K * B; e += 256) {
            const int row = e % K, pi = e / K;
            const float c = sc[pi], s = ss[pi];
            if (s != 0.f) {
              const int p = sp[pi], q = sq[pi];
              const float gp = G[row][p], gq = G[row][q];
              G[row][p] = c * gp - s * gq;
              G[row][q] = fmaf(s, gp, c * gq);
              const float jp = J[row][p], jq = J[row][q];
              J[row][p] = c * jp - s * jq;
              J[row][q] = fmaf(s, jp, c * jq);
            }
          }
          __syncthreads();
          // rows p, q of G (G <- J^T G)
          for (int e = tid; e < K * B; e += 256) {
            const int col = e % K, pi = e / K;
            const float c = sc[pi], s = ss[pi];
            if (s != 0.f) {
              const int p = sp[pi], q = sq[pi];
              const float gp = G[p][col], gq = G[q][col];
              G[p][col] = c * gp - s * gq;
              G[q][col] = fmaf(s, gp, c * gq);
            }
          }
          __syncthreads();
        }

        // 3. W_b <- W_b J, V_b <- V_b J (rows are independent; a row is read before written)
        if (s_rot > 0) {
          for (int pass = 0; pass < 2; ++pass) {
            float* X = pass == 0 ? W : V;
            const int rowsX = pass == 0 ? m : n;
            const long ld = pass == 0 ? m : n;
            for (int row = tid; row < rowsX; row += 256) {
              float x[K];
#pragma unroll
              for (int c = 0; c < K; ++c) x[c] = s_col[c] >= 0 ? __ldcg(X + (long)s_col[c] * ld + row) : 0.f;
#pragma unroll
              for (int c = 0; c < K; ++c) {
                if (s_col[c] < 0) continue;
                float acc = 0.f;
#pragma unroll
                for (int j = 0; j < K; ++j) acc = fmaf(x[j], J[j][c], acc);
                X[(long)s_col[c] * ld + row] = acc;
              }
            }
          }
          flops += 2.0 * K * K * ((double)m + n);
          if (tid == 0) atomicAdd(&a.counters[z * a.max_sweeps + sweep], s_rot);
        }
        __syncthreads();  // shared memory is reused by the next item
      }
      grid.sync();
    }
    sweeps_done = sweep + 1;
    bool all = true;
    for (int z = 0; z < nz; ++z)
      if (bj_ldcg(&a.counters[z * a.max_sweeps + sweep]) != 0) all = false;
    if (all) break;
  }
  if (tid == 0 && flops > 0.0) atomicAdd(&a.t.stat[a.flop_slot], flops);
  if (gthread == 0) {
    for (int z = 0; z < nz; ++z) {
      int used = 0;
      bool conv = false;
      for (int s = 0; s < sweeps_done; ++s) {
        used = s + 1;
        if (bj_ldcg(&a.counters[z * a.max_sweeps + s]) == 0) {
          conv = true;
          break;
        }
      }
      int* is = a.t.istat + z * a.t.nis;
      if (used > is[IS_SWEEPS_MAX]) is[IS_SWEEPS_MAX] = used;
      if (a.count_nonconv && !conv && a.n.eval(a.t, z) > 1) is[IS_NONCONV] += 1;
    }
  }
}

}  // namespace ttm
