// ttm_jac4.cuh -- float32 one-sided Jacobi with two columns per tournament slot, for the
// Swap SVD (Fig. 1C, Eq. eps).
//
// The scalar kernel (ttm_svd.cuh) pairs single columns: n - 1 rounds per sweep, each ending
// at a grid-wide barrier, which sets the cost of a sweep on this part. Here the round-robin
// tournament (Brent & Luk 1985) runs over n/2 slots of two columns each, so a sweep has
// n/2 - 1 rounds. A warp takes one slot pair (four columns, kept in registers, at most 1024
// rows) and visits its six column pairs in three inner rounds of two disjoint pairs:
//   {(0,2), (1,3)}, {(0,3), (1,2)}, {(0,1), (2,3)},
// so every column pair meets at least once per sweep; the two pairs inside a slot meet in
// every round (cheap once they are converged). The rotations are those of the scalar
// kernel (same tests, floors and formulas), and the same rotations are applied to the four
// columns of V, staged in shared memory while the W pairs are worked on.
#pragma once
#include <cooperative_groups.h>
#include "ttm_common.cuh"

namespace cg = cooperative_groups;

namespace ttm {

constexpr int kJ4Warps = 4;      // warps per CTA
constexpr int kJ4MaxN = 1024;    // V columns staged in shared memory

struct Jac4Args {
  Tables t;
  int bw, bv;        // W: m x n float column-major (in/out), V: n x n float column-major (out, from I)
  Dim m, n;
  int nslot_pad_ub;  // even host upper bound of ceil(n / 2)
  int max_sweeps;
  int* counters;     // [nz][max_sweeps] rotations per sweep, zeroed before launch
  double tol, delta; // tests of the scalar kernel
  double* fro2;      // [nz] ||W||_F^2, zeroed before launch
  int flop_slot;
  int count_nonconv;
};

__device__ __forceinline__ void j4_pair(int k, int r, int i, int& p, int& q) {
  if (i == 0) {
    p = k - 1;
    q = r;
  } else {
    p = (r + i) % (k - 1);
    q = (r - i + k - 1) % (k - 1);
  }
}

// R rows per lane: the kernel handles m <= 32 R.
template <int R>
__global__ void __launch_bounds__(kJ4Warps * 32) jacobi4_kernel(Jac4Args a) {
  extern __shared__ float j4_smem[];  // [warp][4][n] V columns
  cg::grid_group grid = cg::this_grid();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const long gthread = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long nthreads = (long)gridDim.x * blockDim.x;
  const long gwarp = (long)wid * gridDim.x + blockIdx.x, nwarps = nthreads >> 5;
  const int nz = a.t.nz;
  float* sV = j4_smem + (long)wid * 4 * kJ4MaxN;

  for (int z = 0; z < nz; ++z) {
    const int n = a.n.eval(a.t, z), m = a.m.eval(a.t, z);
    float* V = reinterpret_cast<float*>(bufp(a.t, z, a.bv));
    for (long e = gthread; e < (long)n * n; e += nthreads) V[e] = (e % n == e / n) ? 1.f : 0.f;
    const float* W = reinterpret_cast<const float*>(bufp(a.t, z, a.bw));
    double f = 0.0;
    for (long e = gthread; e < (long)m * n; e += nthreads) f = fma((double)W[e], (double)W[e], f);
    f = warp_sum(f);
    if (lane == 0 && f != 0.0) atomicAdd(&a.fro2[z], f);
  }
  grid.sync();

  const int half = a.nslot_pad_ub / 2;
  const long items = (long)nz * half;
  double flops = 0.0;
  int sweeps_done = 0;
  for (int sweep = 0; sweep < a.max_sweeps; ++sweep) {
    for (int r = 0; r < a.nslot_pad_ub - 1; ++r) {
      for (long it = gwarp; it < items; it += nwarps) {
        const int z = (int)(it / half), i = (int)(it % half);
        const int n = a.n.eval(a.t, z);
        const int ns = (n + 1) / 2;
        const int nsp = ns + (ns & 1);
        if (i >= nsp / 2 || r >= nsp - 1) continue;
        int P, Q;
        j4_pair(nsp, r, i, P, Q);
        if (P >= ns || Q >= ns) continue;
        if (sweep > 0 && __ldcg(&a.counters[z * a.max_sweeps + sweep - 1]) == 0) continue;
        const int m = a.m.eval(a.t, z);
        float* W = reinterpret_cast<float*>(bufp(a.t, z, a.bw));
        float* V = reinterpret_cast<float*>(bufp(a.t, z, a.bv));
        int col[4] = {2 * P, 2 * P + 1, 2 * Q, 2 * Q + 1};
        bool valid[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) valid[c] = col[c] < n;
        // W columns into registers, V columns into shared memory (used after the W work)
        float x[4][R];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const float* wc = W + (long)col[c] * m;
#pragma unroll
          for (int k = 0; k < R; ++k) {
            const int row = lane + 32 * k;
            x[c][k] = (valid[c] && row < m) ? __ldcg(wc + row) : 0.f;
          }
        }
        for (int c = 0; c < 4; ++c) {
          if (!valid[c]) continue;
          const float* vc = V + (long)col[c] * n;
          for (int row = lane; row < n; row += 32) sV[c * kJ4MaxN + row] = __ldcg(vc + row);
        }
        const double fro = sqrt(__ldcg(&a.fro2[z]));
        float cs[3][2], sn[3][2];
        int nrot = 0;
        const int pp[3][2] = {{0, 1}, {0, 1}, {0, 2}};
        const int qq[3][2] = {{2, 3}, {3, 2}, {1, 3}};
#pragma unroll
        for (int ir = 0; ir < 3; ++ir) {
          float al[2], be[2], ga[2];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int p = pp[ir][h], q = qq[ir][h];
            float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
            for (int k = 0; k < R; ++k) {
              s0 = fmaf(x[p][k], x[p][k], s0);
              s1 = fmaf(x[q][k], x[q][k], s1);
              s2 = fmaf(x[p][k], x[q][k], s2);
            }
            al[h] = s0;
            be[h] = s1;
            ga[h] = s2;
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              al[h] += __shfl_xor_sync(0xffffffffu, al[h], o);
              be[h] += __shfl_xor_sync(0xffffffffu, be[h], o);
              ga[h] += __shfl_xor_sync(0xffffffffu, ga[h], o);
            }
          }
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int p = pp[ir][h], q = qq[ir][h];
            float c = 1.f, s = 0.f;
            const double aga = fabs((double)ga[h]);
            const double big = sqrt((double)fmaxf(al[h], be[h]));
            if (valid[p] && valid[q] && ga[h] != 0.f &&
                aga > a.tol * sqrt((double)al[h]) * sqrt((double)be[h]) && aga > a.delta * big * fro) {
              const float zeta = (be[h] - al[h]) / (2.f * ga[h]);
              const float tt = copysignf(1.f, zeta) / (fabsf(zeta) + hypotf(1.f, zeta));
              c = 1.f / sqrtf(fmaf(tt, tt, 1.f));
              s = c * tt;
              ++nrot;
#pragma unroll
              for (int k = 0; k < R; ++k) {
                const float xp = x[p][k], xq = x[q][k];
                x[p][k] = c * xp - s * xq;
                x[q][k] = fmaf(s, xp, c * xq);
              }
            }
            cs[ir][h] = c;
            sn[ir][h] = s;
          }
          flops += 12.0 * m;
        }
        if (nrot > 0) {
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            if (!valid[c]) continue;
            float* wc = W + (long)col[c] * m;
#pragma unroll
            for (int k = 0; k < R; ++k) {
              const int row = lane + 32 * k;
              if (row < m) wc[row] = x[c][k];
            }
          }
          __syncwarp();
          for (int row = lane; row < n; row += 32) {
            float v[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) v[c] = sV[c * kJ4MaxN + row];
#pragma unroll
            for (int ir = 0; ir < 3; ++ir)
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                const int p = pp[ir][h], q = qq[ir][h];
                const float c = cs[ir][h], s = sn[ir][h];
                if (s != 0.f) {
                  const float vp = v[p], vq = v[q];
                  v[p] = c * vp - s * vq;
                  v[q] = fmaf(s, vp, c * vq);
                }
              }
#pragma unroll
            for (int c = 0; c < 4; ++c)
              if (valid[c]) V[(long)col[c] * n + row] = v[c];
          }
          flops += 12.0 * nrot * ((double)m + n) / 2.0;
          if (lane == 0) atomicAdd(&a.counters[z * a.max_sweeps + sweep], nrot);
        }
        __syncwarp();  // sV is reused by the warp's next item
      }
      grid.sync();
    }
    sweeps_done = sweep + 1;
    bool all = true;
    for (int z = 0; z < nz; ++z)
      if (__ldcg(&a.counters[z * a.max_sweeps + sweep]) != 0) all = false;
    if (all) break;
  }
  if (lane == 0 && flops > 0.0) atomicAdd(&a.t.stat[a.flop_slot], flops);
  if (gthread == 0) {
    for (int z = 0; z < nz; ++z) {
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
    }
  }
}

}  // namespace ttm
