// ttm_common.cuh -- shared device-side data model of the TTM engine.
//
// Every product of a batch owns a row of three tables in device memory:
//   buf  [z][nb]   : pointers to its carriage buffers and workspaces,
//   bond [z][nbd]  : the current value of every bond id (written by the kernels
//                    that create bonds: QR moves, Swap truncations),
//   stat [z][ns]   : float64 statistics (discarded weights, norms, flop counters),
//   istat[z][nis]  : int32 statistics (max bond, Jacobi sweeps, status flags).
// The host walks a static schedule and passes only ids; the kernels read the
// realised bond values, so the whole sweep needs no host synchronisation and can
// be captured in a CUDA graph. Grids are sized by host-side upper bounds and
// blocks beyond the realised sizes exit early. gridDim.z (or a loop) runs over
// the products of a batch.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "ttm.h"

namespace ttm {

struct Tables {
  double** buf;
  int* bond;
  double* stat;
  int* istat;
  int nb, nbd, ns, nis;
  int nz;  // products in this launch
};

__device__ __forceinline__ int bondv(const Tables& t, int z, int id) {
  return id < 0 ? 1 : t.bond[z * t.nbd + id];
}
__device__ __forceinline__ double* bufp(const Tables& t, int z, int id) {
  return t.buf[z * t.nb + id];
}

// istat slots
enum { IS_STATUS = 0, IS_MAX_BOND = 1, IS_SWEEPS_MAX = 2, IS_NONCONV = 3, IS_NFROZEN = 4, IS_NEWTON_BAD = 5,
       IS_ROUND = 6, IS_CAST_EXP = 7, IS_FALLBACK = 8, IS_NEWTON_MORE = 9, IS_NFIXED = 10 };
// stat slots (the per-truncation weights follow from ST_NFIXED)
enum { ST_WSUM = 0, ST_WSQRT = 1, ST_NEWTON_RES = 2, ST_JFLOPS32 = 3, ST_NEWTON_CUR = 4, ST_TRACE = 5,
       ST_JFLOPS = 6, ST_JSWEEPS32 = 7, ST_GFLOPS = 8, ST_NFIXED = 9 };

// Per-SVD diagnostic record (the report's svd_trace): m, n, k, float32 sweeps of passes
// 0, 1, 2, fallback flag.
constexpr int kSvdRec = 8;
enum { SR_M = 0, SR_N = 1, SR_K = 2, SR_SW0 = 3, SR_FALLBACK = 6 };

// Largest correction max(|S_ij|, |E_ij| / 2) of the last Newton step of an SVD for which it
// counts as converged: the error left after a step is of the order of its correction squared,
// so 1e-7 leaves couplings and an orthogonality defect near 1e-14.
constexpr double kNewtonConverged = 1e-7;

// A dimension written as mul * bond[id] (id < 0 means the constant mul).
struct Dim {
  int mul, id;
  __device__ __forceinline__ int eval(const Tables& t, int z) const { return mul * bondv(t, z, id); }
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace ttm
