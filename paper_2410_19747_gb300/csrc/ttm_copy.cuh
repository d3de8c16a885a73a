// ttm_copy.cuh -- strided 2D copies used around the decompositions:
// row-major carriage <-> column-major workspace, the bond-leg exchange of the
// reversed train (Eq. tensor), and plain compaction. A functor maps (product z,
// batch b) to (rows, cols, src view, dst view); sizes come from the bond table.
#pragma once
#include "ttm_common.cuh"
#include "ttm_gemm.cuh"

namespace ttm {

struct CopyDesc {
  int rows, cols;
  MatRef src;
  OutRef dst;
};

// 32 x 32 tiles through shared memory so both sides can be read and written with
// unit stride whichever of the two has it.
template <class F>
__global__ void __launch_bounds__(256) copy2d_kernel(F f, int nbatch) {
  const int z = blockIdx.z / nbatch, b = blockIdx.z % nbatch;
  const CopyDesc c = f(z, b);
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  if (r0 >= c.rows || c0 >= c.cols) return;
  __shared__ double tile[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  const bool src_rowfast = (c.src.cs == 1);
  for (int k = ty; k < 32; k += 8) {
    const int i = src_rowfast ? r0 + k : r0 + tx;
    const int j = src_rowfast ? c0 + tx : c0 + k;
    if (i < c.rows && j < c.cols) {
      const double v = c.src.p[(long)i * c.src.rs + (long)j * c.src.cs];
      if (src_rowfast) tile[k][tx] = v; else tile[tx][k] = v;
    }
  }
  __syncthreads();
  const bool dst_rowfast = (c.dst.cs == 1);
  for (int k = ty; k < 32; k += 8) {
    const int i = dst_rowfast ? r0 + k : r0 + tx;
    const int j = dst_rowfast ? c0 + tx : c0 + k;
    if (i < c.rows && j < c.cols) {
      const double v = dst_rowfast ? tile[k][tx] : tile[tx][k];
      c.dst.p[(long)i * c.dst.rs + (long)j * c.dst.cs] = v;
    }
  }
}

// Carriage [Dl][d][Dr] (row-major m x n, m = Dl*d, n = Dr) -> column-major workspace.
struct RowToColFn {
  Tables t;
  int bsrc, bdst;
  Dim m, n;
  __device__ CopyDesc operator()(int z, int) const {
    const int M = m.eval(t, z), N = n.eval(t, z);
    return CopyDesc{M, N, MatRef{bufp(t, z, bsrc), N, 1}, OutRef{bufp(t, z, bdst), 1, M}};
  }
};

// Column-major m x k workspace -> row-major carriage.
struct ColToRowFn {
  Tables t;
  int bsrc, bdst;
  Dim m, k;
  __device__ CopyDesc operator()(int z, int) const {
    const int M = m.eval(t, z), K = k.eval(t, z);
    return CopyDesc{M, K, MatRef{bufp(t, z, bsrc), 1, M}, OutRef{bufp(t, z, bdst), K, 1}};
  }
};

// Bond-leg exchange: dst[r, s, l] = src[l, s, r] (batch b = s).
struct LegSwapFn {
  Tables t;
  int bsrc, bdst;
  int il, ir;
  int d;
  __device__ CopyDesc operator()(int z, int s) const {
    const int Dl = bondv(t, z, il), Dr = bondv(t, z, ir);
    return CopyDesc{Dl, Dr, MatRef{bufp(t, z, bsrc) + (long)s * Dr, (long)d * Dr, 1},
                    OutRef{bufp(t, z, bdst) + (long)s * Dl, 1, (long)d * Dl}};
  }
};

}  // namespace ttm
