// ttm_tc.cuh -- float64-accurate GEMM on the fifth-generation tensor cores (tcgen05) by
// exact slicing of the operands into bf16 integers (the Ozaki scheme: Ozaki, Ogita, Oishi &
// Rump 2012, error-free splitting of a matrix product into exactly computed partial products).
//
// C = A B with A (M x K) and B (K x N) in float64. Every row r of A is scaled by a power of
// two 2^e_r so that its entries lie in (-1, 1) (every column of B likewise, 2^f_c), and each
// scaled entry x is written as a sum of S signed integer digits,
//     x = sum_t s_t 2^(-6 - 7 t),   |s_t| <= 64,   t = 0 .. S-1,
// every digit exact in bf16. A product of two digits is an integer of magnitude <= 2^12, so
// a K-sum of up to 1024 of them is an integer below 2^24: the tensor core's float32
// accumulator holds it exactly. The partial products of digit levels t + u = l share the
// weight 2^(-12 - 7 l); each level l < S accumulates in its own TMEM accumulator (levels up
// to 3 exactly, the higher ones with a float32 rounding far below float64 resolution of the
// result), and the epilogue combines the levels in float64:
//     C_rc = 2^(e_r + f_c) sum_l 2^(-12 - 7 l) acc_l,
// over the S (S + 1) / 2 digit pairs with t + u < S. With S = 8 the digits carry 55 bits, so
// the result is as accurate as a float64 GEMM. An optional power-of-two scale per K index
// (A diag(2^-q) times diag(2^q) B, mathematically the identity) lets graded operands keep
// relative accuracy per column (W = Theta V with column norms spanning many decades).
//
// Kernels: oz_exp_kernel (row / column exponents), oz_slice_kernel (digits, written in the
// tcgen05 shared-memory layout: K-major, no swizzle, 8 x 16-byte core matrices, so that one
// bulk copy moves a whole tile), oz_gemm_kernel (one CTA per 128 x 64 output tile: a TMA
// producer warp with cp.async.bulk, one thread issuing tcgen05.mma kind::f16 into eight
// TMEM accumulators, four epilogue warps reading them with tcgen05.ld).
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

#include "ttm_common.cuh"
#include "ttm_gemm.cuh"

namespace ttm {

constexpr int kOzMaxS = 8;        // digits per operand (and TMEM accumulators)
constexpr int kOzTM = 128;        // rows of an output tile (UMMA M)
constexpr int kOzTN = 64;         // columns of an output tile (UMMA N)
constexpr int kOzKC = 32;         // K of one pipeline stage
constexpr int kOzKB = 1024;       // K summed exactly in one accumulator block
constexpr int kOzATile = kOzTM * kOzKC * 2;  // bytes of one A digit tile (8 KB)
constexpr int kOzBTile = kOzTN * kOzKC * 2;  // bytes of one B digit tile (4 KB)
constexpr int kOzStages = 2;
constexpr int kOzThreads = 192;   // warps 0-3 epilogue, warp 4 TMA producer, warp 5 MMA issuer
constexpr int kOzExpNone = -100000;  // exponent of an all-zero row or column

__host__ __device__ constexpr int oz_stage_bytes(int S) { return S * (kOzATile + kOzBTile); }
__host__ __device__ constexpr int oz_smem_bytes(int S) { return kOzStages * oz_stage_bytes(S) + 256; }
// TMEM columns of the S accumulators (a power of two, at least 32)
__host__ __device__ constexpr uint32_t oz_tmem_cols(int S) {
  return S * kOzTN <= 32 ? 32u : S * kOzTN <= 64 ? 64u : S * kOzTN <= 128 ? 128u : S * kOzTN <= 256 ? 256u : 512u;
}

// One GEMM of a launch: the float64 problem (from a functor, as for dgemm_kernel) and where
// its digits live.
struct OzWs {
  unsigned char* a;   // digits of A: [S][row tiles of 128][K chunks of 32] tiles of 8 KB
  unsigned char* b;   // digits of B^T: [S][column tiles of 64][K chunks of 32] tiles of 4 KB
  int* ea;            // row exponents of A (M entries)
  int* eb;            // column exponents of B (N entries)
  long a_stride, b_stride, e_stride;  // bytes / ints per (z, batch) problem
  int S;
  int* err;           // set to TTM_ERR_TIMEOUT when a bounded wait gives up
  int kscale_buf;     // buffer id of per-K power-of-two exponents q_k (ints in a double
                      // buffer: A diag(2^-q) times diag(2^q) B), -1 = none
};

__global__ void fill_int_kernel(int* p, long n, int v) {
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) p[e] = v;
}

// Per-column binary exponents q_j of a column-major m x n matrix (frexp of the column's
// largest magnitude; 0 for a zero column), written as ints into a double buffer: the K scale
// that makes W diag(2^-q) have columns of magnitude near 1. One warp per column.
struct ColExpArgs {
  Tables t;
  int bw, bq;
  Dim m, n;
};
__global__ void colexp_kernel(ColExpArgs a) {
  const int z = blockIdx.y;
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  const int n = a.n.eval(a.t, z);
  if (j >= n) return;
  const int m = a.m.eval(a.t, z);
  const double* w = bufp(a.t, z, a.bw) + (long)j * m;
  double mx = 0.0;
  for (int r = lane; r < m; r += 32) mx = fmax(mx, fabs(w[r]));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) {
    int e = 0;
    if (mx > 0.0) frexp(mx, &e);
    reinterpret_cast<int*>(bufp(a.t, z, a.bq))[j] = e;
  }
}

// ---------------------------------------------------------------- operand views
// Operand X (0 = A as R = M rows, 1 = B viewed transposed as R = N rows), both with K columns.
__device__ __forceinline__ double oz_elem(const GemmDesc& g, int which, int r, int k) {
  return which == 0 ? g.A.p[(long)r * g.A.rs + (long)k * g.A.cs] : g.B.p[(long)k * g.B.rs + (long)r * g.B.cs];
}
__device__ __forceinline__ bool oz_r_fast(const GemmDesc& g, int which) {
  return which == 0 ? g.A.rs == 1 : g.B.cs == 1;
}

template <class F>
struct OzArgs {
  F f;
  int nbatch;
  OzWs w;
  double* fl;     // nullptr, or per-product flop accumulators (stride fl_stride)
  int fl_stride;
};

// Exponents: e_r = the binary exponent of max_k |X_rk 2^(-+q_k)| (frexp convention, so the
// scaled row lies in (-1, 1)); kOzExpNone for a zero row. Grid: (K / 32, R / 32, problems),
// block 32 x 8; the 32 x 32 tile is read along the operand's unit stride.
template <class F>
__global__ void oz_exp_kernel(OzArgs<F> a, int which) {
  const int zb = blockIdx.z, z = zb / a.nbatch, b = zb % a.nbatch;
  const GemmDesc g = a.f(z, b);
  const int R = which == 0 ? g.M : g.N, K = g.K;
  const int r0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
  if (R <= 0 || K <= 0 || r0 >= R || k0 >= K) return;
  __shared__ double tile[32][33];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const bool rf = oz_r_fast(g, which);
  const int* q = a.w.kscale_buf >= 0 ? reinterpret_cast<const int*>(bufp(a.f.t, z, a.w.kscale_buf)) : nullptr;
  for (int i = ty; i < 32; i += 8) {
    const int rr = rf ? tx : i, kk = rf ? i : tx;
    const int r = r0 + rr, k = k0 + kk;
    double v = 0.0;
    if (r < R && k < K) {
      v = fabs(oz_elem(g, which, r, k));
      if (q) v = ldexp(v, which == 0 ? -q[k] : q[k]);
    }
    tile[rr][kk] = v;
  }
  __syncthreads();
  if (ty == 0) {
    double m = 0.0;
    for (int kk = 0; kk < 32; ++kk) m = fmax(m, tile[tx][kk]);
    if (m > 0.0 && r0 + tx < R) {
      int e;
      frexp(m, &e);
      int* ex = (which == 0 ? a.w.ea : a.w.eb) + (long)zb * a.w.e_stride;
      atomicMax(ex + r0 + tx, e);
    }
  }
}

// Byte offset of digit t of element (r, k) in the tile layout of an operand with row tiles of
// TR rows: tiles ordered [t][row tile][K chunk]; inside a tile the 8 x 8 core matrices are
// ordered K chunk of 8 outer, row group of 8 inner (leading byte offset TR / 8 * 128 between
// K neighbours, stride byte offset 128 between row neighbours), each core matrix 8 rows of
// 16 contiguous bytes.
template <int TR>
__device__ __forceinline__ long oz_off(int t, int r, int k, int nrt, int nkc) {
  const long tile = ((long)t * nrt + r / TR) * nkc + k / kOzKC;
  const int mi = (r % TR) >> 3, ki = (k % kOzKC) >> 3;
  return tile * (TR * kOzKC * 2) + (ki * (TR / 8) + mi) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// Digits of one operand over its padded extent (zeros outside the matrix). Grid: (Kpad / 32,
// Rpad / 32, problems), block 32 x 8.
template <class F, int TR>
__global__ void oz_slice_kernel(OzArgs<F> a, int which, int rpad, int kpad) {
  const int zb = blockIdx.z, z = zb / a.nbatch, b = zb % a.nbatch;
  const GemmDesc g = a.f(z, b);
  const int R = which == 0 ? g.M : g.N, K = g.K;
  const int r0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
  const int nrt = rpad / TR, nkc = kpad / kOzKC;
  if (r0 >= rpad || k0 >= kpad) return;
  __shared__ double tile[32][33];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const bool rf = oz_r_fast(g, which);
  const int* q = a.w.kscale_buf >= 0 ? reinterpret_cast<const int*>(bufp(a.f.t, z, a.w.kscale_buf)) : nullptr;
  for (int i = ty; i < 32; i += 8) {
    const int rr = rf ? tx : i, kk = rf ? i : tx;
    const int r = r0 + rr, k = k0 + kk;
    double v = 0.0;
    if (R > 0 && K > 0 && r < R && k < K) {
      v = oz_elem(g, which, r, k);
      if (q) v = ldexp(v, which == 0 ? -q[k] : q[k]);
    }
    tile[rr][kk] = v;
  }
  __syncthreads();
  const int* ex = (which == 0 ? a.w.ea : a.w.eb) + (long)zb * a.w.e_stride;
  unsigned char* base = (which == 0 ? a.w.a + zb * a.w.a_stride : a.w.b + zb * a.w.b_stride);
  for (int i = ty; i < 32; i += 8) {
    const int r = r0 + i, k = k0 + tx;
    const int e = (r < R) ? ex[r] : kOzExpNone;
    double x = tile[i][tx];
    // x 2^-e in (-1, 1), times 2^6: the first digit in [-64, 64]
    double rem = (e == kOzExpNone) ? 0.0 : ldexp(x, 6 - e);
    for (int t = 0; t < a.w.S; ++t) {
      const double s = rint(rem);
      rem = (rem - s) * 128.0;
      *reinterpret_cast<__nv_bfloat16*>(base + oz_off<TR>(t, r, k, nrt, nkc)) = __double2bfloat16(s);
    }
  }
}

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// Waits for the phase with the given parity to complete; gives up after limit_ns and
// returns false (the caller records TTM_ERR_TIMEOUT and winds down without trapping).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
  uint32_t done = 0;
  const uint64_t t0 = globaltimer_ns();
  while (true) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (globaltimer_ns() - t0 > limit_ns) return false;
  }
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
// Shared-memory matrix descriptor of tcgen05.mma: start address, leading byte offset (between
// core matrices along K) and stride byte offset (between core matrices along M / N), all in
// 16-byte units; version 1 at bits 46-47; no swizzle.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}
// Instruction descriptor of kind::f16: bf16 A and B (K-major), float32 accumulator, M x N.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
// 32 lanes x 32 consecutive float32 columns of TMEM into 32 registers per thread.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

constexpr uint64_t kOzWaitNs = 2000000000ull;  // 2 s: far beyond any legitimate wait

// ---------------------------------------------------------------- the GEMM
// Grid: (N tiles of 64, M tiles of 128, problems). Dynamic shared memory: oz_smem_bytes(S).
template <class F>
__global__ void __launch_bounds__(kOzThreads, 1) oz_gemm_kernel(OzArgs<F> a, int mpad, int npad, int kpad) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int zb = blockIdx.z, z = zb / a.nbatch, b = zb % a.nbatch;
  const GemmDesc g = a.f(z, b);
  const int m0 = blockIdx.y * kOzTM, n0 = blockIdx.x * kOzTN;
  if (g.M <= 0 || g.N <= 0 || m0 >= g.M || n0 >= g.N) return;   // CTA-uniform exit
  if (m0 == 0 && n0 == 0 && threadIdx.x == 0) gemm_count_flops(a.fl, a.fl_stride, z, g);
  if (g.upper && m0 > n0 + kOzTN - 1) return;
  const int S = a.w.S;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nkc = (g.K + kOzKC - 1) / kOzKC;            // K chunks of this problem
  const int nrtA = mpad / kOzTM, nrtB = npad / kOzTN, nkcp = kpad / kOzKC;
  const int stage_bytes = oz_stage_bytes(S);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kOzStages * stage_bytes);
  // bars: full[2], empty[2], acc_full, acc_empty; then the TMEM address
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 8);
  __shared__ int s_abort;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kOzStages; ++s) {
      mbar_init(smem_u32(&bars[s]), 1);
      mbar_init(smem_u32(&bars[2 + s]), 1);
    }
    mbar_init(smem_u32(&bars[4]), 1);
    mbar_init(smem_u32(&bars[5]), 128);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  const uint32_t tcols = oz_tmem_cols(S);
  __syncwarp();     // warp 0 reconverges after thread 0's barrier set-up (alloc is warp-collective)
  if (warp == 0) {  // TMEM: S accumulators of 64 float32 columns
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(tcols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int nkb = (nkc + (kOzKB / kOzKC) - 1) / (kOzKB / kOzKC);  // exact accumulation blocks

  if (warp == 4) {
    // ---------------- TMA producer: all S digit tiles of A and of B for one K chunk per stage
    if (lane == 0) {
      const unsigned char* Ab = a.w.a + zb * a.w.a_stride;
      const unsigned char* Bb = a.w.b + zb * a.w.b_stride;
      for (int kc = 0; kc < nkc; ++kc) {
        const int s = kc % kOzStages;
        if (kc >= kOzStages && !mbar_wait(smem_u32(&bars[2 + s]), ((kc / kOzStages) - 1) & 1, kOzWaitNs)) {
          atomicExch(&s_abort, 1);
          break;
        }
        if (s_abort) break;
        const uint32_t full = smem_u32(&bars[s]);
        mbar_expect_tx(full, (uint32_t)stage_bytes);
        unsigned char* st = smem + s * stage_bytes;
        for (int t = 0; t < S; ++t) {
          const long ta = ((long)t * nrtA + blockIdx.y) * nkcp + kc;
          bulk_g2s(smem_u32(st + t * kOzATile), Ab + ta * kOzATile, kOzATile, full);
          const long tb = ((long)t * nrtB + blockIdx.x) * nkcp + kc;
          bulk_g2s(smem_u32(st + S * kOzATile + t * kOzBTile), Bb + tb * kOzBTile, kOzBTile, full);
        }
      }
    }
  } else if (warp == 5) {
    // ---------------- MMA issuer: every digit pair (t, u) with t + u < S, two K steps of 16
    if (lane == 0) {
      const uint32_t idesc = umma_idesc_bf16(kOzTM, kOzTN);
      int kc = 0;
      for (int kb = 0; kb < nkb && !s_abort; ++kb) {
        if (kb > 0 && !mbar_wait(smem_u32(&bars[5]), (kb - 1) & 1, kOzWaitNs)) {  // epilogue drained
          atomicExch(&s_abort, 1);
          break;
        }
        tc_fence_after();
        const int kc_end = min(nkc, (kb + 1) * (kOzKB / kOzKC));
        bool first = true;
        for (; kc < kc_end; ++kc) {
          const int s = kc % kOzStages;
          if (!mbar_wait(smem_u32(&bars[s]), (kc / kOzStages) & 1, kOzWaitNs)) {
            atomicExch(&s_abort, 1);
            break;
          }
          tc_fence_after();
          const uint32_t st = smem_u32(smem + s * stage_bytes);
          for (int ks = 0; ks < kOzKC / 16; ++ks) {
            for (int t = 0; t < S; ++t) {
              const uint64_t ad = umma_desc(st + t * kOzATile + ks * 2 * (kOzTM / 8) * 128, (kOzTM / 8) * 128, 128);
              for (int u = 0; u + t < S; ++u) {
                const uint64_t bd =
                    umma_desc(st + S * kOzATile + u * kOzBTile + ks * 2 * (kOzTN / 8) * 128, (kOzTN / 8) * 128, 128);
                // the first step of a block starts every accumulator afresh
                umma_bf16(tmem + (uint32_t)((t + u) * kOzTN), ad, bd, idesc, first ? (t == 0 ? 0u : 1u) : 1u);
              }
            }
            // level l receives its first product from t = 0 (u = l), which zeroes it
            first = false;
          }
          umma_commit(smem_u32(&bars[2 + s]));  // the stage is free once these MMAs are done
        }
        umma_commit(smem_u32(&bars[4]));        // block done: accumulators ready
      }
    }
  } else {
    // ---------------- epilogue: warps 0-3, thread = tile row (TMEM lane)
    const int row = warp * 32 + lane;
    const int gr = m0 + row;
    double acc[kOzTN];
#pragma unroll
    for (int j = 0; j < kOzTN; ++j) acc[j] = 0.0;
    bool ok = true;
    for (int kb = 0; kb < nkb; ++kb) {
      // one lane waits, the warp reconverges before the warp-collective tcgen05.ld
      int got = lane == 0 ? (mbar_wait(smem_u32(&bars[4]), kb & 1, kOzWaitNs) ? 1 : 0) : 0;
      got = __shfl_sync(0xffffffffu, got, 0);
      __syncwarp();
      if (!got) {
        if (lane == 0) atomicExch(&s_abort, 1);
        ok = false;
        break;
      }
      tc_fence_after();
      for (int l = 0; l < S; ++l) {
        const double w = ldexp(1.0, -12 - 7 * l);
#pragma unroll
        for (int h = 0; h < kOzTN / 32; ++h) {
          float v[32];
          tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(l * kOzTN + h * 32), v);
#pragma unroll
          for (int j = 0; j < 32; ++j) acc[h * 32 + j] = fma((double)v[j], w, acc[h * 32 + j]);
        }
      }
      tc_fence_before();
      __syncwarp();
      mbar_arrive(smem_u32(&bars[5]));
    }
    if (ok && gr < g.M) {
      const int* eA = a.w.ea + (long)zb * a.w.e_stride;
      const int* eB = a.w.eb + (long)zb * a.w.e_stride;
      const int er = eA[gr];
#pragma unroll
      for (int j = 0; j < kOzTN; ++j) {  // fully unrolled: acc stays in registers
        const int gc = n0 + j;
        if (gc < g.N) {
          const int ec = eB[gc];
          double v = 0.0;
          if (er != kOzExpNone && ec != kOzExpNone) v = ldexp(acc[j], er + ec);
          double* c = g.C.p + (long)gr * g.C.rs + (long)gc * g.C.cs;
          v *= g.alpha;
          if (g.beta != 0.0) v = fma(g.beta, *c, v);
          *c = v;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (s_abort && threadIdx.x == 0 && a.w.err) atomicExch(a.w.err, (int)TTM_ERR_TIMEOUT);
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols) : "memory");
  }
}

// ---------------------------------------------------------------- host side
inline long oz_cdiv(long a, long b) { return (a + b - 1) / b; }

// Kernel of launch_tc_gemm that last reported an error (for the error message).
inline const char*& tc_failed_step() {
  static thread_local const char* step = "";
  return step;
}

// Digit workspace of one launch of nprob problems with the given upper bounds.
inline size_t tc_ws_bytes(long nprob, int M_ub, int N_ub, int K_ub, int S) {
  const long mpad = oz_cdiv(M_ub, kOzTM) * kOzTM, npad = oz_cdiv(N_ub, kOzTN) * kOzTN;
  const long kpad = oz_cdiv(K_ub > 0 ? K_ub : 1, kOzKC) * kOzKC;
  const long e_ints = mpad > npad ? mpad : npad;
  return (size_t)(nprob * S * (mpad + npad) * kpad * 2 + 2 * nprob * e_ints * (long)sizeof(int) + 256);
}

// Exponents, digits and the tensor-core product of every (z, batch) problem of the functor.
// ws: tc_ws_bytes(nz * nbatch, ...) bytes of device memory; err: int set on a timeout.
template <class F>
cudaError_t launch_tc_gemm(cudaStream_t st, const F& f, int nz, int nbatch, int M_ub, int N_ub, int K_ub, int kscale_buf,
                    int S, unsigned char* ws, int* err, double* fl = nullptr, int fl_stride = 0) {
  const long mpad = oz_cdiv(M_ub, kOzTM) * kOzTM, npad = oz_cdiv(N_ub, kOzTN) * kOzTN;
  const long kpad = oz_cdiv(K_ub > 0 ? K_ub : 1, kOzKC) * kOzKC;
  const long nprob = (long)nz * nbatch;
  const long a_bytes = S * mpad * kpad * 2, b_bytes = S * npad * kpad * 2;
  const long e_ints = mpad > npad ? mpad : npad;
  OzWs w;
  w.a = ws;
  w.b = ws + nprob * a_bytes;
  w.ea = reinterpret_cast<int*>(ws + nprob * (a_bytes + b_bytes));
  w.eb = w.ea + nprob * e_ints;
  w.a_stride = a_bytes;
  w.b_stride = b_bytes;
  w.e_stride = e_ints;
  w.S = S;
  w.err = err;
  w.kscale_buf = kscale_buf;
  OzArgs<F> oa{f, nbatch, w, fl, fl_stride};
  const long ne = 2 * nprob * e_ints;
  // every launch is checked at once: the caller gets the first failing step
  const char*& step = tc_failed_step();
  step = "fill_int_kernel";
  fill_int_kernel<<<(unsigned)oz_cdiv(ne, 256), 256, 0, st>>>(w.ea, ne, kOzExpNone);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  step = "oz_exp_kernel";
  const dim3 blk(32, 8);
  oz_exp_kernel<F><<<dim3((unsigned)oz_cdiv(K_ub, 32), (unsigned)oz_cdiv(M_ub, 32), (unsigned)nprob), blk, 0, st>>>(oa, 0);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  oz_exp_kernel<F><<<dim3((unsigned)oz_cdiv(K_ub, 32), (unsigned)oz_cdiv(N_ub, 32), (unsigned)nprob), blk, 0, st>>>(oa, 1);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  step = "oz_slice_kernel";
  oz_slice_kernel<F, kOzTM><<<dim3((unsigned)(kpad / 32), (unsigned)(mpad / 32), (unsigned)nprob), blk, 0, st>>>(
      oa, 0, (int)mpad, (int)kpad);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  oz_slice_kernel<F, kOzTN><<<dim3((unsigned)(kpad / 32), (unsigned)(npad / 32), (unsigned)nprob), blk, 0, st>>>(
      oa, 1, (int)npad, (int)kpad);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(oz_gemm_kernel<F>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                oz_smem_bytes(kOzMaxS))) != cudaSuccess)
    return e;
  step = "oz_gemm_kernel";
  oz_gemm_kernel<F><<<dim3((unsigned)(npad / kOzTN), (unsigned)(mpad / kOzTM), (unsigned)nprob), kOzThreads,
                      oz_smem_bytes(S), st>>>(oa, (int)mpad, (int)npad, (int)kpad);
  return cudaGetLastError();
}

}  // namespace ttm
