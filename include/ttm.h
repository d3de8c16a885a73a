/*
 * ttm.h -- C ABI of the GB300 (sm_103a) Tensor Train Multiplication library (libttm.so).
 *
 * The library forms the elementwise (Hadamard) product Omega = A o B of two tensor
 * trains by the swap-and-contract sweep of arXiv:2410.19747, Sec. II.B:
 *   - the two trains are concatenated into one chain of length 2N with B reversed
 *     (Eq. tensor; each reversed carriage has its bond legs exchanged);
 *   - carriages with the same site index are joined by the local COPY tensor
 *     (Contract, Eq. contract);
 *   - B's carriages travel left by Swaps: two-site contraction, permutation of the
 *     physical legs, SVD and truncation by Eq. eps (Fig. 1C);
 *   - the chain is kept in mixed canonical gauge with QR gauge moves after every
 *     Contract (the paragraph after Eq. eps).
 * Every step runs in this library's own CUDA kernels on one GPU.
 *
 * Conventions shared by every call:
 *   - A TT of length L with physical dimension d is L cores; core k has shape
 *     [bonds[k]][d][bonds[k+1]], row-major, float64, contiguous; bonds[0] =
 *     bonds[L] = 1 (Eq. TT, Eq. bond).
 *   - Inputs are read-only, stream-ordered on the handle's stream and not
 *     retained after the call returns (host inputs are copied in).
 *   - No call throws or aborts. Every call returns a ttm_status; a message for the
 *     last failure on the calling thread is available from ttm_last_error().
 *   - Device-side waits are bounded; none traps.
 */
#ifndef TTM_H
#define TTM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ttm_handle ttm_handle;

typedef enum {
  TTM_OK = 0,
  TTM_ERR_INVALID_ARG = -1, /* null pointer, eps outside [0,1), L < 1, d < 2 ...      */
  TTM_ERR_SHAPE = -2,       /* boundary bond != 1, bond < 1, A/B mismatch, caller
                               buffer too small                                      */
  TTM_ERR_NOMEM = -3,       /* device allocation failed                              */
  TTM_ERR_WORKSPACE = -4,   /* a caller-sized workspace is too small                 */
  TTM_ERR_NONFINITE = -5,   /* NaN/Inf met in an input (only when checked)           */
  TTM_ERR_CUDA = -6,        /* a CUDA runtime call failed (message has the cause)    */
  TTM_ERR_TIMEOUT = -7,     /* a bounded device-side loop hit its iteration limit    */
  TTM_ERR_RANK_CAP = -8,    /* a bond would exceed the library's supported maximum   */
  TTM_ERR_UNSUPPORTED = -9, /* option combination not supported                      */
  TTM_WARN_NOT_CONVERGED = 1 /* the product was formed, but at least one Swap SVD did not
                               converge (its float64 Jacobi hit the sweep limit): the
                               report's n_nonconverged counts them; the truncation may be
                               suboptimal there                                       */
} ttm_status;

/* Arithmetic of the GEMM-shaped work: the contractions (Theta of every Swap, Contract, the
 * R merge of every gauge move) and the GEMMs inside the Swap SVD (its Newton steps). The
 * Householder QR, the Jacobi rotations, norms and the truncation rule always run on the
 * CUDA cores (float32 Jacobi passes, everything else float64). */
typedef enum {
  TTM_PREC_FP64 = 0,       /* every GEMM on the float64 pipe (the reference form)         */
  TTM_PREC_BF16_SPLIT = 2  /* every GEMM on the tcgen05 tensor cores as the exactly sliced
                              product of bf16 digits (Ozaki scheme): each float64 operand
                              row (column) is scaled by a power of two and split into
                              split_digits digits of 7 bits; the digit products are summed
                              exactly in float32 and combined in float64. 8 digits (the
                              default) give float64 accuracy                             */
} ttm_precision;

typedef enum {
  TTM_LOSS_INNER = 0,   /* f = <W, A o B>                                              */
  TTM_LOSS_SQDIST = 1   /* g = ||A o B - C||^2                                          */
} ttm_loss;

typedef struct {
  int32_t L;            /* number of sites (carriages)                                 */
  int32_t d;            /* physical dimension of every site                            */
  int32_t on_host;      /* 0: cores are device pointers; 1: host pointers (copied in,
                           and for outputs copied out, inside the call)               */
  int32_t reserved;
  int64_t *bonds;       /* L+1 entries, host memory                                    */
  double **cores;       /* L pointers, host array; core k = [bonds[k]][d][bonds[k+1]]  */
} ttm_tt;

typedef struct {
  ttm_precision prec;
  double eps;               /* Eq. eps threshold on the relative discarded weight of every
                               Swap SVD; 0 keeps every singular value                     */
  int64_t chi_max;          /* cap on the bond of every Swap SVD; 0 = unbounded          */
  int64_t chi_out;          /* cap on the output bonds; 0 = none. A product with an
                               output bond above chi_out gets a final TT-SVD rounding that
                               truncates bonds 1..L-1 in order with this cap and the eps
                               rule, leaving the norm on the last core; for a product whose
                               bonds are all within the cap the same sweep keeps every bond
                               (an exact refactorisation; decided per product on the
                               device)                                                    */
  int32_t max_sweeps;       /* sweep limit of the float32 Jacobi passes after the first
                               and of the float64 Jacobi of the Newton fallback; 0 = 20
                               and 40                                                     */
  int32_t use_graph;        /* 1: ttm_multiply / ttm_multiply_batched capture the kernel
                               sequence of a plan (options, shapes, input bonds, arena) into
                               a CUDA graph on first use and replay it while the plan stays
                               the same (input copies are issued before each replay); not
                               with profile_kernels = 1. 0: launch every kernel directly  */
  int32_t check_finite;     /* must be 0 (1 returns TTM_ERR_UNSUPPORTED)                  */
  int32_t profile_kernels;  /* 1: time every GEMM, float32 Jacobi and Householder launch
                               with CUDA events on the handle's stream (fills gemm_ms,
                               jacobi32_ms, jacobi64_ms and qr_ms of the report)          */
  int32_t f32_passes;       /* float32 one-sided Jacobi passes of every Swap SVD: 0 = 3
                               (the first stops after 3 sweeps), 1..8 accepted           */
  int32_t jacobi_kernel;    /* kernel of the float32 passes: 0 = 3 when the Swap matrix
                               has at most 1024 rows, else 1; 1 = one column per
                               tournament slot (n - 1 grid barriers per sweep); 2 = two
                               columns per slot (n/2 - 1 barriers; m, n <= 1024); 3 =
                               blocks of 8 columns held in shared memory, all pairs of a
                               block pair per CTA (about n/8 barriers; m <= 1024); 8 or
                               16 = Gram-based block Jacobi on blocks of that many
                               columns                                                   */
  int32_t newton_steps;     /* float64 Newton steps that finish every Swap SVD after the
                               float32 passes: 0 = 3, 1..8 accepted; an SVD whose last
                               correction is still above 1e-7 takes up to 2 more          */
  int32_t split_digits;     /* digits per operand of TTM_PREC_BF16_SPLIT: 0 = 8, 2..8   */
  int32_t reserved1;        /* must be 0                                                 */
  int64_t env_budget_bytes; /* ttm_backward: device memory for the stored left
                               environments; above it only every ceil(sqrt(L))-th one is
                               kept and the others are recomputed; 0 = 4 GiB            */
} ttm_options;

/* Filled by ttm_multiply. All fields are host values once the call returns. */
typedef struct {
  int32_t status;              /* TTM_OK or TTM_WARN_NOT_CONVERGED                        */
  int32_t jacobi_sweeps_max;   /* largest sweep count of any float32 Jacobi pass          */
  int64_t max_bond;            /* largest bond created by any Swap / QR / Contract       */
  int64_t n_swaps, n_contracts, n_qr;
  double discarded_weight;     /* sum_j w_j, w_j = sum of dropped lambda^2 of truncation j */
  double err_bound;            /* sum_j sqrt(w_j): bound on ||Omega - A o B||_2           */
  double norm_out;             /* ||Omega||_2                                             */
  double flops_counted;        /* model flops of the GEMM-shaped and QR work (Jacobi
                                  iterations excluded), from the realised bonds           */
  double seconds;              /* device time of the call (CUDA events)                  */
  int64_t peak_workspace_bytes;
  int64_t *bond_trace;         /* caller array or NULL: max chain bond after each Contract */
  int64_t bond_trace_len;      /* in: capacity of bond_trace; out: entries written (N)    */
  int64_t n_kernel_launches;   /* kernels this call launched (all products of a batch)   */
  int64_t jacobi_launches;     /* float32 one-sided Jacobi launches                       */
  double gemm_ms;              /* device time of every GEMM-shaped launch, for a
                                  tensor-core GEMM its exponent and digit kernels included
                                  (profile_kernels = 1), else 0                            */
  double newton_residual;      /* largest max(|S_ij|, |E_ij| / 2) of the last Newton step
                                  of any SVD (see ttm_newton.cuh); float64 rounding level
                                  when every SVD converged                                 */
  double jacobi32_ms;          /* device time of the float32 Jacobi passes
                                  (profile_kernels = 1), else 0                           */
  double jacobi32_flops;       /* float32 flops those passes executed (launch-wide)       */
  int64_t n_nonconverged;      /* SVDs that did not converge (see TTM_WARN_NOT_CONVERGED) */
  int64_t n_frozen_pairs;      /* column pairs the last Newton steps left unrotated as
                                  degenerate relative to their coupling                    */
  double gemm_flops;           /* algorithmic flops of the GEMM problems executed (2 M N K;
                                  M (M + 1) K for a symmetric Gram), counted on the device,
                                  launch-wide; problems a predicate left empty count 0      */
  int64_t gemm_launches;       /* GEMMs of the call (launch-wide)                          */
  double qr_ms;                /* device time of the Householder QR launches
                                  (profile_kernels = 1), else 0                            */
  int64_t n_fallback;          /* Swap SVDs whose Newton steps did not reach float64
                                  rounding and were finished by the float64 Jacobi        */
  int64_t jacobi32_sweeps;     /* float32 Jacobi sweeps run, summed over the SVDs (scalar
                                  and resident-block kernels; 0 with the others)          */
  int32_t *svd_trace;          /* caller array or NULL: 8 int32 per SVD in issue order (the
                                  Swaps, then the final rounding): m, n, the kept rank k,
                                  float32 sweeps of passes 0, 1, 2, 1 if the SVD took the
                                  float64 fallback, 0                                     */
  int64_t svd_trace_len;       /* in: capacity of svd_trace in SVDs; out: SVDs written     */
  double jacobi64_ms;          /* device time of the float64 Jacobi of the fallback
                                  (profile_kernels = 1), else 0                            */
} ttm_report;

/* Creates a handle bound to CUDA device `device` and stream `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream). `opt` may be NULL
 * (defaults: FP64, eps = 0, no caps). */
ttm_status ttm_create(ttm_handle **h, int device, void *cuda_stream, const ttm_options *opt);
ttm_status ttm_destroy(ttm_handle *h);
/* Replaces the handle's options. */
ttm_status ttm_set_options(ttm_handle *h, const ttm_options *opt);

/*
 * Omega = A o B (Sec. II.B). A and B must share L and d.
 * out: out->L, out->d are set by the library; out->bonds must point to L+1 host
 * int64 entries (receives the realised output bonds) and out->cores to L host
 * pointer slots. Three output modes:
 *   on_host = 0, cores[0] == NULL : the library writes device pointers into
 *       handle-owned memory, valid until the next multiply on the handle or
 *       ttm_destroy;
 *   on_host = 0, cores[k] != NULL : caller device buffers, each of at least
 *       ttm_output_capacity(...) doubles; the cores are copied there;
 *   on_host = 1                   : caller host buffers of the same capacity.
 * The stored core k is compact: [bonds[k]][d][bonds[k+1]].
 * rep may be NULL. Blocks until the result is host-visible.
 */
ttm_status ttm_multiply(ttm_handle *h, const ttm_tt *A, const ttm_tt *B, ttm_tt *out,
                        ttm_report *rep);

/*
 * n independent products A[i] o B[i] in one batched launch sequence: every kernel of
 * the sweep covers all n products (grid z = product), so products of uneven chi
 * share each launch. All pairs must share L and d. Outputs and reports as in
 * ttm_multiply (n entries each); rep[i].status holds each product's status and the
 * call returns the worst one.
 */
ttm_status ttm_multiply_batched(ttm_handle *h, int32_t n, const ttm_tt *A, const ttm_tt *B,
                                ttm_tt *out, ttm_report *rep);

/* Doubles needed per host output core for the given inputs and options. */
int64_t ttm_output_capacity(const ttm_tt *A, const ttm_tt *B, const ttm_options *opt);

/*
 * Value and gradients of a scalar functional of the product:
 *   TTM_LOSS_INNER : f = <W, A o B>,       W_or_C = W
 *   TTM_LOSS_SQDIST: g = ||A o B - C||^2,  W_or_C = C
 * Environments are contracted over the shared physical index (three layers for
 * <W, A o B>, four for <A o B, A o B>). gradA / gradB have the shapes of A / B
 * (caller device buffers, overwritten); either may be NULL to skip it.
 * *loss_out receives the value (host double).
 */
ttm_status ttm_backward(ttm_handle *h, ttm_loss kind, const ttm_tt *A, const ttm_tt *B,
                        const ttm_tt *W_or_C, double *loss_out, ttm_tt *gradA, ttm_tt *gradB);

/* <X, Y> (two-layer environment) and <W, A o B> (three-layer environment) of device
 * TTs, in float64; the "." product of the paper's error measure Gamma (Sec. III). */
ttm_status ttm_inner(ttm_handle *h, const ttm_tt *X, const ttm_tt *Y, double *out);
ttm_status ttm_inner3(ttm_handle *h, const ttm_tt *W, const ttm_tt *A, const ttm_tt *B,
                      double *out);

/*
 * Allocation-free product (no counterpart in the paper; an addition for callers that
 * cannot allocate device memory). Some callers must not call cudaMalloc once they are
 * running: a host application or plugin that reserves its device memory up front and
 * forbids the heap from growing afterwards, code that runs when device memory is already
 * exhausted, or a caller for which the implicit device-wide synchronisation of
 * cudaMalloc/cudaFree is not acceptable. This entry point computes the same product as
 * ttm_multiply for small trains without any device allocation: all workspace lives in a
 * fixed device array of TTM_NOALLOC_SCRATCH_BYTES bytes that the library defines at file
 * scope (every GPU that loads the library holds it until the process exits).
 *   - A, B: device cores (on_host = 0). out: out->cores[k] must be caller device buffers
 *     of at least ttm_output_capacity(...) doubles each; out->bonds receives the bonds.
 *   - opt may be NULL (defaults as in ttm_create); profile_kernels is ignored.
 *   - cuda_stream: the stream to run on (NULL = legacy default stream). The call blocks
 *     until the result is in `out`.
 *   - A product whose workspace exceeds TTM_NOALLOC_SCRATCH_BYTES is rejected with
 *     TTM_ERR_WORKSPACE before any work is queued.
 *   - The first call on a device (made current by the caller) looks up the device address
 *     of the array; make that first call before any stream capture.
 *   - Every call on a device uses the same array and leaves its contents behind (each call
 *     re-initialises what it reads). Calls whose GPU work overlaps in time on one device
 *     (different streams or host threads) race on the array: serialise them.
 * No cudaMalloc, cudaFree or other allocating routine is called on this path.
 */
#define TTM_NOALLOC_SCRATCH_BYTES (16u << 20)
ttm_status ttm_multiply_noalloc(const ttm_tt *A, const ttm_tt *B, ttm_tt *out, const ttm_options *opt,
                                void *cuda_stream);

/*
 * C = A B for float64 device matrices in column-major order (A: M x K with leading dimension
 * lda >= M, B: K x N with ldb >= K, C: M x N with ldc >= M; 1 <= M, N, K <= 2^20), on the
 * handle's stream, with the GEMM kernels of the product: prec = TTM_PREC_FP64 runs the float64
 * kernel, TTM_PREC_BF16_SPLIT the tensor-core digit product (split_digits of the handle's
 * options). Blocks until C is written. The workspace of the digits is handle-owned.
 */
ttm_status ttm_gemm(ttm_handle *h, ttm_precision prec, int64_t M, int64_t N, int64_t K, const double *A,
                    int64_t lda, const double *B, int64_t ldb, double *C, int64_t ldc);

/* Waits for all work queued on the handle's stream. */
ttm_status ttm_synchronize(ttm_handle *h);
/* Releases the handle-owned output of the last multiply (optional; ttm_destroy frees all). */
ttm_status ttm_tt_free(ttm_handle *h, ttm_tt *t);
/* Message for the last failing call on this thread ("" if none). */
const char *ttm_last_error(void);
/* Library version string. */
const char *ttm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TTM_H */
