// ttm_engine.cuh -- host side of the sweep: plans the static schedule of Sec. II.B
// (Eq. tensor, Contract, Swap, QR gauge moves) once with upper bounds on every bond,
// then walks it again launching the kernels. Both walks run the same code
// (Engine::run), so ids and buffers agree by construction.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <stdexcept>
#include <string>
#include <vector>

#include "ttm.h"
#include "ttm_common.cuh"
#include "ttm_host.hpp"
#include "ttm_copy.cuh"
#include "ttm_gemm.cuh"
#include "ttm_qr.cuh"
#include "ttm_svd.cuh"
#include "ttm_bjac.cuh"
#include "ttm_newton.cuh"
#include "ttm_jac4.cuh"
#include "ttm_jres.cuh"
#include "ttm_tc.cuh"

namespace ttm {

enum StepKind { SK_QR = 0, SK_SWAP = 1, SK_CONTRACT = 2, SK_ROUND = 3 };  // SK_ROUND: final-rounding SVD
struct StepLog {
  int kind;
  int b0, b1, b2, b3;  // bond ids (meaning per kind)
};

class Engine {
 public:
  Engine(HandleState& hs, int Z, const ttm_tt* A, const ttm_tt* B)
      : hs_(hs), Z_(Z), A_(A), B_(B), L_(A[0].L), d_(A[0].d), opt_(hs.opt),
        tc_(hs.opt.prec == TTM_PREC_BF16_SPLIT) {}

  // ------------------------------------------------------------------ planning
  void plan() {
    launch_ = false;
    reset_ids();
    run();
    // sizes
    nchain_ = (int)nbuf_total_;
    nb_ = nchain_ + WS_COUNT;
  }

  size_t bytes_needed() const { return per_product_bytes() * Z_ + table_bytes() + (size_t)tc_bytes_ + 256; }
  // use_graph may capture and replay this plan: only for an arena that persists across calls
  void allow_graph() { graph_ok_ = true; }

  // ------------------------------------------------------------------ execution
  void execute(void* arena, const ttm_options& opt, std::vector<ttm_report>* reps, ttm_tt* outs);

  int L() const { return L_; }
  int d() const { return d_; }
  long max_carriage() const { return carriage_elems_; }

 private:
  enum {
    WS_T = 0, WS_V, WS_NRM, WS_SORT, WS_PERM, WS_TAU, WS_R, WS_Q, WS_W32, WS_V32, WS_X, WS_V2, WS_V3,
    WS_G, WS_W0, WS_V0, WS_W0B, WS_COUNT
  };

  HandleState& hs_;
  int Z_;
  const ttm_tt* A_;
  const ttm_tt* B_;
  int L_, d_;
  ttm_options opt_{};
  bool launch_ = false;
  bool tc_ = false;          // GEMM-shaped work on the tensor cores (TTM_PREC_BF16_SPLIT)
  long tc_bytes_ = 0;        // digit workspace of the largest tensor-core GEMM (planned)
  unsigned char* d_tc_ = nullptr;
  // ids
  std::vector<std::vector<int>> ub_;  // ub_[id][z]
  std::vector<std::vector<int>> exact_;  // exact host values for input bonds, else empty
  std::vector<int> free_bufs_;
  long nbuf_total_ = 0;
  int nchain_ = 0, nb_ = 0;
  int n_trunc_ = 0;
  std::vector<StepLog> log_;
  std::vector<std::vector<int>> trace_ids_;  // chain bond ids after each Contract
  std::vector<int> out_buf_, out_bond_;      // output carriages and their bonds
  // sizes (elements, per product)
  long carriage_elems_ = 1, t_elems_ = 1, v_elems_ = 1, vec_elems_ = 1, r_elems_ = 1, q_elems_ = 1;
  long x_elems_ = 1;  // float64 elements of the X workspace (max(m, n) * n)
  // device tables (launch pass)
  Tables tab_{};
  int* counters_ = nullptr;
  double* fro2_ = nullptr;
  int counter_stride_ = 0;  // ints per Jacobi launch
  int* svd_log_ = nullptr;  // [z][SVD][kSvdRec] per-SVD diagnostics (the report's svd_trace)
  int cur_svd_ = 0;         // index of the SVD being issued
  int* svd_rec(int i) const { return svd_log_ ? svd_log_ + (size_t)i * kSvdRec : nullptr; }
  int svd_stride() const { return std::max(1, n_trunc_planned_) * kSvdRec; }
  int n_trunc_planned_ = 0;
  int jac_launch_ = 0;
  int* d_bond_ = nullptr;
  double** d_buf_ = nullptr;
  double* d_stat_ = nullptr;
  int* d_istat_ = nullptr;
  std::vector<double*> hbuf_;  // host copy of the buffer table

  void reset_ids() {
    gemm_log_.clear();
    ub_.clear();
    exact_.clear();
    free_bufs_.clear();
    nbuf_total_ = 0;
    n_trunc_ = 0;
    log_.clear();
    trace_ids_.clear();
    jac_launch_ = 0;
  }

  int umax(int id) const {
    int m = 1;
    for (int v : ub_[id]) m = std::max(m, v);
    return m;
  }
  int new_bond(const std::vector<int>& ub, const std::vector<int>* exact = nullptr) {
    for (int v : ub)
      if (v > kMaxBond)
        throw Error(TTM_ERR_RANK_CAP, "a bond upper bound reaches " + std::to_string(v) +
                                          " (> " + std::to_string(kMaxBond) + "); set chi_max");
    ub_.push_back(ub);
    exact_.push_back(exact ? *exact : std::vector<int>());
    return (int)ub_.size() - 1;
  }
  int get_buf() {
    if (!free_bufs_.empty()) {
      int b = free_bufs_.back();
      free_bufs_.pop_back();
      return b;
    }
    return (int)nbuf_total_++;
  }
  void put_buf(int b) { free_bufs_.push_back(b); }
  void note_carriage(int il, int ir) {
    for (int z = 0; z < Z_; ++z)
      carriage_elems_ = std::max(carriage_elems_, (long)ub_[il][z] * d_ * ub_[ir][z]);
  }
  int ws(int w) const { return nchain_ + w; }

  size_t per_product_bytes() const {
    long e = (long)nchain_ * carriage_elems_ + 3 * t_elems_ + 5 * v_elems_ + 4 * vec_elems_ + vec_elems_ +
             r_elems_ + q_elems_ + (t_elems_ / 2 + 1) + (v_elems_ / 2 + 1) + x_elems_;
    // every buffer aligned to 256 bytes
    return (size_t)e * 8 + (size_t)(nb_ + 1) * 256;
  }
  size_t table_bytes() const {
    size_t b = 0;
    b += (size_t)Z_ * nb_ * sizeof(double*) + 256;
    b += (size_t)Z_ * ub_.size() * sizeof(int) + 256;
    b += (size_t)Z_ * (ST_NFIXED + n_trunc_) * sizeof(double) + 256;
    b += (size_t)Z_ * IS_NFIXED * sizeof(int) + 256;
    b += (size_t)std::max(1, jac_launch_) * Z_ * counter_sweeps() * sizeof(int) + 256;
    b += (size_t)std::max(1, jac_launch_) * Z_ * sizeof(double) + 256;
    b += (size_t)Z_ * std::max(1, n_trunc_) * kSvdRec * sizeof(int) + 256;
    return b;
  }
  // Sweep counters per product and Jacobi launch: room for the sweep limit of any pass.
  // sweep limit of the float64 Jacobi of the fallback (max_sweeps when set)
  int polish_sweeps() const { return opt_.max_sweeps > 0 ? opt_.max_sweeps : kPolishSweeps; }
  int counter_sweeps() const {
    return std::max(std::max(opt_.max_sweeps, kPolishSweeps), std::max(kF32Sweeps, kF32FirstPassSweeps));
  }
  int f32_passes() const {
    return opt_.f32_passes > 0 ? std::min(opt_.f32_passes, kMaxF32Passes) : kDefaultF32Passes;
  }
  int split_digits() const { return opt_.split_digits > 0 ? opt_.split_digits : kOzMaxS; }
  int newton_steps() const {
    return opt_.newton_steps > 0 ? std::min(opt_.newton_steps, kMaxNewtonSteps) : kDefaultNewtonSteps;
  }

  // grid helpers
  static unsigned cdiv(long a, long b) { return (unsigned)((a + b - 1) / b); }
  // C = A B of every (product, batch index) the functor describes: on the float64 pipe, or
  // (tc_) as the exactly sliced bf16 product on the tensor cores (ttm_tc.cuh). kscale_buf:
  // per-K power-of-two exponents that keep a graded A relatively accurate (tensor cores only).
  // Digit workspace of a tensor-core GEMM with these upper bounds; every GEMM a step may
  // launch is reserved in both walks (the planning walk launches nothing).
  void tc_reserve(int nbatch, int M_ub, int N_ub, int K_ub) {
    if (tc_) tc_bytes_ = std::max(tc_bytes_, (long)tc_ws_bytes((long)Z_ * nbatch, M_ub, N_ub, K_ub, split_digits()));
  }
  // shape: the realised M x N x K of every batch index (for the flop count of the report).
  template <class F>
  void gemm(const F& f, int nbatch, int M_ub, int N_ub, int K_ub, GemmShape shape, int kscale_buf = -1) {
    if (!launch_) {
      tc_reserve(nbatch, M_ub, N_ub, K_ub);
      return;
    }
    if (tc_ && (size_t)tc_bytes_ < tc_ws_bytes((long)Z_ * nbatch, M_ub, N_ub, K_ub, split_digits()))
      throw Error(TTM_ERR_WORKSPACE, "internal: a tensor-core GEMM was not reserved in the plan");
    gemm_log_.push_back(shape);
    timed(0, [&] {
      if (tc_) {
        const cudaError_t e = launch_tc_gemm(hs_.stream, f, Z_, nbatch, M_ub, N_ub, K_ub, kscale_buf,
                                             split_digits(), d_tc_, d_istat_ + IS_STATUS, d_stat_ + ST_GFLOPS,
                                             tab_.ns);
        if (e != cudaSuccess)
          throw Error(TTM_ERR_CUDA, std::string("tensor-core GEMM, ") + tc_failed_step() + ": " + cudaGetErrorString(e));
        launches_ += 6;
      } else {
        dim3 grid(cdiv(N_ub, GT), cdiv(M_ub, GT), (unsigned)(Z_ * nbatch));
        dgemm_kernel<F><<<grid, 256, 0, hs_.stream>>>(f, nbatch, d_stat_ + ST_GFLOPS, tab_.ns);
        TTM_CUDA(cudaGetLastError());
        ++launches_;
      }
    });
  }
  // Predicated copy of a float64 rows x cols buffer (islot < 0: every product).
  void pcopy(int src, int dst, Dim rows, Dim cols, int islot, int want, long n_ub) {
    if (!launch_) return;
    PredCopyArgs pa{tab_, src, dst, rows, cols, islot, want};
    pred_copy_kernel<<<dim3((unsigned)std::min<long>(1024, cdiv(n_ub, 256)), Z_), 256, 0, hs_.stream>>>(pa);
    TTM_CUDA(cudaGetLastError());
    ++launches_;
  }
  // X of a Newton step from G and M (ttm_newton.cuh).
  void newton_x(int g, int mm, int xb, Dim n, int n_ub, int nprov, int eonly, bool last,
                int islot_pred) {
    if (!launch_) return;
    NewtonArgs na{tab_, g, mm, xb, n, ws(WS_SORT), nprov, ST_TRACE, eonly,
                  last ? ST_NEWTON_CUR : -1, last ? IS_NFROZEN : -1, islot_pred};
    dim3 blk(32, 8), grd(cdiv(n_ub, 32), cdiv(n_ub, 8), Z_);
    newton_x_kernel<<<grd, blk, 0, hs_.stream>>>(na);
    TTM_CUDA(cudaGetLastError());
    ++launches_;
  }
  template <class K>
  void launch_small(K kernel, unsigned grid, unsigned block) {
    if (!launch_) return;
    kernel<<<grid, block, 0, hs_.stream>>>(tab_);
    TTM_CUDA(cudaGetLastError());
    ++launches_;
  }
  // Per-column power-of-two exponents of W (the K scale of W X) into the tau workspace.
  void colexp(int wbuf, Dim m, Dim n, int n_ub) {
    if (!launch_) return;
    ColExpArgs ca{tab_, wbuf, ws(WS_TAU), m, n};
    colexp_kernel<<<dim3(cdiv(n_ub, 8), Z_), 256, 0, hs_.stream>>>(ca);
    TTM_CUDA(cudaGetLastError());
    ++launches_;
  }
  template <class F>
  void copy2d(const F& f, int nbatch, int R_ub, int C_ub) {
    if (!launch_) return;
    dim3 grid(cdiv(C_ub, 32), cdiv(R_ub, 32), (unsigned)(Z_ * nbatch));
    copy2d_kernel<F><<<grid, 256, 0, hs_.stream>>>(f, nbatch);
    TTM_CUDA(cudaGetLastError());
    ++launches_;
  }
  void cast(int src, int dst, Dim rows, Dim cols, int to_float, long n_ub) {
    if (!launch_) return;
    CastArgs ca{tab_, src, dst, rows, cols, to_float};
    dim3 g((unsigned)std::min<long>(1024, cdiv(n_ub, 256)), Z_);
    if (to_float == 1) {  // float copies are scaled to max |W| near 1
      reset_cast_exp_kernel<<<cdiv(Z_, 256), 256, 0, hs_.stream>>>(tab_);
      absmax_exp_kernel<<<g, 256, 0, hs_.stream>>>(ca);
      launches_ += 2;
    }
    cast_kernel<<<g, 256, 0, hs_.stream>>>(ca);
    TTM_CUDA(cudaGetLastError());
    ++launches_;
  }
  // Cooperative launch of 256-thread CTAs with one warp per work item (`units` items per round).
  // The kernels hand work item i to warp i / gridDim.x of CTA i % gridDim.x, so a round with
  // fewer items than warps still spreads over every SM; blocks_per_sm = 1 keeps the number of
  // CTAs that meet at each grid-wide barrier at one per SM.
  void coop(void* fn, void* args, int blocks_per_sm, long units) {
    long blocks = std::max(1L, std::min((long)blocks_per_sm * hs_.num_sms, units));
    void* kargs[] = {args};
    TTM_CUDA(cudaLaunchCooperativeKernel(fn, dim3((unsigned)blocks), dim3(256), kargs, 0, hs_.stream));
    ++launches_;
  }
  // Cooperative launch of the two-column-slot Jacobi: at most one CTA of kJ4Warps warps per
  // SM (a grid barrier with few arrivals), work items spread over the SMs first.
  void coop_j4(void* fn, void* args, long units) {
    const size_t smem = (size_t)kJ4Warps * 4 * kJ4MaxN * sizeof(float);
    TTM_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int occ = 0;
    TTM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kJ4Warps * 32, smem));
    if (occ < 1) throw Error(TTM_ERR_UNSUPPORTED, "two-column Jacobi kernel cannot be made resident");
    const long blocks = std::max(1L, std::min((long)hs_.num_sms, units));
    void* kargs[] = {args};
    TTM_CUDA(cudaLaunchCooperativeKernel(fn, dim3((unsigned)blocks), dim3(kJ4Warps * 32), kargs, smem, hs_.stream));
    ++launches_;
  }
  // Cooperative launch of the resident-block Jacobi: one CTA of kJrB warps per block pair,
  // as many as fit (one per SM when the columns fill the shared memory).
  void coop_res(void* fn, void* args, size_t smem, long units) {
    TTM_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int occ = 0;
    TTM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kJrB * 32, smem));
    if (occ < 1) throw Error(TTM_ERR_UNSUPPORTED, "resident-block Jacobi kernel cannot be made resident");
    const long blocks = std::max(1L, std::min((long)occ * hs_.num_sms, units));
    void* kargs[] = {args};
    TTM_CUDA(cudaLaunchCooperativeKernel(fn, dim3((unsigned)blocks), dim3(kJrB * 32), kargs, smem, hs_.stream));
    ++launches_;
  }
  // The resident-block Jacobi for Swap matrices of at most kJrMaxRows rows, instantiated for
  // the rows per lane that cover m_ub.
  template <typename T>
  void jacobi_res(JResArgs& jr, int m_ub, int n_ub, int nblk_pad_ub) {
    const int rows = (m_ub + 31) / 32;
    const int R = rows <= 1 ? 1 : rows <= 2 ? 2 : rows <= 4 ? 4 : rows <= 8 ? 8 : rows <= 16 ? 16 : 32;
    void* fn = R == 1 ? (void*)jacobi_res_kernel<T, kJrB, 1> : R == 2 ? (void*)jacobi_res_kernel<T, kJrB, 2>
             : R == 4 ? (void*)jacobi_res_kernel<T, kJrB, 4> : R == 8 ? (void*)jacobi_res_kernel<T, kJrB, 8>
             : R == 16 ? (void*)jacobi_res_kernel<T, kJrB, 16> : (void*)jacobi_res_kernel<T, kJrB, 32>;
    (void)n_ub;
    const size_t smem = (size_t)2 * kJrB * 32 * R * sizeof(T);
    coop_res(fn, &jr, smem, (long)Z_ * (nblk_pad_ub / 2));
  }
  // co-resident 256-thread CTAs per SM of the block Jacobi kernels (queried on first use)
  int bjac_occ_[2] = {0, 0};
  int bjac_blocks_per_sm(int fb) {
    int& v = bjac_occ_[fb == 8 ? 0 : 1];
    if (v == 0) {
      if (fb == 8)
        TTM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, block_jacobi_kernel<8>, 256, 0));
      else
        TTM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, block_jacobi_kernel<16>, 256, 0));
      if (v < 1) throw Error(TTM_ERR_UNSUPPORTED, "block Jacobi kernel cannot be made resident");
    }
    return v;
  }
  long launches_ = 0;
  int prof_used_ = 0;
  std::vector<int> prof_kind_;  // per event pair: 0 GEMM, 1 float32 Jacobi pass, 2 Householder QR
  std::vector<GemmShape> gemm_log_;  // every GEMM of the launch walk (flop count of the report)
  cudaEvent_t prof_event() {
    if (prof_used_ >= (int)hs_.prof_events.size()) {
      cudaEvent_t e;
      TTM_CUDA(cudaEventCreate(&e));
      hs_.prof_events.push_back(e);
    }
    return hs_.prof_events[prof_used_++];
  }
  // Brackets a Jacobi launch with a pair of events when kernel profiling is on.
  template <class Launch>
  void timed(int kind, Launch&& launch) {
    if (!opt_.profile_kernels) {
      launch();
      return;
    }
    cudaEvent_t e0 = prof_event(), e1 = prof_event();
    prof_kind_.push_back(kind);
    TTM_CUDA(cudaEventRecord(e0, hs_.stream));
    launch();
    TTM_CUDA(cudaEventRecord(e1, hs_.stream));
  }

  // ------------------------------------------------------------------ steps
  void load_core(const ttm_tt* T, int k, int buf);
  void issue_load(const ttm_tt* T, int k, int buf, cudaStream_t st);
  // use_graph: capture the launch walk once per plan, replay it afterwards
  bool graph_ok_ = false;            // set by the caller whose arena persists across calls
  bool defer_loads_ = false;         // capture: input copies are recorded, not captured
  long gemm_launch_count_ = -1;      // replay: the GEMM count of the captured walk
  std::string plan_key(void* arena) const;
  void launch_walk_graph(void* arena, cudaStream_t st, int nchain_planned, int jac_planned);
  void qr_move(int c, int& nx, int bl, int& br, int brr);
  int swap(int x, int y, int bl, int bm, int br, int kind = SK_SWAP);
  void jacobi32(int pass, int slot, Dim m, Dim n, int m_ub, int n_ub, int npad_ub, long pairs, int sweeps);
  void order_and_truncate(int wbuf, Dim m, Dim n, int ibond, int record, int wslot, int n_ub, long cap,
                          int ikeep = -1, int tslot = -1);
  // Final rounding (a7): planned when an output bond can exceed chi_out (the Swap cap is
  // above it, or absent, or an input bond is); the device gate (round_gate_kernel) then
  // truncates only the products whose output has a bond above chi_out.
  bool rounding() const {
    if (opt_.chi_out <= 0) return false;
    if (opt_.chi_max == 0 || opt_.chi_out < opt_.chi_max) return true;
    for (int z = 0; z < Z_; ++z)
      for (int i = 0; i <= L_; ++i)
        if (A_[z].bonds[i] > opt_.chi_out || B_[z].bonds[i] > opt_.chi_out) return true;
    return false;
  }
  void contract(int kb, int mb, int out, int il, int ia, int ir);
  void run();
};

}  // namespace ttm
