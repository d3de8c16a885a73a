// ttm_api.cu -- the C ABI of include/ttm.h and the schedule of the TTM sweep.
//
// Schedule (Sec. II.B): after the preparation (both trains left-canonical, B reversed
// with its bond legs exchanged so the reversed part is right-orthonormal, Eq. tensor),
// site N is contracted across the size-1 junction; then for i = N-1 .. 1 the gauge
// centre is moved by QR from Pi_{i+1} through Pi_N into B's carriage of site i (the
// mover), the mover is swapped leftwards past Pi_N .. Pi_{i+1} (i-1 swaps in the
// paper's count), and finally contracted with A's carriage of site i (Eq. contract).
// That is N contractions and N(N-1)/2 swaps.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "ttm.h"
#include "ttm_engine.cuh"

struct ttm_handle {
  ttm::HandleState s;
  std::vector<double*> last_out;  // device pointers of the last result (into the arena)
};

namespace ttm {

static thread_local std::string g_last_error;

static ttm_status set_err(ttm_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

// ---------------------------------------------------------------- steps

void Engine::load_core(const ttm_tt* T, int k, int buf) {
  if (!launch_) return;
  if (defer_loads_) {  // a captured walk: the copies of every call are issued before the replay
    hs_.graph_loads.push_back(T == A_ ? 0 : 1);
    hs_.graph_loads.push_back(k);
    hs_.graph_loads.push_back(buf);
    return;
  }
  issue_load(T, k, buf, hs_.stream);
}

void Engine::issue_load(const ttm_tt* T, int k, int buf, cudaStream_t st) {
  for (int z = 0; z < Z_; ++z) {
    const ttm_tt& t = T[z];
    const size_t n = (size_t)t.bonds[k] * t.d * t.bonds[k + 1];
    TTM_CUDA(cudaMemcpyAsync(hbuf_[(size_t)z * nb_ + buf], t.cores[k], n * sizeof(double),
                             t.on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st));
  }
}

// Everything that decides the launch walk: the options, the batch shape, every input bond
// and the arena (the captured kernels hold pointers into it).
std::string Engine::plan_key(void* arena) const {
  std::string k((const char*)&opt_, sizeof(opt_));
  auto put = [&](long v) { k.append((const char*)&v, sizeof(v)); };
  put(Z_);
  put(L_);
  put(d_);
  put((long)(size_t)arena);
  put((long)bytes_needed());
  for (int z = 0; z < Z_; ++z)
    for (int i = 0; i <= L_; ++i) {
      put(A_[z].bonds[i]);
      put(B_[z].bonds[i]);
    }
  return k;
}

// use_graph: the first call of a plan runs the launch walk under stream capture (on a private
// stream of the handle; the input copies are recorded instead) and instantiates the graph;
// every call then issues its input copies on st and replays the graph there.
void Engine::launch_walk_graph(void* arena, cudaStream_t st, int nchain_planned, int jac_planned) {
  const std::string key = plan_key(arena);
  if (hs_.graph_exec == nullptr || hs_.graph_key != key) {
    if (hs_.graph_exec) {
      TTM_CUDA(cudaGraphExecDestroy(hs_.graph_exec));
      hs_.graph_exec = nullptr;
    }
    hs_.graph_key.clear();
    hs_.graph_loads.clear();
    if (!hs_.capture_stream) TTM_CUDA(cudaStreamCreateWithFlags(&hs_.capture_stream, cudaStreamNonBlocking));
    const cudaStream_t saved = hs_.stream;
    hs_.stream = hs_.capture_stream;
    defer_loads_ = true;
    cudaGraph_t g = nullptr;
    reset_ids();
    TTM_CUDA(cudaStreamBeginCapture(hs_.capture_stream, cudaStreamCaptureModeRelaxed));
    try {
      run();
      if ((int)nbuf_total_ != nchain_planned || jac_launch_ != jac_planned)
        throw Error(TTM_ERR_INVALID_ARG, "internal: plan and launch walks disagree");
    } catch (...) {
      cudaStreamEndCapture(hs_.capture_stream, &g);
      if (g) cudaGraphDestroy(g);
      hs_.stream = saved;
      defer_loads_ = false;
      throw;
    }
    const cudaError_t ec = cudaStreamEndCapture(hs_.capture_stream, &g);
    hs_.stream = saved;
    defer_loads_ = false;
    TTM_CUDA(ec);
    const cudaError_t ei = cudaGraphInstantiate(&hs_.graph_exec, g, 0);
    cudaGraphDestroy(g);
    TTM_CUDA(ei);
    hs_.graph_key = key;
    hs_.graph_launches = launches_;
    hs_.graph_gemms = (long)gemm_log_.size();
  }
  launches_ = hs_.graph_launches;
  gemm_launch_count_ = hs_.graph_gemms;
  for (size_t q = 0; q + 2 < hs_.graph_loads.size(); q += 3)
    issue_load(hs_.graph_loads[q] == 0 ? A_ : B_, hs_.graph_loads[q + 1], hs_.graph_loads[q + 2], st);
  TTM_CUDA(cudaGraphLaunch(hs_.graph_exec, st));
}

// Gauge move of one carriage (QR after Contract): C [bl][d][br] = Q R; C <- Q; Next <- R Next.
void Engine::qr_move(int c, int& nx, int bl, int& br, int brr) {
  std::vector<int> kub(Z_);
  for (int z = 0; z < Z_; ++z) kub[z] = std::min(d_ * ub_[bl][z], ub_[br][z]);
  const int nbnd = new_bond(kub);
  const int m_ub = d_ * umax(bl), n_ub = umax(br), k_ub = umax(nbnd);
  t_elems_ = std::max(t_elems_, (long)m_ub * n_ub);
  r_elems_ = std::max(r_elems_, (long)k_ub * n_ub);
  q_elems_ = std::max(q_elems_, (long)m_ub * k_ub);
  vec_elems_ = std::max(vec_elems_, (long)k_ub + 1);
  log_.push_back({SK_QR, bl, br, nbnd, brr});
  tc_reserve(1, k_ub, d_ * umax(brr), n_ub);            // R merge
  const int out = get_buf();
  note_carriage(bl, nbnd);
  note_carriage(nbnd, brr);
  if (launch_) {
    const Dim m{d_, bl}, n{1, br};
    copy2d(RowToColFn{tab_, c, ws(WS_T), m, n}, 1, m_ub, n_ub);
    QRArgs qa{tab_, ws(WS_T), ws(WS_TAU), ws(WS_R), ws(WS_Q), m, n, nbnd, n_ub, k_ub};
    timed(2, [&] { coop((void*)householder_kernel, &qa, 1, (long)Z_ * n_ub); });
    copy2d(ColToRowFn{tab_, ws(WS_Q), c, m, Dim{1, nbnd}}, 1, m_ub, k_ub);
    gemm(RMergeFn{tab_, ws(WS_R), nx, out, nbnd, br, brr, d_}, 1, k_ub, d_ * umax(brr), n_ub,
         GemmShape{Dim{1, nbnd}, Dim{d_, brr}, Dim{1, br}, 1, 0});
  }
  put_buf(nx);
  nx = out;
  br = nbnd;
}

// Swap of X [bl][d][bm] and Y [bm][d][br] (Fig. 1C); Y's buffer receives the new left
// carriage (the mover, U Lambda), X's buffer the new right one (V^T). Returns the new bond.
// kind = SK_ROUND is the same truncated two-site SVD with the physical legs left in place
// and the output cap chi_out (the final rounding): Y's buffer then receives the new
// carriage of X's site (U Lambda, leg s) and X's buffer that of Y's site (V^T, leg t).
int Engine::swap(int x, int y, int bl, int bm, int br, int kind) {
  const long cap = kind == SK_ROUND ? opt_.chi_out : opt_.chi_max;
  std::vector<int> kub(Z_);
  for (int z = 0; z < Z_; ++z) {
    int v = std::min(d_ * ub_[bl][z], d_ * ub_[br][z]);
    if (cap > 0) v = std::min<long>(v, cap);
    kub[z] = v;
  }
  const int nbnd = new_bond(kub);
  const int m_ub = d_ * umax(bl), n_ub = d_ * umax(br), k_ub = umax(nbnd);
  t_elems_ = std::max(t_elems_, (long)m_ub * n_ub);
  v_elems_ = std::max(v_elems_, (long)n_ub * n_ub);
  x_elems_ = std::max(x_elems_, (long)std::max(m_ub, n_ub) * n_ub);
  r_elems_ = std::max(r_elems_, (long)n_ub * n_ub);
  vec_elems_ = std::max(vec_elems_, (long)n_ub + 1);
  log_.push_back({kind, bl, bm, br, nbnd});
  note_carriage(bl, nbnd);
  note_carriage(nbnd, br);
  cur_svd_ = n_trunc_;
  const int wslot = ST_NFIXED + n_trunc_++;
  // digit workspace of the tensor-core GEMMs below (sized in the planning walk too)
  tc_reserve(d_ * d_, umax(bl), umax(br), umax(bm));   // Theta
  tc_reserve(1, m_ub, n_ub, n_ub);                      // W X, W V32
  tc_reserve(1, n_ub, n_ub, std::max(m_ub, n_ub));      // Grams of W and V, V X
  const int npass = f32_passes();
  const int sw32 = jac_launch_;
  jac_launch_ += npass;
  const int sw64 = jac_launch_++;          // the fallback's float64 Jacobi
  const int nprov = new_bond(kub);         // provisional rank before the Newton steps
  if (launch_) {
    const Dim m{d_, bl}, n{d_, br};
    const int npad_ub = n_ub + (n_ub & 1);
    const long pairs = (long)Z_ * (npad_ub / 2);
    // 1. Theta = X Y with the physical legs permuted, column-major m x n (Fig. 1C)
    gemm(ThetaFn{tab_, x, y, ws(WS_T), bl, bm, br, d_, kind == SK_ROUND ? 1 : 0}, d_ * d_, umax(bl),
         umax(br), umax(bm), GemmShape{Dim{1, bl}, Dim{1, br}, Dim{1, bm}, d_ * d_, 0});
    // 2. float32 one-sided Jacobi passes. Each runs on a float copy of the current W with V32
    //    starting at I; then W <- W V32 and V <- V V32 in float64, so W = Theta V keeps holding
    //    to float64 rounding (V is orthonormal only to float32 accuracy until step 3). The
    //    first pass works on Theta itself, whose float copy only resolves singular values
    //    above about u32 ||Theta||, so it stops at an absolute floor at that level and after
    //    a few sweeps: it only has to grade W. After it the columns of W are graded (norms
    //    near the singular values), a float copy keeps each column to relative accuracy, and
    //    the next pass (relative test, floor at float64 rounding) resolves the rest of the
    //    spectrum to float32 accuracy.
    int wb = ws(WS_T), wo = ws(WS_X);  // current W (starts as Theta), spare m x n buffer
    int vb = -1;                       // current V (-1: identity)
    std::vector<int> fr = {ws(WS_V), ws(WS_V2), ws(WS_V3), ws(WS_G), ws(WS_R)};  // free n x n buffers
    auto take = [&]() { int b = fr.back(); fr.pop_back(); return b; };
    for (int p = 0; p < npass; ++p) {
      cast(wb, ws(WS_W32), m, n, 1, (long)m_ub * n_ub);
      const int sweeps32 = (p == 0 && npass > 1) ? kF32FirstPassSweeps : (opt_.max_sweeps > 0 ? opt_.max_sweeps : kF32Sweeps);
      jacobi32(p, sw32 + p, m, n, m_ub, n_ub, npad_ub, pairs, sweeps32);
      const int v32 = take();
      cast(ws(WS_V32), v32, n, n, 0, (long)n_ub * n_ub);
      if (p > 0 && tc_) colexp(wb, m, n, n_ub);              // W is graded from pass 1 on
      gemm(ThetaVFn{tab_, wb, v32, wo, m, n}, 1, m_ub, n_ub, n_ub, GemmShape{m, n, n, 1, 0},
           p > 0 && tc_ ? ws(WS_TAU) : -1);  // W <- W V32
      std::swap(wb, wo);
      if (vb < 0) {
        vb = v32;                                              // V = I V32
      } else {
        const int vn = take();
        gemm(ThetaVFn{tab_, vb, v32, vn, n, n}, 1, n_ub, n_ub, n_ub, GemmShape{n, n, n, 1, 0});  // V <- V V32
        fr.push_back(vb);
        fr.push_back(v32);
        vb = vn;
      }
    }
    if (vb < 0) {  // no float32 pass: start from V = I
      vb = take();
      cast(-1, vb, n, n, 2, (long)n_ub * n_ub);
    }
    // 3. float64 Newton steps (ttm_newton.cuh): couplings of W and the orthogonality defect
    //    of V fall quadratically from float32 level to float64 rounding. The provisional
    //    cut (Eq. eps + cap on the current column norms) tells which pairs can matter.
    order_and_truncate(wb, m, n, nprov, 0, -1, n_ub, cap, kind == SK_ROUND ? bm : -1, ST_TRACE);
    pcopy(wb, ws(WS_W0), m, n, -1, 0, (long)m_ub * n_ub);  // the state the fallback restarts from
    pcopy(vb, ws(WS_V0), n, n, -1, 0, (long)n_ub * n_ub);
    const int nsteps = newton_steps();
    for (int s = 0; s < nsteps; ++s) {
      const int g = take(), mm = take(), xb = take();
      gemm(GramFn{tab_, wb, g, m, n}, 1, n_ub, n_ub, m_ub, GemmShape{n, n, m, 1, 1});
      gemm(GramFn{tab_, vb, mm, n, n}, 1, n_ub, n_ub, n_ub, GemmShape{n, n, n, 1, 1});
      newton_x(g, mm, xb, n, n_ub, nprov, 0, s + 1 == nsteps, -1);
      if (tc_) colexp(wb, m, n, n_ub);
      gemm(ThetaVFn{tab_, wb, xb, wo, m, n}, 1, m_ub, n_ub, n_ub, GemmShape{m, n, n, 1, 0},
           tc_ ? ws(WS_TAU) : -1);  // W <- W X
      std::swap(wb, wo);
      gemm(ThetaVFn{tab_, vb, xb, mm, n, n}, 1, n_ub, n_ub, n_ub, GemmShape{n, n, n, 1, 0});  // V <- V X
      fr.push_back(vb);
      fr.push_back(g);
      fr.push_back(xb);
      vb = mm;
    }
    // up to kNewtonExtraSteps more steps for the products whose last correction is still above
    // float64 level (the quadratic convergence from a correction near 0.1 needs five steps);
    // every launch is empty for the others, which keep their W and V
    for (int e = 0; e < kNewtonExtraSteps; ++e) {
      launch_small(newton_more_kernel, cdiv(Z_, 128), 128);
      const int g = take(), mm = take(), xb = take();
      gemm(PredFn<GramFn>{GramFn{tab_, wb, g, m, n}, IS_NEWTON_MORE, 1, tab_}, 1, n_ub, n_ub, m_ub,
           GemmShape{n, n, m, 1, 1});
      gemm(PredFn<GramFn>{GramFn{tab_, vb, mm, n, n}, IS_NEWTON_MORE, 1, tab_}, 1, n_ub, n_ub, n_ub,
           GemmShape{n, n, n, 1, 1});
      newton_x(g, mm, xb, n, n_ub, nprov, 0, true, IS_NEWTON_MORE);
      if (tc_) colexp(wb, m, n, n_ub);
      gemm(PredFn<ThetaVFn>{ThetaVFn{tab_, wb, xb, wo, m, n}, IS_NEWTON_MORE, 1, tab_}, 1, m_ub, n_ub, n_ub,
           GemmShape{m, n, n, 1, 0}, tc_ ? ws(WS_TAU) : -1);  // W <- W X
      pcopy(wb, wo, m, n, IS_NEWTON_MORE, 0, (long)m_ub * n_ub);
      std::swap(wb, wo);
      gemm(PredFn<ThetaVFn>{ThetaVFn{tab_, vb, xb, mm, n, n}, IS_NEWTON_MORE, 1, tab_}, 1, n_ub, n_ub, n_ub,
           GemmShape{n, n, n, 1, 0});  // V <- V X
      pcopy(vb, mm, n, n, IS_NEWTON_MORE, 0, (long)n_ub * n_ub);
      fr.push_back(vb);
      fr.push_back(g);
      fr.push_back(xb);
      vb = mm;
    }
    launch_small(newton_check_kernel, cdiv(Z_, 128), 128);
    // 3b. fallback for the products whose Newton residual stayed above float64 level (every
    //     launch below is empty for the others): restart from the state after the float32
    //     passes, make V orthonormal by two polar steps, and run the float64 one-sided Jacobi
    //     to convergence; then the result replaces the Newton one.
    {
      int fw = ws(WS_W0), fv = ws(WS_V0), fw2 = ws(WS_W0B);
      for (int s = 0; s < 2; ++s) {
        const int mm = take(), xb = take(), vn = take();
        gemm(PredFn<GramFn>{GramFn{tab_, fv, mm, n, n}, IS_FALLBACK, 1, tab_}, 1, n_ub, n_ub, n_ub,
             GemmShape{n, n, n, 1, 1});
        newton_x(mm, mm, xb, n, n_ub, nprov, 1, false, IS_FALLBACK);
        if (tc_) colexp(fw, m, n, n_ub);
        gemm(PredFn<ThetaVFn>{ThetaVFn{tab_, fw, xb, fw2, m, n}, IS_FALLBACK, 1, tab_}, 1, m_ub, n_ub, n_ub,
             GemmShape{m, n, n, 1, 0}, tc_ ? ws(WS_TAU) : -1);
        gemm(PredFn<ThetaVFn>{ThetaVFn{tab_, fv, xb, vn, n, n}, IS_FALLBACK, 1, tab_}, 1, n_ub, n_ub, n_ub,
             GemmShape{n, n, n, 1, 0});
        std::swap(fw, fw2);
        fr.push_back(mm);
        fr.push_back(xb);
        if (fv != ws(WS_V0)) fr.push_back(fv);
        fv = vn;
      }
      HestArgs h64{tab_, fw, fv, m, n, npad_ub, polish_sweeps(), counters_ + (size_t)sw64 * counter_stride_, 1e-10,
                   64 * 1.11e-16, fro2_ + (size_t)sw64 * Z_, 0, ST_JFLOPS, ws(WS_NRM), 1, IS_FALLBACK, -1, nullptr,
                   0, 0};
      if (m_ub <= kJrMaxRows) {  // the resident-block kernel on all pairs of the fallback products
        const int nblk_ub = (n_ub + kJrB - 1) / kJrB;
        const int nblk_pad_ub = nblk_ub + (nblk_ub & 1);
        JResArgs j64{tab_, fw, fv, m, n, nblk_pad_ub, polish_sweeps(), h64.counters, h64.tol, h64.delta, h64.fro2,
                     ST_JFLOPS, ws(WS_NRM), 1, -1, nullptr, 0, 0, 0, IS_FALLBACK};
        timed(3, [&] { jacobi_res<double>(j64, m_ub, n_ub, nblk_pad_ub); });
      } else {
        timed(3, [&] { coop((void*)hestenes_kernel<double>, &h64, 1, pairs); });
      }
      pcopy(fw, wb, m, n, IS_FALLBACK, 1, (long)m_ub * n_ub);
      pcopy(fv, vb, n, n, IS_FALLBACK, 1, (long)n_ub * n_ub);
      if (fv != ws(WS_V0)) fr.push_back(fv);
    }
    // 4. final order by column norm, Eq. eps + cap, new carriages
    order_and_truncate(wb, m, n, nbnd, 1, wslot, n_ub, cap, kind == SK_ROUND ? bm : -1);
    {
      ++launches_;
      GatherArgs ga{tab_, wb, vb, ws(WS_PERM), y, x, bl, br, nbnd, d_};
      dim3 g3(cdiv(std::max(m_ub, n_ub), 128), k_ub, Z_);
      swap_gather_kernel<<<g3, 128, 0, hs_.stream>>>(ga);
      TTM_CUDA(cudaGetLastError());
    }
  }
  return nbnd;
}

// One float32 one-sided Jacobi pass on the W32 workspace (V32 starts at I): by default the
// resident-block kernel (ttm_jres.cuh; one grid barrier per round of block pairs) when the
// columns have at most 1024 rows, else the scalar kernel (one grid barrier per round of
// column pairs); jacobi_kernel selects one explicitly. Pass 0 stops at an absolute floor at float32 rounding of ||W||, later passes at
// float64 rounding.
void Engine::jacobi32(int pass, int slot, Dim m, Dim n, int m_ub, int n_ub, int npad_ub, long pairs,
                      int sweeps) {
  HestArgs h32{tab_, ws(WS_W32), ws(WS_V32), m, n, npad_ub, sweeps,
               counters_ + (size_t)slot * counter_stride_,
               16 * 5.96e-8 * std::sqrt((double)std::max(m_ub, 1)),
               pass == 0 ? 64 * 5.96e-8 : 64 * 1.11e-16,
               fro2_ + (size_t)slot * Z_, 1, ST_JFLOPS32, ws(WS_NRM), 0, -1, ST_JSWEEPS32,
               pass < 3 ? svd_rec(cur_svd_) : nullptr, svd_stride(), SR_SW0 + pass};
  const int jk = opt_.jacobi_kernel;
  const bool fits2 = m_ub <= 32 * 32 && n_ub <= kJ4MaxN;
  if (jk == 3 && m_ub > kJrMaxRows)
    throw Error(TTM_ERR_UNSUPPORTED, "jacobi_kernel = 3 needs Swap matrices of at most 1024 rows");
  if (jk == 3 || (jk == 0 && m_ub <= kJrMaxRows)) {
    const int nblk_ub = (n_ub + kJrB - 1) / kJrB;
    const int nblk_pad_ub = nblk_ub + (nblk_ub & 1);
    JResArgs jr{tab_, ws(WS_W32), ws(WS_V32), m, n, nblk_pad_ub, sweeps, h32.counters, h32.tol, h32.delta,
                h32.fro2, ST_JFLOPS32, ws(WS_NRM), h32.count_nonconv, ST_JSWEEPS32, h32.svd_log, h32.svd_stride,
                h32.svd_field, 1, -1};
    timed(1, [&] { jacobi_res<float>(jr, m_ub, n_ub, nblk_pad_ub); });
    return;
  }
  if (jk == 2 && !fits2)
    throw Error(TTM_ERR_UNSUPPORTED, "jacobi_kernel = 2 needs Swap matrices of at most 1024 x 1024");
  if (jk == 8 || jk == 16) {
    const int fb = jk;
    const int nblk_ub = (n_ub + fb - 1) / fb;
    const int nblk_pad_ub = nblk_ub + (nblk_ub & 1);
    BJacArgs bj{tab_, ws(WS_W32), ws(WS_V32), m, n, nblk_pad_ub, sweeps,
                h32.counters, h32.tol, h32.delta, h32.fro2, ST_JFLOPS32, h32.count_nonconv};
    void* fn = fb == 8 ? (void*)block_jacobi_kernel<8> : (void*)block_jacobi_kernel<16>;
    timed(1, [&] { coop(fn, &bj, bjac_blocks_per_sm(fb), (long)Z_ * (nblk_pad_ub / 2)); });
  } else if (jk == 2) {
    const int ns_ub = (n_ub + 1) / 2;
    const int nsp_ub = ns_ub + (ns_ub & 1);
    Jac4Args ja{tab_, ws(WS_W32), ws(WS_V32), m, n, nsp_ub, sweeps, h32.counters, h32.tol, h32.delta, h32.fro2,
                ST_JFLOPS32, h32.count_nonconv};
    const int rows = (m_ub + 31) / 32;
    void* fn = rows <= 1 ? (void*)jacobi4_kernel<1> : rows <= 2 ? (void*)jacobi4_kernel<2>
             : rows <= 4 ? (void*)jacobi4_kernel<4> : rows <= 8 ? (void*)jacobi4_kernel<8>
             : rows <= 16 ? (void*)jacobi4_kernel<16> : (void*)jacobi4_kernel<32>;
    const long units = (long)Z_ * (nsp_ub / 2);
    timed(1, [&] { coop_j4(fn, &ja, units); });
  } else {
    timed(1, [&] { coop((void*)hestenes_kernel<float>, &h32, 1, pairs); });
  }
}

// Column norms of W (workspace X), descending order, and the rank rule of Eq. eps.
void Engine::order_and_truncate(int wbuf, Dim m, Dim n, int ibond, int record, int wslot, int n_ub,
                                long cap, int ikeep, int tslot) {
  launches_ += 3;
  NormArgs na{tab_, wbuf, ws(WS_NRM), m, n};
  dim3 g(cdiv(n_ub, 8), Z_);
  colnorm_kernel<<<g, 256, 0, hs_.stream>>>(na);
  TTM_CUDA(cudaGetLastError());
  RankArgs ra{tab_, ws(WS_NRM), ws(WS_SORT), ws(WS_PERM), n};
  dim3 g2(cdiv(n_ub, 256), Z_);
  rank_kernel<<<g2, 256, 0, hs_.stream>>>(ra);
  TTM_CUDA(cudaGetLastError());
  TruncArgs ta{tab_, ws(WS_SORT), m, n, ibond, opt_.eps, (int)cap, wslot, record, ikeep, tslot,
               record ? svd_rec(cur_svd_) : nullptr, svd_stride()};
  truncate_kernel<<<Z_, 1024, 0, hs_.stream>>>(ta);
  TTM_CUDA(cudaGetLastError());
}

void Engine::contract(int kb, int mb, int out, int il, int ia, int ir) {
  log_.push_back({SK_CONTRACT, il, ia, ir, 0});
  note_carriage(il, ir);
  gemm(ContractFn{tab_, kb, mb, out, il, ia, ir, d_}, d_, umax(il), umax(ir), umax(ia),
       GemmShape{Dim{1, il}, Dim{1, ir}, Dim{1, ia}, d_, 0});
}

void Engine::run() {
  const int L = L_;
  std::vector<int> a(L), b(L), bA(L + 1), bB(L + 1);
  for (int i = 0; i <= L; ++i) {
    std::vector<int> va(Z_), vb(Z_);
    for (int z = 0; z < Z_; ++z) {
      va[z] = (int)A_[z].bonds[i];
      vb[z] = (int)B_[z].bonds[i];
    }
    bA[i] = new_bond(va, &va);
    bB[i] = new_bond(vb, &vb);
  }
  for (int k = 0; k < L; ++k) {
    a[k] = get_buf();
    b[k] = get_buf();
    note_carriage(bA[k], bA[k + 1]);
    note_carriage(bB[k], bB[k + 1]);
    load_core(A_, k, a[k]);
    load_core(B_, k, b[k]);
  }
  // a1: both trains left-canonical (QR sweeps); the norms end in the last carriages.
  for (int k = 0; k + 1 < L; ++k) qr_move(a[k], a[k + 1], bA[k], bA[k + 1], bA[k + 2]);
  for (int k = 0; k + 1 < L; ++k) qr_move(b[k], b[k + 1], bB[k], bB[k + 1], bB[k + 2]);
  // Eq. tensor: B reversed, each carriage with its bond legs exchanged.
  std::vector<int> mt(L), mtL(L), mtR(L);
  for (int j = 0; j < L; ++j) {
    const int src = b[L - 1 - j];
    const int dst = get_buf();
    const int il = bB[L - 1 - j], ir = bB[L - j];
    note_carriage(ir, il);
    copy2d(LegSwapFn{tab_, src, dst, il, ir, d_}, d_, umax(il), umax(ir));
    put_buf(src);
    mt[j] = dst;
    mtL[j] = ir;
    mtR[j] = il;
  }
  std::vector<int> pi(L + 1), piL(L + 1), piR(L + 1);
  auto record_trace = [&](int i) {
    std::vector<int> ids;
    for (int k = 0; k < i - 1; ++k) ids.push_back(bA[k + 1]);
    for (int j = i; j <= L; ++j) ids.push_back(piR[j]);
    for (int q = L - i + 1; q < L; ++q) ids.push_back(mtR[q]);
    trace_ids_.push_back(ids);
  };
  // a2: site N across the size-1 junction.
  pi[L] = get_buf();
  contract(a[L - 1], mt[0], pi[L], bA[L - 1], bA[L], mtR[0]);
  put_buf(a[L - 1]);
  put_buf(mt[0]);
  piL[L] = bA[L - 1];
  piR[L] = mtR[0];
  record_trace(L);
  for (int i = L - 1; i >= 1; --i) {
    int mv = mt[L - i], mvL = mtL[L - i], mvR = mtR[L - i];
    (void)mvL;
    // a3: centre from Pi_{i+1} through Pi_N into the mover.
    for (int j = i + 1; j <= L; ++j) {
      if (j < L) {
        qr_move(pi[j], pi[j + 1], piL[j], piR[j], piR[j + 1]);
        piL[j + 1] = piR[j];
      } else {
        qr_move(pi[L], mv, piL[L], piR[L], mvR);
        mvL = piR[L];
      }
    }
    // a4 + a5: the mover passes Pi_N .. Pi_{i+1}.
    for (int j = L; j >= i + 1; --j) {
      const int nb = swap(pi[j], mv, piL[j], piR[j], mvR);
      mvL = piL[j];
      const int oldR = mvR;
      mvR = nb;
      piL[j] = nb;
      piR[j] = oldR;
    }
    // a6: Contract with A's carriage of site i.
    const int out = get_buf();
    contract(a[i - 1], mv, out, bA[i - 1], bA[i], mvR);
    put_buf(a[i - 1]);
    put_buf(mv);
    pi[i] = out;
    piL[i] = bA[i - 1];
    piR[i] = mvR;
    record_trace(i);
  }
  // a7: final rounding to chi_out, bond 1 first, as a left-to-right TT-SVD sweep. The
  // sweep leaves Omega right-canonical with the centre on Pi_1. Its mirror (sites reversed,
  // bond legs exchanged, as in Eq. tensor) is left-canonical with the centre on its last
  // site, so truncated two-site SVDs from the mirror's right end (U Lambda to the left,
  // V^T to the right) truncate Omega's bonds 1, 2, ... with the rest of the train
  // orthonormal; then the mirror is undone. The centre ends on Pi_N.
  if (rounding()) {
    // the rounding truncates only products with an output bond above chi_out (reading A4);
    // the others go through the same sweep as exact refactorisations
    if (launch_) {
      std::vector<int> ids;
      for (int j = 1; j < L; ++j) ids.push_back(piR[j]);
      for (size_t c0 = 0; c0 < ids.size(); c0 += 32) {
        RoundGateArgs ra{};
        ra.t = tab_;
        ra.n = (int)std::min<size_t>(32, ids.size() - c0);
        for (int q = 0; q < ra.n; ++q) ra.ids[q] = ids[c0 + q];
        ra.cap = (int)opt_.chi_out;
        round_gate_kernel<<<Z_, 32, 0, hs_.stream>>>(ra);
        TTM_CUDA(cudaGetLastError());
        ++launches_;
      }
    }
    std::vector<int> mb(L + 1), mL(L + 1), mR(L + 1);
    for (int j = 1; j <= L; ++j) {
      const int src = pi[j], dst = get_buf();
      const int il = piL[j], ir = piR[j];
      note_carriage(ir, il);
      copy2d(LegSwapFn{tab_, src, dst, il, ir, d_}, d_, umax(il), umax(ir));
      put_buf(src);
      mb[L + 1 - j] = dst;
      mL[L + 1 - j] = ir;
      mR[L + 1 - j] = il;
    }
    for (int j = L - 1; j >= 1; --j) {
      const int nb = swap(mb[j], mb[j + 1], mL[j], mR[j], mR[j + 1], SK_ROUND);
      std::swap(mb[j], mb[j + 1]);  // the new carriage of mirrored site j sits in the buffer of j + 1
      mR[j] = nb;
      mL[j + 1] = nb;
    }
    for (int j = 1; j <= L; ++j) {
      const int src = mb[L + 1 - j], dst = get_buf();
      const int il = mL[L + 1 - j], ir = mR[L + 1 - j];
      note_carriage(ir, il);
      copy2d(LegSwapFn{tab_, src, dst, il, ir, d_}, d_, umax(il), umax(ir));
      put_buf(src);
      pi[j] = dst;
      piL[j] = ir;
      piR[j] = il;
    }
  }
  out_buf_.assign(pi.begin() + 1, pi.end());
  out_bond_.assign(L + 1, 0);
  out_bond_[0] = piL[1];
  for (int j = 1; j <= L; ++j) out_bond_[j] = piR[j];
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

void Engine::execute(void* arena, const ttm_options& opt, std::vector<ttm_report>* reps, ttm_tt* outs) {
  (void)opt;
  // Layout of the arena: per product [chain buffers | workspaces], then the tables.
  n_trunc_planned_ = n_trunc_;
  char* base = (char*)arena;
  size_t off = 0;
  hbuf_.assign((size_t)Z_ * nb_, nullptr);
  const long ws_elems[] = {t_elems_,   v_elems_, vec_elems_, vec_elems_, vec_elems_,
                           vec_elems_, r_elems_, q_elems_,   t_elems_ / 2 + 1, v_elems_ / 2 + 1,
                           x_elems_,   v_elems_, v_elems_, v_elems_, t_elems_, v_elems_, t_elems_};
  static_assert(sizeof(ws_elems) / sizeof(ws_elems[0]) == WS_COUNT, "one size per workspace");
  for (int z = 0; z < Z_; ++z) {
    for (int bi = 0; bi < nchain_; ++bi) {
      hbuf_[(size_t)z * nb_ + bi] = (double*)(base + off);
      off = align256(off + (size_t)carriage_elems_ * 8);
    }
    for (int w = 0; w < WS_COUNT; ++w) {
      hbuf_[(size_t)z * nb_ + nchain_ + w] = (double*)(base + off);
      off = align256(off + (size_t)ws_elems[w] * 8);
    }
  }
  const int nbd = (int)ub_.size();
  const int ns = ST_NFIXED + n_trunc_;
  const int nis = IS_NFIXED;
  d_buf_ = (double**)(base + off);
  off = align256(off + (size_t)Z_ * nb_ * sizeof(double*));
  d_bond_ = (int*)(base + off);
  off = align256(off + (size_t)Z_ * nbd * sizeof(int));
  d_stat_ = (double*)(base + off);
  off = align256(off + (size_t)Z_ * ns * sizeof(double));
  d_istat_ = (int*)(base + off);
  off = align256(off + (size_t)Z_ * nis * sizeof(int));
  counter_stride_ = Z_ * counter_sweeps();
  counters_ = (int*)(base + off);
  const int n_jac = std::max(1, jac_launch_);
  off = align256(off + (size_t)n_jac * counter_stride_ * sizeof(int));
  fro2_ = (double*)(base + off);
  off = align256(off + (size_t)n_jac * Z_ * sizeof(double));
  d_tc_ = (unsigned char*)(base + off);
  off = align256(off + (size_t)tc_bytes_);
  svd_log_ = (int*)(base + off);
  off = align256(off + (size_t)Z_ * std::max(1, n_trunc_) * kSvdRec * sizeof(int));

  std::vector<int> hb((size_t)Z_ * nbd, 0);
  for (int id = 0; id < nbd; ++id)
    if (!exact_[id].empty())
      for (int z = 0; z < Z_; ++z) hb[(size_t)z * nbd + id] = exact_[id][z];
  cudaStream_t st = hs_.stream;
  if (hs_.ev0) TTM_CUDA(cudaEventRecord(hs_.ev0, st));
  TTM_CUDA(cudaMemcpyAsync(d_buf_, hbuf_.data(), hbuf_.size() * sizeof(double*), cudaMemcpyHostToDevice, st));
  TTM_CUDA(cudaMemcpyAsync(d_bond_, hb.data(), hb.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  TTM_CUDA(cudaMemsetAsync(d_stat_, 0, (size_t)Z_ * ns * sizeof(double), st));
  TTM_CUDA(cudaMemsetAsync(d_istat_, 0, (size_t)Z_ * nis * sizeof(int), st));
  TTM_CUDA(cudaMemsetAsync(counters_, 0, (size_t)n_jac * counter_stride_ * sizeof(int), st));
  TTM_CUDA(cudaMemsetAsync(fro2_, 0, (size_t)n_jac * Z_ * sizeof(double), st));
  TTM_CUDA(cudaMemsetAsync(svd_log_, 0, (size_t)Z_ * std::max(1, n_trunc_) * kSvdRec * sizeof(int), st));
  tab_ = Tables{d_buf_, d_bond_, d_stat_, d_istat_, nb_, nbd, ns, nis, Z_};

  // second walk: launch
  launches_ = 0;
  prof_used_ = 0;
  prof_kind_.clear();
  const int nchain_planned = nchain_;
  const int jac_planned = jac_launch_;
  launch_ = true;
  if (graph_ok_ && opt_.use_graph) {
    launch_walk_graph(arena, st, nchain_planned, jac_planned);
  } else {
    reset_ids();
    run();
    if ((int)nbuf_total_ != nchain_planned || jac_launch_ != jac_planned)
      throw Error(TTM_ERR_INVALID_ARG, "internal: plan and launch walks disagree");
  }
  if (hs_.ev1) TTM_CUDA(cudaEventRecord(hs_.ev1, st));

  // results
  std::vector<int> bonds((size_t)Z_ * nbd);
  std::vector<double> stat((size_t)Z_ * ns);
  std::vector<int> istat((size_t)Z_ * nis);
  TTM_CUDA(cudaMemcpyAsync(bonds.data(), d_bond_, bonds.size() * sizeof(int), cudaMemcpyDeviceToHost, st));
  TTM_CUDA(cudaMemcpyAsync(stat.data(), d_stat_, stat.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  TTM_CUDA(cudaMemcpyAsync(istat.data(), d_istat_, istat.size() * sizeof(int), cudaMemcpyDeviceToHost, st));
  TTM_CUDA(cudaStreamSynchronize(st));
  float ms = 0.f;
  if (hs_.ev0 && hs_.ev1) TTM_CUDA(cudaEventElapsedTime(&ms, hs_.ev0, hs_.ev1));
  double kind_ms[4] = {0.0, 0.0, 0.0, 0.0};  // GEMMs, float32 Jacobi, Householder QR, float64 Jacobi
  for (int q = 0; q + 1 < prof_used_; q += 2) {
    float x = 0.f;
    TTM_CUDA(cudaEventElapsedTime(&x, hs_.prof_events[q], hs_.prof_events[q + 1]));
    kind_ms[prof_kind_[q / 2]] += x;
  }

  for (int z = 0; z < Z_; ++z) {
    const int st_z = istat[(size_t)z * nis + IS_STATUS];
    if (st_z == (int)TTM_ERR_TIMEOUT)
      throw Error(TTM_ERR_TIMEOUT, "a tensor-core pipeline wait hit its time limit");
    if (st_z == (int)TTM_ERR_NONFINITE)
      throw Error(TTM_ERR_NONFINITE, "product " + std::to_string(z) + ": a Swap met a non-finite value");
  }
  for (int z = 0; z < Z_; ++z) {
    auto bv = [&](int id) { return (long)bonds[(size_t)z * nbd + id]; };
    ttm_tt& o = outs[z];
    const bool caller_out = !o.on_host && o.cores[0] != nullptr;
    o.L = L_;
    o.d = d_;
    for (int j = 0; j <= L_; ++j) o.bonds[j] = bv(out_bond_[j]);
    for (int j = 0; j < L_; ++j) {
      double* src = hbuf_[(size_t)z * nb_ + out_buf_[j]];
      const size_t n = (size_t)o.bonds[j] * d_ * o.bonds[j + 1];
      if (o.on_host) {
        TTM_CUDA(cudaMemcpyAsync(o.cores[j], src, n * sizeof(double), cudaMemcpyDeviceToHost, st));
      } else if (caller_out) {
        TTM_CUDA(cudaMemcpyAsync(o.cores[j], src, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
      } else {
        o.cores[j] = src;
      }
    }
    ttm_report& r = (*reps)[z];
    const int64_t* user_trace = r.bond_trace;
    const int64_t trace_cap = r.bond_trace_len;
    int32_t* user_svd = r.svd_trace;
    const int64_t svd_cap = r.svd_trace_len;
    std::memset(&r, 0, sizeof(r));
    r.status = TTM_OK;
    r.jacobi_sweeps_max = istat[(size_t)z * nis + IS_SWEEPS_MAX];
    long maxb = 0;
    for (int id = 0; id < nbd; ++id) maxb = std::max(maxb, bv(id));
    r.max_bond = maxb;
    double fl = 0.0;
    for (const StepLog& s : log_) {
      if (s.kind == SK_SWAP || s.kind == SK_ROUND) {
        if (s.kind == SK_SWAP) r.n_swaps++;
        const double Dl = bv(s.b0), Dm = bv(s.b1), Dr = bv(s.b2), k = bv(s.b3);
        const double m = d_ * Dl, n = d_ * Dr;
        fl += 2.0 * d_ * d_ * Dl * Dm * Dr;            // Theta
        fl += 2.0 * m * n * n + 2.0 * m * n * k;       // Gram-equivalent + U formation (SVD model)
      } else if (s.kind == SK_CONTRACT) {
        r.n_contracts++;
        fl += 2.0 * d_ * (double)bv(s.b0) * bv(s.b1) * bv(s.b2);
      } else {
        r.n_qr++;
        const double m = d_ * (double)bv(s.b0), n = bv(s.b1), k = bv(s.b2), rr = bv(s.b3);
        const double p = std::max(m, n), q = std::min(m, n);
        fl += 2.0 * p * q * q - 2.0 / 3.0 * q * q * q;  // factorisation
        fl += 2.0 * m * k * k - 2.0 / 3.0 * k * k * k;  // explicit Q
        fl += 2.0 * k * n * d_ * rr;                     // R merge
      }
    }
    r.flops_counted = fl;
    r.discarded_weight = stat[(size_t)z * ns + ST_WSUM];
    r.err_bound = stat[(size_t)z * ns + ST_WSQRT];
    r.seconds = ms * 1e-3;
    r.peak_workspace_bytes = (int64_t)bytes_needed();
    r.newton_residual = stat[(size_t)z * ns + ST_NEWTON_RES];
    r.n_nonconverged = istat[(size_t)z * nis + IS_NONCONV];
    r.n_fallback = istat[(size_t)z * nis + IS_NEWTON_BAD];
    r.n_frozen_pairs = istat[(size_t)z * nis + IS_NFROZEN];
    if (r.n_nonconverged > 0) r.status = TTM_WARN_NOT_CONVERGED;  // result formed; optimality not guaranteed
    r.n_kernel_launches = launches_;
    r.jacobi_launches = jac_launch_;
    r.gemm_ms = kind_ms[0];
    r.jacobi32_ms = kind_ms[1];
    r.qr_ms = kind_ms[2];
    r.jacobi64_ms = kind_ms[3];
    r.jacobi32_flops = stat[(size_t)0 * ns + ST_JFLOPS32];
    r.jacobi32_sweeps = (int64_t)stat[(size_t)z * ns + ST_JSWEEPS32];
    r.gemm_launches = gemm_launch_count_ >= 0 ? (int64_t)gemm_launch_count_ : (int64_t)gemm_log_.size();
    double gf = 0.0;  // counted on the device per executed problem; launch-wide like the others
    for (int zz = 0; zz < Z_; ++zz) gf += stat[(size_t)zz * ns + ST_GFLOPS];
    r.gemm_flops = gf;
    if (user_svd && svd_cap > 0) {
      const int64_t nrec = std::min<int64_t>(svd_cap, n_trunc_);
      std::vector<int> tmp((size_t)nrec * kSvdRec);
      TTM_CUDA(cudaMemcpy(tmp.data(), svd_log_ + (size_t)z * svd_stride(), tmp.size() * sizeof(int),
                          cudaMemcpyDeviceToHost));
      for (size_t q = 0; q < tmp.size(); ++q) user_svd[q] = tmp[q];
      r.svd_trace_len = nrec;
    }
    r.svd_trace = user_svd;
    r.bond_trace = (int64_t*)user_trace;
    r.bond_trace_len = 0;
    if (user_trace) {
      const int64_t nt = std::min<int64_t>(trace_cap, (int64_t)trace_ids_.size());
      for (int64_t q = 0; q < nt; ++q) {
        long mb = 1;
        for (int id : trace_ids_[q]) mb = std::max(mb, bv(id));
        r.bond_trace[q] = mb;
      }
      r.bond_trace_len = nt;
    }
  }
  // norm of the output: the norm of the centre carriage (Pi_1 after the sweep, Pi_N after
  // the final rounding); every other carriage is orthonormal on the side facing away from it
  const int centre = rounding() ? L_ - 1 : 0;
  for (int z = 0; z < Z_; ++z) {
    const ttm_tt& o = outs[z];
    const size_t n = (size_t)o.bonds[centre] * d_ * o.bonds[centre + 1];
    std::vector<double> c0(n);
    TTM_CUDA(cudaMemcpy(c0.data(), hbuf_[(size_t)z * nb_ + out_buf_[centre]], n * sizeof(double),
                        cudaMemcpyDeviceToHost));
    double s = 0.0;
    for (double v : c0) s += v * v;
    (*reps)[z].norm_out = std::sqrt(s);
  }
  TTM_CUDA(cudaStreamSynchronize(st));
}

// ---------------------------------------------------------------- validation

static ttm_status check_tt(const ttm_tt* t, const char* name, bool need_cores) {
  if (!t) return set_err(TTM_ERR_INVALID_ARG, std::string(name) + " is NULL");
  if (t->L < 1) return set_err(TTM_ERR_INVALID_ARG, std::string(name) + ": L < 1");
  if (t->d < 2) return set_err(TTM_ERR_INVALID_ARG, std::string(name) + ": d < 2");
  if (!t->bonds) return set_err(TTM_ERR_INVALID_ARG, std::string(name) + ": bonds is NULL");
  if (need_cores && !t->cores) return set_err(TTM_ERR_INVALID_ARG, std::string(name) + ": cores is NULL");
  if (t->bonds[0] != 1 || t->bonds[t->L] != 1)
    return set_err(TTM_ERR_SHAPE, std::string(name) + ": boundary bonds must be 1");
  // Bonds above the unfolding bound min(d^i, d^(L-i)) are redundant but valid (a TTM output
  // can carry them next to the ends of the train), so only positivity is required.
  for (int i = 0; i <= t->L; ++i) {
    if (t->bonds[i] < 1)
      return set_err(TTM_ERR_SHAPE, std::string(name) + ": bond " + std::to_string(i) + " = " +
                                        std::to_string(t->bonds[i]) + " is below 1");
    if (t->bonds[i] > kMaxBond) return set_err(TTM_ERR_RANK_CAP, std::string(name) + ": bond too large");
  }
  if (need_cores)
    for (int k = 0; k < t->L; ++k)
      if (!t->cores[k]) return set_err(TTM_ERR_INVALID_ARG, std::string(name) + ": core " + std::to_string(k) + " is NULL");
  return TTM_OK;
}

static ttm_status check_opts(const ttm_options& o) {
  if (!(o.eps >= 0.0 && o.eps < 1.0)) return set_err(TTM_ERR_INVALID_ARG, "eps must lie in [0, 1)");
  if (o.chi_max < 0 || o.chi_out < 0) return set_err(TTM_ERR_INVALID_ARG, "negative cap");
  if (o.prec != TTM_PREC_FP64 && o.prec != TTM_PREC_BF16_SPLIT)
    return set_err(TTM_ERR_INVALID_ARG, "unknown precision mode");
  if (o.use_graph != 0 && o.use_graph != 1) return set_err(TTM_ERR_INVALID_ARG, "use_graph must be 0 or 1");
  if (o.use_graph && o.profile_kernels)
    return set_err(TTM_ERR_UNSUPPORTED, "use_graph = 1 cannot be combined with profile_kernels = 1");
  if (o.check_finite != 0) return set_err(TTM_ERR_UNSUPPORTED, "check_finite is not built (must be 0)");
  if (o.f32_passes < 0 || o.f32_passes > kMaxF32Passes)
    return set_err(TTM_ERR_INVALID_ARG, "f32_passes must lie in [0, 8]");
  if (o.jacobi_kernel != 0 && o.jacobi_kernel != 1 && o.jacobi_kernel != 2 && o.jacobi_kernel != 3 &&
      o.jacobi_kernel != 8 && o.jacobi_kernel != 16)
    return set_err(TTM_ERR_INVALID_ARG, "jacobi_kernel must be 0, 1, 2, 3, 8 or 16");
  if (o.newton_steps < 0 || o.newton_steps > kMaxNewtonSteps)
    return set_err(TTM_ERR_INVALID_ARG, "newton_steps must lie in [0, 8]");
  if (o.max_sweeps < 0 || o.max_sweeps > 1000) return set_err(TTM_ERR_INVALID_ARG, "max_sweeps must lie in [0, 1000]");
  if (o.reserved1 != 0) return set_err(TTM_ERR_INVALID_ARG, "reserved option field must be 0");
  if (o.env_budget_bytes < 0) return set_err(TTM_ERR_INVALID_ARG, "env_budget_bytes must be >= 0");
  if (o.split_digits != 0 && (o.split_digits < 2 || o.split_digits > kOzMaxS))
    return set_err(TTM_ERR_INVALID_ARG, "split_digits must be 0 or lie in [2, 8]");
  return TTM_OK;
}

static ttm_options default_options() {
  ttm_options o;
  std::memset(&o, 0, sizeof(o));
  o.prec = TTM_PREC_FP64;
  return o;
}

static ttm_status multiply_impl(ttm_handle* h, int32_t n, const ttm_tt* A, const ttm_tt* B, ttm_tt* out,
                                ttm_report* rep) {
  if (!h) return set_err(TTM_ERR_INVALID_ARG, "handle is NULL");
  if (n < 1 || !A || !B || !out) return set_err(TTM_ERR_INVALID_ARG, "null argument or n < 1");
  ttm_status s = check_opts(h->s.opt);
  if (s != TTM_OK) return s;
  for (int i = 0; i < n; ++i) {
    if ((s = check_tt(&A[i], "A", true)) != TTM_OK) return s;
    if ((s = check_tt(&B[i], "B", true)) != TTM_OK) return s;
    if (A[i].L != B[i].L || A[i].d != B[i].d) return set_err(TTM_ERR_SHAPE, "A and B differ in L or d");
    if (A[i].L != A[0].L || A[i].d != A[0].d) return set_err(TTM_ERR_SHAPE, "batch items differ in L or d");
    if (!out[i].bonds || !out[i].cores) return set_err(TTM_ERR_INVALID_ARG, "out bonds/cores arrays are NULL");
  }
  try {
    TTM_CUDA(cudaSetDevice(h->s.device));
    Engine e(h->s, n, A, B);
    e.allow_graph();  // the handle's arena persists across calls
    e.plan();
    h->s.arena.ensure(e.bytes_needed());
    std::vector<ttm_report> reps(n);
    for (int i = 0; i < n; ++i) {
      std::memset(&reps[i], 0, sizeof(ttm_report));
      if (rep) {
        reps[i].bond_trace = rep[i].bond_trace;
        reps[i].bond_trace_len = rep[i].bond_trace_len;
        reps[i].svd_trace = rep[i].svd_trace;
        reps[i].svd_trace_len = rep[i].svd_trace_len;
      }
    }
    e.execute(h->s.arena.ptr, h->s.opt, &reps, out);
    if (rep)
      for (int i = 0; i < n; ++i) rep[i] = reps[i];
    for (int i = 0; i < n; ++i)
      if (reps[i].status == TTM_WARN_NOT_CONVERGED)
        return set_err(TTM_WARN_NOT_CONVERGED, "product " + std::to_string(i) + ": " +
                                                   std::to_string(reps[i].n_nonconverged) +
                                                   " Swap SVD(s) did not converge");
  } catch (const Error& err) {
    return set_err(err.status, err.what());
  } catch (const std::exception& ex) {
    return set_err(TTM_ERR_INVALID_ARG, ex.what());
  }
  return TTM_OK;
}

}  // namespace ttm

using namespace ttm;

extern "C" {

ttm_status ttm_create(ttm_handle** h, int device, void* cuda_stream, const ttm_options* opt) {
  if (!h) return set_err(TTM_ERR_INVALID_ARG, "h is NULL");
  *h = nullptr;
  ttm_options o = opt ? *opt : default_options();
  ttm_status s = check_opts(o);
  if (s != TTM_OK) return s;
  ttm_handle* H = new (std::nothrow) ttm_handle();
  if (!H) return set_err(TTM_ERR_NOMEM, "host allocation failed");
  try {
    TTM_CUDA(cudaSetDevice(device));
    H->s.device = device;
    H->s.stream = (cudaStream_t)cuda_stream;
    H->s.opt = o;
    TTM_CUDA(cudaDeviceGetAttribute(&H->s.num_sms, cudaDevAttrMultiProcessorCount, device));
    TTM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&H->s.coop_hest32, hestenes_kernel<float>, 256, 0));
    TTM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&H->s.coop_hest, hestenes_kernel<double>, 256, 0));
    TTM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&H->s.coop_qr, householder_kernel, 256, 0));
    int coop = 0;
    TTM_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device));
    if (!coop) throw Error(TTM_ERR_UNSUPPORTED, "device lacks cooperative launch");
    TTM_CUDA(cudaEventCreate(&H->s.ev0));
    TTM_CUDA(cudaEventCreate(&H->s.ev1));
  } catch (const Error& err) {
    delete H;
    return set_err(err.status, err.what());
  }
  *h = H;
  return TTM_OK;
}

ttm_status ttm_destroy(ttm_handle* h) {
  if (!h) return TTM_OK;
  cudaSetDevice(h->s.device);
  if (h->s.stream) cudaStreamSynchronize(h->s.stream);
  else cudaDeviceSynchronize();
  if (h->s.ev0) cudaEventDestroy(h->s.ev0);
  if (h->s.ev1) cudaEventDestroy(h->s.ev1);
  delete h;
  return TTM_OK;
}

ttm_status ttm_set_options(ttm_handle* h, const ttm_options* opt) {
  if (!h || !opt) return set_err(TTM_ERR_INVALID_ARG, "null argument");
  ttm_status s = check_opts(*opt);
  if (s != TTM_OK) return s;
  h->s.opt = *opt;
  return TTM_OK;
}

ttm_status ttm_multiply(ttm_handle* h, const ttm_tt* A, const ttm_tt* B, ttm_tt* out, ttm_report* rep) {
  return multiply_impl(h, 1, A, B, out, rep);
}

ttm_status ttm_multiply_batched(ttm_handle* h, int32_t n, const ttm_tt* A, const ttm_tt* B, ttm_tt* out,
                                ttm_report* rep) {
  return multiply_impl(h, n, A, B, out, rep);
}

int64_t ttm_output_capacity(const ttm_tt* A, const ttm_tt* B, const ttm_options* opt) {
  if (check_tt(A, "A", false) != TTM_OK || check_tt(B, "B", false) != TTM_OK) return -1;
  if (A->L != B->L || A->d != B->d) return -1;
  ttm_options o = opt ? *opt : default_options();
  try {
    HandleState hs;
    hs.opt = o;
    Engine e(hs, 1, A, B);
    e.plan();
    return e.max_carriage();
  } catch (...) {
    return -1;
  }
}

static ttm_status check_env_tt(const ttm_tt* t, const char* name, int L, int d) {
  ttm_status s = check_tt(t, name, true);
  if (s != TTM_OK) return s;
  if (t->on_host) return set_err(TTM_ERR_UNSUPPORTED, std::string(name) + ": environments take device cores");
  if (t->L != L || t->d != d) return set_err(TTM_ERR_SHAPE, std::string(name) + ": L or d differs");
  return TTM_OK;
}

ttm_status ttm_backward(ttm_handle* h, ttm_loss kind, const ttm_tt* A, const ttm_tt* B, const ttm_tt* WC,
                        double* loss_out, ttm_tt* gradA, ttm_tt* gradB) {
  if (!h || !A || !B || !WC || !loss_out) return set_err(TTM_ERR_INVALID_ARG, "null argument");
  if (kind != TTM_LOSS_INNER && kind != TTM_LOSS_SQDIST) return set_err(TTM_ERR_INVALID_ARG, "unknown loss");
  ttm_status s;
  if ((s = check_env_tt(A, "A", A->L, A->d)) != TTM_OK) return s;
  if ((s = check_env_tt(B, "B", A->L, A->d)) != TTM_OK) return s;
  if ((s = check_env_tt(WC, "W_or_C", A->L, A->d)) != TTM_OK) return s;
  for (ttm_tt* g : {gradA, gradB}) {
    if (!g) continue;
    const ttm_tt* ref = (g == gradA) ? A : B;
    if ((s = check_env_tt(g, "grad", A->L, A->d)) != TTM_OK) return s;
    for (int i = 0; i <= A->L; ++i)
      if (g->bonds[i] != ref->bonds[i]) return set_err(TTM_ERR_SHAPE, "gradient bonds differ from the train's");
  }
  try {
    TTM_CUDA(cudaSetDevice(h->s.device));
    *loss_out = env_backward(h->s, h->s.env_arena, (int)kind, *A, *B, *WC, gradA, gradB);
    TTM_CUDA(h->s.stream ? cudaStreamSynchronize(h->s.stream) : cudaDeviceSynchronize());
  } catch (const Error& err) {
    return set_err(err.status, err.what());
  }
  return TTM_OK;
}

ttm_status ttm_inner(ttm_handle* h, const ttm_tt* X, const ttm_tt* Y, double* outv) {
  if (!h || !X || !Y || !outv) return set_err(TTM_ERR_INVALID_ARG, "null argument");
  ttm_status s;
  if ((s = check_env_tt(X, "X", X->L, X->d)) != TTM_OK) return s;
  if ((s = check_env_tt(Y, "Y", X->L, X->d)) != TTM_OK) return s;
  try {
    TTM_CUDA(cudaSetDevice(h->s.device));
    *outv = env_inner(h->s, h->s.env_arena, *X, *Y);
  } catch (const Error& err) {
    return set_err(err.status, err.what());
  }
  return TTM_OK;
}

ttm_status ttm_inner3(ttm_handle* h, const ttm_tt* W, const ttm_tt* A, const ttm_tt* B, double* outv) {
  if (!h || !W || !A || !B || !outv) return set_err(TTM_ERR_INVALID_ARG, "null argument");
  ttm_status s;
  if ((s = check_env_tt(W, "W", W->L, W->d)) != TTM_OK) return s;
  if ((s = check_env_tt(A, "A", W->L, W->d)) != TTM_OK) return s;
  if ((s = check_env_tt(B, "B", W->L, W->d)) != TTM_OK) return s;
  try {
    TTM_CUDA(cudaSetDevice(h->s.device));
    *outv = env_inner3(h->s, h->s.env_arena, *W, *A, *B);
  } catch (const Error& err) {
    return set_err(err.status, err.what());
  }
  return TTM_OK;
}

ttm_status ttm_synchronize(ttm_handle* h) {
  if (!h) return set_err(TTM_ERR_INVALID_ARG, "handle is NULL");
  cudaError_t e = h->s.stream ? cudaStreamSynchronize(h->s.stream) : cudaDeviceSynchronize();
  if (e != cudaSuccess) return set_err(TTM_ERR_CUDA, cudaGetErrorString(e));
  return TTM_OK;
}

ttm_status ttm_tt_free(ttm_handle* h, ttm_tt* t) {
  if (!h) return set_err(TTM_ERR_INVALID_ARG, "handle is NULL");
  if (t && !t->on_host && t->cores)
    for (int k = 0; k < t->L; ++k) t->cores[k] = nullptr;
  return TTM_OK;
}

// ---------------------------------------------------------------- allocation-free product

// Workspace of ttm_multiply_noalloc: a fixed array in device memory, defined at file scope.
// Host code must not use the symbol as an address (on the host it names a stand-in);
// the device address comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[TTM_NOALLOC_SCRATCH_BYTES];

namespace {
struct NoAllocDevice {
  bool ready = false;
  void* scratch = nullptr;
  int num_sms = 0, coop_hest32 = 0, coop_hest = 0, coop_qr = 0;
};
std::mutex g_noalloc_mu;
NoAllocDevice g_noalloc_dev[64];
}  // namespace

ttm_status ttm_multiply_noalloc(const ttm_tt* A, const ttm_tt* B, ttm_tt* out, const ttm_options* opt,
                                void* cuda_stream) {
  if (!A || !B || !out) return set_err(TTM_ERR_INVALID_ARG, "null argument");
  ttm_options o = opt ? *opt : default_options();
  o.profile_kernels = 0;
  ttm_status s = check_opts(o);
  if (s != TTM_OK) return s;
  if ((s = check_tt(A, "A", true)) != TTM_OK) return s;
  if ((s = check_tt(B, "B", true)) != TTM_OK) return s;
  if (A->L != B->L || A->d != B->d) return set_err(TTM_ERR_SHAPE, "A and B differ in L or d");
  if (A->on_host || B->on_host || out->on_host)
    return set_err(TTM_ERR_UNSUPPORTED, "the allocation-free product takes device cores only");
  if (!out->bonds || !out->cores) return set_err(TTM_ERR_INVALID_ARG, "out bonds/cores arrays are NULL");
  for (int k = 0; k < A->L; ++k)
    if (!out->cores[k]) return set_err(TTM_ERR_INVALID_ARG, "out->cores must be caller device buffers");
  try {
    int dev = 0;
    TTM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) throw Error(TTM_ERR_UNSUPPORTED, "device index above 63");
    NoAllocDevice info;
    {
      std::lock_guard<std::mutex> lock(g_noalloc_mu);
      NoAllocDevice& nd = g_noalloc_dev[dev];
      if (!nd.ready) {
        void* p = nullptr;
        TTM_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        TTM_CUDA(cudaDeviceGetAttribute(&nd.num_sms, cudaDevAttrMultiProcessorCount, dev));
        TTM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nd.coop_hest32, hestenes_kernel<float>, 256, 0));
        TTM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nd.coop_hest, hestenes_kernel<double>, 256, 0));
        TTM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nd.coop_qr, householder_kernel, 256, 0));
        nd.scratch = p;
        nd.ready = true;
      }
      info = nd;
    }
    HandleState hs;  // no arena is ever allocated through it on this path, and no events
    hs.device = dev;
    hs.stream = (cudaStream_t)cuda_stream;
    hs.opt = o;
    hs.num_sms = info.num_sms;
    hs.coop_hest32 = info.coop_hest32;
    hs.coop_hest = info.coop_hest;
    hs.coop_qr = info.coop_qr;
    Engine e(hs, 1, A, B);
    e.plan();
    const size_t need = e.bytes_needed();
    if (need > (size_t)TTM_NOALLOC_SCRATCH_BYTES)
      throw Error(TTM_ERR_WORKSPACE, "the product needs " + std::to_string(need) +
                                         " bytes of workspace; the allocation-free path has " +
                                         std::to_string((size_t)TTM_NOALLOC_SCRATCH_BYTES));
    std::vector<ttm_report> reps(1);
    std::memset(&reps[0], 0, sizeof(ttm_report));
    e.execute(info.scratch, o, &reps, out);
    if (reps[0].status == TTM_WARN_NOT_CONVERGED)
      return set_err(TTM_WARN_NOT_CONVERGED, std::to_string(reps[0].n_nonconverged) +
                                                 " Swap SVD(s) did not converge");
  } catch (const Error& err) {
    return set_err(err.status, err.what());
  } catch (const std::exception& ex) {
    return set_err(TTM_ERR_INVALID_ARG, ex.what());
  }
  return TTM_OK;
}

// ---------------------------------------------------------------- plain GEMM

namespace {
// C = A B with column-major device matrices (one problem per launch).
struct RawGemmFn {
  Tables t;
  int M, N, K;
  const double* A;
  long lda;
  const double* B;
  long ldb;
  double* C;
  long ldc;
  __device__ GemmDesc operator()(int, int) const {
    GemmDesc g;
    g.M = M; g.N = N; g.K = K;
    g.A = MatRef{A, 1, lda};
    g.B = MatRef{B, 1, ldb};
    g.C = OutRef{C, 1, ldc};
    g.alpha = 1.0; g.beta = 0.0; g.upper = 0;
    return g;
  }
};
}  // namespace

ttm_status ttm_gemm(ttm_handle* h, ttm_precision prec, int64_t M, int64_t N, int64_t K, const double* A, int64_t lda,
                    const double* B, int64_t ldb, double* C, int64_t ldc) {
  if (!h || !A || !B || !C) return set_err(TTM_ERR_INVALID_ARG, "null argument");
  if (M < 1 || N < 1 || K < 1 || M > (1 << 20) || N > (1 << 20) || K > (1 << 20))
    return set_err(TTM_ERR_SHAPE, "M, N, K must lie in [1, 2^20]");
  if (lda < M || ldb < K || ldc < M) return set_err(TTM_ERR_SHAPE, "leading dimension below the row count");
  if (prec != TTM_PREC_FP64 && prec != TTM_PREC_BF16_SPLIT) return set_err(TTM_ERR_INVALID_ARG, "unknown precision mode");
  try {
    TTM_CUDA(cudaSetDevice(h->s.device));
    Tables t{};
    RawGemmFn f{t, (int)M, (int)N, (int)K, A, (long)lda, B, (long)ldb, C, (long)ldc};
    cudaStream_t st = h->s.stream;
    if (prec == TTM_PREC_FP64) {
      dim3 grid((unsigned)((N + GT - 1) / GT), (unsigned)((M + GT - 1) / GT), 1);
      dgemm_kernel<RawGemmFn><<<grid, 256, 0, st>>>(f, 1);
      TTM_CUDA(cudaGetLastError());
    } else {
      const int S = h->s.opt.split_digits > 0 ? h->s.opt.split_digits : kOzMaxS;
      const size_t need = tc_ws_bytes(1, (int)M, (int)N, (int)K, S) + 256;
      h->s.env_arena.ensure(need);
      unsigned char* ws = (unsigned char*)h->s.env_arena.ptr;
      int* err = (int*)(ws + need - 256);
      TTM_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
      TTM_CUDA(launch_tc_gemm(st, f, 1, 1, (int)M, (int)N, (int)K, -1, S, ws, err));
      int herr = 0;
      TTM_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
      TTM_CUDA(cudaStreamSynchronize(st));
      if (herr != 0) throw Error(TTM_ERR_TIMEOUT, "a tensor-core pipeline wait hit its time limit");
    }
    TTM_CUDA(st ? cudaStreamSynchronize(st) : cudaDeviceSynchronize());
  } catch (const Error& err) {
    return set_err(err.status, err.what());
  }
  return TTM_OK;
}

const char* ttm_last_error(void) { return g_last_error.c_str(); }

const char* ttm_version(void) { return "ttm-gb300 0.1 (sm_103a)"; }

}  // extern "C"
