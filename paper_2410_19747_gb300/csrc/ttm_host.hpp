// ttm_host.hpp -- host-side types shared by the translation units of libttm.so:
// the internal exception carrying a ttm_status, the CUDA error check, the grow-only
// device arena and the per-handle state.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <stdexcept>
#include <string>
#include <vector>

#include "ttm.h"

namespace ttm {

struct Error : std::runtime_error {
  ttm_status status;
  Error(ttm_status s, const std::string& m) : std::runtime_error(m), status(s) {}
};

#define TTM_CUDA(call)                                                                    \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      throw ::ttm::Error(TTM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_) + \
                                           " (" + __FILE__ + ":" + std::to_string(__LINE__) + ")"); \
  } while (0)

constexpr int kMaxBond = 8192;         // largest bond the planner accepts
constexpr int kDefaultF32Passes = 3;   // float32 Jacobi passes of every Swap SVD
constexpr int kMaxF32Passes = 8;
constexpr int kF32Sweeps = 20;         // sweep limit of the later float32 passes (the Newton steps
                                        // finish what they leave; 20 instead of 30 measured 6 % faster
                                        // at chi = 512 with the same fallbacks and result)
constexpr int kDefaultNewtonSteps = 3; // float64 Newton steps after the float32 passes
constexpr int kNewtonExtraSteps = 2;   // further steps for an SVD whose last correction is above 1e-7
constexpr int kMaxNewtonSteps = 8;
constexpr int kPolishSweeps = 40;      // sweep limit of the float64 Jacobi of the fallback
// Sweep limit of the first float32 pass: it only has to grade W (the next pass redoes the
// whole Jacobi on the graded W), so its refining sweeps are dropped.
constexpr int kF32FirstPassSweeps = 3;

struct DeviceArena {
  void* ptr = nullptr;
  size_t bytes = 0;
  void ensure(size_t need) {
    if (need <= bytes) return;
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
    cudaError_t e = cudaMalloc(&ptr, need);
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw Error(TTM_ERR_NOMEM, "device allocation of " + std::to_string(need) + " bytes failed");
    }
    bytes = need;
  }
  ~DeviceArena() {
    if (ptr) cudaFree(ptr);
  }
};

// Per-handle state.
struct HandleState {
  int device = 0;
  cudaStream_t stream = nullptr;
  ttm_options opt{};
  int num_sms = 0;
  int coop_hest32 = 0, coop_hest = 0, coop_qr = 0;  // co-resident blocks per SM (cooperative kernels)
  DeviceArena arena;      // sweep buffers and workspaces
  DeviceArena env_arena;  // environments of ttm_inner / ttm_inner3 / ttm_backward
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::vector<cudaEvent_t> prof_events;  // pairs around Jacobi launches (profile_kernels)
  // use_graph = 1: the launch walk of the last plan, captured once into a CUDA graph and
  // replayed while the plan (options, shapes, input bonds, arena) stays the same
  cudaStream_t capture_stream = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  std::string graph_key;
  std::vector<int> graph_loads;          // (input: 0 = A, 1 = B; core k; buffer) per input copy
  long graph_launches = 0, graph_gemms = 0;
  ~HandleState() {
    for (cudaEvent_t e : prof_events) cudaEventDestroy(e);
    if (graph_exec) cudaGraphExecDestroy(graph_exec);
    if (capture_stream) cudaStreamDestroy(capture_stream);
  }
};


// Environment drivers (ttm_env.cu).
double env_inner(HandleState& hs, DeviceArena& ar, const ttm_tt& X, const ttm_tt& Y);
double env_inner3(HandleState& hs, DeviceArena& ar, const ttm_tt& W, const ttm_tt& A, const ttm_tt& B);
double env_backward(HandleState& hs, DeviceArena& ar, int kind, const ttm_tt& A, const ttm_tt& B,
                    const ttm_tt& WC, const ttm_tt* gA, const ttm_tt* gB);

}  // namespace ttm
