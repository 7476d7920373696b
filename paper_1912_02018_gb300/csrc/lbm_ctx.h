// Host-side state of one simulation context, shared by the C-ABI translation units
// (lbm_api.cu: creation, stepping, state I/O, batches; lbm_adjoint_api.cu: the adjoint).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "lbm.h"
#include "lbm_internal.h"

struct lbm_adjoint_work;

struct lbm_ctx {
  lbm::Geo geo{};
  lbm::Phys ph{};
  lbm::Dev dev{};
  lbm_domain dom{};
  lbm_cylinder cyl{};
  lbm_params prm{};
  lbm_allocator alloc{};
  bool has_alloc = false;
  cudaStream_t stream = nullptr;
  int device = 0;
  int cur = 0;   // buffer index of f* and the outlet side values
  int tcur = 0;  // buffer index of T
  int psi_pending = 0;  // dev.psi_next holds psi of the next step (made by the last energy pass)
  int64_t steps = 0;
  int64_t launches = 0;
  bool f64 = false;
  double Tc = 0, pc = 0, p_sat = 0, h_fg = 0, lambda_v = 0;
  std::vector<void*> blocks;
  size_t bytes = 0;
  std::string err = "no error";
  // per-launch timing
  struct Pending {
    int kernel;
    cudaEvent_t e0, e1;
  };
  bool prof = false;
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  double prof_ms[lbm::kNumKernels] = {};
  int64_t prof_n[lbm::kNumKernels] = {};
  cudaEvent_t open_ev = nullptr;
  bool batch_owned = false;  // stepped only through its lbm_batch
  // wall temperature: typed [ny][pitch] plane (values at the solid nodes) and, for an angular
  // profile, each solid node's two knots and interpolation weight
  void* wallT = nullptr;
  int n_wall = 0;
  std::vector<int> wall_node, wall_k0, wall_k1;  // wall_node: y * nx + x
  std::vector<double> wall_t;
  lbm_adjoint_work* adjw = nullptr;  // buffers of the adjoint window (created on first use)
  // staged restores (lbm_stage_state_native / lbm_take_staged), made on first use: a copy
  // stream, the staging buffers of f, T and the outlet rows, and two events: copied (the
  // staged state has landed) and released (the context's stream no longer uses the buffers
  // that became the staging buffers at the last take)
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_copied = nullptr, ev_released = nullptr;
  void* stage_f = nullptr;
  void* stage_T = nullptr;
  void* stage_side = nullptr;
  int staged = 0;  // 0: nothing staged; else 1 + (1 if the outlet rows were staged)
  int64_t staged_steps = -1;
};

namespace lbm {
namespace host {

// Record an error message on the context (or the thread's creation error) and return st.
lbm_status fail(lbm_ctx* ctx, lbm_status st, const char* fmt, ...);
// Device allocation through the context's allocator (or cudaMalloc), freed by dfree_all.
void* dalloc(lbm_ctx* c, size_t bytes);
void dfree_all(lbm_ctx* c);
// Synchronise the context's stream and turn latched kernel fault bits into a status.
lbm_status check_status(lbm_ctx* c);
// Free the adjoint window's buffers (no-op when none were made).
void adjoint_release(lbm_ctx* c);

}  // namespace host
}  // namespace lbm

#define LBM_CUDA(ctx, call)                                                                            \
  do {                                                                                                 \
    cudaError_t e_ = (call);                                                                           \
    if (e_ != cudaSuccess) return lbm::host::fail((ctx), LBM_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)
