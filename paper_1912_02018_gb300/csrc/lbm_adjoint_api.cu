// Host side of the adjoint entry points of include/lbm.h: one reverse step at the current
// state (lbm_adjoint_step) and the checkpointed window (lbm_adjoint_window).  The forward
// steps and every reverse step run in the kernels of lbm_kernels.cuh and lbm_adjoint.cuh.
//
// Window of n steps, checkpoint every K steps: the forward pass advances the context and
// copies its state (f*, T, outlet side values) at the start of each segment.  The reverse
// pass takes the segments last to first: it recomputes the segment from its checkpoint into
// K + 1 state slots (keeping rho, psi and u of every collision), then runs the reverse steps
// last to first.  Memory: (K + 1) states and psi fields, K sets of rho, u and the stage-1
// temperature, one state per checkpoint and 30 adjoint work planes.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <map>
#include <tuple>
#include <vector>

#include "lbm.h"
#include "lbm_ctx.h"
#include "lbm_internal.h"

using namespace lbm::host;

struct lbm_adjoint_work {
  int K = 0, nseg = 0;
  std::vector<void*> blocks;
  std::vector<void*> sf, sT, sside;         // K + 1 state slots
  std::vector<void*> arho, apsi, aux, auy;  // K sets of collision fields
  std::vector<void*> aT1;                   // K stage-1 temperatures of the recomputed energy passes
  std::vector<void*> cf, cT, cside;         // nseg checkpoints
  void *fb[2] = {}, *Tb[2] = {}, *sb[2] = {};
  void *Tb1 = nullptr, *ub[2] = {}, *lamb = nullptr, *rhob = nullptr;
  void *fpb = nullptr, *fmb[2] = {}, *psib = nullptr;
  double *gw = nullptr, *uin = nullptr, *hf = nullptr;
  // a segment's recompute and reverse steps replayed from a CUDA graph on a private stream,
  // ordered after and before the context's stream by events; one graph per (length, starting
  // ping-pong parity, heat-flux weight)
  cudaStream_t gs = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  std::map<std::tuple<int, int, double>, cudaGraphExec_t> graphs;
};

namespace {

void* walloc(lbm_ctx* c, lbm_adjoint_work* w, size_t bytes) {
  bytes = (bytes + 255) & ~size_t(255);
  void* p = nullptr;
  if (c->has_alloc) {
    p = c->alloc.alloc(bytes, c->alloc.user);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) w->blocks.push_back(p);
  return p;
}

size_t elem(const lbm_ctx* c) { return c->f64 ? sizeof(double) : sizeof(float); }

lbm_status prepare(lbm_ctx* c, int K, int nseg) {
  if (c->adjw && c->adjw->K >= K && c->adjw->nseg >= nseg) return LBM_OK;
  adjoint_release(c);
  lbm_adjoint_work* w = new lbm_adjoint_work();
  c->adjw = w;
  w->K = K;
  w->nseg = nseg;
  const size_t es = elem(c), plane = (size_t)c->geo.plane * es, fs = 9 * plane, ss = 3 * (size_t)c->geo.ny * es;
  bool ok = true;
  auto A = [&](size_t b) {
    void* p = walloc(c, w, b);
    ok = ok && p;
    return p;
  };
  for (int j = 0; j <= K; ++j) {
    w->sf.push_back(A(fs));
    w->sT.push_back(A(plane));
    w->sside.push_back(A(ss));
  }
  for (int j = 0; j < K; ++j) {
    char* ruv = static_cast<char*>(A(3 * plane));  // rho, u_x, u_y as consecutive planes (one TMA map)
    w->arho.push_back(ruv);
    w->aux.push_back(ruv ? ruv + plane : nullptr);
    w->auy.push_back(ruv ? ruv + 2 * plane : nullptr);
    w->aT1.push_back(A(plane));
  }
  for (int j = 0; j <= K; ++j) w->apsi.push_back(A(plane));  // psi of slot K comes from the last energy pass
  for (int s = 0; s < nseg; ++s) {
    w->cf.push_back(A(fs));
    w->cT.push_back(A(plane));
    w->cside.push_back(A(ss));
  }
  for (int k = 0; k < 2; ++k) {
    w->fb[k] = A(fs);
    w->Tb[k] = A(plane);
    w->sb[k] = A(ss);
    w->ub[k] = A(plane);
    w->fmb[k] = A(plane);
  }
  w->Tb1 = A(plane);
  w->lamb = A(plane);
  w->rhob = A(plane);
  w->fpb = A(fs);
  w->psib = A(plane);
  w->gw = static_cast<double*>(A((size_t)c->geo.plane * sizeof(double)));
  w->uin = static_cast<double*>(A((size_t)c->geo.ny * sizeof(double)));
  w->hf = static_cast<double*>(A(4 * sizeof(double)));
  if (!ok) {
    adjoint_release(c);
    return fail(c, LBM_ENOMEM, "device allocation for the adjoint (K = %d, %d checkpoints) failed", K, nseg);
  }
  if ((c->f64 ? lbm::adjoint_setup_f64() : lbm::adjoint_setup_f32()) < 0)
    return fail(c, LBM_ECUDA, "adjoint kernel set-up failed: %s", cudaGetErrorString(cudaGetLastError()));
  return LBM_OK;
}

// Forward step of slot j into slot j + 1, keeping the collision fields of slot j.  Within a
// segment the energy pass of step j makes psi of step j + 1, so only the first step runs the psi
// pass.
int forward_slot(lbm_ctx* c, lbm_adjoint_work* w, int j, cudaStream_t st) {
  lbm::Dev v = c->dev;
  v.f[0] = w->sf[j];
  v.f[1] = w->sf[j + 1];
  v.T[0] = w->sT[j];
  v.T[1] = w->sT[j + 1];
  v.side[0] = w->sside[j];
  v.side[1] = w->sside[j + 1];
  v.rho = w->arho[j];
  v.psi = w->apsi[j];
  v.psi_next = w->apsi[j + 1];
  v.ux = w->aux[j];
  v.uy = w->auy[j];
  v.hf = w->hf;
  v.nb = 0;  // the recompute needs no heat-flux sample
  v.t1_out = w->aT1[j];
  // plain launches inside the segment's graph: programmatic dependent launch of its many small
  // passes (512 x 256: one wave each) measured slower there
  v.pdl = 0;
  int flipped = 0;
  lbm::PsiChain chain{j > 0 ? 1 : 0, 1, 0};
  const int k = c->f64 ? lbm::step_f64(c->geo, c->ph, v, 0, 0, 1, 1, c->prm.psi_mode, st, nullptr, &flipped, &chain)
                       : lbm::step_f32(c->geo, c->ph, v, 0, 0, 1, 1, c->prm.psi_mode, c->prm.storage, st, nullptr,
                                       &flipped, &chain);
  return k < 0 || !flipped ? -1 : k;
}

template <typename C>
lbm::AdjArgs<C> make_args(lbm_ctx* c, lbm_adjoint_work* w, int j, int ping, double wq) {
  lbm::AdjArgs<C> a{};
  a.g = c->geo;
  a.ph = c->ph;
  a.mask = c->dev.mask;
  a.f = static_cast<const C*>(w->sf[j]);
  a.T = static_cast<const C*>(w->sT[j]);
  a.side = static_cast<const C*>(w->sside[j]);
  a.rho = static_cast<const C*>(w->arho[j]);
  a.psi = static_cast<const C*>(w->apsi[j]);
  a.ux = static_cast<const C*>(w->aux[j]);
  a.uy = static_cast<const C*>(w->auy[j]);
  a.T1 = static_cast<const C*>(w->aT1[j]);
  a.fb_in = static_cast<const C*>(w->fb[ping]);
  a.Tb_in = static_cast<const C*>(w->Tb[ping]);
  a.sb_in = static_cast<const C*>(w->sb[ping]);
  a.fb_out = static_cast<C*>(w->fb[ping ^ 1]);
  a.Tb_out = static_cast<C*>(w->Tb[ping ^ 1]);
  a.sb_out = static_cast<C*>(w->sb[ping ^ 1]);
  a.Tb1 = static_cast<C*>(w->Tb1);
  a.ub[0] = static_cast<C*>(w->ub[0]);
  a.ub[1] = static_cast<C*>(w->ub[1]);
  a.lamb = static_cast<C*>(w->lamb);
  a.rhob = static_cast<C*>(w->rhob);
  a.fpb = static_cast<C*>(w->fpb);
  a.fmb[0] = static_cast<C*>(w->fmb[0]);
  a.fmb[1] = static_cast<C*>(w->fmb[1]);
  a.psib = static_cast<C*>(w->psib);
  a.gw = w->gw;
  a.uin = w->uin;
  a.wq = (C)wq;
  a.do_hf = c->dev.nb > 0 && wq != 0.0;
  return a;
}

int reverse_slot(lbm_ctx* c, lbm_adjoint_work* w, int j, int ping, double wq, cudaStream_t st) {
  return c->f64 ? lbm::adjoint_step_f64(make_args<double>(c, w, j, ping, wq), st)
                : lbm::adjoint_step_f32(make_args<float>(c, w, j, ping, wq), st);
}

// Recompute a segment of len steps from state slot 0 and run its reverse steps, the first with
// adjoint buffers [ping]; on stream st.  Returns false on a launch error.
bool segment_launches(lbm_ctx* c, lbm_adjoint_work* w, int len, int ping, double wq, cudaStream_t st) {
  for (int j = 0; j < len; ++j)
    if (forward_slot(c, w, j, st) < 0) return false;
  for (int j = len - 1; j >= 0; --j) {
    if (reverse_slot(c, w, j, ping, wq, st) < 0) return false;
    ping ^= 1;
  }
  return true;
}

// The same from a cached CUDA graph (captured on first use).
lbm_status segment_graph(lbm_ctx* c, lbm_adjoint_work* w, int len, int ping, double wq) {
  if (!w->gs) {
    LBM_CUDA(c, cudaStreamCreateWithFlags(&w->gs, cudaStreamNonBlocking));
    LBM_CUDA(c, cudaEventCreateWithFlags(&w->ev_in, cudaEventDisableTiming));
    LBM_CUDA(c, cudaEventCreateWithFlags(&w->ev_out, cudaEventDisableTiming));
  }
  const auto key = std::make_tuple(len, ping, wq);
  auto it = w->graphs.find(key);
  if (it == w->graphs.end()) {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    LBM_CUDA(c, cudaStreamBeginCapture(w->gs, cudaStreamCaptureModeThreadLocal));
    const bool ok = segment_launches(c, w, len, ping, wq, w->gs);
    const cudaError_t e = cudaStreamEndCapture(w->gs, &graph);
    if (!ok || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return fail(c, LBM_ECUDA, "capture of the adjoint segment failed: %s", cudaGetErrorString(cudaGetLastError()));
    }
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) return fail(c, LBM_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(ei));
    it = w->graphs.emplace(key, exec).first;
  }
  LBM_CUDA(c, cudaEventRecord(w->ev_in, c->stream));
  LBM_CUDA(c, cudaStreamWaitEvent(w->gs, w->ev_in, 0));
  LBM_CUDA(c, cudaGraphLaunch(it->second, w->gs));
  LBM_CUDA(c, cudaEventRecord(w->ev_out, w->gs));
  LBM_CUDA(c, cudaStreamWaitEvent(c->stream, w->ev_out, 0));
  return LBM_OK;
}
int aux(lbm_ctx* c, int op, const void* src, void* dst) {
  return c->f64 ? lbm::adjoint_aux_f64(op, c->geo, c->dev.mask, src, dst, c->stream)
                : lbm::adjoint_aux_f32(op, c->geo, c->dev.mask, src, dst, c->stream);
}

// Copy the context's current state into state slot / checkpoint buffers.
lbm_status copy_state(lbm_ctx* c, void* f, void* T, void* side, bool to_ctx) {
  const size_t es = elem(c), plane = (size_t)c->geo.plane * es;
  void* cf = c->dev.f[c->cur];
  void* cT = c->dev.T[c->tcur];
  void* cs = c->dev.side[c->cur];
  auto cp = [&](void* dst, const void* src, size_t b) {
    return cudaMemcpyAsync(dst, src, b, cudaMemcpyDeviceToDevice, c->stream);
  };
  if (to_ctx) {
    LBM_CUDA(c, cp(cf, f, 9 * plane));
    LBM_CUDA(c, cp(cT, T, plane));
    LBM_CUDA(c, cp(cs, side, 3 * (size_t)c->geo.ny * es));
  } else {
    LBM_CUDA(c, cp(f, cf, 9 * plane));
    LBM_CUDA(c, cp(T, cT, plane));
    LBM_CUDA(c, cp(side, cs, 3 * (size_t)c->geo.ny * es));
  }
  return LBM_OK;
}
lbm_status copy_slot(lbm_ctx* c, void* df, void* dT, void* ds, const void* sf, const void* sT, const void* ss) {
  const size_t es = elem(c), plane = (size_t)c->geo.plane * es;
  LBM_CUDA(c, cudaMemcpyAsync(df, sf, 9 * plane, cudaMemcpyDeviceToDevice, c->stream));
  LBM_CUDA(c, cudaMemcpyAsync(dT, sT, plane, cudaMemcpyDeviceToDevice, c->stream));
  LBM_CUDA(c, cudaMemcpyAsync(ds, ss, 3 * (size_t)c->geo.ny * es, cudaMemcpyDeviceToDevice, c->stream));
  return LBM_OK;
}

lbm_status zero_adjoint(lbm_ctx* c, lbm_adjoint_work* w, int ping) {
  const size_t es = elem(c), plane = (size_t)c->geo.plane * es;
  LBM_CUDA(c, cudaMemsetAsync(w->fb[ping], 0, 9 * plane, c->stream));
  LBM_CUDA(c, cudaMemsetAsync(w->Tb[ping], 0, plane, c->stream));
  for (int k = 0; k < 2; ++k) LBM_CUDA(c, cudaMemsetAsync(w->sb[k], 0, 3 * (size_t)c->geo.ny * es, c->stream));
  LBM_CUDA(c, cudaMemsetAsync(w->gw, 0, (size_t)c->geo.plane * sizeof(double), c->stream));
  LBM_CUDA(c, cudaMemsetAsync(w->uin, 0, (size_t)c->geo.ny * sizeof(double), c->stream));
  return LBM_OK;
}

// Dense host doubles <-> typed device planes (through the context's staging buffer).
lbm_status upload_planes(lbm_ctx* c, const double* src, void* dst, int nplanes) {
  const size_t M = (size_t)c->geo.nx * c->geo.ny, es = elem(c);
  for (int p = 0; p < nplanes; ++p) {
    char* d = static_cast<char*>(dst) + (size_t)p * c->geo.plane * es;
    if (!src) {
      LBM_CUDA(c, cudaMemsetAsync(d, 0, (size_t)c->geo.plane * es, c->stream));
      continue;
    }
    LBM_CUDA(c, cudaMemcpyAsync(c->dev.stage, src + p * M, M * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    if (aux(c, 2, c->dev.stage, d) < 0) return fail(c, LBM_ECUDA, "plane upload failed");
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
  }
  return LBM_OK;
}
lbm_status download_planes(lbm_ctx* c, const void* src, double* dst, int nplanes) {
  const size_t M = (size_t)c->geo.nx * c->geo.ny, es = elem(c);
  for (int p = 0; p < nplanes && dst; ++p) {
    const char* s = static_cast<const char*>(src) + (size_t)p * c->geo.plane * es;
    if (aux(c, 3, s, c->dev.stage) < 0) return fail(c, LBM_ECUDA, "plane download failed");
    LBM_CUDA(c, cudaMemcpyAsync(dst + p * M, c->dev.stage, M * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
  }
  return LBM_OK;
}
lbm_status side_io(lbm_ctx* c, void* dev, double* host, bool up) {
  const size_t n = 3 * (size_t)c->geo.ny;
  if (c->f64) {
    if (up) LBM_CUDA(c, cudaMemcpyAsync(dev, host, n * 8, cudaMemcpyHostToDevice, c->stream));
    else LBM_CUDA(c, cudaMemcpyAsync(host, dev, n * 8, cudaMemcpyDeviceToHost, c->stream));
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
  }
  std::vector<float> t(n);
  if (up) {
    for (size_t i = 0; i < n; ++i) t[i] = (float)host[i];
    LBM_CUDA(c, cudaMemcpyAsync(dev, t.data(), n * 4, cudaMemcpyHostToDevice, c->stream));
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
  } else {
    LBM_CUDA(c, cudaMemcpyAsync(t.data(), dev, n * 4, cudaMemcpyDeviceToHost, c->stream));
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    for (size_t i = 0; i < n; ++i) host[i] = t[i];
  }
  return LBM_OK;
}

// gw (pitched doubles) -> dense host array; uin rows -> their sum.
lbm_status read_params(lbm_ctx* c, lbm_adjoint_work* w, std::vector<double>& gw, double& duin) {
  const lbm::Geo& g = c->geo;
  gw.assign((size_t)g.nx * g.ny, 0.0);
  std::vector<double> u(g.ny);
  LBM_CUDA(c, cudaMemcpy2DAsync(gw.data(), g.nx * sizeof(double), w->gw, g.pitch * sizeof(double),
                                g.nx * sizeof(double), g.ny, cudaMemcpyDeviceToHost, c->stream));
  LBM_CUDA(c, cudaMemcpyAsync(u.data(), w->uin, g.ny * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  LBM_CUDA(c, cudaStreamSynchronize(c->stream));
  duin = 0.0;
  for (double v : u) duin += v;
  return LBM_OK;
}

lbm_status check_adjoint_ctx(lbm_ctx* c) {
  if (c->batch_owned) return fail(c, LBM_ESTATE, "this domain belongs to a batch");
  if (!c->prm.energy) return fail(c, LBM_EINVAL, "the adjoint needs the energy equation (energy = 1)");
  if (c->dom.walls != 0 || c->prm.body_fx != 0.0)
    return fail(c, LBM_EINVAL, "the adjoint differentiates the cylinder flow: no flat walls, no body force");
  if (c->prm.collision != LBM_COLL_CM) return fail(c, LBM_EINVAL, "the adjoint differentiates the CM collision");
  if (!c->f64 && c->prm.storage != LBM_STORE_F32)
    return fail(c, LBM_EINVAL, "the FP32 adjoint needs storage = LBM_STORE_F32");
  if (c->steps < c->prm.warmup_steps)
    return fail(c, LBM_ESTATE, "the adjoint needs every step to apply the force (step %lld < warm-up %lld)",
                (long long)c->steps, (long long)c->prm.warmup_steps);
  return LBM_OK;
}

}  // namespace

namespace lbm {
namespace host {
void adjoint_release(lbm_ctx* c) {
  if (!c->adjw) return;
  cudaStreamSynchronize(c->stream);
  for (auto& kv : c->adjw->graphs) cudaGraphExecDestroy(kv.second);
  if (c->adjw->gs) {
    cudaStreamSynchronize(c->adjw->gs);
    cudaStreamDestroy(c->adjw->gs);
  }
  if (c->adjw->ev_in) cudaEventDestroy(c->adjw->ev_in);
  if (c->adjw->ev_out) cudaEventDestroy(c->adjw->ev_out);
  for (void* p : c->adjw->blocks) {
    if (c->has_alloc) c->alloc.free(p, c->alloc.user);
    else cudaFree(p);
  }
  delete c->adjw;
  c->adjw = nullptr;
}
}  // namespace host
}  // namespace lbm

extern "C" {

lbm_status lbm_adjoint_step(lbm_ctx* c, const double* fb, const double* Tb, const double* sb, double q_weight,
                            double* fb_out, double* Tb_out, double* sb_out, double* dJ_dTw, double* dJ_du_in) {
  if (!c) return LBM_EINVAL;
  lbm_status st = check_adjoint_ctx(c);
  if (st != LBM_OK) return st;
  if ((st = prepare(c, 1, 0)) != LBM_OK) return st;
  lbm_adjoint_work* w = c->adjw;
  if ((st = copy_state(c, w->sf[0], w->sT[0], w->sside[0], false)) != LBM_OK) return st;
  if (forward_slot(c, w, 0, c->stream) < 0) return fail(c, LBM_ECUDA, "forward step of the adjoint failed");
  if ((st = zero_adjoint(c, w, 0)) != LBM_OK) return st;
  if ((st = upload_planes(c, fb, w->fb[0], 9)) != LBM_OK) return st;
  if ((st = upload_planes(c, Tb, w->Tb[0], 1)) != LBM_OK) return st;
  if (sb && (st = side_io(c, w->sb[0], const_cast<double*>(sb), true)) != LBM_OK) return st;
  const double wq = c->dev.nb > 0 ? q_weight / c->dev.nb : 0.0;
  if (reverse_slot(c, w, 0, 0, wq, c->stream) < 0) return fail(c, LBM_ECUDA, "reverse step failed");
  if ((st = download_planes(c, w->fb[1], fb_out, 9)) != LBM_OK) return st;
  if ((st = download_planes(c, w->Tb[1], Tb_out, 1)) != LBM_OK) return st;
  if (sb_out && (st = side_io(c, w->sb[1], sb_out, false)) != LBM_OK) return st;
  std::vector<double> gw;
  double duin;
  if ((st = read_params(c, w, gw, duin)) != LBM_OK) return st;
  if (dJ_dTw) std::memcpy(dJ_dTw, gw.data(), gw.size() * sizeof(double));
  if (dJ_du_in) *dJ_du_in = duin;
  return check_status(c);
}

lbm_status lbm_adjoint_window(lbm_ctx* c, int64_t n, int32_t ckpt_every, lbm_window_grad* out) {
  if (!c || !out) return LBM_EINVAL;
  if (n < 1 || ckpt_every < 1) return fail(c, LBM_EINVAL, "n_steps and ckpt_every must be >= 1");
  lbm_status st = check_adjoint_ctx(c);
  if (st != LBM_OK) return st;
  const int K = (int)std::min<int64_t>(ckpt_every, n);
  const int nseg = (int)((n + K - 1) / K);
  if ((st = prepare(c, K, nseg)) != LBM_OK) return st;
  lbm_adjoint_work* w = c->adjw;
  // forward: the wall at its temperature, then the segments with their checkpoints
  if (aux(c, 0, c->wallT, c->dev.T[c->tcur]) < 0) return fail(c, LBM_ECUDA, "wall reset failed");
  c->psi_pending = 0;  // T at the wall may have changed
  double hf0[4], hf1[4];
  LBM_CUDA(c, cudaMemcpyAsync(hf0, c->dev.hf, sizeof(hf0), cudaMemcpyDeviceToHost, c->stream));
  for (int s = 0; s < nseg; ++s) {
    if ((st = copy_state(c, w->cf[s], w->cT[s], w->cside[s], false)) != LBM_OK) return st;
    if ((st = lbm_step(c, std::min<int64_t>(K, n - (int64_t)s * K))) != LBM_OK) return st;
  }
  LBM_CUDA(c, cudaMemcpyAsync(hf1, c->dev.hf, sizeof(hf1), cudaMemcpyDeviceToHost, c->stream));
  if ((st = check_status(c)) != LBM_OK) return st;
  out->J = (hf1[1] - hf0[1]) / (double)n;
  // reverse: segments last to first, each recomputed from its checkpoint
  const double wq = c->dev.nb > 0 ? 1.0 / ((double)n * c->dev.nb) : 0.0;
  int ping = 0;
  if ((st = zero_adjoint(c, w, 0)) != LBM_OK) return st;
  for (int s = nseg - 1; s >= 0; --s) {
    const int len = (int)std::min<int64_t>(K, n - (int64_t)s * K);
    if ((st = copy_slot(c, w->sf[0], w->sT[0], w->sside[0], w->cf[s], w->cT[s], w->cside[s])) != LBM_OK) return st;
    if ((st = segment_graph(c, w, len, ping, wq)) != LBM_OK) return st;
    ping ^= len & 1;
    c->launches += 7 * (int64_t)len + 1;
  }
  if (aux(c, 1, w->Tb[ping], w->gw) < 0) return fail(c, LBM_ECUDA, "wall seed failed");
  std::vector<double> gw;
  double duin;
  if ((st = read_params(c, w, gw, duin)) != LBM_OK) return st;
  if ((st = check_status(c)) != LBM_OK) return st;
  double sum = 0.0;  // gw is zero away from the solid nodes
  for (double v : gw) sum += v;
  out->dJ_dsuperheat = c->Tc * sum;
  out->dJ_du_in = duin;
  if (out->dJ_dwall_dT && c->n_wall > 0) {
    std::fill(out->dJ_dwall_dT, out->dJ_dwall_dT + c->n_wall, 0.0);
    for (size_t k = 0; k < c->wall_node.size(); ++k) {
      const double v = c->Tc * gw[c->wall_node[k]];
      out->dJ_dwall_dT[c->wall_k0[k]] += (1.0 - c->wall_t[k]) * v;
      out->dJ_dwall_dT[c->wall_k1[k]] += c->wall_t[k] * v;
    }
  }
  if (out->dJ_dTw) std::memcpy(out->dJ_dTw, gw.data(), gw.size() * sizeof(double));
  return LBM_OK;
}

}  // extern "C"
