// Host side of the C ABI declared in include/lbm.h: parameter validation, the
// derived thermodynamic constants (Peng-Robinson EOS and Maxwell's rule, Sec. II.C and
// Sec. III.D of arXiv:1912.02018), the cylinder geometry tables (Sec. IV.A), device
// memory, the step loop and state I/O.  All compute of a step runs in the kernels of
// lbm_kernels.cuh; nothing here falls back to the CPU.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "lbm.h"
#include "lbm_internal.h"
#include "lbm_ctx.h"

namespace lbm {
const char* const kKernelNames[kNumKernels] = {"k_rho_psi", "k_collide", "k_energy", "k_export", "k_import"};
}  // namespace lbm

namespace {

thread_local std::string g_create_error;

// ---------------------------------------------------------------- thermodynamics (host, FP64)
// Peng-Robinson EOS, Eq. (eos): p = rho R T/(1 - b rho) - a phi(T) rho^2/(1 + 2 b rho - b^2 rho^2).
struct PengRobinson {
  double a, b, R, kappa, Tc;

  double phi(double T) const {
    double s = 1.0 + kappa * (1.0 - std::sqrt(T / Tc));
    return s * s;
  }
  double p(double rho, double T) const {
    return rho * R * T / (1.0 - b * rho) - a * phi(T) * rho * rho / (1.0 + 2.0 * b * rho - b * b * rho * rho);
  }
  double dp_drho(double rho, double T) const {
    double D = 1.0 + 2.0 * b * rho - b * b * rho * rho;
    double dD = 2.0 * b - 2.0 * b * b * rho;
    double x = 1.0 - b * rho;
    return R * T / (x * x) - a * phi(T) * (2.0 * rho * D - rho * rho * dD) / (D * D);
  }
  // Antiderivative of p with respect to the specific volume v = 1/rho:
  // int RT/(v-b) dv = RT ln(v-b);  int dv/((v+b)^2 - 2b^2) = ln((v+b-sqrt2 b)/(v+b+sqrt2 b)) / (2 sqrt2 b).
  double p_dv(double v, double T) const {
    const double s2 = std::sqrt(2.0);
    return R * T * std::log(v - b) - a * phi(T) / (2.0 * s2 * b) * std::log((v + b - s2 * b) / (v + b + s2 * b));
  }
  // Density where p = target on a monotonic branch [lo, hi] (bisection to the last bit).
  double branch_root(double target, double lo, double hi, double T) const {
    double flo = p(lo, T) - target;
    for (int it = 0; it < 200; ++it) {
      double mid = 0.5 * (lo + hi);
      if (mid <= lo || mid >= hi) break;
      double fm = p(mid, T) - target;
      if ((fm < 0.0) == (flo < 0.0)) {
        lo = mid;
        flo = fm;
      } else {
        hi = mid;
      }
    }
    return 0.5 * (lo + hi);
  }
  // Maxwell's equal-area rule: p(rho_v) = p(rho_l) = p_s and int_{v_l}^{v_v} p dv = p_s (v_v - v_l).
  bool maxwell(double T, double& rho_v, double& rho_l, double& p_s) const {
    const int n = 4000;
    const double top = 1.0 / b;
    double roots[2];
    int nr = 0;
    double prev = dp_drho(0.5 / n * top, T);
    for (int k = 1; k < n && nr < 2; ++k) {
      double r1 = (k + 0.5) / n * top;
      double cur = dp_drho(r1, T);
      if ((cur < 0.0) != (prev < 0.0)) {
        double lo = (k - 0.5) / n * top, hi = r1, flo = prev;
        for (int it = 0; it < 200; ++it) {
          double mid = 0.5 * (lo + hi);
          if (mid <= lo || mid >= hi) break;
          double fm = dp_drho(mid, T);
          if ((fm < 0.0) == (flo < 0.0)) {
            lo = mid;
            flo = fm;
          } else {
            hi = mid;
          }
        }
        roots[nr++] = 0.5 * (lo + hi);
      }
      prev = cur;
    }
    if (nr != 2) return false;
    const double ra = roots[0], rb = roots[1];
    const double p_hi = p(ra, T);
    double p_lo = p(rb, T);
    if (p_lo < 1e-10 * p_hi) p_lo = 1e-10 * p_hi;
    auto area = [&](double ps, double& rv, double& rl) {
      rv = branch_root(ps, 0.0, ra, T);
      rl = branch_root(ps, rb, (1.0 - 1e-12) * top, T);
      double vv = 1.0 / rv, vl = 1.0 / rl;
      return (p_dv(vv, T) - p_dv(vl, T)) - ps * (vv - vl);
    };
    double lo = p_lo + 1e-14 * (p_hi - p_lo), hi = p_hi - 1e-14 * (p_hi - p_lo), rv, rl;
    double alo = area(lo, rv, rl);
    for (int it = 0; it < 200; ++it) {
      double mid = 0.5 * (lo + hi);
      if (mid <= lo || mid >= hi) break;
      double am = area(mid, rv, rl);
      if ((am < 0.0) == (alo < 0.0)) {
        lo = mid;
        alo = am;
      } else {
        hi = mid;
      }
    }
    p_s = 0.5 * (lo + hi);
    area(p_s, rho_v, rho_l);
    return rho_v > 0.0 && rho_l > rho_v;
  }
};

}  // namespace

struct lbm_batch {
  std::vector<lbm_ctx*> ctx;
  cudaStream_t stream = nullptr;   // the caller's stream
  cudaStream_t gstream = nullptr;  // capture and replay stream of the graphs
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  bool f64 = false;
  int variant = 0;
  int cur = 0, tcur = 0;
  long long steps = 0, max_warmup = 0;
  std::vector<lbm::BatchDomain> h_doms;
  lbm::BatchDomain* d_doms = nullptr;
  int* d_maps = nullptr;  // psi map, collision map, energy map (each at most max_tiles)
  int max_tiles = 0;
  int nb_psi = 0, nb_coll = 0, nb_en = 0;
  bool use_graph = true;
  cudaGraphExec_t gexec = nullptr;
  int g_cur = -1, g_tcur = -1, g_variant = -1;
  int g_launches[2] = {0, 0};    // launches of the two captured steps
  std::vector<void*> psi_buf[2]; // per domain: psi of the state with population parity 0 / 1
  std::vector<lbm::DomainMaps> hmaps;  // per domain: tensor maps for the current tile variant
  std::string err = "no error";
};

namespace lbm {
namespace host {

lbm_status fail(lbm_ctx* ctx, lbm_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (ctx) ctx->err = buf;
  else g_create_error = buf;
  return st;
}

void* dalloc(lbm_ctx* c, size_t bytes) {
  bytes = (bytes + 255) & ~size_t(255);
  void* p = nullptr;
  if (c->has_alloc) {
    p = c->alloc.alloc(bytes, c->alloc.user);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) {
    c->blocks.push_back(p);
    c->bytes += bytes;
  }
  return p;
}

void dfree_all(lbm_ctx* c) {
  for (void* p : c->blocks) {
    if (c->has_alloc) c->alloc.free(p, c->alloc.user);
    else cudaFree(p);
  }
  c->blocks.clear();
  c->bytes = 0;
  adjoint_release(c);
}

lbm_status check_status(lbm_ctx* c) {
  int st = 0;
  LBM_CUDA(c, cudaMemcpyAsync(&st, c->dev.status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  LBM_CUDA(c, cudaStreamSynchronize(c->stream));
  if (st & 1) return fail(c, LBM_EUNSTABLE, "non-finite or non-positive density or velocity in the collision");
  if (st & 2) return fail(c, LBM_EUNSTABLE, "pseudopotential radicand <= 0 (Eq. potential) at some node");
  if (st & lbm::kStatusTimeoutCollide)
    return fail(c, LBM_ETIMEOUT, "a collision tile's shared-memory copy did not complete in time");
  if (st & lbm::kStatusTimeoutEnergy)
    return fail(c, LBM_ETIMEOUT, "an energy tile's shared-memory copy did not complete in time");
  return LBM_OK;
}

// A restored state supersedes the one that latched a fault: clear the fault bits and the
// heat-flux bookkeeping of the energy pass (a tile stopped by a timed-out wait leaves its
// completion counter short).
void clear_latched(lbm_ctx* c) {
  const lbm::Dev& d = c->dev;
  cudaMemsetAsync(d.status, 0, sizeof(int), c->stream);
  cudaMemsetAsync(d.counter, 0, sizeof(unsigned), c->stream);
  cudaMemsetAsync(d.partial, 0, sizeof(double) * lbm::energy_blocks(c->geo.nx, c->geo.ny), c->stream);
}

}  // namespace host
}  // namespace lbm

namespace {

using namespace lbm::host;

void hook_before(void* self, int k) {
  lbm_ctx* c = static_cast<lbm_ctx*>(self);
  cudaEvent_t e;
  if (!c->pool.empty()) {
    e = c->pool.back();
    c->pool.pop_back();
  } else {
    cudaEventCreate(&e);
  }
  cudaEventRecord(e, c->stream);
  c->open_ev = e;
  (void)k;
}

void hook_after(void* self, int k) {
  lbm_ctx* c = static_cast<lbm_ctx*>(self);
  cudaEvent_t e;
  if (!c->pool.empty()) {
    e = c->pool.back();
    c->pool.pop_back();
  } else {
    cudaEventCreate(&e);
  }
  cudaEventRecord(e, c->stream);
  c->pending.push_back({k, c->open_ev, e});
}

int do_export(lbm_ctx* c, int which, double* dst) {
  return c->f64 ? lbm::export_f64(c->geo, c->ph, c->dev, c->cur, c->tcur, which, dst, c->stream)
                : lbm::export_f32(c->geo, c->ph, c->dev, c->cur, c->tcur, which, c->prm.storage, dst, c->stream);
}
int do_import(lbm_ctx* c, int which, const double* src) {
  return c->f64 ? lbm::import_f64(c->geo, c->ph, c->dev, c->cur, c->tcur, which, src, c->stream)
                : lbm::import_f32(c->geo, c->ph, c->dev, c->cur, c->tcur, which, c->prm.storage, src, c->stream);
}

}  // namespace

using namespace lbm::host;

extern "C" {

lbm_status lbm_create(const lbm_domain* domain, const lbm_cylinder* cyl, const lbm_params* params,
                      const lbm_init* init, const lbm_allocator* alloc, void* cuda_stream, lbm_ctx** out) {
  g_create_error = "no error";
  if (!domain || !cyl || !params || !out) return fail(nullptr, LBM_EINVAL, "NULL domain, cylinder, params or out");
  *out = nullptr;
  const lbm_domain& D = *domain;
  const lbm_params& P = *params;
  if (D.nx < 5 || D.ny < 5) return fail(nullptr, LBM_EINVAL, "nx and ny must be >= 5 (got %d x %d)", D.nx, D.ny);
  if (9ll * D.ny * ((D.nx + 31) / 32 * 32) >= (1ll << 31))
    return fail(nullptr, LBM_EINVAL, "lattice too large: 9 ny pitch must stay below 2^31");
  if (P.compute_f64 && P.storage != LBM_STORE_F64)
    return fail(nullptr, LBM_EINVAL, "compute_f64 = 1 needs storage = LBM_STORE_F64");
  if (!P.compute_f64 && P.storage != LBM_STORE_F32 && P.storage != LBM_STORE_F64 && P.storage != LBM_STORE_F16S)
    return fail(nullptr, LBM_EINVAL, "storage must be LBM_STORE_F64, LBM_STORE_F32 or LBM_STORE_F16S");
  if (P.psi_mode < 0 || P.psi_mode > 2) return fail(nullptr, LBM_EINVAL, "psi_mode must be 0, 1 or 2");
  if (D.walls & ~3) return fail(nullptr, LBM_EINVAL, "walls takes bit 0 (x = 0) and bit 1 (y = 0, ny-1) only");
  if ((D.walls & 1) && D.periodic_x) return fail(nullptr, LBM_EINVAL, "a wall at x = 0 needs periodic_x = 0");
  if (!std::isfinite(P.body_fx)) return fail(nullptr, LBM_EINVAL, "body_fx must be finite");
  if (P.collision != LBM_COLL_CM && P.collision != LBM_COLL_BGK)
    return fail(nullptr, LBM_EINVAL, "collision must be LBM_COLL_CM (0) or LBM_COLL_BGK (1)");
  if (P.reserved != 0) return fail(nullptr, LBM_EINVAL, "lbm_params.reserved must be 0");
  if (!(P.a > 0 && P.b > 0 && P.R > 0)) return fail(nullptr, LBM_EINVAL, "EOS constants a, b, R must be > 0");
  if (P.G > 0) return fail(nullptr, LBM_EINVAL, "G must be <= 0 (Eq. potential needs G < 0; 0 = single phase)");
  if (!(P.Tr_sat > 0 && P.Tr_sat < 1)) return fail(nullptr, LBM_EINVAL, "Tr_sat must lie in (0, 1)");
  if (!(P.c_v > 0 && P.Pr_l > 0 && P.Pr_v > 0 && P.nu_ratio > 0))
    return fail(nullptr, LBM_EINVAL, "c_v, Pr_l, Pr_v and nu_ratio must be > 0");
  const bool has_cyl = cyl->D > 0;
  if (has_cyl) {
    const double r = 0.5 * cyl->D;
    if (!D.periodic_x && (cyl->xc - r < 3.0 || cyl->xc + r > D.nx - 4.0))
      return fail(nullptr, LBM_EINVAL, "cylinder must stay 3 nodes away from the inlet and outlet");
    if (2.0 * r + 4.0 > D.ny) return fail(nullptr, LBM_EINVAL, "cylinder does not fit across the channel");
  }

  lbm_ctx* c = new lbm_ctx();
  c->dom = D;
  c->cyl = *cyl;
  c->prm = P;
  c->f64 = P.compute_f64 != 0;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  if (alloc && alloc->alloc && alloc->free) {
    c->alloc = *alloc;
    c->has_alloc = true;
  }
  cudaGetDevice(&c->device);

  // derived constants, Sec. II.C and Sec. IV.A
  PengRobinson eos;
  eos.a = P.a;
  eos.b = P.b;
  eos.R = P.R;
  eos.kappa = 0.37464 + 1.54226 * P.acentric - 0.26992 * P.acentric * P.acentric;
  eos.Tc = 0.0778 * P.a / (0.4572 * P.b * P.R);
  c->Tc = eos.Tc;
  c->pc = 0.0778 * P.R * eos.Tc / P.b;
  const double T_sat = P.Tr_sat * eos.Tc;
  const double T_wall = T_sat + cyl->superheat_Tc * eos.Tc;
  double rho_v, rho_l, p_s;
  if (!eos.maxwell(T_sat, rho_v, rho_l, p_s)) {
    delete c;
    return fail(nullptr, LBM_EINVAL, "no liquid-vapour coexistence at T_sat = %g", T_sat);
  }
  c->p_sat = p_s;
  {
    // latent heat from the EOS (Sec. IV.A), read as Clausius-Clapeyron: h_fg = T (1/rho_v - 1/rho_l)
    // dp_sat/dT, the slope of the coexistence pressure by a central difference (steps of 1e-5 T)
    double rv, rl, pp, pm;
    const double dT = 1e-5 * T_sat;
    c->h_fg = (eos.maxwell(T_sat + dT, rv, rl, pp) && eos.maxwell(T_sat - dT, rv, rl, pm))
                  ? T_sat * (1.0 / rho_v - 1.0 / rho_l) * (pp - pm) / (2.0 * dT)
                  : 0.0;
  }
  lbm::Phys& phys = c->ph;
  lbm::PhysC<double>& ph = phys.d;
  ph.a = P.a;
  ph.b = P.b;
  ph.R = P.R;
  ph.kappa = eos.kappa;
  ph.Tc = eos.Tc;
  ph.G = P.G;
  ph.sigma = P.sigma;
  ph.T_sat = T_sat;
  ph.T_wall = T_wall;
  ph.rho_l = rho_l;
  ph.rho_v = rho_v;
  ph.rho_s = cyl->rho_solid > 0 ? cyl->rho_solid : rho_l;
  ph.nu_l = P.nu_l > 0 ? P.nu_l : (P.Re > 0 ? P.u_in * cyl->D / P.Re : 0.0);
  ph.nu_v = ph.nu_l / P.nu_ratio;
  ph.alpha_l = ph.nu_l / P.Pr_l;
  ph.alpha_v = ph.nu_v / P.Pr_v;
  ph.c_v = P.c_v;
  ph.g = P.g >= 0 ? P.g : (has_cyl ? P.u_in * P.u_in / (16.0 * cyl->D) : 0.0);
  ph.body_fx = P.body_fx;
  ph.u_in = P.u_in;
  ph.U_out = P.outlet_U >= 0 ? P.outlet_U : P.u_in;
  ph.U_k = ph.U_out / (1.0 + ph.U_out);
  c->lambda_v = rho_v * P.c_v * ph.alpha_v;
  {
    lbm::PhysC<float>& pf = phys.f;
    pf.a = (float)ph.a, pf.b = (float)ph.b, pf.R = (float)ph.R, pf.kappa = (float)ph.kappa, pf.Tc = (float)ph.Tc;
    pf.G = (float)ph.G, pf.sigma = (float)ph.sigma, pf.T_sat = (float)ph.T_sat, pf.T_wall = (float)ph.T_wall;
    pf.rho_l = (float)ph.rho_l, pf.rho_v = (float)ph.rho_v, pf.rho_s = (float)ph.rho_s;
    pf.nu_l = (float)ph.nu_l, pf.nu_v = (float)ph.nu_v, pf.alpha_l = (float)ph.alpha_l, pf.alpha_v = (float)ph.alpha_v;
    pf.c_v = (float)ph.c_v, pf.g = (float)ph.g, pf.u_in = (float)ph.u_in, pf.U_out = (float)ph.U_out;
    pf.U_k = (float)ph.U_k;
    pf.body_fx = (float)ph.body_fx;
  }
  auto split = [](double v) {
    lbm::F2 r;
    r.hi = (float)v;
    r.lo = (float)(v - (double)r.hi);
    return r;
  };
  phys.a2 = split(P.a);
  phys.b2 = split(P.b);
  phys.R2 = split(P.R);
  phys.kappa2 = split(eos.kappa);
  phys.K12 = split(1.0 + eos.kappa);
  phys.invTc2 = split(1.0 / eos.Tc);
  phys.cs22 = split(1.0 / 3.0);
  phys.k2 = split(P.G != 0 ? 2.0 / (P.G * (1.0 / 3.0)) : 0.0);
  {
    const double k = P.G != 0 ? 2.0 / (P.G * (1.0 / 3.0)) : 0.0;
    phys.kR2 = split(k * P.R);
    phys.ka2 = split(k * P.a);
    phys.k32 = split(k / 3.0);
  }
  phys.dpdT_c1 = (float)(eos.kappa * (1.0 + eos.kappa));
  phys.dpdT_c2 = (float)(eos.kappa * eos.kappa / eos.Tc);
  {
    static const double W[9] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                                1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
    for (int i = 0; i < 9; ++i) phys.pop_shift[i] = (float)(W[i] * rho_l);
  }
  for (double nu : {ph.nu_l, ph.nu_v}) {
    const double omega = 1.0 / (nu * 3.0 + 0.5);
    if (!(nu > 0) || !(omega > 0 && omega < 2)) {
      delete c;
      return fail(nullptr, LBM_EINVAL, "relaxation rate outside (0, 2): nu_l = %g, nu_v = %g", ph.nu_l, ph.nu_v);
    }
  }
  if (P.G != 0) {
    const double cs2 = 1.0 / 3.0;
    for (double T : {T_sat, T_wall})
      for (int k = 0; k <= 64; ++k) {
        const double r = rho_v + (rho_l - rho_v) * k / 64.0;
        if (!((eos.p(r, T) - r * cs2) / (P.G * cs2) > 0)) {
          delete c;
          return fail(nullptr, LBM_EINVAL, "psi radicand <= 0 at rho = %g, T = %g (Eq. potential)", r, T);
        }
      }
  }

  // geometry
  lbm::Geo& g = c->geo;
  g.nx = D.nx;
  g.ny = D.ny;
  g.pitch = (D.nx + 31) / 32 * 32;
  g.periodic_x = D.periodic_x ? 1 : 0;
  g.plane = g.ny * g.pitch;
  g.xc = cyl->xc;
  g.yc = cyl->yc;
  g.r = has_cyl ? 0.5 * cyl->D : -1.0;
  const long long plane = g.plane;
  std::vector<uint8_t> mask(plane, 0);
  auto cyl_at = [&](int x, int y) {
    if (!has_cyl) return false;
    double dx = x - g.xc, dy = y - g.yc;
    return dx * dx + dy * dy <= g.r * g.r;
  };
  // the flat walls: the column x = 0 (bit 0) and the rows y = 0, ny - 1 (bit 1)
  auto solid_at = [&](int x, int y) {
    return ((D.walls & 1) && x == 0) || ((D.walls & 2) && (y == 0 || y == g.ny - 1)) || cyl_at(x, y);
  };
  for (int y = 0; y < g.ny; ++y)
    for (int x = 0; x < g.nx; ++x)
      if (solid_at(x, y)) mask[(long long)y * g.pitch + x] = lbm::kSolid;
  std::vector<int> bnode;
  std::vector<double> bnx, bny;
  static const int CX[9] = {0, 1, -1, 0, 0, 1, -1, 1, -1};
  static const int CY[9] = {0, 0, 0, 1, -1, 1, -1, -1, 1};
  for (int y = 0; y < g.ny; ++y)
    for (int x = 0; x < g.nx; ++x) {
      const long long id = (long long)y * g.pitch + x;
      if (mask[id] & lbm::kSolid) continue;
      bool near = false, near_cyl = false;
      for (int i = 1; i < 9; ++i) {
        int sx = x - CX[i], sy = (y - CY[i] + g.ny) % g.ny;
        if (g.periodic_x) sx = (sx + g.nx) % g.nx;
        if (sx < 0 || sx >= g.nx) continue;
        if (mask[(long long)sy * g.pitch + sx] & lbm::kSolid) {
          near = true;
          near_cyl = near_cyl || cyl_at(sx, sy);
        }
      }
      if (near) {
        // outward normal: from the cylinder centre, else that of the flat wall
        mask[id] |= lbm::kNearWall;
        double nxv = 1.0, nyv = 0.0;
        if ((D.walls & 2) && y == 1) nxv = 0.0, nyv = 1.0;
        if ((D.walls & 2) && y == g.ny - 2) nxv = 0.0, nyv = -1.0;
        if (near_cyl) {
          double dx = x - g.xc, dy = y - g.yc, rr = std::sqrt(dx * dx + dy * dy);
          nxv = dx / rr;
          nyv = dy / rr;
        }
        bnode.push_back((int)id);
        bnx.push_back(nxv);
        bny.push_back(nyv);
      }
    }

  // link fractions of the near-wall nodes (Bouzidi), in double with the device's operation order
  std::vector<int> widx(plane, -1);
  std::vector<double> wq;
  for (int y = 0; y < g.ny; ++y)
    for (int x = 0; x < g.nx; ++x) {
      const long long id = (long long)y * g.pitch + x;
      if (!(mask[id] & lbm::kNearWall)) continue;
      widx[id] = (int)(wq.size() / 8);
      for (int i = 1; i < 9; ++i) {
        int sx = x - CX[i], sy = (y - CY[i] + g.ny) % g.ny;
        if (g.periodic_x) sx = (sx + g.nx) % g.nx;
        double q = -1.0;
        if (sx >= 0 && sx < g.nx && (mask[(long long)sy * g.pitch + sx] & lbm::kSolid) && !cyl_at(sx, sy)) {
          q = 0.5;  // a flat wall's surface lies halfway between its nodes and the fluid's
        } else if (sx >= 0 && sx < g.nx && (mask[(long long)sy * g.pitch + sx] & lbm::kSolid)) {
          const int cx = -CX[i], cy = -CY[i];
          const double dx = x - g.xc, dy = y - g.yc, r = g.r;
          const double A = (double)(cx * cx + cy * cy);
          const double B = dx * cx + dy * cy;
          const double C0 = dx * dx + dy * dy - r * r;
          q = (-B - std::sqrt(B * B - A * C0)) / A;
        }
        wq.push_back(q);
      }
    }

  // fluid nodes with a solid node within 2 nodes in x and y (the adjoint's slow pull path)
  for (int y = 0; y < g.ny; ++y)
    for (int x = 0; x < g.nx; ++x) {
      const long long id = (long long)y * g.pitch + x;
      if (mask[id] & lbm::kSolid) continue;
      bool near2 = false;
      for (int dy = -2; dy <= 2 && !near2; ++dy)
        for (int dx = -2; dx <= 2 && !near2; ++dx) {
          int sx = x + dx;
          const int sy = ((y + dy) % g.ny + g.ny) % g.ny;
          if (g.periodic_x) sx = ((sx % g.nx) + g.nx) % g.nx;
          if (sx < 0 || sx >= g.nx) continue;
          near2 = (mask[(long long)sy * g.pitch + sx] & lbm::kSolid) != 0;
        }
      if (near2) mask[id] |= lbm::kNear2;
    }

  // energy tiles (32 x 8 and 32 x 16) that hold a near-wall node: they alone sum heat flux
  int wall_tiles[2] = {0, 0};
  for (int h = 0; h < 2; ++h) {
    const int TY = h == 0 ? 8 : 16;
    for (int ty = 0; ty * TY < g.ny; ++ty)
      for (int tx = 0; tx * 32 < g.nx; ++tx) {
        bool any = false;
        for (int y = ty * TY; y < std::min(g.ny, ty * TY + TY) && !any; ++y)
          for (int x = tx * 32; x < std::min(g.nx, tx * 32 + 32) && !any; ++x)
            any = (mask[(long long)y * g.pitch + x] & lbm::kNearWall) != 0;
        wall_tiles[h] += any ? 1 : 0;
      }
  }

  // device memory
  const size_t es = c->f64 ? sizeof(double) : sizeof(float);  // compute-type fields
  const size_t ps = P.storage == LBM_STORE_F64 ? 8 : (P.storage == LBM_STORE_F16S ? 2 : 4);  // populations
  const size_t N = (size_t)plane;
  lbm::Dev& d = c->dev;
  d.f[0] = dalloc(c, 9 * N * ps);
  d.f[1] = dalloc(c, 9 * N * ps);
  d.T[0] = dalloc(c, N * es);
  d.T[1] = dalloc(c, N * es);
  d.psi = dalloc(c, N * es);
  d.psi_next = dalloc(c, N * es);
  // rho, u_x, u_y as three consecutive planes: one 3D tensor map stages all three
  d.rho = dalloc(c, 3 * N * es);
  d.ux = d.rho ? static_cast<char*>(d.rho) + N * es : nullptr;
  d.uy = d.rho ? static_cast<char*>(d.rho) + 2 * N * es : nullptr;
  d.side[0] = dalloc(c, 3 * (size_t)g.ny * es);
  d.side[1] = dalloc(c, 3 * (size_t)g.ny * es);
  d.partial = static_cast<double*>(dalloc(c, sizeof(double) * lbm::energy_blocks(g.nx, g.ny)));
  d.counter = static_cast<unsigned*>(dalloc(c, sizeof(unsigned)));
  d.wall_tiles[0] = wall_tiles[0];
  d.wall_tiles[1] = wall_tiles[1];
  uint8_t* dmask = static_cast<uint8_t*>(dalloc(c, N));
  d.mask = dmask;
  d.nb = (int)bnode.size();
  {
    const char* e = std::getenv("LBM_TMA");
    d.tma = (e && e[0] == '0' && e[1] == 0) ? 0 : 1;
  }
  {
    const char* e = std::getenv("LBM_PDL");
    d.pdl = (e && e[0] == '0' && e[1] == 0) ? 0 : 1;
  }
  d.f_ready = 0;
  static_assert(lbm::kCollCM == LBM_COLL_CM && lbm::kCollBGK == LBM_COLL_BGK, "collision operator codes");
  d.collision = P.collision;
  int* dbn = static_cast<int*>(dalloc(c, sizeof(int) * (bnode.size() + 1)));
  double* dbv = static_cast<double*>(dalloc(c, sizeof(double) * (2 * bnode.size() + 1)));
  d.bnode = dbn;
  d.bn = dbv;
  d.hf = static_cast<double*>(dalloc(c, 4 * sizeof(double)));
  d.status = static_cast<int*>(dalloc(c, sizeof(int)));
  int* dwidx = static_cast<int*>(dalloc(c, sizeof(int) * N));
  void* dwq = dalloc(c, es * (wq.size() + 8));
  double* dwn = static_cast<double*>(dalloc(c, sizeof(double) * (2 * bnode.size() + 2)));
  g.wall_idx = dwidx;
  g.wall_q = dwq;
  g.wall_n = dwn;
  // staging planes for host I/O: a whole state (9 populations, T) and the outlet rows in one copy
  d.stage = static_cast<double*>(dalloc(c, sizeof(double) * ((size_t)g.nx * g.ny * 10 + 3 * (size_t)g.ny)));
  if (!d.f[0] || !d.f[1] || !d.T[0] || !d.T[1] || !d.psi || !d.psi_next || !d.rho || !d.ux || !d.uy || !d.side[0] ||
      !d.side[1] || !d.partial || !d.counter || !dmask || !dbn || !dbv || !d.hf || !d.status || !d.stage ||
      !dwidx || !dwq || !dwn) {
    dfree_all(c);
    delete c;
    return fail(nullptr, LBM_ENOMEM, "device allocation failed");
  }
  std::vector<double> bnv(bnx);
  bnv.insert(bnv.end(), bny.begin(), bny.end());
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t r) {
    if (e == cudaSuccess && r != cudaSuccess) e = r;
  };
  chk(cudaMemsetAsync(d.psi, 0, N * es, c->stream));
  chk(cudaMemsetAsync(d.psi_next, 0, N * es, c->stream));
  for (void* p : {d.side[0], d.side[1]}) chk(cudaMemsetAsync(p, 0, 3 * g.ny * es, c->stream));
  chk(cudaMemsetAsync(d.hf, 0, 4 * sizeof(double), c->stream));
  chk(cudaMemsetAsync(d.status, 0, sizeof(int), c->stream));
  chk(cudaMemsetAsync(d.counter, 0, sizeof(unsigned), c->stream));
  chk(cudaMemsetAsync(d.partial, 0, sizeof(double) * lbm::energy_blocks(g.nx, g.ny), c->stream));
  chk(cudaMemcpyAsync(dmask, mask.data(), N, cudaMemcpyHostToDevice, c->stream));
  chk(cudaMemcpyAsync(dwidx, widx.data(), sizeof(int) * N, cudaMemcpyHostToDevice, c->stream));
  std::vector<double> wn;  // near-wall rows are the boundary list in the same order
  for (size_t b = 0; b < bnode.size(); ++b) {
    wn.push_back(bnx[b]);
    wn.push_back(bny[b]);
  }
  if (!wn.empty()) chk(cudaMemcpyAsync(dwn, wn.data(), sizeof(double) * wn.size(), cudaMemcpyHostToDevice, c->stream));
  std::vector<float> wqf(wq.begin(), wq.end());
  if (!wq.empty())
    chk(cudaMemcpyAsync(dwq, c->f64 ? (const void*)wq.data() : (const void*)wqf.data(), es * wq.size(),
                        cudaMemcpyHostToDevice, c->stream));
  if (!bnode.empty()) {
    chk(cudaMemcpyAsync(dbn, bnode.data(), sizeof(int) * bnode.size(), cudaMemcpyHostToDevice, c->stream));
    chk(cudaMemcpyAsync(dbv, bnv.data(), sizeof(double) * bnv.size(), cudaMemcpyHostToDevice, c->stream));
  }
  // optional initial fields, staged through the export buffer (6 dense planes); the sixth holds
  // the wall temperature of the solid nodes when an angular profile is given
  const size_t M = (size_t)g.nx * g.ny;
  std::vector<double> wallT;
  c->cyl.wall_dT = nullptr;  // the knots are used here only
  if (has_cyl && cyl->n_wall > 0 && cyl->wall_dT) {
    wallT.assign(M, ph.T_wall);
    c->n_wall = cyl->n_wall;
    const double two_pi = 2.0 * std::acos(-1.0);
    for (int y = 0; y < g.ny; ++y)
      for (int x = 0; x < g.nx; ++x) {
        if (!cyl_at(x, y)) continue;  // the profile is the cylinder's; flat walls stay at T_w
        double s = std::atan2(y - g.yc, x - g.xc) / two_pi;
        if (s < 0.0) s += 1.0;
        const double pos = s * cyl->n_wall, fl = std::floor(pos), t = pos - fl;
        const int k0 = ((int)fl) % cyl->n_wall, k1 = (k0 + 1) % cyl->n_wall;
        const double dlt = (1.0 - t) * cyl->wall_dT[k0] + t * cyl->wall_dT[k1];
        wallT[(size_t)y * g.nx + x] = ph.T_wall + dlt * eos.Tc;
        c->wall_node.push_back(y * g.nx + x);
        c->wall_k0.push_back(k0);
        c->wall_k1.push_back(k1);
        c->wall_t.push_back(t);
      }
  }
  const double* src[6] = {init ? init->rho : nullptr, init ? init->drho : nullptr, init ? init->ux : nullptr,
                          init ? init->uy : nullptr, init ? init->T : nullptr,
                          wallT.empty() ? nullptr : wallT.data()};
  const double* dsrc[6] = {};
  for (int k = 0; k < 6; ++k)
    if (src[k]) {
      chk(cudaMemcpyAsync(d.stage + k * M, src[k], M * sizeof(double), cudaMemcpyHostToDevice, c->stream));
      dsrc[k] = d.stage + k * M;
    }
  const int ok = c->f64 ? lbm::init_f64(g, phys, d, dsrc[0], dsrc[1], dsrc[2], dsrc[3], dsrc[4], dsrc[5], P.seed,
                                        P.noise_amp, c->stream)
                        : lbm::init_f32(g, phys, d, dsrc[0], dsrc[1], dsrc[2], dsrc[3], dsrc[4], dsrc[5], P.seed,
                                        P.noise_amp, P.storage, c->stream);
  if (ok < 0) chk(cudaGetLastError());
  chk(cudaMemcpyAsync(d.f[1], d.f[0], 9 * N * ps, cudaMemcpyDeviceToDevice, c->stream));
  chk(cudaMemcpyAsync(d.T[1], d.T[0], N * es, cudaMemcpyDeviceToDevice, c->stream));
  chk(cudaMemcpyAsync(d.side[1], d.side[0], 3 * g.ny * es, cudaMemcpyDeviceToDevice, c->stream));
  // the wall temperature of the solid nodes, kept for the adjoint window
  c->wallT = dalloc(c, N * es);
  if (c->wallT) chk(cudaMemcpyAsync(c->wallT, d.T[0], N * es, cudaMemcpyDeviceToDevice, c->stream));
  else chk(cudaErrorMemoryAllocation);
  chk(cudaStreamSynchronize(c->stream));
  if (e != cudaSuccess) {
    std::string m = cudaGetErrorString(e);
    dfree_all(c);
    delete c;
    return fail(nullptr, LBM_ECUDA, "initialisation failed: %s", m.c_str());
  }
  c->launches = 1;
  *out = c;
  return LBM_OK;
}

lbm_status lbm_step(lbm_ctx* c, int64_t n) {
  if (!c) return LBM_EINVAL;
  if (c->batch_owned) return fail(c, LBM_ESTATE, "this domain belongs to a batch; step it with lbm_batch_step");
  if (n < 0) return fail(c, LBM_EINVAL, "negative step count");
  lbm::LaunchHook hook{hook_before, hook_after, c};
  const lbm::LaunchHook* hk = c->prof ? &hook : nullptr;
  int energy_last = 0;
  for (int64_t s = 0; s < n; ++s) {
    const int forcing = c->steps >= c->prm.warmup_steps;
    int flipped = 0;
    // psi of this step may already have been made by the last energy pass (into psi_next)
    if (c->psi_pending) std::swap(c->dev.psi, c->dev.psi_next);
    lbm::PsiChain chain{c->psi_pending, 1, 0};
    // from the second step of a call on, the kernel before the collision is the last step's
    // energy pass, which leaves the populations alone
    c->dev.f_ready = s > 0 && energy_last;
    const int k = c->f64 ? lbm::step_f64(c->geo, c->ph, c->dev, c->cur, c->tcur, forcing, c->prm.energy,
                                         c->prm.psi_mode, c->stream, hk, &flipped, &chain)
                         : lbm::step_f32(c->geo, c->ph, c->dev, c->cur, c->tcur, forcing, c->prm.energy,
                                         c->prm.psi_mode, c->prm.storage, c->stream, hk, &flipped, &chain);
    c->psi_pending = chain.made;
    c->dev.starve = 0;  // the test hook of lbm_inject_fault covers one step
    c->dev.f_ready = 0;
    energy_last = flipped;
    if (k < 0) return fail(c, LBM_ECUDA, "kernel launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    c->launches += k;
    c->cur ^= 1;
    c->tcur ^= flipped;
    c->steps++;
  }
  return LBM_OK;
}

lbm_status lbm_sync(lbm_ctx* c) {
  if (!c) return LBM_EINVAL;
  return check_status(c);
}

lbm_status lbm_wall_heat_flux(lbm_ctx* c, double* q_now, double* q_mean, double* q_std, double* nu_mean,
                              int64_t* n_samples) {
  if (!c) return LBM_EINVAL;
  double hf[4];
  LBM_CUDA(c, cudaMemcpyAsync(hf, c->dev.hf, sizeof(hf), cudaMemcpyDeviceToHost, c->stream));
  lbm_status st = check_status(c);
  if (st != LBM_OK) return st;
  const double cnt = hf[3];
  const double mean = cnt > 0 ? hf[1] / cnt : 0.0;
  double var = cnt > 0 ? hf[2] / cnt - mean * mean : 0.0;
  if (var < 0) var = 0;
  const double dT = c->ph.d.T_wall - c->ph.d.T_sat;
  if (q_now) *q_now = hf[0];
  if (q_mean) *q_mean = mean;
  if (q_std) *q_std = std::sqrt(var);
  if (nu_mean) *nu_mean = (cnt > 0 && dT > 0) ? mean * c->cyl.D / (c->lambda_v * dT) : 0.0;
  if (n_samples) *n_samples = (int64_t)cnt;
  return LBM_OK;
}

lbm_status lbm_reset_heat_flux(lbm_ctx* c) {
  if (!c) return LBM_EINVAL;
  LBM_CUDA(c, cudaMemsetAsync(c->dev.hf, 0, 4 * sizeof(double), c->stream));
  return LBM_OK;
}

lbm_status lbm_fields(lbm_ctx* c, uint32_t mask, void* dst, size_t bytes, int dst_on_device) {
  if (!c || !dst) return LBM_EINVAL;
  const size_t M = (size_t)c->geo.nx * c->geo.ny;
  int planes = 0;
  for (int b = 0; b < 8; ++b) planes += (mask >> b) & 1u;
  if (mask >> 8) return fail(c, LBM_EINVAL, "unknown field bits 0x%x", mask);
  if (bytes < planes * M * sizeof(double)) return fail(c, LBM_EINVAL, "dst too small for %d planes", planes);
  // the force planes are those of the last collision: with forcing unless it was a warm-up step
  const int forcing = c->steps > 0 && c->steps - 1 >= c->prm.warmup_steps;
  // every requested field into its staging plane, then one copy
  int k = 0;
  for (int b = 0; b < 8; ++b) {
    if (!((mask >> b) & 1u)) continue;
    const int which = b < 6 ? b : 30 + (b - 6) + 2 * forcing;
    if (do_export(c, which, c->dev.stage + k * M) < 0) return fail(c, LBM_ECUDA, "export kernel failed");
    c->launches++;
    ++k;
  }
  if (k)
    LBM_CUDA(c, cudaMemcpyAsync(dst, c->dev.stage, k * M * sizeof(double),
                                dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  return check_status(c);
}

lbm_status lbm_get_state(lbm_ctx* c, double* f, double* T, double* side, int64_t* steps) {
  if (!c) return LBM_EINVAL;
  const size_t M = (size_t)c->geo.nx * c->geo.ny;
  double* st = c->dev.stage;
  if (f) {
    for (int i = 0; i < 9; ++i)
      if (do_export(c, 10 + i, st + i * M) < 0) return fail(c, LBM_ECUDA, "export kernel failed");
    LBM_CUDA(c, cudaMemcpyAsync(f, st, 9 * M * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  }
  if (T) {
    if (do_export(c, 3, st + 9 * M) < 0) return fail(c, LBM_ECUDA, "export kernel failed");
    LBM_CUDA(c, cudaMemcpyAsync(T, st + 9 * M, M * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  }
  if (side) {
    for (int j = 0; j < 3; ++j)
      if (do_export(c, 20 + j, st + 10 * M + j * c->geo.ny) < 0) return fail(c, LBM_ECUDA, "export kernel failed");
    LBM_CUDA(c, cudaMemcpyAsync(side, st + 10 * M, 3 * c->geo.ny * sizeof(double), cudaMemcpyDeviceToHost,
                                c->stream));
  }
  if (steps) *steps = c->steps;
  return check_status(c);
}

lbm_status lbm_set_state(lbm_ctx* c, const double* f, const double* T, const double* side, int64_t steps) {
  if (!c) return LBM_EINVAL;
  c->psi_pending = 0;  // the state changes: psi of the next step is no longer known
  clear_latched(c);
  const size_t M = (size_t)c->geo.nx * c->geo.ny;
  double* st = c->dev.stage;
  // one copy per part into the staging planes, then the conversions; the stream orders them
  if (f) {
    LBM_CUDA(c, cudaMemcpyAsync(st, f, 9 * M * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    for (int i = 0; i < 9; ++i)
      if (do_import(c, 10 + i, st + i * M) < 0) return fail(c, LBM_ECUDA, "import kernel failed");
  }
  if (T) {
    LBM_CUDA(c, cudaMemcpyAsync(st + 9 * M, T, M * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    if (do_import(c, 3, st + 9 * M) < 0) return fail(c, LBM_ECUDA, "import kernel failed");
  }
  if (side) {
    LBM_CUDA(c, cudaMemcpyAsync(st + 10 * M, side, 3 * c->geo.ny * sizeof(double), cudaMemcpyHostToDevice,
                                c->stream));
    for (int j = 0; j < 3; ++j)
      if (do_import(c, 20 + j, st + 10 * M + j * c->geo.ny) < 0) return fail(c, LBM_ECUDA, "import kernel failed");
  }
  if (steps >= 0) c->steps = steps;
  return check_status(c);
}

// Native checkpoints: the device layout is [plane][ny][pitch], consecutive planes back to back,
// so a set of planes is one 2D copy of (planes * ny) rows.
static lbm_status native_io(lbm_ctx* c, void* f, void* T, void* side, bool up) {
  const lbm::Geo& g = c->geo;
  const size_t es = c->f64 ? sizeof(double) : sizeof(float);
  const size_t ps = c->prm.storage == LBM_STORE_F64 ? 8 : (c->prm.storage == LBM_STORE_F16S ? 2 : 4);
  const cudaMemcpyKind kind = up ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost;
  auto copy2d = [&](void* host, void* dev, size_t elem, size_t rows) {
    const size_t hp = g.nx * elem, dp = g.pitch * elem;
    return up ? cudaMemcpy2DAsync(dev, dp, host, hp, hp, rows, kind, c->stream)
              : cudaMemcpy2DAsync(host, hp, dev, dp, hp, rows, kind, c->stream);
  };
  if (f) LBM_CUDA(c, copy2d(f, c->dev.f[c->cur], ps, 9 * (size_t)g.ny));
  if (T) LBM_CUDA(c, copy2d(T, c->dev.T[c->tcur], es, g.ny));
  if (side) {
    const size_t b = 3 * (size_t)g.ny * es;
    LBM_CUDA(c, up ? cudaMemcpyAsync(c->dev.side[c->cur], side, b, kind, c->stream)
                   : cudaMemcpyAsync(side, c->dev.side[c->cur], b, kind, c->stream));
  }
  return check_status(c);
}

lbm_status lbm_get_state_native(lbm_ctx* c, void* f, void* T, void* side, int64_t* steps) {
  if (!c) return LBM_EINVAL;
  if (steps) *steps = c->steps;
  return native_io(c, f, T, side, false);
}

lbm_status lbm_set_state_native(lbm_ctx* c, const void* f, const void* T, const void* side, int64_t steps) {
  if (!c) return LBM_EINVAL;
  c->psi_pending = 0;  // the state changes: psi of the next step is no longer known
  clear_latched(c);
  if (steps >= 0) c->steps = steps;
  return native_io(c, const_cast<void*>(f), const_cast<void*>(T), const_cast<void*>(side), true);
}

lbm_status lbm_stage_state_native(lbm_ctx* c, const void* f, const void* T, const void* side, int64_t steps) {
  if (!c || !f || !T) return LBM_EINVAL;
  if (c->batch_owned) return fail(c, LBM_ESTATE, "this domain belongs to a batch");
  const lbm::Geo& g = c->geo;
  const size_t es = c->f64 ? sizeof(double) : sizeof(float);
  const size_t ps = c->prm.storage == LBM_STORE_F64 ? 8 : (c->prm.storage == LBM_STORE_F16S ? 2 : 4);
  const size_t N = (size_t)g.plane;
  if (!c->copy_stream) {
    c->stage_f = dalloc(c, 9 * N * ps);
    c->stage_T = dalloc(c, N * es);
    c->stage_side = dalloc(c, 3 * (size_t)g.ny * es);
    if (!c->stage_f || !c->stage_T || !c->stage_side)
      return fail(c, LBM_ENOMEM, "device allocation of the staging buffers failed");
    // the pitch's padding columns are never read; zero them once all the same
    LBM_CUDA(c, cudaMemsetAsync(c->stage_f, 0, 9 * N * ps, c->stream));
    LBM_CUDA(c, cudaMemsetAsync(c->stage_T, 0, N * es, c->stream));
    LBM_CUDA(c, cudaEventCreateWithFlags(&c->ev_copied, cudaEventDisableTiming));
    LBM_CUDA(c, cudaEventCreateWithFlags(&c->ev_released, cudaEventDisableTiming));
    LBM_CUDA(c, cudaEventRecord(c->ev_released, c->stream));  // after the zeroing
    LBM_CUDA(c, cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
  }
  // the staging buffers may still be in use by work the context's stream had before the last take
  LBM_CUDA(c, cudaStreamWaitEvent(c->copy_stream, c->ev_released, 0));
  const size_t hpf = g.nx * ps, dpf = g.pitch * ps, hpt = g.nx * es, dpt = g.pitch * es;
  LBM_CUDA(c, cudaMemcpy2DAsync(c->stage_f, dpf, f, hpf, hpf, 9 * (size_t)g.ny, cudaMemcpyHostToDevice,
                                c->copy_stream));
  LBM_CUDA(c, cudaMemcpy2DAsync(c->stage_T, dpt, T, hpt, hpt, g.ny, cudaMemcpyHostToDevice, c->copy_stream));
  if (side)
    LBM_CUDA(c, cudaMemcpyAsync(c->stage_side, side, 3 * (size_t)g.ny * es, cudaMemcpyHostToDevice, c->copy_stream));
  LBM_CUDA(c, cudaEventRecord(c->ev_copied, c->copy_stream));
  c->staged = side ? 2 : 1;
  c->staged_steps = steps;
  return LBM_OK;
}

lbm_status lbm_take_staged(lbm_ctx* c) {
  if (!c) return LBM_EINVAL;
  if (!c->staged) return fail(c, LBM_ESTATE, "no state is staged (lbm_stage_state_native)");
  LBM_CUDA(c, cudaStreamWaitEvent(c->stream, c->ev_copied, 0));
  lbm::Dev& d = c->dev;
  // the staged buffers become the current state; the current ones become the staging buffers
  std::swap(d.f[c->cur], c->stage_f);
  std::swap(d.T[c->tcur], c->stage_T);
  if (c->staged == 2) std::swap(d.side[c->cur], c->stage_side);
  // everything the context's stream has so far may use the buffers now held for staging
  LBM_CUDA(c, cudaEventRecord(c->ev_released, c->stream));
  c->staged = 0;
  c->psi_pending = 0;  // the state changes: psi of the next step is no longer known
  clear_latched(c);
  if (c->staged_steps >= 0) c->steps = c->staged_steps;
  return LBM_OK;
}

lbm_status lbm_info(lbm_ctx* c, lbm_info_t* info) {
  if (!c || !info) return LBM_EINVAL;
  info->Tc = c->Tc;
  info->pc = c->pc;
  info->T_sat = c->ph.d.T_sat;
  info->T_wall = c->ph.d.T_wall;
  info->rho_l = c->ph.d.rho_l;
  info->rho_v = c->ph.d.rho_v;
  info->p_sat = c->p_sat;
  info->h_fg = c->h_fg;
  info->nu_l = c->ph.d.nu_l;
  info->nu_v = c->ph.d.nu_v;
  info->alpha_l = c->ph.d.alpha_l;
  info->alpha_v = c->ph.d.alpha_v;
  info->lambda_v = c->lambda_v;
  info->g = c->ph.d.g;
  info->outlet_U = c->ph.d.U_out;
  info->steps = c->steps;
  info->n_boundary = c->dev.nb;
  info->kernel_launches = c->launches;
  info->device_bytes = (int64_t)c->bytes;
  return LBM_OK;
}

lbm_status lbm_profile(lbm_ctx* c, int enable) {
  if (!c) return LBM_EINVAL;
  if (enable && !c->prof) {
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    for (auto& p : c->pending) {
      c->pool.push_back(p.e0);
      c->pool.push_back(p.e1);
    }
    c->pending.clear();
    for (int k = 0; k < lbm::kNumKernels; ++k) {
      c->prof_ms[k] = 0;
      c->prof_n[k] = 0;
    }
  }
  c->prof = enable != 0;
  return LBM_OK;
}

lbm_status lbm_profile_read(lbm_ctx* c, const char** names, int64_t* launches, double* total_ms, int32_t max_kernels,
                            int32_t* n_kernels) {
  if (!c) return LBM_EINVAL;
  LBM_CUDA(c, cudaStreamSynchronize(c->stream));
  for (auto& p : c->pending) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, p.e0, p.e1) == cudaSuccess) {
      c->prof_ms[p.kernel] += ms;
      c->prof_n[p.kernel] += 1;
    }
    c->pool.push_back(p.e0);
    c->pool.push_back(p.e1);
  }
  c->pending.clear();
  for (int k = 0; k < lbm::kNumKernels && k < max_kernels; ++k) {
    if (names) names[k] = lbm::kKernelNames[k];
    if (launches) launches[k] = c->prof_n[k];
    if (total_ms) total_ms[k] = c->prof_ms[k];
  }
  if (n_kernels) *n_kernels = lbm::kNumKernels;
  return LBM_OK;
}

lbm_status lbm_inject_fault(lbm_ctx* c, int32_t kind) {
  if (!c) return LBM_EINVAL;
  if (kind != LBM_FAULT_STARVE_COLLIDE && kind != LBM_FAULT_STARVE_ENERGY)
    return fail(c, LBM_EINVAL, "unknown fault kind %d", (int)kind);
  if (!c->dev.tma) return fail(c, LBM_ESTATE, "no tile of this context is staged by TMA (LBM_TMA=0)");
  if (kind == LBM_FAULT_STARVE_ENERGY && !c->prm.energy)
    return fail(c, LBM_ESTATE, "this context runs no energy pass");
  c->dev.starve = kind == LBM_FAULT_STARVE_COLLIDE ? lbm::kStarveCollide : lbm::kStarveEnergy;
  return LBM_OK;
}

const char* lbm_last_error(const lbm_ctx* c) { return c ? c->err.c_str() : g_create_error.c_str(); }

void lbm_destroy(lbm_ctx* c) {
  if (!c || c->batch_owned) return;
  cudaStreamSynchronize(c->stream);
  if (c->copy_stream) {
    cudaStreamSynchronize(c->copy_stream);
    cudaStreamDestroy(c->copy_stream);
    cudaEventDestroy(c->ev_copied);
    cudaEventDestroy(c->ev_released);
  }
  for (auto& p : c->pending) {
    cudaEventDestroy(p.e0);
    cudaEventDestroy(p.e1);
  }
  for (auto e : c->pool) cudaEventDestroy(e);
  dfree_all(c);
  delete c;
}


// ---------------------------------------------------------------- batches

static lbm_status batch_fail(lbm_batch* b, lbm_status st, const char* msg) {
  if (b) b->err = msg;
  g_create_error = msg;
  return st;
}

// Tile numbering of every pass for the current variant, and the block -> domain maps.
static lbm_status batch_layout(lbm_batch* b) {
  int cty, ety;
  lbm::batch_variant(b->variant, b->f64, cty, ety);
  std::vector<int> mp, mc, me;
  for (size_t k = 0; k < b->ctx.size(); ++k) {
    lbm::BatchDomain& D = b->h_doms[k];
    const lbm::Geo& g = D.g;
    const int ntx = (g.nx + 31) / 32;
    D.psi_first = (int)mp.size();
    D.psi_ntx = ntx;
    mp.insert(mp.end(), (size_t)ntx * ((g.ny + 7) / 8), (int)k);
    D.coll_first = (int)mc.size();
    D.coll_ntx = ntx;
    mc.insert(mc.end(), (size_t)ntx * ((g.ny + cty - 1) / cty), (int)k);
    D.en_first = (int)me.size();
    D.en_ntx = ntx;
    D.en_nblocks = ntx * ((g.ny + ety - 1) / ety);
    me.insert(me.end(), (size_t)D.en_nblocks, (int)k);
    // TMA maps for this variant's tiles (plain loads for the domain when one cannot be made)
    if (b->f64) lbm::batch_maps_f64(D, b->hmaps[k], cty, ety);
    else lbm::batch_maps_f32(D, b->hmaps[k], cty, ety);
  }
  b->nb_psi = (int)mp.size();
  b->nb_coll = (int)mc.size();
  b->nb_en = (int)me.size();
  if (b->nb_psi > b->max_tiles || b->nb_coll > b->max_tiles || b->nb_en > b->max_tiles)
    return batch_fail(b, LBM_ESTATE, "batch tile maps larger than allocated");
  cudaError_t e = cudaMemcpyAsync(b->d_doms, b->h_doms.data(), sizeof(lbm::BatchDomain) * b->h_doms.size(),
                                  cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_maps, mp.data(), sizeof(int) * mp.size(), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_maps + b->max_tiles, mc.data(), sizeof(int) * mc.size(), cudaMemcpyHostToDevice,
                        b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_maps + 2 * b->max_tiles, me.data(), sizeof(int) * me.size(), cudaMemcpyHostToDevice,
                        b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return batch_fail(b, LBM_ECUDA, cudaGetErrorString(e));
  return LBM_OK;
}

// psi of the current state is unknown for some two-phase domain (creation, or a state set
// through the API): the next step starts with the psi pass
static bool batch_needs_psi(const lbm_batch* b) {
  for (const lbm_ctx* c : b->ctx)
    if (!c->psi_pending && c->ph.d.G != 0.0) return true;
  return false;
}

static int batch_launch(lbm_batch* b, cudaStream_t s) {
  const int* m = b->d_maps;
  const int need_psi = batch_needs_psi(b) ? 1 : 0;
  const int nd = (int)b->h_doms.size();
  return b->f64 ? lbm::batch_step_f64(b->variant, b->d_doms, m, b->nb_psi, m + b->max_tiles, b->nb_coll,
                                      m + 2 * b->max_tiles, b->nb_en, b->cur, b->tcur, b->steps, need_psi,
                                      b->h_doms.data(), b->hmaps.data(), nd, s)
                : lbm::batch_step_f32(b->variant, b->d_doms, m, b->nb_psi, m + b->max_tiles, b->nb_coll,
                                      m + 2 * b->max_tiles, b->nb_en, b->cur, b->tcur, b->steps, need_psi,
                                      b->h_doms.data(), b->hmaps.data(), nd, s);
}

// After a batched step: the energy pass has made psi of the new state in buffer b->cur; each
// domain's context sees the buffers as a single-domain step leaves them (psi: the one the
// step's collision used, psi_next: the pending one)
static void batch_advance(lbm_batch* b, int launches) {
  b->cur ^= 1;
  b->tcur ^= 1;
  b->steps++;
  for (size_t k = 0; k < b->ctx.size(); ++k) {
    lbm_ctx* c = b->ctx[k];
    c->cur = b->cur;
    c->tcur = b->tcur;
    c->steps = b->steps;
    c->launches += launches;
    c->dev.psi = b->psi_buf[b->cur ^ 1][k];
    c->dev.psi_next = b->psi_buf[b->cur][k];
    c->psi_pending = 1;
  }
}


lbm_status lbm_batch_create(int32_t n, const lbm_domain* domains, const lbm_cylinder* cyls, const lbm_params* params,
                            const lbm_allocator* alloc, void* cuda_stream, lbm_batch** out) {
  if (n < 1 || !domains || !cyls || !params || !out) return batch_fail(nullptr, LBM_EINVAL, "bad batch arguments");
  *out = nullptr;
  for (int k = 0; k < n; ++k) {
    if (params[k].compute_f64 != params[0].compute_f64)
      return batch_fail(nullptr, LBM_EINVAL, "all domains of a batch must share compute_f64");
    const int want = params[k].compute_f64 ? LBM_STORE_F64 : LBM_STORE_F32;
    if (params[k].storage != want || params[k].psi_mode != 0)
      return batch_fail(nullptr, LBM_EINVAL, "batches need storage F32 (FP32) or F64 (FP64 build) and psi_mode 0");
    if (params[k].collision != LBM_COLL_CM) return batch_fail(nullptr, LBM_EINVAL, "batches use the CM collision");
  }
  lbm_batch* b = new lbm_batch();
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  b->f64 = params[0].compute_f64 != 0;
  for (int k = 0; k < n; ++k) {
    lbm_ctx* c = nullptr;
    lbm_status st = lbm_create(&domains[k], &cyls[k], &params[k], nullptr, alloc, cuda_stream, &c);
    if (st != LBM_OK) {
      std::string m = "domain " + std::to_string(k) + ": " + g_create_error;
      for (lbm_ctx* x : b->ctx) {
        x->batch_owned = false;
        lbm_destroy(x);
      }
      delete b;
      return batch_fail(nullptr, st, m.c_str());
    }
    c->batch_owned = true;
    b->ctx.push_back(c);
    lbm::BatchDomain D{};
    D.g = c->geo;
    D.ph = c->ph;
    D.d = c->dev;  // psi, psi_next: the buffers of population parity 0 and 1
    b->psi_buf[0].push_back(c->dev.psi);
    b->psi_buf[1].push_back(c->dev.psi_next);
    D.warmup = params[k].warmup_steps;
    D.energy = params[k].energy;
    b->h_doms.push_back(D);
    b->max_warmup = std::max<long long>(b->max_warmup, params[k].warmup_steps);
    b->max_tiles += ((domains[k].nx + 31) / 32) * ((domains[k].ny + 7) / 8);
  }
  b->hmaps.resize(b->h_doms.size());
  cudaError_t e = cudaMalloc(&b->d_doms, sizeof(lbm::BatchDomain) * n);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_maps, sizeof(int) * 3 * (size_t)b->max_tiles);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->gstream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    std::string m = cudaGetErrorString(e);
    lbm_batch_destroy(b);
    return batch_fail(nullptr, LBM_ENOMEM, m.c_str());
  }
  lbm_status st = batch_layout(b);
  if (st != LBM_OK) {
    std::string m = b->err;
    lbm_batch_destroy(b);
    return batch_fail(nullptr, st, m.c_str());
  }
  *out = b;
  return LBM_OK;
}

lbm_status lbm_batch_step(lbm_batch* b, int64_t n) {
  if (!b) return LBM_EINVAL;
  if (n < 0) return batch_fail(b, LBM_EINVAL, "negative step count");
  int64_t s = 0;
  // eager steps until every domain is past its warm-up (the graph bakes in the step counter)
  // and psi of the current state is known (the graph holds no psi pass)
  while (s < n && (b->steps < b->max_warmup || !b->use_graph || n - s < 2 || batch_needs_psi(b))) {
    const int k = batch_launch(b, b->stream);
    if (k < 0) return batch_fail(b, LBM_ECUDA, cudaGetErrorString(cudaGetLastError()));
    batch_advance(b, k);
    ++s;
  }
  if (s + 1 >= n) {
    if (s < n) {
      const int k = batch_launch(b, b->stream);
      if (k < 0) return batch_fail(b, LBM_ECUDA, cudaGetErrorString(cudaGetLastError()));
      batch_advance(b, k);
    }
    return LBM_OK;
  }
  // pairs of steps from a CUDA graph captured for the current buffer parity and variant
  if (!b->gexec || b->g_cur != b->cur || b->g_tcur != b->tcur || b->g_variant != b->variant) {
    if (b->gexec) {
      cudaGraphExecDestroy(b->gexec);
      b->gexec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(b->gstream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return batch_fail(b, LBM_ECUDA, "stream capture failed to begin");
    const int c0 = b->cur, t0 = b->tcur;
    const long long s0 = b->steps;
    int k1 = batch_launch(b, b->gstream);
    b->cur ^= 1;
    b->tcur ^= 1;
    b->steps++;
    int k2 = batch_launch(b, b->gstream);
    b->cur = c0;
    b->tcur = t0;
    b->steps = s0;
    cudaError_t e = cudaStreamEndCapture(b->gstream, &graph);
    if (k1 < 0 || k2 < 0 || e != cudaSuccess) return batch_fail(b, LBM_ECUDA, "graph capture failed");
    e = cudaGraphInstantiate(&b->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return batch_fail(b, LBM_ECUDA, cudaGetErrorString(e));
    b->g_cur = b->cur;
    b->g_tcur = b->tcur;
    b->g_variant = b->variant;
    b->g_launches[0] = k1;
    b->g_launches[1] = k2;
  }
  if (cudaEventRecord(b->ev_in, b->stream) != cudaSuccess || cudaStreamWaitEvent(b->gstream, b->ev_in, 0) != cudaSuccess)
    return batch_fail(b, LBM_ECUDA, "event ordering failed");
  for (; s + 2 <= n; s += 2) {
    if (cudaGraphLaunch(b->gexec, b->gstream) != cudaSuccess) return batch_fail(b, LBM_ECUDA, "graph launch failed");
    batch_advance(b, b->g_launches[0]);
    batch_advance(b, b->g_launches[1]);
  }
  if (cudaEventRecord(b->ev_out, b->gstream) != cudaSuccess || cudaStreamWaitEvent(b->stream, b->ev_out, 0) != cudaSuccess)
    return batch_fail(b, LBM_ECUDA, "event ordering failed");
  if (s < n) {
    const int k = batch_launch(b, b->stream);
    if (k < 0) return batch_fail(b, LBM_ECUDA, cudaGetErrorString(cudaGetLastError()));
    batch_advance(b, k);
  }
  return LBM_OK;
}

}  // extern "C"

namespace {

// Tuning cache: the variant chosen for a set of domains on a kind of device, kept for the
// process and, when the environment names a file in LBM_TUNE_CACHE, in that file (lines
// "<16 hex digits of the key> <variant>", appended as choices are made).
std::mutex g_tune_mu;
std::map<unsigned long long, int>* g_tune = nullptr;

unsigned long long fnv1a(unsigned long long h, const void* p, size_t n) {
  const unsigned char* c = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < n; ++i) h = (h ^ c[i]) * 1099511628211ull;
  return h;
}

unsigned long long tune_key(const lbm_batch* b) {
  unsigned long long h = 1469598103934665603ull;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp pr;
  if (cudaGetDeviceProperties(&pr, dev) == cudaSuccess) {
    h = fnv1a(h, pr.name, std::strlen(pr.name));
    h = fnv1a(h, &pr.major, sizeof(pr.major));
    h = fnv1a(h, &pr.minor, sizeof(pr.minor));
    h = fnv1a(h, &pr.multiProcessorCount, sizeof(pr.multiProcessorCount));
  }
  const int f64 = b->f64 ? 1 : 0;
  h = fnv1a(h, &f64, sizeof(f64));
  for (const lbm_ctx* c : b->ctx) {
    const int dims[6] = {c->dom.nx, c->dom.ny, c->dom.periodic_x, c->dom.walls, c->prm.energy, c->prm.G != 0.0};
    const double cyl[3] = {c->cyl.D, c->cyl.xc, c->cyl.yc};
    h = fnv1a(h, dims, sizeof(dims));
    h = fnv1a(h, cyl, sizeof(cyl));
  }
  return h;
}

std::map<unsigned long long, int>& tune_table() {
  if (!g_tune) {
    g_tune = new std::map<unsigned long long, int>();
    if (const char* path = std::getenv("LBM_TUNE_CACHE")) {
      if (FILE* f = std::fopen(path, "r")) {
        unsigned long long k;
        int v;
        while (std::fscanf(f, "%llx %d", &k, &v) == 2) (*g_tune)[k] = v;
        std::fclose(f);
      }
    }
  }
  return *g_tune;
}

void tune_store(unsigned long long key, int v) {
  tune_table()[key] = v;
  if (const char* path = std::getenv("LBM_TUNE_CACHE")) {
    if (FILE* f = std::fopen(path, "a")) {
      std::fprintf(f, "%016llx %d\n", key, v);
      std::fclose(f);
    }
  }
}

}  // namespace

extern "C" {

lbm_status lbm_batch_tune(lbm_batch* b, int32_t steps_per_variant, int32_t* variant) {
  if (!b || steps_per_variant < 1) return LBM_EINVAL;
  const int nv = b->f64 ? 2 : lbm::kBatchVariants;
  const unsigned long long key = tune_key(b);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto& t = tune_table();
    auto it = t.find(key);
    if (it != t.end() && it->second >= 0 && it->second < nv) {  // chosen before: no timing, no steps
      b->variant = it->second;
      if (variant) *variant = b->variant;
      return batch_layout(b);
    }
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // two interleaved rounds over the variants; each variant keeps its faster round
  float ms_of[lbm::kBatchVariants];
  for (int v = 0; v < nv; ++v) ms_of[v] = 1e30f;
  for (int round = 0; round < 2; ++round)
    for (int v = 0; v < nv; ++v) {
      b->variant = v;
      lbm_status st = batch_layout(b);
      if (st != LBM_OK) return st;
      cudaEventRecord(e0, b->stream);
      for (int s = 0; s < steps_per_variant; ++s) {
        const int k = batch_launch(b, b->stream);
        if (k < 0) return batch_fail(b, LBM_ECUDA, cudaGetErrorString(cudaGetLastError()));
        batch_advance(b, k);
      }
      cudaEventRecord(e1, b->stream);
      cudaEventSynchronize(e1);
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < ms_of[v]) ms_of[v] = ms;
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  int best = 0;
  for (int v = 1; v < nv; ++v)
    if (ms_of[v] < ms_of[best]) best = v;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_store(key, best);
  }
  b->variant = best;
  lbm_status st = batch_layout(b);
  if (variant) *variant = best;
  return st;
}

lbm_status lbm_batch_graph(lbm_batch* b, int enable) {
  if (!b) return LBM_EINVAL;
  b->use_graph = enable != 0;
  return LBM_OK;
}

lbm_status lbm_batch_domain(lbm_batch* b, int32_t i, lbm_ctx** ctx) {
  if (!b || !ctx || i < 0 || i >= (int32_t)b->ctx.size()) return LBM_EINVAL;
  *ctx = b->ctx[i];
  return LBM_OK;
}

void lbm_batch_destroy(lbm_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->gstream) cudaStreamSynchronize(b->gstream);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  if (b->gstream) cudaStreamDestroy(b->gstream);
  if (b->d_doms) cudaFree(b->d_doms);
  if (b->d_maps) cudaFree(b->d_maps);
  for (lbm_ctx* c : b->ctx) {
    c->batch_owned = false;
    lbm_destroy(c);
  }
  delete b;
}

}  // extern "C"
