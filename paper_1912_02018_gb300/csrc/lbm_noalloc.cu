// Allocation-free wall heat flux: lbm_wall_heat_flux_noalloc (declared in include/lbm.h).
//
// The same quantity as the heat-flux part of the energy kernel -- the mean over the fluid
// nodes next to the cylinder of -lambda(rho) grad T . n, grad T the isotropic 24-neighbour
// gradient -- computed from fields the caller passes in, without a context and without
// allocating.  Its only working memory is the file-scope array below: one (sum, count)
// pair per thread block plus a completion counter.  Every GPU that loads the library
// holds this array until the process exits.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "lbm.h"

namespace {

constexpr int kTX = 32, kTY = 8, kThreads = kTX * kTY;
constexpr int kMaxBlocks = 32768;  // tiles of 32 x 8 nodes: up to 8,388,608 lattice nodes per call
constexpr int kMaxDevices = 64;

// Scratch: [0, kMaxBlocks) partial sums, [kMaxBlocks, 2 kMaxBlocks) partial counts,
// then the completion counter (as a double-sized slot).  512 KiB + 8 B per device.
static __device__ __align__(256) double g_scratch[2 * kMaxBlocks + 1];

struct Consts {
  int nx, ny, periodic_x;
  double xc, yc, r;
  double rho_l, rho_v, alpha_l, alpha_v, c_v;
};

__device__ __forceinline__ int wrap_mod(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}
__device__ __forceinline__ bool solid_at(const Consts& k, int x, int y) {
  const double dx = x - k.xc, dy = y - k.yc;
  return dx * dx + dy * dy <= k.r * k.r;
}
__device__ __forceinline__ double field_at(const Consts& k, const double* f, int x, int y) {
  y = wrap_mod(y, k.ny);
  if (k.periodic_x) x = wrap_mod(x, k.nx);
  else x = x < 0 ? 0 : (x >= k.nx ? k.nx - 1 : x);
  return f[y * k.nx + x];
}

// One block per 32 x 8 tile; the last block to finish sums the per-block partials in block
// order and writes the mean.  scratch: g_scratch's device address (host-side lookup).
__global__ void __launch_bounds__(kThreads)
    k_wall_flux_noalloc(Consts k, const double* __restrict__ T, const double* __restrict__ rho, double* scratch,
                        double* q_out) {
  __shared__ double red_s[kThreads / 32], red_c[kThreads / 32];
  __shared__ int last;
  const int x = blockIdx.x * kTX + threadIdx.x % kTX, y = blockIdx.y * kTY + threadIdx.x / kTX;
  double q = 0.0, c = 0.0;
  if (x < k.nx && y < k.ny && !solid_at(k, x, y)) {
    bool near = false;
    for (int i = 1; i < 9 && !near; ++i) {
      const int cx = (i == 1 || i == 5 || i == 7) ? 1 : ((i == 2 || i == 6 || i == 8) ? -1 : 0);
      const int cy = (i == 3 || i == 5 || i == 8) ? 1 : ((i == 4 || i == 6 || i == 7) ? -1 : 0);
      int sx = x - cx;
      const int sy = wrap_mod(y - cy, k.ny);
      if (k.periodic_x) sx = wrap_mod(sx, k.nx);
      if (sx >= 0 && sx < k.nx) near = solid_at(k, sx, sy);
    }
    if (near) {
      // isotropic gradient over the 12 pairs (e, -e) of the 24-neighbour stencil
      const int ex[12] = {1, 2, -2, -1, 0, 1, 2, -2, -1, 0, 1, 2};
      const int ey[12] = {0, 0, 1, 1, 1, 1, 1, 2, 2, 2, 2, 2};
      double gx = 0.0, gy = 0.0;
      for (int p = 0; p < 12; ++p) {
        const int e2 = ex[p] * ex[p] + ey[p] * ey[p];
        const double w = e2 == 1 ? 4.0 / 21.0 : e2 == 2 ? 4.0 / 45.0 : e2 == 4 ? 1.0 / 60.0
                       : e2 == 5 ? 2.0 / 315.0 : 1.0 / 5040.0;
        const double d = field_at(k, T, x + ex[p], y + ey[p]) - field_at(k, T, x - ex[p], y - ey[p]);
        gx += w * d * ex[p];
        gy += w * d * ey[p];
      }
      const double r0 = rho[y * k.nx + x];
      double ph = k.rho_l > k.rho_v ? (r0 - k.rho_v) / (k.rho_l - k.rho_v) : 1.0;
      ph = ph < 0.0 ? 0.0 : (ph > 1.0 ? 1.0 : ph);
      const double lam = r0 * k.c_v * (k.alpha_v + ph * (k.alpha_l - k.alpha_v));
      const double dx = x - k.xc, dy = y - k.yc, rr = sqrt(dx * dx + dy * dy);
      q = -lam * (gx * (dx / rr) + gy * (dy / rr));
      c = 1.0;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    q += __shfl_down_sync(0xffffffffu, q, o);
    c += __shfl_down_sync(0xffffffffu, c, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red_s[threadIdx.x >> 5] = q;
    red_c[threadIdx.x >> 5] = c;
  }
  __syncthreads();
  const int nblocks = gridDim.x * gridDim.y, bid = blockIdx.y * gridDim.x + blockIdx.x;
  unsigned* counter = reinterpret_cast<unsigned*>(scratch + 2 * kMaxBlocks);
  if (threadIdx.x == 0) {
    double s = 0.0, n = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) {
      s += red_s[w];
      n += red_c[w];
    }
    scratch[bid] = s;
    scratch[kMaxBlocks + bid] = n;
    __threadfence();
    last = atomicInc(counter, nblocks - 1) == (unsigned)(nblocks - 1);
  }
  __syncthreads();
  if (last) {
    __threadfence();
    double s = 0.0, n = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += kThreads) {
      s += __ldcg(&scratch[i]);
      n += __ldcg(&scratch[kMaxBlocks + i]);
    }
    for (int o = 16; o > 0; o >>= 1) {
      s += __shfl_down_sync(0xffffffffu, s, o);
      n += __shfl_down_sync(0xffffffffu, n, o);
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
      red_s[threadIdx.x >> 5] = s;
      red_c[threadIdx.x >> 5] = n;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double ts = 0.0, tn = 0.0;
      for (int w = 0; w < kThreads / 32; ++w) {
        ts += red_s[w];
        tn += red_c[w];
      }
      *q_out = tn > 0.0 ? ts / tn : 0.0;
    }
  }
}

// Per-device address of g_scratch, looked up once per device (and CUDA context) with that device current.
std::mutex g_mu;
double* g_addr[kMaxDevices] = {};
unsigned long long g_ctx_id[kMaxDevices] = {};  // the CUDA context the address was looked up in

// Unique id of the calling thread's current CUDA context (0 if it cannot be had): the driver's
// cuCtxGetCurrent and cuCtxGetId, reached through the runtime's driver entry points.  A device
// reset (cudaDeviceReset) destroys the primary context and unloads the library's device code,
// so an address looked up in the old context is stale; the new context has a new id.
unsigned long long current_ctx_id() {
  using GetCurrent = CUresult (*)(CUcontext*);
  using GetId = CUresult (*)(CUcontext, unsigned long long*);
  static GetCurrent get_current = []() -> GetCurrent {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    return cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
                   q == cudaDriverEntryPointSuccess
               ? reinterpret_cast<GetCurrent>(p)
               : nullptr;
  }();
  static GetId get_id = []() -> GetId {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    return cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
                   q == cudaDriverEntryPointSuccess
               ? reinterpret_cast<GetId>(p)
               : nullptr;
  }();
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (get_current && get_id && get_current(&ctx) == CUDA_SUCCESS && ctx && get_id(ctx, &id) == CUDA_SUCCESS) return id;
  return 0;
}

// Peng-Robinson EOS and Maxwell's equal-area rule at T, on the host (no allocation).
struct Eos {
  double a, b, R, kappa, Tc;
  double phi(double T) const {
    const double s = 1.0 + kappa * (1.0 - std::sqrt(T / Tc));
    return s * s;
  }
  double p(double r, double T) const {
    return r * R * T / (1.0 - b * r) - a * phi(T) * r * r / (1.0 + 2.0 * b * r - b * b * r * r);
  }
  double dp(double r, double T) const {
    const double D = 1.0 + 2.0 * b * r - b * b * r * r, dD = 2.0 * b - 2.0 * b * b * r, x = 1.0 - b * r;
    return R * T / (x * x) - a * phi(T) * (2.0 * r * D - r * r * dD) / (D * D);
  }
  double p_dv(double v, double T) const {
    const double s2 = std::sqrt(2.0);
    return R * T * std::log(v - b) - a * phi(T) / (2.0 * s2 * b) * std::log((v + b - s2 * b) / (v + b + s2 * b));
  }
  template <class F>
  static double bisect(F f, double lo, double hi) {
    const double flo = f(lo);
    for (int it = 0; it < 200; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (mid <= lo || mid >= hi) break;
      if ((f(mid) < 0.0) == (flo < 0.0)) lo = mid;
      else hi = mid;
    }
    return 0.5 * (lo + hi);
  }
  bool maxwell(double T, double& rv, double& rl) const {
    const int n = 4000;
    const double top = 1.0 / b;
    double roots[2];
    int nr = 0;
    double prev = dp(0.5 / n * top, T);
    for (int k = 1; k < n && nr < 2; ++k) {
      const double r1 = (k + 0.5) / n * top, cur = dp(r1, T);
      if ((cur < 0.0) != (prev < 0.0))
        roots[nr++] = bisect([&](double r) { return dp(r, T); }, (k - 0.5) / n * top, r1);
      prev = cur;
    }
    if (nr != 2) return false;
    const double ra = roots[0], rb = roots[1], p_hi = p(ra, T);
    double p_lo = p(rb, T);
    if (p_lo < 1e-10 * p_hi) p_lo = 1e-10 * p_hi;
    auto area = [&](double ps) {
      const double v = bisect([&](double r) { return p(r, T) - ps; }, 0.0, ra);
      const double l = bisect([&](double r) { return p(r, T) - ps; }, rb, (1.0 - 1e-12) * top);
      rv = v;
      rl = l;
      return (p_dv(1.0 / v, T) - p_dv(1.0 / l, T)) - ps * (1.0 / v - 1.0 / l);
    };
    const double ps = bisect(area, p_lo + 1e-14 * (p_hi - p_lo), p_hi - 1e-14 * (p_hi - p_lo));
    area(ps);
    return rv > 0.0 && rl > rv;
  }
};

}  // namespace

extern "C" lbm_status lbm_wall_heat_flux_noalloc(const lbm_domain* dom, const lbm_cylinder* cyl,
                                                 const lbm_params* P, const double* T, const double* rho,
                                                 double* q_out, void* cuda_stream) {
  if (!dom || !cyl || !P || !T || !rho || !q_out) return LBM_EINVAL;
  if (dom->nx < 5 || dom->ny < 5 || !(cyl->D > 0) || dom->walls != 0) return LBM_EINVAL;  // the cylinder alone
  const int bx = (dom->nx + kTX - 1) / kTX, by = (dom->ny + kTY - 1) / kTY;
  if ((long long)bx * by > kMaxBlocks) return LBM_EINVAL;  // more than 8,388,608 nodes: beyond the scratch
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LBM_ECUDA;
  double* scratch;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    // set-up, once per device and context: the device address of the scratch array
    const unsigned long long id = g_addr[dev] ? current_ctx_id() : 0;
    if (!g_addr[dev] || id != g_ctx_id[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess) return LBM_ECUDA;
      g_addr[dev] = static_cast<double*>(p);
      g_ctx_id[dev] = current_ctx_id();  // the lookup made the device's context current
    }
    scratch = g_addr[dev];
  }
  // constants the energy equation uses for lambda(rho), Sec. II.C and Sec. IV.A
  Eos e;
  e.a = P->a;
  e.b = P->b;
  e.R = P->R;
  e.kappa = 0.37464 + 1.54226 * P->acentric - 0.26992 * P->acentric * P->acentric;
  e.Tc = 0.0778 * P->a / (0.4572 * P->b * P->R);
  Consts k;
  if (!e.maxwell(P->Tr_sat * e.Tc, k.rho_v, k.rho_l)) return LBM_EINVAL;
  const double nu_l = P->nu_l > 0 ? P->nu_l : (P->Re > 0 ? P->u_in * cyl->D / P->Re : 0.0);
  if (!(nu_l > 0) || !(P->nu_ratio > 0) || !(P->Pr_l > 0) || !(P->Pr_v > 0)) return LBM_EINVAL;
  k.nx = dom->nx;
  k.ny = dom->ny;
  k.periodic_x = dom->periodic_x ? 1 : 0;
  k.xc = cyl->xc;
  k.yc = cyl->yc;
  k.r = 0.5 * cyl->D;
  k.alpha_l = nu_l / P->Pr_l;
  k.alpha_v = nu_l / P->nu_ratio / P->Pr_v;
  k.c_v = P->c_v;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  // the completion counter must start at zero on every call
  if (cudaMemsetAsync(scratch + 2 * kMaxBlocks, 0, sizeof(double), s) != cudaSuccess) return LBM_ECUDA;
  k_wall_flux_noalloc<<<dim3(bx, by), kThreads, 0, s>>>(k, T, rho, scratch, q_out);
  return cudaPeekAtLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}
