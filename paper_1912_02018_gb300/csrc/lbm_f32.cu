// FP32 instantiation of the step kernels: float populations and float arithmetic
// (FMA contraction allowed); psi is still evaluated in FP64 and the wall heat flux is
// accumulated in FP64.
#include "lbm_kernels.cuh"

namespace lbm {

int step_f32(const Geo& g, const Phys& ph, const Dev& d, int cur, int forcing, int energy, cudaStream_t s,
             const LaunchHook* hook) {
  return step_impl<float, float>(g, ph, d, cur, forcing, energy, s, hook);
}
int export_f32(const Geo& g, const Dev& d, int cur, int which, double* dst, cudaStream_t s) {
  return export_impl<float, float>(g, d, cur, which, dst, s);
}
int import_f32(const Geo& g, const Dev& d, int cur, int which, const double* src, cudaStream_t s) {
  return import_impl<float, float>(g, d, cur, which, src, s);
}
int init_f32(const Geo& g, const Phys& ph, const Dev& d, const double* rho0, const double* drho, const double* ux0,
             const double* uy0, const double* T0, unsigned long long seed, double amp, cudaStream_t s) {
  return init_impl<float, float>(g, ph, d, rho0, drho, ux0, uy0, T0, seed, amp, s);
}

}  // namespace lbm
