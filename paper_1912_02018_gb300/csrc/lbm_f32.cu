// FP32 instantiation of the step kernels: float populations and float arithmetic
// (FMA contraction allowed).  psi is evaluated in double-float arithmetic by default
// (IEEE FP64 or plain FP32 on request) and the wall heat flux is accumulated in FP64.
#include "lbm_kernels.cuh"

namespace lbm {

int step_f32(const Geo& g, const Phys& ph, const Dev& d, int cur, int tcur, int forcing, int energy, int psi_mode,
             cudaStream_t s, const LaunchHook* hook, int* t_flipped) {
  switch (psi_mode) {
    case kPsiF64: return step_impl<float, float, kPsiF64>(g, ph, d, cur, tcur, forcing, energy, s, hook, t_flipped);
    case kPsiF32: return step_impl<float, float, kPsiF32>(g, ph, d, cur, tcur, forcing, energy, s, hook, t_flipped);
    default: return step_impl<float, float, kPsiDF>(g, ph, d, cur, tcur, forcing, energy, s, hook, t_flipped);
  }
}
int export_f32(const Geo& g, const Dev& d, int cur, int tcur, int which, double* dst, cudaStream_t s) {
  return export_impl<float, float>(g, d, cur, tcur, which, dst, s);
}
int import_f32(const Geo& g, const Dev& d, int cur, int tcur, int which, const double* src, cudaStream_t s) {
  return import_impl<float, float>(g, d, cur, tcur, which, src, s);
}
int init_f32(const Geo& g, const Phys& ph, const Dev& d, const double* rho0, const double* drho, const double* ux0,
             const double* uy0, const double* T0, unsigned long long seed, double amp, cudaStream_t s) {
  return init_impl<float, float>(g, ph, d, rho0, drho, ux0, uy0, T0, seed, amp, s);
}

}  // namespace lbm
