// FP64 instantiation of the step kernels: double populations and double arithmetic.
// Built with --fmad=false so that every product and sum is rounded separately, in the
// order the kernels spell out (the paper's equations term by term).
#include "lbm_kernels.cuh"

namespace lbm {

int step_f64(const Geo& g, const Phys& ph, const Dev& d, int cur, int tcur, int forcing, int energy, int psi_mode,
             cudaStream_t s, const LaunchHook* hook, int* t_flipped, PsiChain* chain) {
  (void)psi_mode;  // the FP64 build always evaluates psi in IEEE FP64
  return step_impl<double, double, kPsiF64>(g, ph, d, cur, tcur, forcing, energy, s, hook, t_flipped, chain);
}
int export_f64(const Geo& g, const Phys& ph, const Dev& d, int cur, int tcur, int which, double* dst, cudaStream_t s) {
  return export_impl<double, double>(g, ph, d, cur, tcur, which, dst, s);
}
int import_f64(const Geo& g, const Phys& ph, const Dev& d, int cur, int tcur, int which, const double* src,
               cudaStream_t s) {
  return import_impl<double, double>(g, ph, d, cur, tcur, which, src, s);
}
int init_f64(const Geo& g, const Phys& ph, const Dev& d, const double* rho0, const double* drho, const double* ux0,
             const double* uy0, const double* T0, const double* Tw, unsigned long long seed, double amp, cudaStream_t s) {
  return init_impl<double, double>(g, ph, d, rho0, drho, ux0, uy0, T0, Tw, seed, amp, s);
}

bool batch_maps_f64(BatchDomain& D, DomainMaps& m, int cty, int ety) {
  return kern::batch_maps_impl<double, double>(D, m, cty, ety);
}

int batch_step_f64(int variant, const BatchDomain* doms, const int* mp, int np, const int* mc, int nc,
                   const int* me, int ne, int cur, int tcur, long long step, int need_psi,
                   const BatchDomain* hd, const DomainMaps* hm, int nd, cudaStream_t s) {
  switch (variant & 1) {
    case 1: return kern::batch_step_impl<double, double, kPsiF64, 16, 8>(doms, mp, np, mc, nc, me, ne, cur, tcur, step, need_psi, hd, hm, nd, s);
    default: return kern::batch_step_impl<double, double, kPsiF64, 8, 8>(doms, mp, np, mc, nc, me, ne, cur, tcur, step, need_psi, hd, hm, nd, s);
  }
}

}  // namespace lbm
