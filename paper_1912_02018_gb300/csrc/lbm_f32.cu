// FP32-compute instantiation of the step kernels (FMA contraction allowed), for populations
// stored as FP64, FP32 or shifted FP16.  psi is evaluated in double-float arithmetic by default
// (IEEE FP64 or plain FP32 on request) and the wall heat flux is accumulated in FP64.
#include "lbm.h"
#include "lbm_adjoint.cuh"
#include "lbm_kernels.cuh"

namespace lbm {

namespace {
template <typename S>
int step_s(const Geo& g, const Phys& ph, const Dev& d, int cur, int tcur, int forcing, int energy, int psi_mode,
           cudaStream_t s, const LaunchHook* hook, int* t_flipped, PsiChain* chain) {
  switch (psi_mode) {
    case kPsiF64: return step_impl<float, S, kPsiF64>(g, ph, d, cur, tcur, forcing, energy, s, hook, t_flipped, chain);
    case kPsiF32: return step_impl<float, S, kPsiF32>(g, ph, d, cur, tcur, forcing, energy, s, hook, t_flipped, chain);
    default: return step_impl<float, S, kPsiDF>(g, ph, d, cur, tcur, forcing, energy, s, hook, t_flipped, chain);
  }
}
}  // namespace

int step_f32(const Geo& g, const Phys& ph, const Dev& d, int cur, int tcur, int forcing, int energy, int psi_mode,
             int storage, cudaStream_t s, const LaunchHook* hook, int* t_flipped, PsiChain* chain) {
  switch (storage) {
    case LBM_STORE_F64: return step_s<double>(g, ph, d, cur, tcur, forcing, energy, psi_mode, s, hook, t_flipped, chain);
    case LBM_STORE_F16S: return step_s<__half>(g, ph, d, cur, tcur, forcing, energy, psi_mode, s, hook, t_flipped, chain);
    default: return step_s<float>(g, ph, d, cur, tcur, forcing, energy, psi_mode, s, hook, t_flipped, chain);
  }
}
int export_f32(const Geo& g, const Phys& ph, const Dev& d, int cur, int tcur, int which, int storage, double* dst,
               cudaStream_t s) {
  switch (storage) {
    case LBM_STORE_F64: return export_impl<float, double>(g, ph, d, cur, tcur, which, dst, s);
    case LBM_STORE_F16S: return export_impl<float, __half>(g, ph, d, cur, tcur, which, dst, s);
    default: return export_impl<float, float>(g, ph, d, cur, tcur, which, dst, s);
  }
}
int import_f32(const Geo& g, const Phys& ph, const Dev& d, int cur, int tcur, int which, int storage,
               const double* src, cudaStream_t s) {
  switch (storage) {
    case LBM_STORE_F64: return import_impl<float, double>(g, ph, d, cur, tcur, which, src, s);
    case LBM_STORE_F16S: return import_impl<float, __half>(g, ph, d, cur, tcur, which, src, s);
    default: return import_impl<float, float>(g, ph, d, cur, tcur, which, src, s);
  }
}
int init_f32(const Geo& g, const Phys& ph, const Dev& d, const double* rho0, const double* drho, const double* ux0,
             const double* uy0, const double* T0, const double* Tw, unsigned long long seed, double amp, int storage, cudaStream_t s) {
  switch (storage) {
    case LBM_STORE_F64: return init_impl<float, double>(g, ph, d, rho0, drho, ux0, uy0, T0, Tw, seed, amp, s);
    case LBM_STORE_F16S: return init_impl<float, __half>(g, ph, d, rho0, drho, ux0, uy0, T0, Tw, seed, amp, s);
    default: return init_impl<float, float>(g, ph, d, rho0, drho, ux0, uy0, T0, Tw, seed, amp, s);
  }
}

bool batch_maps_f32(BatchDomain& D, DomainMaps& m, int cty, int ety) {
  return kern::batch_maps_impl<float, float>(D, m, cty, ety);
}

int batch_step_f32(int variant, const BatchDomain* doms, const int* mp, int np, const int* mc, int nc,
                   const int* me, int ne, int cur, int tcur, long long step, int need_psi,
                   const BatchDomain* hd, const DomainMaps* hm, int nd, cudaStream_t s) {
  switch (variant) {
    case 1: return kern::batch_step_impl<float, float, kPsiDF, 16, 16>(doms, mp, np, mc, nc, me, ne, cur, tcur, step, need_psi, hd, hm, nd, s);
    case 2: return kern::batch_step_impl<float, float, kPsiDF, 8, 8>(doms, mp, np, mc, nc, me, ne, cur, tcur, step, need_psi, hd, hm, nd, s);
    case 3: return kern::batch_step_impl<float, float, kPsiDF, 16, 8>(doms, mp, np, mc, nc, me, ne, cur, tcur, step, need_psi, hd, hm, nd, s);
    default: return kern::batch_step_impl<float, float, kPsiDF, 8, 16>(doms, mp, np, mc, nc, me, ne, cur, tcur, step, need_psi, hd, hm, nd, s);
  }
}

int adjoint_step_f32(const AdjArgs<float>& a, cudaStream_t s) { return adj::adjoint_step_impl<float>(a, s); }
int adjoint_setup_f32() { return adj::adjoint_setup_impl<float>(); }
int adjoint_aux_f32(int op, const Geo& g, const uint8_t* mask, const void* src, void* dst, cudaStream_t s) {
  const dim3 blk(32, 8), grd((g.nx + 31) / 32, (g.ny + 7) / 8);
  switch (op) {
    case 0: adj::k_impose_wall<float><<<grd, blk, 0, s>>>(g, mask, static_cast<const float*>(src), static_cast<float*>(dst)); break;
    case 1: adj::k_adj_wall_seed<float><<<grd, blk, 0, s>>>(g, mask, static_cast<const float*>(src), static_cast<double*>(dst)); break;
    case 2: adj::k_dense_to_plane<float><<<grd, blk, 0, s>>>(g, static_cast<const double*>(src), static_cast<float*>(dst)); break;
    case 3: adj::k_plane_to_dense<float><<<grd, blk, 0, s>>>(g, static_cast<const float*>(src), static_cast<double*>(dst)); break;
    default: return -1;
  }
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace lbm
