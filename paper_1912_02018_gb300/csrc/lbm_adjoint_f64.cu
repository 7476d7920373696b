// FP64 instantiation of the reverse-step kernels of the adjoint window.  Unlike the forward
// kernels (lbm_f64.cu, no contraction, so that they round like the oracle), these are built with
// FMA contraction: the reverse step is held to the gradient oracle at 1e-10, not bit for bit, and
// a fused multiply-add is one FP64 operation instead of two on GB300's 1/64-rate FP64 pipe.
#include "lbm_adjoint.cuh"

namespace lbm {

int adjoint_step_f64(const AdjArgs<double>& a, cudaStream_t s) { return adj::adjoint_step_impl<double>(a, s); }
int adjoint_setup_f64() { return adj::adjoint_setup_impl<double>(); }
int adjoint_aux_f64(int op, const Geo& g, const uint8_t* mask, const void* src, void* dst, cudaStream_t s) {
  const dim3 blk(32, 8), grd((g.nx + 31) / 32, (g.ny + 7) / 8);
  switch (op) {
    case 0: adj::k_impose_wall<double><<<grd, blk, 0, s>>>(g, mask, static_cast<const double*>(src), static_cast<double*>(dst)); break;
    case 1: adj::k_adj_wall_seed<double><<<grd, blk, 0, s>>>(g, mask, static_cast<const double*>(src), static_cast<double*>(dst)); break;
    case 2: adj::k_dense_to_plane<double><<<grd, blk, 0, s>>>(g, static_cast<const double*>(src), static_cast<double*>(dst)); break;
    case 3: adj::k_plane_to_dense<double><<<grd, blk, 0, s>>>(g, static_cast<const double*>(src), static_cast<double*>(dst)); break;
    default: return -1;
  }
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace lbm
