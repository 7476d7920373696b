// Tensor-memory-accelerator (TMA) staging of lattice tiles into shared memory, sm_90+ PTX:
// one elected thread arms an mbarrier with the expected byte count and issues tiled bulk
// copies (cp.async.bulk.tensor) that complete on it; the block waits on the barrier's phase
// with a bounded number of tries.  Host side: tensor maps of the [planes][ny][pitch] fields,
// encoded through the driver entry point the runtime exposes (no link against libcuda).
//
// Copy rules kept by every caller: the tile's first column times the element size is a
// multiple of 16 bytes, the box's inner extent is a multiple of 16 bytes, base addresses are
// 16-byte aligned and row/plane strides multiples of 16 bytes; coordinates past the lattice
// are read as zeros (callers use TMA only where the box lies inside the lattice).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace lbm {
namespace tma {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void bar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  // make the initialised barrier visible to the async proxy that completes the copies
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void bar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool bar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// Bounded wait for phase `parity` of the barrier: false if it did not complete in `tries`.
__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity, int tries) {
  for (int i = 0; i < tries; ++i)
    if (bar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(smem_addr(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ void load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
      : "memory");
}

// Tries of the bounded wait: each try blocks for a hardware-defined slice; a tile copy takes
// a few microseconds, the bound a fraction of a second.
constexpr int kWaitTries = 1 << 18;
// The bound of a tile starved on purpose by the test hook (lbm_inject_fault).
constexpr int kStarveTries = 64;

template <typename E>
struct DType;
template <>
struct DType<float> {
  static constexpr CUtensorMapDataType v = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
};
template <>
struct DType<double> {
  static constexpr CUtensorMapDataType v = CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
};
template <>
struct DType<__half> {
  static constexpr CUtensorMapDataType v = CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
};

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

inline EncodeTiled encoder() {
  static EncodeTiled fn = []() -> EncodeTiled {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return reinterpret_cast<EncodeTiled>(p);
  }();
  return fn;
}

// Tensor map of `planes` planes of nx x ny elements (row pitch `pitch` elements, plane
// stride `plane` elements) with box (bx, by, planes); planes == 1 gives a 2D map.  False if
// the encoder is unavailable or any copy rule is not met (the caller then loads without TMA).
template <typename E>
bool encode(CUtensorMap* map, const void* base, int nx, int ny, int pitch, long long plane, int planes, int bx,
            int by) {
  const EncodeTiled fn = encoder();
  if (!fn || !base || (reinterpret_cast<uintptr_t>(base) & 15) != 0) return false;
  if ((bx * sizeof(E)) % 16 != 0 || (pitch * sizeof(E)) % 16 != 0 || (plane * sizeof(E)) % 16 != 0) return false;
  if (bx > 256 || by > 256 || planes > 256) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)planes};
  const cuuint64_t strides[2] = {(cuuint64_t)pitch * sizeof(E), (cuuint64_t)plane * sizeof(E)};
  const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)planes};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(map, DType<E>::v, planes > 1 ? 3 : 2, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace tma
}  // namespace lbm
