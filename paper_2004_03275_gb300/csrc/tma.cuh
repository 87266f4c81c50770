// Tensor-memory-accelerator (TMA) helpers.
//
// Host: a 2D float32 tensor map (cuTensorMapEncodeTiled, reached through the
// runtime's driver entry point, so the library does not link the driver library).
// Device: one bulk tensor copy global -> shared with mbarrier completion
// (cp.async.bulk.tensor + mbarrier.arrive.expect_tx), and a bounded wait on the
// barrier phase so that a copy that never lands cannot hang the kernel.
//
// Rules the callers keep: the shared destination is 128-byte aligned, the inner
// (x) coordinate times 4 bytes is a multiple of 16 (it is 0 here), the global base
// is 16-byte aligned and the row stride a multiple of 16 bytes, and the byte count
// given to expect_tx equals the box size.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace amrgpu {

// host: rows x cols float32 tensor, row stride cols * 4 bytes, box of br rows x bc columns
inline cudaError_t encode_tmap_2d(CUtensorMap* map, const float* base, uint64_t rows, uint64_t cols, uint32_t bc,
                                  uint32_t br) {
  using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static Encode fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p) return cudaErrorNotSupported;
    fn = reinterpret_cast<Encode>(p);
  }
  if ((reinterpret_cast<uintptr_t>(base) & 15) || ((cols * sizeof(float)) & 15) || ((bc * sizeof(float)) & 15))
    return cudaErrorInvalidValue;
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {cols * sizeof(float)};
  cuuint32_t box[2] = {bc, br};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

namespace tma {

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// order this thread's earlier generic shared-memory accesses before later async-proxy writes
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// one arrival that also announces `bytes` of transaction for the current phase
__device__ __forceinline__ void bar_expect(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ bool bar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// wait for the phase `parity` to complete; false after `limit` attempts (each try_wait
// itself suspends for a bounded, implementation-defined time)
__device__ __forceinline__ bool bar_wait(uint64_t* bar, unsigned parity, int limit) {
  for (int i = 0; i < limit; ++i)
    if (bar_try_wait(bar, parity)) return true;
  return false;
}

}  // namespace tma
}  // namespace amrgpu
