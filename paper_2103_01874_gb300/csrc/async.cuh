// Asynchronous global -> shared copies (cp.async, sm_80+ PTX), so that a CTA
// can put a whole tile of loads in flight before it waits once.
#pragma once
#include <cuda_runtime.h>

namespace ppe {

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
// 8-byte copy (float2-sized elements)
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_addr(smem)), "l"(gmem) : "memory");
}
// 16-byte copy (double2-sized elements); both addresses 16-byte aligned
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(smem)), "l"(gmem) : "memory");
}
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
  if (BYTES == 16) cp_async16(smem, gmem);
  else cp_async8(smem, gmem);
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

}  // namespace ppe
