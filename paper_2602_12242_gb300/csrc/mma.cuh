// Helpers shared by the conv-net kernels (cnn.cu) and the DFT-as-GEMM stage
// (dftgemm.cu): BF16 conversion and cp.async.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace mx {

typedef unsigned short bf16_t;

__device__ __forceinline__ bf16_t f2bf(float f) {
  const __nv_bfloat16_raw r = __float2bfloat16_rn(f);
  return r.x;
}
__device__ __forceinline__ float bf2f(bf16_t h) {
  __nv_bfloat16_raw r;
  r.x = h;
  return __bfloat162float(r);
}
__device__ __forceinline__ uint32_t pack2(float a, float b) {
  return (uint32_t)f2bf(a) | ((uint32_t)f2bf(b) << 16);
}
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp_async16(uint32_t saddr, const void* g, bool valid) {
  const int n = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(saddr), "l"(g), "r"(n));
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n" ::);
  asm volatile("cp.async.wait_group 0;\n" ::);
}


}  // namespace mx
