// mma.cuh -- warp-level tensor-core helpers shared by the surrogate's GEMM kernels:
// ldmatrix fragment loads from shared memory, the m16n8k16 BF16 MMA with FP32
// accumulation, 16-byte cp.async, and GELU with its derivative (erf form, by a published
// rational-exponential approximation of erf).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace chem {

// Phi(x) = (1 + erf(x / sqrt 2)) / 2 (the standard normal distribution function) and
// exp(-x^2 / 2), from erf(u) = 1 - (a1 t + a2 t^2 + a3 t^3 + a4 t^4 + a5 t^5) e^(-u^2),
// t = 1 / (1 + p u), u >= 0 (Abramowitz & Stegun 7.1.26, |error| <= 1.5e-7).  For x < 0
// the tail 1 - erf(u) = poly e^(-u^2) is returned directly instead of cancelling 1 + erf,
// so Phi keeps a relative accuracy below BF16's there (0.16 % at x = -5).  One reciprocal and one exponential
// (the fast hardware approximations) and five FMAs.
__device__ __forceinline__ float phi_cdf(float x, float &e) {
  const float u = fabsf(x) * 0.70710678118654752f;
  const float t = __fdividef(1.0f, fmaf(0.3275911f, u, 1.0f));
  float p = fmaf(t, 1.061405429f, -1.453152027f);
  p = fmaf(t, p, 1.421413741f);
  p = fmaf(t, p, -0.284496736f);
  p = fmaf(t, p, 0.254829592f);
  p *= t;
  e = __expf(-u * u);
  const float tail = 0.5f * p * e;  // (1 - erf(u)) / 2
  return x >= 0.0f ? 1.0f - tail : tail;
}

__device__ __forceinline__ float gelu_f(float x) {
  float e;
  return x * phi_cdf(x, e);
}

// GELU'(x) = Phi(x) + x phi(x), phi(x) = exp(-x^2 / 2) / sqrt(2 pi)
__device__ __forceinline__ float gelu_grad_f(float x) {
  float e;
  const float c = phi_cdf(x, e);
  return fmaf(x * 0.39894228040143268f, e, c);
}

__device__ __forceinline__ void ldmatrix_x4(uint32_t (&r)[4], const void *smem) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

__device__ __forceinline__ void ldmatrix_x2(uint32_t (&r)[2], const void *smem) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n"
               : "=r"(r[0]), "=r"(r[1])
               : "r"(a));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(a), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

}  // namespace chem
