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

__device__ __forceinline__ float rcp_approx_f(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ float ex2_approx_f(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// GELU(x) = x Phi(x) with the same approximation, arranged for the fewest operations:
// x Phi(x) = max(x, 0) - |x| (1 - erf(u)) / 2 for either sign (u = |x| / sqrt 2), and
// (1 - erf(u)) / 2 = t Q(t) e^(-x^2 / 2) with Q the halved polynomial, so
// GELU = fma(-(|x| t) Q(t), 2^(-x^2 / (2 ln 2)), max(x, 0)).  For x < 0 the max is 0 and
// the result is one product (no cancellation, the tail keeps its relative accuracy); for
// x >= 0 it is x minus a tail below x / 2.  One reciprocal, one base-2 exponential (the
// hardware approximations), four FMAs for Q and five further multiplies or FMAs.
__device__ __forceinline__ float gelu_f(float x) {
  const float ax = fabsf(x);
  const float t = rcp_approx_f(fmaf(0.3275911f * 0.70710678118654752f, ax, 1.0f));
  float q = fmaf(t, 0.5307027145f, -0.7265760135f);  // a5 / 2, a4 / 2
  q = fmaf(t, q, 0.7107068705f);                      // a3 / 2
  q = fmaf(t, q, -0.142248368f);                      // a2 / 2
  q = fmaf(t, q, 0.127414796f);                       // a1 / 2
  const float e = ex2_approx_f(x * (x * -0.72134752044448170f));  // e^(-x^2 / 2)
  return fmaf(-(ax * t) * q, e, fmaxf(x, 0.0f));
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
