// fastmath.cuh -- table-driven fp64 exp and log for the FP64-pipe-bound kernels.
//
// On GB300 the FP64 pipe issues 2 lanes per clock per SM, and a library fp64 exp takes
// about 20 of those slots (log about 37).  The right-hand side needs ~38 exponentials
// and ~5 logarithms, so these two functions dominate its FP64 cost.  The versions here
// follow Tang's table-driven methods (ACM TOMS 15 (1989) 144-157 for exp, 16 (1990)
// 378-400 for log) with Taylor polynomials, in about 10 FP64 operations each; the
// exponent and table-index arithmetic runs on the integer pipe and the 64-entry tables
// live in shared memory.  Accuracy is about 1 ulp on the ranges used (checked against the
// CUDA library functions by the GPU tests through chem_diag_math).
#pragma once

#include <cstdint>

#include "math_tables.cuh"

namespace chem {

// Per-block copies of the tables: divergent table reads from shared memory cost far
// less latency than L1 round trips.  Every kernel that calls exp_t / log_t fills them
// first with load_math_tables() (all threads, then a barrier).
__shared__ double s_exp2_64[64];
__shared__ double s_log_inv[65];
__shared__ double s_log_tab[65];
__shared__ double s_log_tab_m1[65];

__device__ __forceinline__ void load_math_tables() {
  for (int i = threadIdx.x; i < 65; i += blockDim.x) {
    if (i < 64) s_exp2_64[i] = k_exp2_64[i];
    s_log_inv[i] = k_log_inv[i];
    s_log_tab[i] = k_log_tab[i];
    s_log_tab_m1[i] = k_log_tab_m1[i];
  }
  __syncthreads();
}

// exp(x).  Exact to ~1 ulp for x in [-708, 709]; the table index k is clamped with
// integer min/max and the 2^m scale is applied by a multiply, so arguments outside
// that range still give +inf above and a value below 1e-290 in magnitude below,
// with no fp64 compares.  Kept out of line: the right-hand side calls it ~38 times,
// and one shared copy keeps the kernel's code within the instruction cache (measured
// 4 % faster than inlining it on GB300).
static __device__ __noinline__ double exp_t(double x) {
  const double kShift = 6755399441055744.0;  // 1.5 * 2^52: rounds to an integer in the low bits
  const double t = fma(x, kInvLn2x64, kShift);
  const int k = min(max(__double2loint(t), -65408), 65471);  // 2^(k>>6) stays a normal double
  const double kd = (double)k;
  double r = fma(-kd, kLn2d64Hi, x);
  r = fma(-kd, kLn2d64Lo, r);
  // e^r - 1 = r + r^2/2 + r^3/6 + r^4/24 + r^5/120 + r^6/720, |r| <= ln2/128
  double p = fma(r, 1.0 / 720.0, 1.0 / 120.0);
  p = fma(r, p, 1.0 / 24.0);
  p = fma(r, p, 1.0 / 6.0);
  p = fma(r, p, 0.5);
  p = fma(r, p, 1.0);
  p = r * p;
  const double tj = s_exp2_64[k & 63];
  const double scale = __hiloint2double(((k >> 6) + 1023) << 20, 0);
  return fma(tj, p, tj) * scale;
}

// log(x) for positive normal finite x (the kernels' arguments: temperatures, F_cent,
// Pr); zero, subnormal, negative, inf and NaN inputs fall back to the library log via
// an integer test of the exponent field.
__device__ __forceinline__ double log_t(double x) {
  const long long bits = __double_as_longlong(x);
  const int ef = (int)(bits >> 52);  // sign and biased exponent
  if (ef <= 0 || ef >= 0x7ff) return log(x);
  const int ex = ef - 1023;
  const long long mb = bits & 0x000fffffffffffffLL;
  const int j = (int)(((mb >> 45) + 1) >> 1);  // nearest 64th of the fraction, 0..64
  const double f = __longlong_as_double(mb | 0x3ff0000000000000LL);
  const double r = fma(f, s_log_inv[j], -1.0);  // |r| <= 1/128
  // log1p(r) = r - r^2/2 + r^3/3 - r^4/4 + r^5/5 - r^6/6 + r^7/7
  double q = fma(r, 1.0 / 7.0, -1.0 / 6.0);
  q = fma(r, q, 1.0 / 5.0);
  q = fma(r, q, -0.25);
  q = fma(r, q, 1.0 / 3.0);
  q = fma(r, q, -0.5);
  const double r2 = r * r;
  const double l1p = fma(r2, q, r);
  // inputs in [0.5, 1): -ln(2 c_j) from the second table, no e ln2 term to cancel against
  if (ex == -1) return s_log_tab_m1[j] + l1p;
  const double e = (double)ex;
  return fma(e, kLn2Hi, s_log_tab[j] + fma(e, kLn2Lo, l1p));
}

__device__ __forceinline__ double log10_t(double x) { return log_t(x) * kInvLn10; }
__device__ __forceinline__ double exp10_t(double x) { return exp_t(x * kLn10); }

}  // namespace chem
