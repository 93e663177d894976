// fastmath.cuh -- fp64 device math for the FP64-pipe-bound kernels: table-driven exp
// and log, Newton-Raphson reciprocals, and fp32 <-> fp64 conversions, compares and
// clamps on the integer pipe.
//
// On GB300 the FP64 pipe issues 2 lanes per clock per SM, and a library fp64 exp takes
// about 20 of those slots (log about 37).  The right-hand side needs ~38 exponentials
// and ~5 logarithms, so these two functions dominate its FP64 cost.  The versions here
// follow Tang's table-driven methods (ACM TOMS 15 (1989) 144-157 for exp, 16 (1990)
// 378-400 for log) with Taylor polynomials, in about 10 FP64 operations each; the
// exponent and table-index arithmetic runs on the integer pipe and the 128-entry (exp)
// and 65-entry (log) tables live in shared memory.  Accuracy is about 1 ulp on the
// ranges used (checked against the CUDA library functions by the GPU tests through
// chem_diag_math).
#pragma once

#include <cstdint>

#include "math_tables.cuh"

namespace chem {

// Per-block copies of the tables: divergent table reads from shared memory cost far
// less latency than L1 round trips.  Every kernel that calls exp_t / log_t fills them
// first with load_math_tables() (all threads, then a barrier).
__shared__ double s_exp2_128[128];
__shared__ double s_log_inv[65];
__shared__ double s_log_tab[65];
__shared__ double s_log_tab_m1[65];

__device__ __forceinline__ void load_math_tables() {
  for (int i = threadIdx.x; i < 128; i += blockDim.x) {
    s_exp2_128[i] = k_exp2_128[i];
    if (i < 65) {
      s_log_inv[i] = k_log_inv[i];
      s_log_tab[i] = k_log_tab[i];
      s_log_tab_m1[i] = k_log_tab_m1[i];
    }
  }
  __syncthreads();
}

// exp(x).  About 1 ulp for x in [-708, 709]: x = (128 m + j) ln2/128 + r, |r| <= ln2/256,
// e^r - 1 by its degree-5 Taylor polynomial (truncation below 6e-19 relative), and the
// scale 2^m added to the exponent field of the table entry 2^(j/128) on the integer
// pipe (10 FP64-pipe operations in all).  Arguments beyond +-710 are first clamped there
// on the integer pipe, so they still give +inf above and a positive value below 1e-307
// below, however large; a NaN stays NaN.  Kept out of line: the right-hand side calls it
// ~38 times, and one shared copy keeps the kernel's code within the instruction cache
// (measured 4 % faster than inlining it on GB300).
static __device__ __noinline__ double exp_t(double x) {
  const long long kLim = 0x40863000'00000000LL;  // 710.0
  const long long b = __double_as_longlong(x);
  const long long ab = b & 0x7fffffffffffffffLL;
  if (ab > kLim && ab <= 0x7ff0000000000000LL) x = __longlong_as_double((b & (long long)0x8000000000000000ULL) | kLim);
  const double kShift = 6755399441055744.0;  // 1.5 * 2^52: rounds to an integer in the low bits
  const double t = fma(x, kInvLn2x128, kShift);
  const int k = min(max(__double2loint(t), -130816), 130943);  // 2^(k>>7) stays a normal double
  const double kd = (double)k;
  double r = fma(-kd, kLn2d128Hi, x);
  r = fma(-kd, kLn2d128Lo, r);
  // e^r - 1 = r + r^2/2 + r^3/6 + r^4/24 + r^5/120
  double p = fma(r, 1.0 / 120.0, 1.0 / 24.0);
  p = fma(r, p, 1.0 / 6.0);
  p = fma(r, p, 0.5);
  p = fma(r, p, 1.0);
  p = r * p;
  const double tj = s_exp2_128[k & 127];
  const double ts = __hiloint2double(__double2hiint(tj) + ((k >> 7) << 20), __double2loint(tj));
  return fma(ts, p, ts);
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

// ---- fp32 <-> fp64 conversions on the integer pipe ----
// On GB300 a cvt between fp32 and fp64 takes an FP64-pipe slot, the same as a DFMA
// (measured), and the mixed-precision right-hand side converts ~50 values per
// evaluation.  These two build the IEEE-754 bit patterns with integer operations
// instead.  Both give a signed zero for magnitudes below the fp32 normal range
// (2^-126) and keep infinities and NaNs.

// fp32 -> fp64: exact for normal numbers
__device__ __forceinline__ double f2d(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t a = u & 0x7fffffffu;
  uint32_t hi = (a >> 3) + 0x38000000u;     // exponent bias 127 -> 1023
  if (a >= 0x7f800000u) hi |= 0x7ff00000u;  // inf / NaN: all-ones exponent
  const bool tiny = a < 0x00800000u;
  hi = tiny ? 0u : hi;
  const uint32_t lo = tiny ? 0u : (u << 29);
  return __hiloint2double((int)(hi | (u & 0x80000000u)), (int)lo);
}

// fp64 -> fp32, rounded to nearest (ties to even); |d| >= 2^128 gives inf
__device__ __forceinline__ float d2f(double d) {
  const uint32_t hi = (uint32_t)__double2hiint(d), lo = (uint32_t)__double2loint(d);
  const uint32_t a = hi & 0x7fffffffu;
  uint32_t r = ((a - 0x38000000u) << 3) | (lo >> 29);  // exponent bias 1023 -> 127, 23 bits
  const uint32_t guard = (lo >> 28) & 1u;
  const uint32_t sticky = (lo & 0x0fffffffu) != 0u;
  r += guard & (sticky | (r & 1u));  // a carry out of the fraction bumps the exponent
  r = a >= 0x47f00000u ? 0x7f800000u : r;
  r = (a > 0x7ff00000u || (a == 0x7ff00000u && lo != 0u)) ? 0x7fc00000u : r;
  r = a < 0x38100000u ? 0u : r;
  return __uint_as_float(r | (hi & 0x80000000u));
}

// ---- fp64 reciprocals ----
// An IEEE fp64 divide costs ~9 FP64-pipe slots on GB300 (measured).  Here 1/x starts
// from the hardware approximation rcp.approx.ftz.f64 and takes Newton-Raphson steps
// r <- r + r (1 - x r), each of which squares the relative error (the approximation's
// is near 2^-20): one step for a relative error near 2^-40 (Newton's derivative), two
// for a result within an ulp or two.  x must be finite, nonzero and normal (0 gives
// NaN).
__device__ __forceinline__ double rcp_approx(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  return r;
}
__device__ __forceinline__ double rcp1(double x) {
  const double r = rcp_approx(x);
  return fma(r, fma(-x, r, 1.0), r);
}
__device__ __forceinline__ double rcp2(double x) {
  const double r = rcp1(x);
  return fma(r, fma(-x, r, 1.0), r);
}

// ---- fp64 tests and selects on the integer pipe ----
// x positive, finite and normal
__device__ __forceinline__ bool pos_normal(double x) {
  return (uint32_t)__double2hiint(x) - 0x00100000u < 0x7fe00000u;
}
// a >= b for non-negative a, b (the bit patterns of non-negative doubles are ordered)
__device__ __forceinline__ bool ge_nonneg(double a, double b) {
  return __double_as_longlong(a) >= __double_as_longlong(b);
}
// max(|a|, |b|); a NaN operand gives NaN
__device__ __forceinline__ double max_abs(double a, double b) {
  const long long x = __double_as_longlong(a) & 0x7fffffffffffffffLL;
  const long long y = __double_as_longlong(b) & 0x7fffffffffffffffLL;
  return __longlong_as_double(x > y ? x : y);
}
// max(x, 0) (negative values, -0 and NaNs with the sign bit set give +0)
__device__ __forceinline__ double clamp_nonneg(double x) {
  const long long b = __double_as_longlong(x);
  return __longlong_as_double(b & ~(b >> 63));
}

// x clamped to [-lim, lim] for lim > 0 (a NaN gives +-lim)
__device__ __forceinline__ double clamp_abs(double x, double lim) {
  const long long b = __double_as_longlong(x);
  const long long l = __double_as_longlong(lim);
  return (b & 0x7fffffffffffffffLL) > l ? __longlong_as_double((b & (long long)0x8000000000000000ULL) | l) : x;
}

// x = hi + lo for an fp64 x of magnitude below 2^12: hi is x truncated to a multiple of
// 2^-12 (at most 24 significant bits, so exact in fp32) and lo = x - hi (|lo| < 2^-12)
// rounded to fp32, an absolute error below 2^-37.  A signed sum of a few such hi parts
// whose magnitude stays below 2^12 is exact in fp32, so an fp64 sum with heavy
// cancellation (ln K_c from Gibbs functions of magnitude up to a few hundred) is
// assembled in fp32 to within an ulp of the result plus ~1e-11.
__device__ __forceinline__ void split_hilo(double x, float &hi, float &lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int n = 40 - ((int)((b >> 52) & 0x7ff) - 1023);  // fraction bits worth < 2^-12
  const unsigned long long mask = n >= 53 ? 0ull : (n <= 0 ? ~0ull : (~0ull << n));
  const double h = __longlong_as_double((long long)(b & mask));
  hi = d2f(h);
  lo = d2f(x - h);
}

}  // namespace chem
