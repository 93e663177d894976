// rhs_mixed.cuh -- mixed-precision right-hand side of one constant-(rho, e) cell.
//
// The same right-hand side as rhs.cuh (Eq. 10, 14-16), split by precision:
//   fp64: the temperature solve (Newton on the mixture NASA-7 coefficients), ln T, 1/T,
//         the Gibbs functions g_k / RT and ln(R_u T / p_ref);
//   fp32: forward rate coefficients, third-body sums, Troe fall-off, reverse rates
//         k_r = exp(ln k_f + ln(1 / K_c)), the law-of-mass-action products, production
//         rates and F.
// The equilibrium exponents ln(1 / K_c,j) = sum_k nu_jk g_k + (sum_k nu_jk) ln(R_u T / p_ref)
// are the fp64 sums rounded once to fp32: each fp64 term is split into an fp32 hi part
// on a 2^-12 grid (whose sums are exact in fp32) and an fp32 lo part, so the sum needs
// no fp64 add.  The fp32 work runs on the FMA/MUFU pipes, 64x the FP64 pipe's throughput
// on GB300; what stays in fp64 is the part whose accuracy decides the temperature and
// the equilibrium state, and the conversions between the two run on the integer pipe.
#pragma once

#include "rhs.cuh"

namespace chem {

struct RateInputsF {
  float lnT, invT, T, ctot;
  float c[NSP];
};

// fp32 transcendentals and divisions of the rate expressions: the CUDA library's
// accurate functions for the integrator, or its fast intrinsics (hardware base-2
// exponential and logarithm, approximate division; relative errors ~1e-6 on these
// arguments) for the error test's estimator, which compares with a tolerance of ~5e-4 T.
template <bool FAST>
__device__ __forceinline__ float exp_r(float x) {
  if constexpr (FAST) return __expf(x); else return expf(x);
}
template <bool FAST>
__device__ __forceinline__ float log_r(float x) {
  if constexpr (FAST) return __logf(x); else return logf(x);
}
template <bool FAST>
__device__ __forceinline__ float log10_r(float x) {
  if constexpr (FAST) return __log10f(x); else return log10f(x);
}
template <bool FAST>
__device__ __forceinline__ float exp10_r(float x) {
  if constexpr (FAST) return __exp10f(x); else return exp10f(x);
}
template <bool FAST>
__device__ __forceinline__ float div_r(float a, float b) {
  if constexpr (FAST) return __fdividef(a, b); else return a / b;
}

template <int J, bool FAST>
__device__ __forceinline__ float troe_F_f32(const MechTables &mt, float T, float invT, float Pr) {
  constexpr int n = kRx[J].troe_n;
  if constexpr (n == 0) {
    return 1.0f;
  } else {
    const float a = mt.f.troe_a[J];
    float Fc = (1.0f - a) * exp_r<FAST>(-T * mt.f.troe_i3[J]) + a * exp_r<FAST>(-T * mt.f.troe_i1[J]);
    if constexpr (n == 4) Fc += exp_r<FAST>(-mt.f.troe_T2[J] * invT);
    const float lFc = log10_r<FAST>(Fc);
    const float cc = -0.4f - 0.67f * lFc;
    const float nn = 0.75f - 1.27f * lFc;
    const float x = log10_r<FAST>(Pr) + cc;
    const float f1 = div_r<FAST>(x, nn - 0.14f * x);
    return exp10_r<FAST>(div_r<FAST>(lFc, 1.0f + f1 * f1));
  }
}

// The ingredients of ln(1/K_c,j) = sum_k nu_jk g_k + (sum_k nu_jk) ln(R_u T / p_ref).
// GibbsHL (mixed variant): the fp64 g_k / RT and ln(R_u T / p_ref) as fp32 hi/lo pairs
// (split_hilo); the hi parts sum exactly in fp32 and the lo parts carry the rest, so
// the fp32 ln(1/K_c) is the fp64 sum rounded once (to within ~1e-11) without an fp64
// add per term.  GibbsF (the error test's all-fp32 right-hand side): plain fp32.
struct GibbsHL {
  float h[NSP], l[NSP];
  float rh, rl;
};
struct GibbsF {
  float g[NSP];
  float r;
};

// g_k / RT = a1 (1 - ln T) - a2 T / 2 - ... - a5 T^4 / 20 + a6 / T - a7 (NASA-7, with the
// coefficients pre-combined per range into gc) and ln(R_u T / p_ref), evaluated in fp64
// and split into fp32 hi/lo pairs.
__device__ __forceinline__ void gibbs_hl(const MechTables &mt, double T, double lnT, double invT, GibbsHL &g) {
  const double oml = 1.0 - lnT;
  const int range = ge_nonneg(T, mt.T_mid);
#pragma unroll
  for (int k = 0; k < NSP; ++k) {
    const double *gc = mt.gc[range][k];
    const double gk = fma(T, fma(T, fma(T, fma(T, gc[4], gc[3]), gc[2]), gc[1]), fma(gc[5], invT, gc[6]));
    split_hilo(fma(gc[0], oml, gk), g.h[k], g.l[k]);
  }
  split_hilo(lnT + mt.ln_R_over_Pref, g.rh, g.rl);
}

// The same functions evaluated entirely in fp32 (the error test's right-hand side).
__device__ __forceinline__ void gibbs_f(const MechTables &mt, float T, float lnT, float invT, GibbsF &g) {
  const float oml = 1.0f - lnT;
  const int range = T >= mt.f.T_mid;
#pragma unroll
  for (int k = 0; k < NSP; ++k) {
    const float *gc = mt.f.gc[range][k];
    const float gk = fmaf(T, fmaf(T, fmaf(T, fmaf(T, gc[4], gc[3]), gc[2]), gc[1]), fmaf(gc[5], invT, gc[6]));
    g.g[k] = fmaf(gc[0], oml, gk);
  }
  g.r = lnT + mt.f.ln_R_over_Pref;
}

template <int J>
__device__ __forceinline__ float ln_inv_kc(const GibbsHL &g) {
  constexpr RxStruct R = kRx[J];
  constexpr int dnu = n_prod(R) - n_reac(R);
  float h = g.h[R.p0] - g.h[R.r0], l = g.l[R.p0] - g.l[R.r0];
  if constexpr (R.p1 >= 0) { h += g.h[R.p1]; l += g.l[R.p1]; }
  if constexpr (R.r1 >= 0) { h -= g.h[R.r1]; l -= g.l[R.r1]; }
  if constexpr (dnu == 1) { h += g.rh; l += g.rl; }
  if constexpr (dnu == -1) { h -= g.rh; l -= g.rl; }
  return h + l;
}

template <int J>
__device__ __forceinline__ float ln_inv_kc(const GibbsF &g) {
  constexpr RxStruct R = kRx[J];
  constexpr int dnu = n_prod(R) - n_reac(R);
  float q = g.g[R.p0] - g.g[R.r0];
  if constexpr (R.p1 >= 0) q += g.g[R.p1];
  if constexpr (R.r1 >= 0) q -= g.g[R.r1];
  if constexpr (dnu == 1) q += g.r;
  if constexpr (dnu == -1) q -= g.r;
  return q;
}

template <int J, bool FAST, typename Gibbs>
__device__ __forceinline__ void reaction_mixed(const MechTables &mt, const RateInputsF &in,
                                               const Gibbs &g, float (&wdot)[NSP]) {
  constexpr RxStruct R = kRx[J];
  float lnkf = fmaf(mt.f.beta[J], in.lnT, mt.f.lnA[J]) - mt.f.Ta[J] * in.invT;
  float kf = mt.kconst[J] == 1 ? mt.f.A[J] : exp_r<FAST>(lnkf);
  float M = 0.0f;
  if constexpr (R.type != ELEM) {
    M = in.ctot;
    if (mt.has_eff[J]) {
#pragma unroll
      for (int k = 0; k < NSP; ++k) M = fmaf(mt.f.effm1[J][k], in.c[k], M);
    }
  }
  if constexpr (R.type == FALLOFF) {
    const float k0 = exp_r<FAST>(fmaf(mt.f.beta0[J], in.lnT, mt.f.lnA0[J]) - mt.f.Ta0[J] * in.invT);
    const float Pr = div_r<FAST>(k0 * M, kf);
    kf = (Pr > 0.0f) ? kf * div_r<FAST>(Pr, 1.0f + Pr) * troe_F_f32<J, FAST>(mt, in.T, in.invT, Pr) : 0.0f;
    lnkf = log_r<FAST>(kf);
  }
  float qf = kf * in.c[R.r0];
  if constexpr (R.r1 >= 0) qf *= in.c[R.r1];
  float q = qf;
  if (mt.reversible[J]) {
    const float kr = (kf > 0.0f) ? exp_r<FAST>(lnkf + ln_inv_kc<J>(g)) : 0.0f;
    float qr = kr * in.c[R.p0];
    if constexpr (R.p1 >= 0) qr *= in.c[R.p1];
    q = qf - qr;
  }
  if constexpr (R.type == THIRD_BODY) q *= M;
  wdot[R.r0] -= q;
  if constexpr (R.r1 >= 0) wdot[R.r1] -= q;
  wdot[R.p0] += q;
  if constexpr (R.p1 >= 0) wdot[R.p1] += q;
}

template <bool FAST, typename Gibbs, int... J>
__device__ __forceinline__ void all_reactions_mixed(const MechTables &mt, const RateInputsF &in,
                                                    const Gibbs &g, float (&wdot)[NSP],
                                                    std::integer_sequence<int, J...>) {
  (reaction_mixed<J, FAST, Gibbs>(mt, in, g, wdot), ...);
}

// dY/dt (fp32) of one cell at fixed (rho, e) from the fp32 stage state U.
// T: in = Newton guess, out = solved T (fp64).  Returns false when the solve fails.
__device__ __forceinline__ bool cell_rhs_mixed(const MechTables &mt, const float (&U)[NSP],
                                               float rho_f, float invRho_f, double eR, double &T,
                                               float (&F)[NSP]) {
  double Y[NSP];
#pragma unroll
  for (int k = 0; k < NSP; ++k) Y[k] = f2d(U[k]);
  if (!solve_T(mt, Y, eR, T)) return false;
  const double lnT = log_t(T);
  const double invT = rcp1(T);
  GibbsHL g;
  gibbs_hl(mt, T, lnT, invT, g);
  RateInputsF in;
  in.lnT = d2f(lnT);
  in.invT = d2f(invT);
  in.T = d2f(T);
  float ctot = 0.0f, wdot[NSP];
#pragma unroll
  for (int k = 0; k < NSP; ++k) {
    in.c[k] = fmaxf(rho_f * U[k] * mt.f.invW[k], 0.0f);
    ctot += in.c[k];
    wdot[k] = 0.0f;
  }
  in.ctot = ctot;
  all_reactions_mixed<false>(mt, in, g, wdot, std::make_integer_sequence<int, NRX>{});
#pragma unroll
  for (int k = 0; k < NSP; ++k) F[k] = wdot[k] * mt.f.W[k] * invRho_f;
  return true;
}

// Temperature from e/R_u and Y/W entirely in fp32 (for the error test): Newton from T
// (1500 K if not positive and finite), |dT| <= 2e-6 T within 12 iterations; false on
// no convergence or a non-positive / non-finite iterate (the test then rejects).
__device__ __forceinline__ bool solve_T_f32(const MechTables &mt, const float (&yw)[NSP], float eR, float &T) {
  float Tn = (isfinite(T) && T > 0.0f) ? T : 1500.0f;
  int range = -1;
  float m[6], d[5];
  for (int it = 0; it < 12; ++it) {
    const int r = Tn >= mt.f.T_mid;
    if (r != range) {
      range = r;
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        float s = 0.0f;
#pragma unroll
        for (int k = 0; k < NSP; ++k) s = fmaf(yw[k], mt.f.ec[range][k][i], s);
        m[i] = s;
      }
      d[0] = m[0];
      d[1] = 2.0f * m[1];
      d[2] = 3.0f * m[2];
      d[3] = 4.0f * m[3];
      d[4] = 5.0f * m[4];
    }
    const float eT = fmaf(Tn, fmaf(Tn, fmaf(Tn, fmaf(Tn, fmaf(Tn, m[4], m[3]), m[2]), m[1]), m[0]), m[5]);
    const float cv = fmaf(Tn, fmaf(Tn, fmaf(Tn, fmaf(Tn, d[4], d[3]), d[2]), d[1]), d[0]);
    const float dT = __fdividef(eT - eR, cv);
    Tn -= dT;
    if (!isfinite(Tn) || Tn <= 0.0f) return false;
    if (fabsf(dT) <= 2e-6f * Tn) {
      T = Tn;
      return true;
    }
  }
  return false;
}

// dY/dt of one cell entirely in fp32 (temperature, Gibbs functions and ln(1/K_c)
// included) with the fast intrinsics: the right-hand side of the surrogate's error test,
// an estimator that needs relative accuracy far coarser than fp32's.  T: in = guess, out = solved T.
__device__ __forceinline__ bool cell_rhs_f32(const MechTables &mt, const float (&U)[NSP], float rho,
                                             float invRho, float eR, float &T, float (&F)[NSP]) {
  float yw[NSP];
#pragma unroll
  for (int k = 0; k < NSP; ++k) yw[k] = U[k] * mt.f.invW[k];
  if (!solve_T_f32(mt, yw, eR, T)) return false;
  const float lnT = __logf(T);
  const float invT = __fdividef(1.0f, T);
  GibbsF g;
  gibbs_f(mt, T, lnT, invT, g);
  RateInputsF in;
  in.lnT = lnT;
  in.invT = invT;
  in.T = T;
  float ctot = 0.0f, wdot[NSP];
#pragma unroll
  for (int k = 0; k < NSP; ++k) {
    in.c[k] = fmaxf(rho * yw[k], 0.0f);
    ctot += in.c[k];
    wdot[k] = 0.0f;
  }
  in.ctot = ctot;
  all_reactions_mixed<true>(mt, in, g, wdot, std::make_integer_sequence<int, NRX>{});
#pragma unroll
  for (int k = 0; k < NSP; ++k) F[k] = wdot[k] * mt.f.W[k] * invRho;
  return true;
}

}  // namespace chem
