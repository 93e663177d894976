// rhs.cuh -- device right-hand side dY/dt of one constant-(rho, e) cell.
//
// Per evaluation: temperature from (e, Y) by Newton on NASA-7 (Eq. 10; calculate_T of
// Table 1), species Gibbs functions, Arrhenius / third-body / Troe forward rates,
// reverse rates from equilibrium constants (Sec. 2.1.2), law of mass action (Eq. 16),
// and F_k = W_k wdot_k / rho (Eq. 14, 20 at constant density).
//
// Arithmetic layout (the FP64 pipe of GB300 issues 2 lanes/clk/SM, so every fp64
// operation counts):
//   - exponentials and logarithms are the table-driven exp_t / log_t (fastmath.cuh);
//   - g_k / RT comes from one combined NASA-7 polynomial per species (6 FMAs);
//   - Newton works on mixture coefficients m_i = sum_k Y_k (ec_ki / W_k), assembled once
//     per evaluation (54 FMAs), so each iteration is two Horner chains and a reciprocal;
//   - equilibrium constants come from per-species G_k = exp(-g_k / RT):
//     1/K_c,j = prod_reactants G * prod_products (1/G) * (R_u T / p_ref)^(sum nu), i.e.
//     9 exponentials + 9 reciprocals per evaluation instead of one exponential per
//     reaction; with a_k = c_k / G_k the net rate of progress is
//     k_f (prod_reactants c - prod_reactants G * prod_products a * (R_u T / p_ref)^(sum nu)),
//     one FMA for the reverse direction;
//   - reciprocals are Newton-Raphson-refined hardware approximations (rcp1 / rcp2), ~3.5
//     and ~5.7 FP64-pipe slots against ~9 for an IEEE divide; compares, clamps and
//     fp32 <-> fp64 conversions run on the integer pipe (fastmath.cuh);
//   - forward rates are exp(ln A + beta ln T - Ta / T), one exponential per reaction
//     (none for temperature-independent rates or A T^-1, A T^-2 with no activation).
#pragma once

#include <cmath>
#include <utility>

#include "fastmath.cuh"
#include "mech.cuh"

namespace chem {

// Mixture internal-energy coefficients from mass fractions, shifted by the target:
// e/R_u - eR = T (m0 + T (m1 + T (m2 + T (m3 + T m4)))) + m5
__device__ __forceinline__ void mix_ecoef(const MechTables &mt, int range, const double (&Y)[NSP],
                                          double eR, double (&m)[6]) {
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < NSP; ++k) s = fma(Y[k], mt.ecw[range][k][i], s);
    m[i] = s;
  }
  m[5] -= eR;
}

__device__ __forceinline__ double e_over_R(const double (&m)[6], double T) {
  return fma(T, fma(T, fma(T, fma(T, fma(T, m[4], m[3]), m[2]), m[1]), m[0]), m[5]);
}

// cv/R = d(e/R)/dT from the scaled coefficients d = {m0, 2 m1, 3 m2, 4 m3, 5 m4}
__device__ __forceinline__ double cv_over_R(const double (&d)[5], double T) {
  return fma(T, fma(T, fma(T, fma(T, d[4], d[3]), d[2]), d[1]), d[0]);
}

__device__ __forceinline__ void cv_coef(const double (&m)[6], double (&d)[5]) {
  d[0] = m[0];
  d[1] = 2.0 * m[1];
  d[2] = 3.0 * m[2];
  d[3] = 4.0 * m[3];
  d[4] = 5.0 * m[4];
}

// Temperature from e/R_u and the mass fractions Y.  T: in = starting guess (1500 K if not
// positive and finite), out = root.  Newton stops at |dT| <= 1e-12 T, or as soon as the
// quadratic convergence bound guarantees that (dT^2 <= newton_sq T: the remaining error
// is then below 1e-12 T / 2), within 30 iterations; on a non-positive / non-finite
// iterate or no convergence, bisection on [200, 6000] K.  The step divides by c_v through
// a reciprocal with relative error ~2^-40 (a perturbed Newton step converges the same
// way), the stop test runs in fp32 on the rounded dT and T (it only decides when to
// stop), and the range and sign tests run on the integer pipe.
__device__ __forceinline__ bool solve_T(const MechTables &mt, const double (&Y)[NSP], double eR,
                                        double &T) {
  double Tn = pos_normal(T) ? T : 1500.0;
  int range = ge_nonneg(Tn, mt.T_mid);
  double m[6], d[5];
  mix_ecoef(mt, range, Y, eR, m);
  cv_coef(m, d);
  for (int it = 0; it < 30; ++it) {
    const int r = ge_nonneg(Tn, mt.T_mid);
    if (r != range) {
      range = r;
      mix_ecoef(mt, range, Y, eR, m);
      cv_coef(m, d);
    }
    const double dT = e_over_R(m, Tn) * rcp1(cv_over_R(d, Tn));
    Tn -= dT;
    if (!pos_normal(Tn)) break;
    const float dTf = d2f(dT), Tf = d2f(Tn);
    if (fabsf(dTf) <= 1e-12f * Tf || dTf * dTf <= mt.f.newton_sq * Tf) {
      T = Tn;
      return true;
    }
  }
  // bracketed fallback
  double lo = 200.0, hi = 6000.0, mlo[6], mhi[6];
  mix_ecoef(mt, lo >= mt.T_mid, Y, eR, mlo);
  mix_ecoef(mt, hi >= mt.T_mid, Y, eR, mhi);
  if (e_over_R(mlo, lo) > 0.0 || e_over_R(mhi, hi) < 0.0) return false;
  for (int it = 0; it < 200 && hi - lo > 1e-13 * hi; ++it) {
    const double mid = 0.5 * (lo + hi);
    mix_ecoef(mt, mid >= mt.T_mid, Y, eR, m);
    if (e_over_R(m, mid) > 0.0) hi = mid; else lo = mid;
  }
  T = 0.5 * (lo + hi);
  return true;
}

// Quantities shared by every reaction of one evaluation.
struct RateInputs {
  double lnT, invT, RTP, PRT, ctot;
  double c[NSP];   // clamped concentrations, mol/m^3
  double G[NSP];   // exp(-g_k / (R_u T))
  double iG[NSP];  // 1 / G_k (with the one-way fluxes) or c_k / G_k (net rates only)
};

// Troe broadening factor (Gilbert, Luther & Troe 1983).
template <int J>
__device__ __forceinline__ double troe_F(const MechTables &mt, double T, double invT, double Pr) {
  constexpr int n = kRx[J].troe_n;
  if constexpr (n == 0) {
    return 1.0;
  } else {
    const double a = mt.troe_a[J];
    double Fc = (1.0 - a) * exp_t(-T * mt.troe_i3[J]) + a * exp_t(-T * mt.troe_i1[J]);
    if constexpr (n == 4) Fc += exp_t(-mt.troe_T2[J] * invT);
    const double lFc = log10_t(Fc);
    const double cc = -0.4 - 0.67 * lFc;
    const double nn = 0.75 - 1.27 * lFc;
    const double x = log10_t(Pr) + cc;
    const double f1 = x * rcp2(nn - 0.14 * x);
    return exp10_t(lFc / (1.0 + f1 * f1));
  }
}

// Rate of progress of reaction J added into wdot (law of mass action, Eq. 16).  With
// kDestr, the one-way fluxes that consume each species are also summed into dflux
// (used by the stiffness probe: consumption rate per unit concentration).
template <int J, bool kDestr = false>
__device__ __forceinline__ void reaction(const MechTables &mt, const RateInputs &in, double T,
                                         double (&wdot)[NSP], double *dflux = nullptr) {
  constexpr RxStruct R = kRx[J];
  constexpr int dnu = n_prod(R) - n_reac(R);
  static_assert(dnu >= -1 && dnu <= 1, "compiled structure assumes |sum nu| <= 1");
  // kconst: 0 Arrhenius exponential; 1 constant (b = Ea = 0); 2, 3: A T^-1, A T^-2 (Ea = 0)
  const int kc = mt.kconst[J];
  double kf;
  if (kc == 0) kf = exp_t(fma(mt.beta[J], in.lnT, mt.lnA[J]) - mt.Ta[J] * in.invT);
  else if (kc == 1) kf = mt.A[J];
  else if (kc == 2) kf = mt.A[J] * in.invT;
  else kf = mt.A[J] * in.invT * in.invT;
  double M = 0.0;
  if constexpr (R.type != ELEM) {
    M = in.ctot;
    if (mt.has_eff[J]) {
#pragma unroll
      for (int k = 0; k < NSP; ++k)
        if ((mt.eff_mask[J] >> k) & 1) M = fma(mt.effm1[J][k], in.c[k], M);
    }
  }
  if constexpr (R.type == FALLOFF) {
    const double k0 = exp_t(fma(mt.beta0[J], in.lnT, mt.lnA0[J]) - mt.Ta0[J] * in.invT);
    const double Pr = k0 * M * rcp2(kf);
    kf = (Pr > 0.0) ? kf * (Pr * rcp2(1.0 + Pr)) * troe_F<J>(mt, T, in.invT, Pr) : 0.0;
  }
  double q;
  if constexpr (kDestr) {
    double qf = kf * in.c[R.r0];
    if constexpr (R.r1 >= 0) qf *= in.c[R.r1];
    double qr = 0.0;
    q = qf;
    if (mt.reversible[J]) {
      double kr = kf * in.G[R.r0];
      if constexpr (R.r1 >= 0) kr *= in.G[R.r1];
      kr *= in.iG[R.p0];
      if constexpr (R.p1 >= 0) kr *= in.iG[R.p1];
      if constexpr (dnu == 1) kr *= in.RTP;
      if constexpr (dnu == -1) kr *= in.PRT;
      qr = kr * in.c[R.p0];
      if constexpr (R.p1 >= 0) qr *= in.c[R.p1];
      q = qf - qr;
    }
    const double m = (R.type == THIRD_BODY) ? M : 1.0;
    dflux[R.r0] += m * qf;
    if constexpr (R.r1 >= 0) dflux[R.r1] += m * qf;
    dflux[R.p0] += m * qr;
    if constexpr (R.p1 >= 0) dflux[R.p1] += m * qr;
  } else {
    // q = k_f (prod c_reactants - prod G_reactants prod (c / G)_products (R_u T / p)^dnu),
    // the same net rate as k_f prod c - k_r prod c with k_r = k_f / K_c
    double cf = in.c[R.r0];
    if constexpr (R.r1 >= 0) cf *= in.c[R.r1];
    if (mt.reversible[J]) {
      double gr = in.G[R.r0];
      if constexpr (R.r1 >= 0) gr *= in.G[R.r1];
      if constexpr (dnu == 1) gr *= in.RTP;
      if constexpr (dnu == -1) gr *= in.PRT;
      double ap = in.iG[R.p0];
      if constexpr (R.p1 >= 0) ap *= in.iG[R.p1];
      cf = fma(-gr, ap, cf);
    }
    q = kf * cf;
  }
  if constexpr (R.type == THIRD_BODY) q *= M;
  wdot[R.r0] -= q;
  if constexpr (R.r1 >= 0) wdot[R.r1] -= q;
  wdot[R.p0] += q;
  if constexpr (R.p1 >= 0) wdot[R.p1] += q;
}

template <bool kDestr, int... J>
__device__ __forceinline__ void all_reactions(const MechTables &mt, const RateInputs &in, double T,
                                              double (&wdot)[NSP], double *dflux,
                                              std::integer_sequence<int, J...>) {
  (reaction<J, kDestr>(mt, in, T, wdot, dflux), ...);
}

// Molar production rates wdot (mol/m^3/s) at temperature T and clamped concentrations c.
// kDestr: also the consumption fluxes per species into dflux (zeroed here).
template <bool kDestr = false>
__device__ __forceinline__ void production_rates(const MechTables &mt, double T,
                                                 const double (&c)[NSP], double (&wdot)[NSP],
                                                 double *dflux = nullptr) {
  RateInputs in;
  in.lnT = log_t(T);
  in.invT = rcp2(T);
  in.RTP = (R_U / P_REF) * T;
  in.PRT = (P_REF / R_U) * in.invT;
  const double oml = 1.0 - in.lnT;
  const int range = ge_nonneg(T, mt.T_mid);
  double ctot = 0.0;
#pragma unroll
  for (int k = 0; k < NSP; ++k) {
    in.c[k] = c[k];
    ctot += c[k];
    const double *gc = mt.gc[range][k];
    double g = fma(T, fma(T, fma(T, fma(T, gc[4], gc[3]), gc[2]), gc[1]), fma(gc[5], in.invT, gc[6]));
    g = fma(gc[0], oml, g);
    // clamp keeps G finite far outside the tables' range
    g = clamp_abs(g, 700.0);
    in.G[k] = exp_t(-g);
    in.iG[k] = kDestr ? rcp2(in.G[k]) : c[k] * rcp2(in.G[k]);
    wdot[k] = 0.0;
    if constexpr (kDestr) dflux[k] = 0.0;
  }
  in.ctot = ctot;
  all_reactions<kDestr>(mt, in, T, wdot, dflux, std::make_integer_sequence<int, NRX>{});
}

// dY/dt of one cell at fixed (rho, e).  T: in = Newton guess, out = solved T.
// Returns false when the temperature solve fails.
__device__ __forceinline__ bool cell_rhs(const MechTables &mt, const double (&Y)[NSP], double rho,
                                         double invRho, double eR, double &T, double (&F)[NSP]) {
  if (!solve_T(mt, Y, eR, T)) return false;
  double c[NSP], wdot[NSP];
#pragma unroll
  for (int k = 0; k < NSP; ++k) c[k] = clamp_nonneg(rho * (Y[k] * mt.invW[k]));
  production_rates(mt, T, c, wdot);
#pragma unroll
  for (int k = 0; k < NSP; ++k) F[k] = wdot[k] * mt.W[k] * invRho;
  return true;
}

}  // namespace chem
