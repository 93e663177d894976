/*
 * Plain FP64 CPU oracle for the per-cell chemistry integrator.
 *
 * TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the CPU-baseline leg
 * of the benchmark call this library; the GPU product path never does, and this file
 * shares no code, header or table with it.  It is written to be checked by eye
 * against the paper, not to be fast: scalar loops, library exp/log/pow, no reordering.
 *
 * Each cell is a constant-density, constant-internal-energy adiabatic reactor: the
 * chemical source term of Eq. 14 changes only the partial densities, so rho and e
 * stay fixed while the mass fractions Y_k evolve.  What is computed:
 *   - species thermo from NASA-7 tables, and the mixture internal energy of Eq. 10;
 *   - temperature from (e, Y) by Newton-Raphson (the calculate_T kernel of Table 1),
 *     with a bisection fallback;
 *   - molar production rates by the law of mass action (Eq. 15-16), Arrhenius
 *     forward rates and reverse rates from the equilibrium constant (Sec. 2.1.2),
 *     plus third-body and Troe fall-off reactions;
 *   - the five-stage fourth-order low-storage RK of Eq. 21 (two registers U, X plus
 *     the error register of the embedded third-order scheme, Sec. 2.2.3), with the
 *     RK4(3)5[2R+]C coefficients of the paper's ref. [37];
 *   - the WRMS step-size controller of Eq. 22.
 *
 * Readings where the paper is silent (all documented with the design):
 *   integrated variables are the 9 mass fractions at fixed rho, e; the WRMS norm runs
 *   over them with |u_i| = max(|y_n,i|, |y_n+1,i|); h_max / h_min of Eq. 22 act as
 *   growth / shrink factors 5 and 1/5; a step is accepted iff ||e|| <= 1; h0 = dt;
 *   h is clipped to land on dt; the loop ends when dt - t <= 1e-12 dt; at most
 *   max_steps attempts, h < 1e-15 dt is an underflow; concentrations are clamped at
 *   zero inside the rate evaluation only; Newton stops at |dT| <= 1e-12 T within 30
 *   iterations, then bisects on [200, 6000] K; a trial stage with no temperature root
 *   or a non-finite error estimate rejects the attempt with the factor 1/5, while no
 *   root at the accepted state ends the cell (status 3).
 * Units are SI: kg/mol, J/mol, mol/m^3, Pa, s.
 */
#include <math.h>
#include <stdlib.h>
#include <stdint.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXSP 16
#define OR_MAXRX 64
#define OR_NEL 3

static const double R_U = 8.31446261815324;  /* J/(mol K) */
static const double P_REF = 101325.0;        /* Pa, standard state of the equilibrium constant */

/* The mechanism, as marshalled by the Python side of the oracle. */
typedef struct {
  int32_t nsp, nrx;
  double W[OR_MAXSP];                 /* molar mass, kg/mol */
  int32_t ncomp[OR_MAXSP][OR_NEL];    /* element counts H, O, N */
  double Tmid[OR_MAXSP];              /* NASA-7 range switch */
  double alo[OR_MAXSP][7];            /* NASA-7 coefficients below Tmid */
  double ahi[OR_MAXSP][7];            /* NASA-7 coefficients at and above Tmid */
  int32_t rtype[OR_MAXRX];            /* 0 elementary, 1 third body, 2 fall-off */
  int32_t nuf[OR_MAXRX][OR_MAXSP];    /* reactant stoichiometric coefficients */
  int32_t nur[OR_MAXRX][OR_MAXSP];    /* product stoichiometric coefficients */
  double A[OR_MAXRX], b[OR_MAXRX], Ea[OR_MAXRX];     /* Arrhenius (high-pressure limit) */
  double A0[OR_MAXRX], b0[OR_MAXRX], Ea0[OR_MAXRX];  /* low-pressure limit (fall-off) */
  double troe[OR_MAXRX][4];           /* alpha, T***, T*, T** */
  int32_t troe_n[OR_MAXRX];           /* 0 Lindemann, 3 or 4 Troe parameters */
  double eff[OR_MAXRX][OR_MAXSP];     /* third-body efficiencies */
  int32_t reversible[OR_MAXRX];
} omech;

/* ------------------------------------------------------------------ thermo (Eq. 10) */

static const double *nasa(const omech *m, int k, double T) {
  return (T < m->Tmid[k]) ? m->alo[k] : m->ahi[k];
}

/* cp/R = a1 + a2 T + a3 T^2 + a4 T^3 + a5 T^4 */
double oracle_cp_R(const omech *m, int k, double T) {
  const double *a = nasa(m, k, T);
  return a[0] + a[1] * T + a[2] * T * T + a[3] * T * T * T + a[4] * T * T * T * T;
}

/* h/(RT) = a1 + a2 T/2 + a3 T^2/3 + a4 T^3/4 + a5 T^4/5 + a6/T */
double oracle_h_RT(const omech *m, int k, double T) {
  const double *a = nasa(m, k, T);
  return a[0] + a[1] * T / 2.0 + a[2] * T * T / 3.0 + a[3] * T * T * T / 4.0 +
         a[4] * T * T * T * T / 5.0 + a[5] / T;
}

/* s/R = a1 ln T + a2 T + a3 T^2/2 + a4 T^3/3 + a5 T^4/4 + a7  (at P_REF) */
double oracle_s_R(const omech *m, int k, double T) {
  const double *a = nasa(m, k, T);
  return a[0] * log(T) + a[1] * T + a[2] * T * T / 2.0 + a[3] * T * T * T / 3.0 +
         a[4] * T * T * T * T / 4.0 + a[6];
}

/* Mixture specific internal energy, J/kg: e = sum_k Y_k (h_k - R_u T) / W_k (Eq. 10
 * with p/rho = R_u T sum_k Y_k/W_k). */
double oracle_e_mix(const omech *m, const double *Y, double T) {
  double e = 0.0;
  for (int k = 0; k < m->nsp; ++k)
    e += Y[k] * (oracle_h_RT(m, k, T) * R_U * T - R_U * T) / m->W[k];
  return e;
}

/* Mixture specific heat at constant volume, J/(kg K): sum_k Y_k (cp_k - R_u) / W_k */
double oracle_cv_mix(const omech *m, const double *Y, double T) {
  double cv = 0.0;
  for (int k = 0; k < m->nsp; ++k)
    cv += Y[k] * (oracle_cp_R(m, k, T) * R_U - R_U) / m->W[k];
  return cv;
}

/* T from (e, Y) by bisection on [200, 6000] K.  Returns 0 on success. */
int oracle_T_from_e_bisect(const omech *m, const double *Y, double e, double *T_out) {
  double lo = 200.0, hi = 6000.0;
  if (oracle_e_mix(m, Y, lo) - e > 0.0 || oracle_e_mix(m, Y, hi) - e < 0.0) return 3;
  for (int it = 0; it < 200 && hi - lo > 1e-13 * hi; ++it) {
    double mid = 0.5 * (lo + hi);
    if (oracle_e_mix(m, Y, mid) - e > 0.0) hi = mid; else lo = mid;
  }
  *T_out = 0.5 * (lo + hi);
  return 0;
}

/* T from (e, Y) by Newton-Raphson, T <- T - (e(T) - e) / cv(T), started from Tguess
 * (1500 K when Tguess is not a positive finite number).  Stops when |dT| <= 1e-12 T;
 * after 30 iterations, or on a non-positive or non-finite iterate, falls back to
 * bisection.  Returns 0 on success, 3 on failure. */
int oracle_T_from_e(const omech *m, const double *Y, double e, double Tguess, double *T_out,
                    int32_t *iters) {
  double T = (isfinite(Tguess) && Tguess > 0.0) ? Tguess : 1500.0;
  for (int it = 1; it <= 30; ++it) {
    double f = oracle_e_mix(m, Y, T) - e;
    double d = oracle_cv_mix(m, Y, T);
    double dT = f / d;
    T = T - dT;
    if (!isfinite(T) || T <= 0.0) break;
    if (fabs(dT) <= 1e-12 * fabs(T)) {
      *T_out = T;
      if (iters) *iters = it;
      return 0;
    }
  }
  if (iters) *iters = -1;
  return oracle_T_from_e_bisect(m, Y, e, T_out);
}

/* ---------------------------------------------------------- kinetics (Eq. 15-16) */

static double ipow(double x, int n) {
  double r = 1.0;
  for (int i = 0; i < n; ++i) r *= x;
  return r;
}

/* Third-body concentration of reaction j: [M] = sum_k eff_jk c_k */
static double third_body(const omech *m, int j, const double *c) {
  double M = 0.0;
  for (int k = 0; k < m->nsp; ++k) M += m->eff[j][k] * c[k];
  return M;
}

/* Troe broadening factor F(Pr, T) (Gilbert, Luther & Troe 1983); 1 for Lindemann. */
double oracle_troe_F(const omech *m, int j, double T, double Pr) {
  if (m->troe_n[j] == 0) return 1.0;
  const double *p = m->troe[j];
  double Fcent = (1.0 - p[0]) * exp(-T / p[1]) + p[0] * exp(-T / p[2]);
  if (m->troe_n[j] == 4) Fcent += exp(-p[3] / T);
  double logFc = log10(Fcent);
  double cc = -0.4 - 0.67 * logFc;
  double nn = 0.75 - 1.27 * logFc;
  double x = log10(Pr) + cc;
  double f1 = x / (nn - 0.14 * x);
  double logF = logFc / (1.0 + f1 * f1);
  return pow(10.0, logF);
}

/* Forward and reverse rate coefficients of every reaction at T, given the clamped
 * concentrations c (needed for the fall-off pressure dependence).
 * Forward: k = A T^b exp(-Ea/(R_u T)); for fall-off, k = k_inf Pr/(1+Pr) F with
 * Pr = k0 [M] / k_inf.  Reverse: k_r = k_f / K_c with
 * K_c = exp(-sum_k nu_jk g_k/(R_u T)) (P_REF/(R_u T))^(sum_k nu_jk), nu = nu'' - nu'. */
void oracle_rate_constants(const omech *m, double T, const double *c, double *kf, double *kr) {
  double g[OR_MAXSP];
  for (int k = 0; k < m->nsp; ++k) g[k] = oracle_h_RT(m, k, T) - oracle_s_R(m, k, T);
  for (int j = 0; j < m->nrx; ++j) {
    double k_inf = m->A[j] * pow(T, m->b[j]) * exp(-m->Ea[j] / (R_U * T));
    double k = k_inf;
    if (m->rtype[j] == 2) {
      double k0 = m->A0[j] * pow(T, m->b0[j]) * exp(-m->Ea0[j] / (R_U * T));
      double Pr = k0 * third_body(m, j, c) / k_inf;
      k = (Pr > 0.0) ? k_inf * (Pr / (1.0 + Pr)) * oracle_troe_F(m, j, T, Pr) : 0.0;
    }
    kf[j] = k;
    double dG = 0.0;
    int dnu = 0;
    for (int s = 0; s < m->nsp; ++s) {
      int nu = m->nur[j][s] - m->nuf[j][s];
      dG += nu * g[s];
      dnu += nu;
    }
    double Kc = exp(-dG) * pow(P_REF / (R_U * T), (double)dnu);
    kr[j] = m->reversible[j] ? k / Kc : 0.0;
  }
}

/* Forward and reverse rates of progress (mol/m^3/s) of every reaction:
 * q_f = k_f prod c^nu', q_r = k_r prod c^nu'', both times [M] for third-body reactions. */
void oracle_progress(const omech *m, double rho, double T, const double *Y, double *qf, double *qr) {
  double c[OR_MAXSP], kf[OR_MAXRX], kr[OR_MAXRX];
  for (int k = 0; k < m->nsp; ++k) {
    double ck = rho * Y[k] / m->W[k];
    c[k] = ck > 0.0 ? ck : 0.0;
  }
  oracle_rate_constants(m, T, c, kf, kr);
  for (int j = 0; j < m->nrx; ++j) {
    double f = kf[j], r = kr[j];
    for (int k = 0; k < m->nsp; ++k) {
      f *= ipow(c[k], m->nuf[j][k]);
      r *= ipow(c[k], m->nur[j][k]);
    }
    if (m->rtype[j] == 1) {
      double M = third_body(m, j, c);
      f *= M;
      r *= M;
    }
    qf[j] = f;
    qr[j] = r;
  }
}

/* Molar production rates (Eq. 16): wdot_k = sum_j (nu''_jk - nu'_jk) (q_f,j - q_r,j). */
void oracle_wdot(const omech *m, double rho, double T, const double *Y, double *wdot) {
  double qf[OR_MAXRX], qr[OR_MAXRX];
  oracle_progress(m, rho, T, Y, qf, qr);
  for (int k = 0; k < m->nsp; ++k) wdot[k] = 0.0;
  for (int j = 0; j < m->nrx; ++j)
    for (int k = 0; k < m->nsp; ++k)
      wdot[k] += (double)(m->nur[j][k] - m->nuf[j][k]) * (qf[j] - qr[j]);
}

/* Conserved state from (T, p, Y): rho = p Wbar / (R_u T), e = e(T, Y). */
void oracle_state_from_TPY(const omech *m, int64_t n, const double *T, const double *p,
                           const double *Y, int64_t ld, double *rho, double *e) {
  for (int64_t i = 0; i < n; ++i) {
    double y[OR_MAXSP], inv_w = 0.0;
    for (int k = 0; k < m->nsp; ++k) {
      y[k] = Y[k * ld + i];
      inv_w += y[k] / m->W[k];
    }
    rho[i] = p[i] / (R_U * T[i] * inv_w);
    e[i] = oracle_e_mix(m, y, T[i]);
  }
}

/* ------------------------------------------- low-storage RK (Eq. 21) and control */

/* RK4(3)5[2R+]C of the paper's ref. [37]: sub-diagonal a_{i+1,i}, weights b and the
 * embedded third-order weights bhat.  All other a_{i,j} (j < i-1) equal b_j. */
static const double LS_A[4] = {
    970286171893.0 / 4311952581923.0, 6584761158862.0 / 12103376702013.0,
    2251764453980.0 / 15575788980749.0, 26877169314380.0 / 34165994151039.0};
static const double LS_B[5] = {
    1153189308089.0 / 22510343858157.0, 1772645290293.0 / 4653164025191.0,
    -1672844663538.0 / 4480602732383.0, 2114624349019.0 / 3568978502595.0,
    5198255086312.0 / 14908931495163.0};
static const double LS_BH[5] = {
    1016888040809.0 / 7410784769900.0, 11231460423587.0 / 58533540763752.0,
    -1563879915014.0 / 6823010717585.0, 606302364029.0 / 971179775848.0,
    1097981568119.0 / 3980877426909.0};

void oracle_lsrk_coefficients(double *a, double *b, double *bh) {
  for (int i = 0; i < 4; ++i) a[i] = LS_A[i];
  for (int i = 0; i < 5; ++i) { b[i] = LS_B[i]; bh[i] = LS_BH[i]; }
}

#define OR_MAXN 32
typedef int (*rhs_fn)(void *ctx, const double *y, double *f);

/* One step of Eq. 21 from X (overwritten with y_n+1).  Register 1 holds U (the stage
 * input), register 2 holds X; F is the stage derivative; E accumulates the embedded
 * error sum_i (b_i - bhat_i) h F_i.  Returns 0, or the 1-based stage whose RHS failed. */
static int lsrk_step(int n, rhs_fn f, void *ctx, double h, double *X, double *E) {
  double U[OR_MAXN], F[OR_MAXN];
  for (int i = 0; i < n; ++i) { U[i] = X[i]; E[i] = 0.0; }
  for (int s = 0; s < 5; ++s) {
    if (f(ctx, U, F)) return s + 1;
    for (int i = 0; i < n; ++i) E[i] += (LS_B[s] - LS_BH[s]) * h * F[i];
    double a = (s < 4) ? LS_A[s] : 0.0;
    for (int i = 0; i < n; ++i) {
      U[i] = X[i] + a * h * F[i];               /* register 1 */
      X[i] = U[i] + (LS_B[s] - a) * h * F[i];   /* register 2 */
    }
  }
  return 0;
}

/* ------------------------------------ conventional (full-storage) explicit RK */

/* An explicit Runge-Kutta tableau in Butcher form: stage i evaluates k_i = f(U_i) at
 * U_i = y_n + h sum_{j<i} a_ij k_j; the step keeps every k_i and ends with
 * y_n+1 = y_n + h sum_i b_i k_i and the embedded error estimate h sum_i (b_i - bhat_i) k_i.
 * expo is the controller exponent 1/(q+1), q the order of the error estimate's leading
 * term minus one. */
#define OR_MAXSTAGE 6
typedef struct {
  int s;
  double a[OR_MAXSTAGE][OR_MAXSTAGE], b[OR_MAXSTAGE], bh[OR_MAXSTAGE];
  double expo;
} butcher;

/* The method of Eq. 21 written in Butcher form: the two-register recursion
 * U = X + a_{i+1,i} h F, X = U + (b_i - a_{i+1,i}) h F leaves every earlier stage in X
 * with its weight b_j, so a_ij = b_j for j < i-1 and a_{i,i-1} is the sub-diagonal
 * coefficient (Sec. 2.2.3; ref. [37]). */
static butcher lsrk_full_tableau(void) {
  butcher t;
  memset(&t, 0, sizeof t);
  t.s = 5;
  for (int i = 1; i < 5; ++i) {
    for (int j = 0; j < i - 1; ++j) t.a[i][j] = LS_B[j];
    t.a[i][i - 1] = LS_A[i - 1];
  }
  for (int i = 0; i < 5; ++i) { t.b[i] = LS_B[i]; t.bh[i] = LS_BH[i]; }
  t.expo = 0.25;
  return t;
}

/* Fehlberg's embedded 4(5) pair (RKF45, the paper's ref. [36]; Fehlberg, NASA TR R-315,
 * 1969): six stages, the fourth-order solution is propagated (b) and the fifth-order one
 * (bhat) estimates its error, whose leading term is O(h^5): exponent 1/5. */
static butcher rkf45_tableau(void) {
  butcher t;
  memset(&t, 0, sizeof t);
  t.s = 6;
  t.a[1][0] = 1.0 / 4.0;
  t.a[2][0] = 3.0 / 32.0; t.a[2][1] = 9.0 / 32.0;
  t.a[3][0] = 1932.0 / 2197.0; t.a[3][1] = -7200.0 / 2197.0; t.a[3][2] = 7296.0 / 2197.0;
  t.a[4][0] = 439.0 / 216.0; t.a[4][1] = -8.0; t.a[4][2] = 3680.0 / 513.0; t.a[4][3] = -845.0 / 4104.0;
  t.a[5][0] = -8.0 / 27.0; t.a[5][1] = 2.0; t.a[5][2] = -3544.0 / 2565.0; t.a[5][3] = 1859.0 / 4104.0;
  t.a[5][4] = -11.0 / 40.0;
  const double b4[6] = {25.0 / 216.0, 0.0, 1408.0 / 2565.0, 2197.0 / 4104.0, -1.0 / 5.0, 0.0};
  const double b5[6] = {16.0 / 135.0, 0.0, 6656.0 / 12825.0, 28561.0 / 56430.0, -9.0 / 50.0, 2.0 / 55.0};
  for (int i = 0; i < 6; ++i) { t.b[i] = b4[i]; t.bh[i] = b5[i]; }
  t.expo = 0.2;
  return t;
}

/* The integration schemes: 0 the two-register method of Eq. 21, 1 the same tableau with
 * full k-storage, 2 RKF45 with full k-storage. */
static butcher scheme_tableau(int scheme) {
  return scheme == 2 ? rkf45_tableau() : lsrk_full_tableau();
}

void oracle_butcher(int32_t scheme, int32_t *s, double *a, double *b, double *bh, double *expo) {
  butcher t = scheme_tableau(scheme);
  *s = t.s;
  for (int i = 0; i < OR_MAXSTAGE; ++i) {
    for (int j = 0; j < OR_MAXSTAGE; ++j) a[i * OR_MAXSTAGE + j] = t.a[i][j];
    b[i] = t.b[i];
    bh[i] = t.bh[i];
  }
  *expo = t.expo;
}

/* One step of tableau t from X (overwritten with y_n+1), every stage derivative kept.
 * Returns 0, or the 1-based stage whose RHS failed. */
static int butcher_step(int n, rhs_fn f, void *ctx, const butcher *t, double h, double *X, double *E) {
  double K[OR_MAXSTAGE][OR_MAXN], U[OR_MAXN];
  for (int i = 0; i < t->s; ++i) {
    for (int k = 0; k < n; ++k) {
      double acc = 0.0;
      for (int j = 0; j < i; ++j) acc += t->a[i][j] * K[j][k];
      U[k] = X[k] + h * acc;
    }
    if (f(ctx, U, K[i])) return i + 1;
  }
  for (int k = 0; k < n; ++k) {
    double sb = 0.0, se = 0.0;
    for (int i = 0; i < t->s; ++i) {
      sb += t->b[i] * K[i][k];
      se += (t->b[i] - t->bh[i]) * K[i][k];
    }
    X[k] += h * sb;
    E[k] = h * se;
  }
  return 0;
}

/* One step of scheme 0, 1 or 2; exponent of its controller in *expo. */
static int scheme_step(int scheme, int n, rhs_fn f, void *ctx, double h, double *X, double *E,
                       double *expo) {
  if (scheme == 0) {
    *expo = 0.25;
    return lsrk_step(n, f, ctx, h, X, E);
  }
  butcher t = scheme_tableau(scheme);
  *expo = t.expo;
  return butcher_step(n, f, ctx, &t, h, X, E);
}

/* WRMS error of Eq. 22 over n components, |u_i| = max(|y_n,i|, |y_n+1,i|). */
static double wrms(int n, const double *E, const double *Xold, const double *Xnew, double rtol,
                   double atol) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) {
    double u = fmax(fabs(Xold[i]), fabs(Xnew[i]));
    double w = E[i] / (rtol * u + atol);
    s += w * w;
  }
  return sqrt(s / n);
}

typedef struct {
  int32_t status, nacc, nrej;
  double margin; /* min over attempted steps of |err - 1| */
  double h_next; /* the controller's next step after the last attempt */
} adapt_out;

/* Adaptive integration of y' = f(y) over [0, dt] with the Eq. 22 controller.
 * Optional logs (h, err, accepted) of every attempted step. */
/* on_event (nullable) is told when an attempt begins (0) and when one is rejected (1),
 * so that a right-hand side with state of its own (the temperature warm start of a
 * chemistry cell) can return it to the accepted state together with X. */
static void integrate_adaptive(int scheme, int n, rhs_fn f, void *ctx, double dt, double rtol,
                               double atol, double h0, int32_t max_steps, double *X, adapt_out *out,
                               double *log_h, double *log_err, int32_t *log_acc, int32_t max_log,
                               void (*on_event)(void *ctx, int ev)) {
  double t = 0.0, h = (h0 > 0.0) ? h0 : dt;
  double Xs[OR_MAXN], E[OR_MAXN];
  out->status = 0; out->nacc = 0; out->nrej = 0; out->margin = INFINITY; out->h_next = h;
  while (dt - t > 1e-12 * dt) {
    if (out->nacc + out->nrej >= max_steps) { out->status = 1; break; }
    if (h < 1e-15 * dt) { out->status = 2; break; }
    if (h > dt - t) h = dt - t;
    for (int i = 0; i < n; ++i) Xs[i] = X[i];
    int k = out->nacc + out->nrej;
    if (on_event) on_event(ctx, 0);
    /* A trial stage (2..5) whose RHS fails (no temperature root) or an error estimate
     * that is not finite rejects the attempt with the smallest factor 1/5; a failure
     * at stage 1, the accepted state itself, ends the cell with status 3. */
    double expo = 0.25;
    int failed = scheme_step(scheme, n, f, ctx, h, X, E, &expo);
    if (failed == 1) {
      for (int i = 0; i < n; ++i) X[i] = Xs[i];
      out->status = 3;
      break;
    }
    double err = failed ? NAN : wrms(n, E, Xs, X, rtol, atol);
    if (!isfinite(err)) {
      for (int i = 0; i < n; ++i) X[i] = Xs[i];
      if (on_event) on_event(ctx, 1);
      if (k < max_log) { log_h[k] = h; log_err[k] = err; log_acc[k] = 0; }
      out->nrej++;
      h = h * 0.2;
      continue;
    }
    double fac = (err == 0.0) ? 5.0 : fmin(5.0, fmax(0.2, 0.9 * pow(1.0 / err, expo)));
    if (k < max_log) { log_h[k] = h; log_err[k] = err; log_acc[k] = err <= 1.0; }
    if (fabs(err - 1.0) < out->margin) out->margin = fabs(err - 1.0);
    if (err <= 1.0) {
      t += h;
      out->nacc++;
    } else {
      for (int i = 0; i < n; ++i) X[i] = Xs[i];
      if (on_event) on_event(ctx, 1);
      out->nrej++;
    }
    h = h * fac;
  }
  out->h_next = h;
}

/* ------------------------------------------------------------ test problems */

typedef struct { int n; const double *M; } linear_ctx;

static int linear_rhs(void *vctx, const double *y, double *f) {
  const linear_ctx *c = (const linear_ctx *)vctx;
  for (int i = 0; i < c->n; ++i) {
    double s = 0.0;
    for (int j = 0; j < c->n; ++j) s += c->M[i * c->n + j] * y[j];
    f[i] = s;
  }
  return 0;
}

/* One Eq. 21 step of y' = M y (M row-major n x n): y is overwritten with y_n+1 and E
 * receives the embedded error estimate. */
void oracle_linear_step(int32_t n, const double *M, double h, double *y, double *E) {
  linear_ctx c = {n, M};
  lsrk_step(n, linear_rhs, &c, h, y, E);
}

/* The same step with scheme 0, 1 or 2. */
void oracle_linear_step_scheme(int32_t scheme, int32_t n, const double *M, double h, double *y,
                               double *E) {
  linear_ctx c = {n, M};
  double expo;
  scheme_step(scheme, n, linear_rhs, &c, h, y, E, &expo);
}

/* Adaptive integration of y' = M y over [0, dt]; logs every attempted step.
 * out4 = {status, accepted, rejected}; returns the number of attempts. */
int32_t oracle_linear_integrate(int32_t n, const double *M, double *y, double dt, double rtol,
                                double atol, double h0, int32_t max_steps, double *log_h,
                                double *log_err, int32_t *log_acc, int32_t max_log, int32_t *out3) {
  linear_ctx c = {n, M};
  adapt_out o;
  integrate_adaptive(0, n, linear_rhs, &c, dt, rtol, atol, h0, max_steps, y, &o, log_h, log_err,
                     log_acc, max_log, NULL);
  out3[0] = o.status; out3[1] = o.nacc; out3[2] = o.nrej;
  return o.nacc + o.nrej;
}

static int quadratic_rhs(void *vctx, const double *y, double *f) {
  (void)vctx;
  f[0] = -y[0] * y[0];
  return 0;
}

/* Fixed-step integration of y' = -y^2 from y0 over nsteps steps of h, propagating either
 * the fourth-order solution (embedded = 0) or the third-order embedded one (X - E). */
double oracle_quadratic_fixed(double y0, double h, int32_t nsteps, int32_t embedded) {
  double X[1] = {y0}, E[1];
  for (int s = 0; s < nsteps; ++s) {
    lsrk_step(1, quadratic_rhs, NULL, h, X, E);
    if (embedded) X[0] -= E[0];
  }
  return X[0];
}

/* The same with scheme 0, 1 or 2 (embedded: propagate y_n+1 - E, the solution of the
 * bhat weights). */
double oracle_quadratic_fixed_scheme(int32_t scheme, double y0, double h, int32_t nsteps,
                                     int32_t embedded) {
  double X[1] = {y0}, E[1], expo;
  for (int s = 0; s < nsteps; ++s) {
    scheme_step(scheme, 1, quadratic_rhs, NULL, h, X, E, &expo);
    if (embedded) X[0] -= E[0];
  }
  return X[0];
}

/* ------------------------------------------------------------ chemistry cells */

typedef struct {
  const omech *m;
  double rho, e, T;  /* T: last Newton result, the next warm start */
  double T_acc;      /* temperature of the accepted state (stage 1 of the attempt) */
  int first;         /* the next evaluation is stage 1 of an attempt */
} chem_cell;

/* A rejected attempt returns the cell to its accepted state: X (restored by the
 * integrator) and the temperature warm start with it, so the next Newton solve starts
 * from that state's own temperature, not from a trial stage's. */
static void chem_event(void *vctx, int ev) {
  chem_cell *cc = (chem_cell *)vctx;
  if (ev == 0) cc->first = 1;
  else cc->T = cc->T_acc;
}

/* dY_k/dt = W_k wdot_k / rho at fixed (rho, e); T from Newton on (e, Y). */
static int chem_rhs(void *vctx, const double *Y, double *F) {
  chem_cell *cc = (chem_cell *)vctx;
  double T, w[OR_MAXSP];
  if (oracle_T_from_e(cc->m, Y, cc->e, cc->T, &T, NULL)) return 1;
  cc->T = T;
  if (cc->first) { cc->T_acc = T; cc->first = 0; }
  oracle_wdot(cc->m, cc->rho, T, Y, w);
  for (int k = 0; k < cc->m->nsp; ++k) F[k] = cc->m->W[k] * w[k] / cc->rho;
  return 0;
}

/* dY/dt of one cell at (rho, e, Y), T solved from Tguess; the solved T is returned. */
double oracle_chem_rhs(const omech *m, double rho, double e, const double *Y, double Tguess,
                       double *F) {
  chem_cell cc = {m, rho, e, Tguess, Tguess, 0};
  if (chem_rhs(&cc, Y, F)) return NAN;
  return cc.T;
}

/* Integrate n independent cells over dt (the hot path's reference).
 * Y: species planes Y[k * ldY + i], advanced in place.  T: in = Newton guess (or NaN),
 * out = temperature of the final state.  h0: per-cell initial step (NULL -> dt).
 * Per cell out: status (0 ok, 1 max steps, 2 h underflow, 3 Newton failure,
 * 4 non-finite), attempted steps, accepted steps, the smallest |err - 1| seen
 * (used to classify cells whose accept/reject decisions sit on a rounding knife-edge)
 * and the controller's next step h_out (to carry into a following call). */
int32_t oracle_integrate_scheme(int32_t scheme, const omech *m, int64_t n, const double *rho,
                                const double *e, double *Y, int64_t ldY, double *T, double dt,
                                double rtol, double atol, const double *h0, int32_t max_steps,
                                int32_t *status, int32_t *nsteps, int32_t *naccept, double *margin,
                                double *h_out, int32_t nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 8)
#else
  (void)nthreads;
#endif
  for (int64_t i = 0; i < n; ++i) {
    double X[OR_MAXN];
    for (int k = 0; k < m->nsp; ++k) X[k] = Y[k * ldY + i];
    chem_cell cc = {m, rho[i], e[i], T[i], T[i], 0};
    adapt_out o;
    int bad_input = !(isfinite(rho[i]) && rho[i] > 0.0 && isfinite(e[i]));
    for (int k = 0; k < m->nsp; ++k) bad_input |= !isfinite(X[k]);
    if (bad_input) {
      o.status = 4; o.nacc = 0; o.nrej = 0; o.margin = INFINITY;
      o.h_next = (h0 && isfinite(h0[i]) && h0[i] > 0.0) ? h0[i] : dt;
    } else {
      double hi = (h0 && isfinite(h0[i]) && h0[i] > 0.0) ? h0[i] : 0.0;
      integrate_adaptive(scheme, m->nsp, chem_rhs, &cc, dt, rtol, atol, hi, max_steps, X,
                         &o, NULL, NULL, NULL, 0, chem_event);
    }
    double Tout = NAN;
    if (o.status != 4 && oracle_T_from_e(m, X, e[i], cc.T, &Tout, NULL) != 0) {
      if (o.status == 0) o.status = 3;
      Tout = NAN;
    }
    for (int k = 0; k < m->nsp; ++k) Y[k * ldY + i] = X[k];
    T[i] = Tout;
    if (status) status[i] = o.status;
    if (nsteps) nsteps[i] = o.nacc + o.nrej;
    if (naccept) naccept[i] = o.nacc;
    if (margin) margin[i] = o.margin;
    if (h_out) h_out[i] = o.h_next;
  }
  return 0;
}

/* The integration of the two-register method of Eq. 21 (scheme 0). */
int32_t oracle_integrate(const omech *m, int64_t n, const double *rho, const double *e, double *Y,
                         int64_t ldY, double *T, double dt, double rtol, double atol,
                         const double *h0, int32_t max_steps, int32_t *status, int32_t *nsteps,
                         int32_t *naccept, double *margin, double *h_out, int32_t nthreads) {
  return oracle_integrate_scheme(0, m, n, rho, e, Y, ldY, T, dt, rtol, atol, h0, max_steps, status,
                                 nsteps, naccept, margin, h_out, nthreads);
}

/* Fixed-step integration of one cell (nsteps steps of h, no error control), recording
 * T after every step in T_trace[nsteps]; used for the step-halving ignition-delay check. */
int32_t oracle_chem_fixed(const omech *m, double rho, double e, double *Y, double Tguess, double h,
                          int32_t nsteps, double *T_trace) {
  chem_cell cc = {m, rho, e, Tguess, Tguess, 0};
  double E[OR_MAXN];
  for (int s = 0; s < nsteps; ++s) {
    if (lsrk_step(m->nsp, chem_rhs, &cc, h, Y, E)) return 3;
    double T;
    if (oracle_T_from_e(m, Y, e, cc.T, &T, NULL)) return 3;
    T_trace[s] = T;
  }
  return 0;
}

/* ------------------------------------------- 1D reactive Euler and Strang splitting */

/* The operator on either side of the chemistry in the paper's split scheme (Sec. 2.2.1,
 * Strang splitting of the reactive Euler equations, Eq. 14 without transport): a
 * minimal 1D finite-volume step for the conserved state U = (rho, rho u, rho E,
 * rho Y_k) of n cells of width dx.  Second-order MUSCL reconstruction of the primitive
 * variables (rho, u, p, Y_k) with minmod-limited slopes, the HLL flux with Davis wave
 * speeds, and the two-stage SSP Runge-Kutta (Heun) step in time.  A face whose
 * reconstructed density or pressure is not positive falls back to the cell averages.
 * Boundaries: 0 transmissive (zero gradient), 1 reflecting wall.  Thermo of Eq. 10:
 * p = rho R_u T sum_k Y_k / W_k with T from e = E - u^2/2 by Newton (oracle_T_from_e). */

typedef struct { double rho, u, p, Y[OR_MAXSP], T; } prim1d;

static double mix_inv_w(const omech *m, const double *Y) {
  double s = 0.0;
  for (int k = 0; k < m->nsp; ++k) s += Y[k] / m->W[k];
  return s;
}

/* Sound speed squared gamma p / rho with gamma = cp / cv of the mixture at T. */
static double sound2(const omech *m, const prim1d *w) {
  double cv = oracle_cv_mix(m, w->Y, w->T);
  double cp = cv + R_U * mix_inv_w(m, w->Y);
  return cp / cv * w->p / w->rho;
}

/* Primitive state of cell i from the conserved planes; T starts from Tguess.  Returns 0
 * or 3 when no temperature root exists. */
static int cons_to_prim(const omech *m, const double *rho, const double *rhou, const double *rhoE,
                        const double *rhoY, int64_t ld, int64_t i, double Tguess, prim1d *w) {
  w->rho = rho[i];
  w->u = rhou[i] / rho[i];
  for (int k = 0; k < m->nsp; ++k) w->Y[k] = rhoY[k * ld + i] / rho[i];
  double e = rhoE[i] / rho[i] - 0.5 * w->u * w->u;
  if (oracle_T_from_e(m, w->Y, e, Tguess, &w->T, NULL)) return 3;
  w->p = rho[i] * R_U * w->T * mix_inv_w(m, w->Y);
  return 0;
}

/* Physical flux of a primitive state (T known from p, rho, Y). */
static void euler_flux(const omech *m, const prim1d *w, double *F) {
  double e = oracle_e_mix(m, w->Y, w->T);
  double E = e + 0.5 * w->u * w->u;
  F[0] = w->rho * w->u;
  F[1] = w->rho * w->u * w->u + w->p;
  F[2] = (w->rho * E + w->p) * w->u;
  for (int k = 0; k < m->nsp; ++k) F[3 + k] = w->rho * w->Y[k] * w->u;
}

static void prim_to_cons(const omech *m, const prim1d *w, double *U) {
  double e = oracle_e_mix(m, w->Y, w->T);
  U[0] = w->rho;
  U[1] = w->rho * w->u;
  U[2] = w->rho * (e + 0.5 * w->u * w->u);
  for (int k = 0; k < m->nsp; ++k) U[3 + k] = w->rho * w->Y[k];
}

static double minmod(double a, double b) {
  if (a * b <= 0.0) return 0.0;
  return fabs(a) < fabs(b) ? a : b;
}

/* Ghost or interior primitive state of index j in [-2, n+1]. */
static prim1d ghost(const prim1d *W, int64_t n, int64_t j, int bcl, int bcr) {
  prim1d g;
  if (j < 0) {
    g = W[-j - 1];                       /* mirror: -1 -> 0, -2 -> 1 */
    if (bcl == 0) g = W[0];
    else g.u = -g.u;
  } else if (j >= n) {
    g = W[2 * n - 1 - j];                /* n -> n-1, n+1 -> n-2 */
    if (bcr == 0) g = W[n - 1];
    else g.u = -g.u;
  } else {
    g = W[j];
  }
  return g;
}

/* HLL flux at the face between reconstructed states L and R (primitive; T set). */
static void hll(const omech *m, const prim1d *L, const prim1d *R, double *F) {
  int nv = 3 + m->nsp;
  double FL[3 + OR_MAXSP], FR[3 + OR_MAXSP], UL[3 + OR_MAXSP], UR[3 + OR_MAXSP];
  double cL = sqrt(sound2(m, L)), cR = sqrt(sound2(m, R));
  double SL = fmin(L->u - cL, R->u - cR), SR = fmax(L->u + cL, R->u + cR);
  euler_flux(m, L, FL);
  euler_flux(m, R, FR);
  if (SL >= 0.0) { for (int v = 0; v < nv; ++v) F[v] = FL[v]; return; }
  if (SR <= 0.0) { for (int v = 0; v < nv; ++v) F[v] = FR[v]; return; }
  prim_to_cons(m, L, UL);
  prim_to_cons(m, R, UR);
  for (int v = 0; v < nv; ++v)
    F[v] = (SR * FL[v] - SL * FR[v] + SL * SR * (UR[v] - UL[v])) / (SR - SL);
}

/* Reconstructed face state from cell state c with slope s, offset +-1/2; T from p. */
static prim1d face_state(const omech *m, const prim1d *c, const prim1d *s, double half) {
  prim1d f;
  f.rho = c->rho + half * s->rho;
  f.u = c->u + half * s->u;
  f.p = c->p + half * s->p;
  for (int k = 0; k < m->nsp; ++k) f.Y[k] = c->Y[k] + half * s->Y[k];
  f.T = f.p / (f.rho * R_U * mix_inv_w(m, f.Y));
  return f;
}

static prim1d slope(const omech *m, const prim1d *a, const prim1d *b, const prim1d *c) {
  prim1d s;
  s.rho = minmod(b->rho - a->rho, c->rho - b->rho);
  s.u = minmod(b->u - a->u, c->u - b->u);
  s.p = minmod(b->p - a->p, c->p - b->p);
  for (int k = 0; k < m->nsp; ++k) s.Y[k] = minmod(b->Y[k] - a->Y[k], c->Y[k] - b->Y[k]);
  s.T = 0.0;
  return s;
}

/* dU/dt of every cell (the flux divergence) from the primitive states W. */
static void euler_rhs(const omech *m, int64_t n, double dx, int bcl, int bcr, const prim1d *W, double *dU) {
  int nv = 3 + m->nsp;
  double Fr[3 + OR_MAXSP];
  for (int64_t f = 0; f <= n; ++f) {     /* face f between cells f-1 and f */
    prim1d a = ghost(W, n, f - 2, bcl, bcr), b = ghost(W, n, f - 1, bcl, bcr);
    prim1d c = ghost(W, n, f, bcl, bcr), d = ghost(W, n, f + 1, bcl, bcr);
    prim1d sb = slope(m, &a, &b, &c), sc = slope(m, &b, &c, &d);
    prim1d L = face_state(m, &b, &sb, 0.5), R = face_state(m, &c, &sc, -0.5);
    if (!(L.rho > 0.0 && L.p > 0.0 && R.rho > 0.0 && R.p > 0.0)) { L = b; R = c; }
    hll(m, &L, &R, Fr);
    if (f > 0)
      for (int v = 0; v < nv; ++v) dU[(f - 1) * nv + v] -= Fr[v] / dx;
    if (f < n)
      for (int v = 0; v < nv; ++v) dU[f * nv + v] = Fr[v] / dx;
  }
}

/* One SSP-RK2 step of the 1D Euler equations over dt (planes updated in place; T: in =
 * Newton start, out = temperature of the new state).  Returns 0, or 3 when a
 * temperature solve failed (state unchanged). */
int32_t oracle_euler1d_step(const omech *m, int64_t n, double dx, double dt, int32_t bcl, int32_t bcr,
                            double *rho, double *rhou, double *rhoE, double *rhoY, int64_t ld, double *T) {
  int nv = 3 + m->nsp;
  prim1d *W = (prim1d *)malloc(sizeof(prim1d) * (size_t)n);
  double *U0 = (double *)malloc(sizeof(double) * (size_t)(n * nv));
  double *U1 = (double *)malloc(sizeof(double) * (size_t)(n * nv));
  double *dU = (double *)malloc(sizeof(double) * (size_t)(n * nv));
  int32_t rc = 0;
  for (int64_t i = 0; i < n; ++i) {
    U0[i * nv + 0] = rho[i]; U0[i * nv + 1] = rhou[i]; U0[i * nv + 2] = rhoE[i];
    for (int k = 0; k < m->nsp; ++k) U0[i * nv + 3 + k] = rhoY[k * ld + i];
  }
  double *Tw = (double *)malloc(sizeof(double) * (size_t)n);
  for (int64_t i = 0; i < n; ++i) Tw[i] = T[i];
  for (int stage = 0; stage < 2 && rc == 0; ++stage) {
    const double *U = stage == 0 ? U0 : U1;
    for (int64_t i = 0; i < n && rc == 0; ++i) {
      double r = U[i * nv], ru = U[i * nv + 1], rE = U[i * nv + 2], rY[OR_MAXSP];
      for (int k = 0; k < m->nsp; ++k) rY[k] = U[i * nv + 3 + k];
      rc = cons_to_prim(m, &r, &ru, &rE, rY, 1, 0, Tw[i], &W[i]);
      Tw[i] = W[i].T;
    }
    if (rc) break;
    euler_rhs(m, n, dx, bcl, bcr, W, dU);
    for (int64_t j = 0; j < n * nv; ++j) {
      if (stage == 0) U1[j] = U0[j] + dt * dU[j];
      else U1[j] = 0.5 * U0[j] + 0.5 * (U1[j] + dt * dU[j]);
    }
  }
  if (rc == 0) {
    for (int64_t i = 0; i < n && rc == 0; ++i) {
      prim1d w;
      double rY[OR_MAXSP];
      for (int k = 0; k < m->nsp; ++k) rY[k] = U1[i * nv + 3 + k];
      rc = cons_to_prim(m, &U1[i * nv], &U1[i * nv + 1], &U1[i * nv + 2], rY, 1, 0, Tw[i], &w);
      Tw[i] = w.T;
    }
  }
  if (rc == 0) {
    for (int64_t i = 0; i < n; ++i) {
      rho[i] = U1[i * nv]; rhou[i] = U1[i * nv + 1]; rhoE[i] = U1[i * nv + 2];
      for (int k = 0; k < m->nsp; ++k) rhoY[k * ld + i] = U1[i * nv + 3 + k];
      T[i] = Tw[i];
    }
  }
  free(W); free(U0); free(U1); free(dU); free(Tw);
  return rc;
}

/* Largest |u| + c over the cells (the CFL speed); T: Newton starts (not modified). */
double oracle_euler1d_max_speed(const omech *m, int64_t n, const double *rho, const double *rhou,
                                const double *rhoE, const double *rhoY, int64_t ld, const double *T) {
  double smax = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    prim1d w;
    if (cons_to_prim(m, rho, rhou, rhoE, rhoY, ld, i, T[i], &w)) return NAN;
    smax = fmax(smax, fabs(w.u) + sqrt(sound2(m, &w)));
  }
  return smax;
}

/* One Strang-split step (Sec. 2.2.1): chemistry over dt/2 at fixed (rho, e) of every
 * cell, the Euler step over dt, chemistry over dt/2 again.  The chemistry is
 * oracle_integrate (Eq. 20-22) on Y = rho Y / rho with e = E - u^2/2; rho E and rho u do
 * not change in a chemistry half-step.  Returns 0, or the first nonzero per-cell status
 * / Euler code. */
int32_t oracle_strang_step(const omech *m, int64_t n, double dx, double dt, int32_t bcl, int32_t bcr,
                           double rtol, double atol, double *rho, double *rhou, double *rhoE,
                           double *rhoY, int64_t ld, double *T, int32_t nthreads) {
  double *e = (double *)malloc(sizeof(double) * (size_t)n);
  double *Y = (double *)malloc(sizeof(double) * (size_t)(n * m->nsp));
  int32_t *st = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  int32_t rc = 0;
  for (int half = 0; half < 2 && rc == 0; ++half) {
    if (half == 1) {
      rc = oracle_euler1d_step(m, n, dx, dt, bcl, bcr, rho, rhou, rhoE, rhoY, ld, T);
      if (rc) break;
    }
    for (int64_t i = 0; i < n; ++i) {
      double u = rhou[i] / rho[i];
      e[i] = rhoE[i] / rho[i] - 0.5 * u * u;
      for (int k = 0; k < m->nsp; ++k) Y[k * n + i] = rhoY[k * ld + i] / rho[i];
    }
    oracle_integrate(m, n, rho, e, Y, n, T, 0.5 * dt, rtol, atol, NULL, 100000, st, NULL, NULL, NULL, NULL,
                     nthreads);
    for (int64_t i = 0; i < n; ++i) {
      if (st[i] && !rc) rc = st[i];
      for (int k = 0; k < m->nsp; ++k) rhoY[k * ld + i] = rho[i] * Y[k * n + i];
    }
  }
  free(e); free(Y); free(st);
  return rc;
}

int32_t oracle_max_species(void) { return OR_MAXSP; }
int32_t oracle_max_reactions(void) { return OR_MAXRX; }
int32_t oracle_struct_size(void) { return (int32_t)sizeof(omech); }
