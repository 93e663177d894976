// cell.cuh -- one cell's low-storage RK integration (Eq. 21-22, Sec. 2.2.3), split into
// begin / attempt / finish so that both the one-pass kernel (a loop per thread) and the
// persistent work-stealing kernel (one attempt per iteration, lanes refilled as cells
// finish) run the same arithmetic.
//
// Per cell the integrator keeps four register vectors of NSP values: the solution
// register X (y_n advancing to y_n+1), the stage register U (input of the next
// right-hand side), the error register E (sum_i (b_i - bhat_i) h F_i, the embedded
// third-order estimate) and the saved y_n for a rejected step; F is transient.  That is
// the two-register scheme of Eq. 21 plus the error register the paper adds, plus the
// copy any rejecting controller needs.  The stage loop stays rolled (coefficients from
// __constant__), so the right-hand side is inlined once.
//
// Controller (Eq. 22): ||e|| = sqrt(mean_k (E_k / (rtol max(|y_n,k|, |y_n+1,k|) + atol))^2);
// accept iff ||e|| <= 1; h <- h min(5, max(0.2, 0.9 ||e||^(-1/4))); h is clipped to land
// on dt; the loop ends when dt - t <= 1e-12 dt; attempted steps are capped; h below
// 1e-15 dt is an underflow.  A trial stage whose temperature solve fails rejects the
// attempt with factor 1/5; a failure at stage 1 (the accepted state) ends the cell.
//
// Variants: V = CHEM_VARIANT_FP64, every register fp64; V = CHEM_VARIANT_MIXED, the stage
// register U and the stage derivative F are fp32 (cell_rhs_mixed) while X, y_n, E, the
// WRMS norm and the controller stay fp64.
#pragma once

#include <math_constants.h>

#include <type_traits>

#include "internal.cuh"
#include "rhs.cuh"
#include "rhs_mixed.cuh"

namespace chem {

// RK4(3)5[2R+]C (Kennedy, Carpenter & Lewis 2000): a_{s+1,s} (0 after the last
// stage), b_s and b_s - bhat_s.  One copy per translation unit.
static __constant__ double c_ls_a[5] = {
    970286171893.0 / 4311952581923.0, 6584761158862.0 / 12103376702013.0,
    2251764453980.0 / 15575788980749.0, 26877169314380.0 / 34165994151039.0, 0.0};
static __constant__ double c_ls_b[5] = {
    1153189308089.0 / 22510343858157.0, 1772645290293.0 / 4653164025191.0,
    -1672844663538.0 / 4480602732383.0, 2114624349019.0 / 3568978502595.0,
    5198255086312.0 / 14908931495163.0};
static __constant__ double c_ls_e[5] = {
    1153189308089.0 / 22510343858157.0 - 1016888040809.0 / 7410784769900.0,
    1772645290293.0 / 4653164025191.0 - 11231460423587.0 / 58533540763752.0,
    -1672844663538.0 / 4480602732383.0 - -1563879915014.0 / 6823010717585.0,
    2114624349019.0 / 3568978502595.0 - 606302364029.0 / 971179775848.0,
    5198255086312.0 / 14908931495163.0 - 1097981568119.0 / 3980877426909.0};

// Conventional explicit RK with full k-storage, the comparators of the two-register
// scheme (the paper's "standard explicit" methods, Sec. 2.2.3 and Sec. 4.2.2): stage i
// evaluates k_i = f(y_n + h sum_{j<i} a_ij k_j) and every k_i is kept until
// y_n+1 = y_n + h sum_i b_i k_i and the error h sum_i (b_i - bhat_i) k_i are formed.
// Table 0: the RK4(3)5[2R+]C tableau above in Butcher form (the two-register recursion
// leaves a_ij = b_j for j < i-1); table 1: Fehlberg's RKF45 (NASA TR R-315, 1969), the
// fourth-order solution propagated and the fifth-order one estimating its error.
static __constant__ double c_fs_a[2][6][6] = {
    {{0.0},
     {970286171893.0 / 4311952581923.0},
     {1153189308089.0 / 22510343858157.0, 6584761158862.0 / 12103376702013.0},
     {1153189308089.0 / 22510343858157.0, 1772645290293.0 / 4653164025191.0,
      2251764453980.0 / 15575788980749.0},
     {1153189308089.0 / 22510343858157.0, 1772645290293.0 / 4653164025191.0,
      -1672844663538.0 / 4480602732383.0, 26877169314380.0 / 34165994151039.0},
     {0.0}},
    {{0.0},
     {1.0 / 4.0},
     {3.0 / 32.0, 9.0 / 32.0},
     {1932.0 / 2197.0, -7200.0 / 2197.0, 7296.0 / 2197.0},
     {439.0 / 216.0, -8.0, 3680.0 / 513.0, -845.0 / 4104.0},
     {-8.0 / 27.0, 2.0, -3544.0 / 2565.0, 1859.0 / 4104.0, -11.0 / 40.0}}};
static __constant__ double c_fs_b[2][6] = {
    {1153189308089.0 / 22510343858157.0, 1772645290293.0 / 4653164025191.0,
     -1672844663538.0 / 4480602732383.0, 2114624349019.0 / 3568978502595.0,
     5198255086312.0 / 14908931495163.0, 0.0},
    {25.0 / 216.0, 0.0, 1408.0 / 2565.0, 2197.0 / 4104.0, -1.0 / 5.0, 0.0}};
static __constant__ double c_fs_e[2][6] = {
    {1153189308089.0 / 22510343858157.0 - 1016888040809.0 / 7410784769900.0,
     1772645290293.0 / 4653164025191.0 - 11231460423587.0 / 58533540763752.0,
     -1672844663538.0 / 4480602732383.0 - -1563879915014.0 / 6823010717585.0,
     2114624349019.0 / 3568978502595.0 - 606302364029.0 / 971179775848.0,
     5198255086312.0 / 14908931495163.0 - 1097981568119.0 / 3980877426909.0, 0.0},
    {25.0 / 216.0 - 16.0 / 135.0, 0.0, 1408.0 / 2565.0 - 6656.0 / 12825.0,
     2197.0 / 4104.0 - 28561.0 / 56430.0, -1.0 / 5.0 - -9.0 / 50.0, 0.0 - 2.0 / 55.0}};

struct CellState {
  double X[NSP];
  double T, h, t, dt;
  double rho, invRho, eR;
  float rho_f, invRho_f;
  int nacc, nrej, nrhs, status;
  bool done;
};

// Set up a cell for integration over [0, dt] from (rho, e, X, T guess, h0).
__device__ __forceinline__ void cell_begin(CellState &c, double rho, double e, double dt) {
  bool bad = !(isfinite(rho) && rho > 0.0 && isfinite(e));
#pragma unroll
  for (int k = 0; k < NSP; ++k) bad |= !isfinite(c.X[k]);
  c.rho = rho;
  c.invRho = 1.0 / rho;
  c.rho_f = (float)rho;
  c.invRho_f = (float)c.invRho;
  c.eR = e / R_U;
  c.t = 0.0;
  c.dt = dt;
  c.status = CHEM_CELL_OK;
  c.done = false;
  if (!(isfinite(c.h) && c.h > 0.0)) c.h = dt;
  if (bad) {
    c.status = CHEM_CELL_NONFINITE;
    c.T = CUDART_NAN;
    c.done = true;
  }
}

// One attempted step (or the end of the integration).  Sets c.done when the cell has
// reached dt or hit a limit.
template <int V>
__device__ __forceinline__ void cell_attempt(const MechTables &mt, CellState &c,
                                             const StepParams &p) {
  constexpr bool kMixed = V == CHEM_VARIANT_MIXED;
  using SReal = std::conditional_t<kMixed, float, double>;
  const double dt = c.dt;
  if (!(dt - c.t > 1e-12 * dt)) { c.done = true; return; }
  if (c.nacc + c.nrej >= p.max_steps) { c.status = CHEM_CELL_MAX_STEPS; c.done = true; return; }
  if (c.h < 1e-15 * dt) { c.status = CHEM_CELL_H_UNDERFLOW; c.done = true; return; }
  double h = c.h;
  if (h > dt - c.t) h = dt - c.t;
  double Xs[NSP], E[NSP];
  SReal U[NSP];
#pragma unroll
  for (int k = 0; k < NSP; ++k) {
    Xs[k] = c.X[k];
    if constexpr (kMixed) U[k] = d2f(c.X[k]);
    else U[k] = c.X[k];
    E[k] = 0.0;
  }
  int failed = 0;
  double Tacc = c.T;  // temperature of the accepted state, set by stage 1
#pragma unroll 1
  for (int s = 0; s < 5; ++s) {
    SReal F[NSP];
    ++c.nrhs;
    bool ok;
    if constexpr (kMixed) ok = cell_rhs_mixed(mt, U, c.rho_f, c.invRho_f, c.eR, c.T, F);
    else ok = cell_rhs(mt, U, c.rho, c.invRho, c.eR, c.T, F);
    if (!ok) { failed = s + 1; break; }
    if (s == 0) Tacc = c.T;
    const double ha = h * c_ls_a[s], hb = h * c_ls_b[s], he = h * c_ls_e[s];
    if constexpr (kMixed) {
      const float ha_f = d2f(ha);
#pragma unroll
      for (int k = 0; k < NSP; ++k) {
        U[k] = fmaf(ha_f, F[k], d2f(c.X[k]));
        const double Fk = f2d(F[k]);
        E[k] = fma(he, Fk, E[k]);
        c.X[k] = fma(hb, Fk, c.X[k]);
      }
    } else {
#pragma unroll
      for (int k = 0; k < NSP; ++k) {
        E[k] = fma(he, F[k], E[k]);
        U[k] = fma(ha, F[k], c.X[k]);
        c.X[k] = fma(hb, F[k], c.X[k]);
      }
    }
  }
  if (failed == 1) {
#pragma unroll
    for (int k = 0; k < NSP; ++k) c.X[k] = Xs[k];
    c.status = CHEM_CELL_NEWTON_FAIL;
    c.done = true;
    return;
  }
  // WRMS norm; the weights' reciprocals are Newton-Raphson-refined (two steps, within
  // 2 ulp, in the fp64 variant; one step, ~2^-40 relative, in the mixed one, whose fp32
  // stages perturb the estimate far more)
  double err = CUDART_NAN;
  if (!failed) {
    double sum = 0.0;
#pragma unroll
    for (int k = 0; k < NSP; ++k) {
      const double den = fma(p.rtol, max_abs(Xs[k], c.X[k]), p.atol);
      const double w = E[k] * (kMixed ? rcp1(den) : rcp2(den));
      sum = fma(w, w, sum);
    }
    err = sqrt(sum * (1.0 / NSP));
  }
  // a rejected attempt returns the cell to its accepted state, the temperature warm
  // start included (a trial stage's temperature can sit near another root of e(T) of the
  // extrapolated polynomials)
  if (!isfinite(err)) {
#pragma unroll
    for (int k = 0; k < NSP; ++k) c.X[k] = Xs[k];
    c.T = Tacc;
    ++c.nrej;
    c.h = h * 0.2;
    return;
  }
  // the step factor stays IEEE fp64: an explicit scheme at its stability limit grows a
  // perturbation of h along its weakly unstable modes into another rejection sequence
  const double fac = (err == 0.0) ? 5.0 : fmin(5.0, fmax(0.2, 0.9 / sqrt(sqrt(err))));
  if (err <= 1.0) {
    c.t += h;
    ++c.nacc;
  } else {
#pragma unroll
    for (int k = 0; k < NSP; ++k) c.X[k] = Xs[k];
    c.T = Tacc;
    ++c.nrej;
  }
  c.h = h * fac;
}

// One attempted step of a full-storage scheme (CHEM_SCHEME_FULL_STORAGE: table 0, five
// stages; CHEM_SCHEME_RKF45: table 1, six stages).  The same controller as cell_attempt
// with the table's exponent (1/4 and 1/5).  The stage loop stays rolled (the right-hand
// side is inlined once); the stage derivatives live in a register array indexed by
// compile-time constants, written through predicated moves, so the k-storage costs
// registers (and spills), not local-memory indexing.
template <int V, int SCH>
__device__ __forceinline__ void cell_attempt_full(const MechTables &mt, CellState &c,
                                                  const StepParams &p) {
  constexpr bool kMixed = V == CHEM_VARIANT_MIXED;
  constexpr int TB = SCH == CHEM_SCHEME_RKF45 ? 1 : 0;
  constexpr int S = SCH == CHEM_SCHEME_RKF45 ? 6 : 5;
  using SReal = std::conditional_t<kMixed, float, double>;
  const double dt = c.dt;
  if (!(dt - c.t > 1e-12 * dt)) { c.done = true; return; }
  if (c.nacc + c.nrej >= p.max_steps) { c.status = CHEM_CELL_MAX_STEPS; c.done = true; return; }
  if (c.h < 1e-15 * dt) { c.status = CHEM_CELL_H_UNDERFLOW; c.done = true; return; }
  double h = c.h;
  if (h > dt - c.t) h = dt - c.t;
  SReal K[S][NSP];
#pragma unroll
  for (int j = 0; j < S; ++j)
#pragma unroll
    for (int k = 0; k < NSP; ++k) K[j][k] = SReal(0);
  int failed = 0;
  double Tacc = c.T;
#pragma unroll 1
  for (int s = 0; s < S; ++s) {
    SReal U[NSP], F[NSP];
#pragma unroll
    for (int k = 0; k < NSP; ++k) {
      if constexpr (kMixed) {
        float acc = 0.0f;
#pragma unroll
        for (int j = 0; j < S - 1; ++j)
          if (j < s) acc = fmaf(d2f(h * c_fs_a[TB][s][j]), K[j][k], acc);
        U[k] = d2f(c.X[k]) + acc;
      } else {
        double acc = 0.0;
#pragma unroll
        for (int j = 0; j < S - 1; ++j)
          if (j < s) acc = fma(c_fs_a[TB][s][j], K[j][k], acc);
        U[k] = fma(h, acc, c.X[k]);
      }
    }
    ++c.nrhs;
    bool ok;
    if constexpr (kMixed) ok = cell_rhs_mixed(mt, U, c.rho_f, c.invRho_f, c.eR, c.T, F);
    else ok = cell_rhs(mt, U, c.rho, c.invRho, c.eR, c.T, F);
    if (!ok) { failed = s + 1; break; }
    if (s == 0) Tacc = c.T;
#pragma unroll
    for (int j = 0; j < S; ++j)
      if (j == s) {
#pragma unroll
        for (int k = 0; k < NSP; ++k) K[j][k] = F[k];
      }
  }
  if (failed == 1) {
    c.status = CHEM_CELL_NEWTON_FAIL;
    c.done = true;
    return;
  }
  double Xn[NSP], E[NSP];
  double err = CUDART_NAN;
  if (!failed) {
    double sum = 0.0;
#pragma unroll
    for (int k = 0; k < NSP; ++k) {
      double sb = 0.0, se = 0.0;
#pragma unroll
      for (int j = 0; j < S; ++j) {
        const double Kj = kMixed ? f2d((float)K[j][k]) : (double)K[j][k];
        sb = fma(c_fs_b[TB][j], Kj, sb);
        se = fma(c_fs_e[TB][j], Kj, se);
      }
      Xn[k] = fma(h, sb, c.X[k]);
      E[k] = h * se;
      const double den = fma(p.rtol, max_abs(c.X[k], Xn[k]), p.atol);
      const double w = E[k] * (kMixed ? rcp1(den) : rcp2(den));
      sum = fma(w, w, sum);
    }
    err = sqrt(sum * (1.0 / NSP));
  }
  if (!isfinite(err)) {
    c.T = Tacc;
    ++c.nrej;
    c.h = h * 0.2;
    return;
  }
  double fac;
  if (err == 0.0) fac = 5.0;
  else if constexpr (TB == 1) fac = fmin(5.0, fmax(0.2, 0.9 * pow(err, -0.2)));
  else fac = fmin(5.0, fmax(0.2, 0.9 / sqrt(sqrt(err))));
  if (err <= 1.0) {
#pragma unroll
    for (int k = 0; k < NSP; ++k) c.X[k] = Xn[k];
    c.t += h;
    ++c.nacc;
  } else {
    c.T = Tacc;
    ++c.nrej;
  }
  c.h = h * fac;
}

// Temperature of the final state (fp64 Newton); a failure marks the cell.
__device__ __forceinline__ void cell_finish(const MechTables &mt, CellState &c) {
  if (c.status == CHEM_CELL_NONFINITE) return;
  if (!solve_T(mt, c.X, c.eR, c.T)) {
    if (c.status == CHEM_CELL_OK) c.status = CHEM_CELL_NEWTON_FAIL;
    c.T = CUDART_NAN;
  }
}

__device__ __forceinline__ long long warp_sum(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ int warp_max(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Warp-aggregated statistics: one atomic per counter per warp.  Every lane of the warp
// must call it (no early return in the kernels).  cells/status_count count the cells
// this lane finished (persistent lanes finish several).
__device__ __forceinline__ void accumulate_stats(chem_stats *st, int cells, int nacc, int nrej,
                                                 int nrhs, int maxsteps, const int (&hist)[6]) {
  const int lane = threadIdx.x & 31;
  const long long wc = warp_sum(cells);
  const long long acc = warp_sum(nacc);
  const long long rej = warp_sum(nrej);
  const long long rhs = warp_sum(nrhs);
  const int mx = warp_max(maxsteps);
  long long wh[6];
#pragma unroll
  for (int s = 0; s < 6; ++s) wh[s] = warp_sum(hist[s]);
  if (lane == 0 && wc > 0) {
    atomicAdd(reinterpret_cast<unsigned long long *>(&st->cells), (unsigned long long)wc);
    atomicAdd(reinterpret_cast<unsigned long long *>(&st->accepted), (unsigned long long)acc);
    atomicAdd(reinterpret_cast<unsigned long long *>(&st->rejected), (unsigned long long)rej);
    atomicAdd(reinterpret_cast<unsigned long long *>(&st->rhs_evals), (unsigned long long)rhs);
    atomicMax(reinterpret_cast<unsigned long long *>(&st->max_steps_cell), (unsigned long long)mx);
#pragma unroll
    for (int s = 0; s < 6; ++s)
      if (wh[s]) atomicAdd(reinterpret_cast<unsigned long long *>(&st->status_count[s]),
                           (unsigned long long)wh[s]);
  }
}

}  // namespace chem
