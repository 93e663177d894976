// integrate.cu -- per-cell low-storage RK integration kernels (Eq. 21-22, Sec. 2.2.3).
//
// One thread per cell (Sec. 4.1.2).  Per cell the integrator keeps four register
// vectors of NSP fp64 values: the solution register X (y_n advancing to y_n+1), the
// stage register U (input of the next right-hand side), the error register E
// (sum_i (b_i - bhat_i) h F_i, the embedded third-order estimate) and the saved
// y_n for a rejected step; F is transient.  That is the two-register scheme of Eq. 21
// plus the error register the paper adds, plus the copy any rejecting controller
// needs.  The stage loop stays rolled (its coefficients come from __constant__), so
// the right-hand side is inlined once.
//
// Controller (Eq. 22): ||e|| = sqrt(mean_k (E_k / (rtol max(|y_n,k|, |y_n+1,k|) + atol))^2);
// accept iff ||e|| <= 1; h <- h min(5, max(0.2, 0.9 ||e||^(-1/4))); h is clipped to land
// on dt; the loop ends when dt - t <= 1e-12 dt; attempted steps are capped; h below
// 1e-15 dt is an underflow.  A trial stage whose temperature solve fails rejects the
// attempt with factor 1/5; a failure at stage 1 (the accepted state) ends the cell.
#include <cuda_runtime.h>
#include <math_constants.h>

#include <type_traits>

#include "internal.cuh"
#include "rhs.cuh"
#include "rhs_mixed.cuh"

namespace chem {

// RK4(3)5[2R+]C (Kennedy, Carpenter & Lewis 2000): a_{s+1,s} (0 after the last
// stage), b_s and b_s - bhat_s.
__constant__ double c_ls_a[5] = {
    970286171893.0 / 4311952581923.0, 6584761158862.0 / 12103376702013.0,
    2251764453980.0 / 15575788980749.0, 26877169314380.0 / 34165994151039.0, 0.0};
__constant__ double c_ls_b[5] = {
    1153189308089.0 / 22510343858157.0, 1772645290293.0 / 4653164025191.0,
    -1672844663538.0 / 4480602732383.0, 2114624349019.0 / 3568978502595.0,
    5198255086312.0 / 14908931495163.0};
__constant__ double c_ls_e[5] = {
    1153189308089.0 / 22510343858157.0 - 1016888040809.0 / 7410784769900.0,
    1772645290293.0 / 4653164025191.0 - 11231460423587.0 / 58533540763752.0,
    -1672844663538.0 / 4480602732383.0 - -1563879915014.0 / 6823010717585.0,
    2114624349019.0 / 3568978502595.0 - 606302364029.0 / 971179775848.0,
    5198255086312.0 / 14908931495163.0 - 1097981568119.0 / 3980877426909.0};

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
// must call it (no early return in the kernels).
__device__ __forceinline__ void accumulate_stats(chem_stats *st, bool live, int nacc, int nrej,
                                                 int nrhs, int status) {
  const int lane = threadIdx.x & 31;
  const long long cells = warp_sum(live ? 1 : 0);
  const long long acc = warp_sum(nacc);
  const long long rej = warp_sum(nrej);
  const long long rhs = warp_sum(nrhs);
  const int mx = warp_max(nacc + nrej);
  long long hist[6];
#pragma unroll
  for (int s = 0; s < 6; ++s) hist[s] = warp_sum(live && status == s ? 1 : 0);
  if (lane == 0 && cells > 0) {
    atomicAdd(reinterpret_cast<unsigned long long *>(&st->cells), (unsigned long long)cells);
    atomicAdd(reinterpret_cast<unsigned long long *>(&st->accepted), (unsigned long long)acc);
    atomicAdd(reinterpret_cast<unsigned long long *>(&st->rejected), (unsigned long long)rej);
    atomicAdd(reinterpret_cast<unsigned long long *>(&st->rhs_evals), (unsigned long long)rhs);
    atomicMax(reinterpret_cast<unsigned long long *>(&st->max_steps_cell), (unsigned long long)mx);
#pragma unroll
    for (int s = 0; s < 6; ++s)
      if (hist[s]) atomicAdd(reinterpret_cast<unsigned long long *>(&st->status_count[s]),
                             (unsigned long long)hist[s]);
  }
}

// Integrate one cell in place.  Returns the status; counts attempts and RHS calls.
// V = CHEM_VARIANT_FP64: every register fp64.  V = CHEM_VARIANT_MIXED: the stage
// register U and the stage derivative F are fp32 (cell_rhs_mixed); the solution X, the
// saved y_n, the error register E, the WRMS norm and the controller stay fp64.
template <int V>
__device__ __forceinline__ int integrate_cell(const MechTables &mt, double rho, double e,
                                              double (&X)[NSP], double &T, double &h,
                                              const StepParams &p, int &nacc, int &nrej,
                                              int &nrhs) {
  constexpr bool kMixed = V == CHEM_VARIANT_MIXED;
  using SReal = std::conditional_t<kMixed, float, double>;
  bool bad = !(isfinite(rho) && rho > 0.0 && isfinite(e));
#pragma unroll
  for (int k = 0; k < NSP; ++k) bad |= !isfinite(X[k]);
  if (bad) {
    T = CUDART_NAN;
    return CHEM_CELL_NONFINITE;
  }
  const double dt = p.dt;
  const double invRho = 1.0 / rho;
  const float rho_f = (float)rho, invRho_f = (float)invRho;
  const double eR = e / R_U;
  int status = CHEM_CELL_OK;
  double t = 0.0;
  while (dt - t > 1e-12 * dt) {
    if (nacc + nrej >= p.max_steps) { status = CHEM_CELL_MAX_STEPS; break; }
    if (h < 1e-15 * dt) { status = CHEM_CELL_H_UNDERFLOW; break; }
    if (h > dt - t) h = dt - t;
    double Xs[NSP], E[NSP];
    SReal U[NSP];
#pragma unroll
    for (int k = 0; k < NSP; ++k) { Xs[k] = X[k]; U[k] = (SReal)X[k]; E[k] = 0.0; }
    int failed = 0;
#pragma unroll 1
    for (int s = 0; s < 5; ++s) {
      SReal F[NSP];
      ++nrhs;
      bool ok;
      if constexpr (kMixed) ok = cell_rhs_mixed(mt, U, rho_f, invRho_f, eR, T, F);
      else ok = cell_rhs(mt, U, rho, invRho, eR, T, F);
      if (!ok) { failed = s + 1; break; }
      const double ha = h * c_ls_a[s], hb = h * c_ls_b[s], he = h * c_ls_e[s];
      if constexpr (kMixed) {
        const float ha_f = (float)ha;
#pragma unroll
        for (int k = 0; k < NSP; ++k) {
          U[k] = fmaf(ha_f, F[k], (float)X[k]);
          const double Fk = (double)F[k];
          E[k] = fma(he, Fk, E[k]);
          X[k] = fma(hb, Fk, X[k]);
        }
      } else {
#pragma unroll
        for (int k = 0; k < NSP; ++k) {
          E[k] = fma(he, F[k], E[k]);
          U[k] = fma(ha, F[k], X[k]);
          X[k] = fma(hb, F[k], X[k]);
        }
      }
    }
    if (failed == 1) {
#pragma unroll
      for (int k = 0; k < NSP; ++k) X[k] = Xs[k];
      status = CHEM_CELL_NEWTON_FAIL;
      break;
    }
    double err = CUDART_NAN;
    if (!failed) {
      double sum = 0.0;
#pragma unroll
      for (int k = 0; k < NSP; ++k) {
        const double w = E[k] / fma(p.rtol, fmax(fabs(Xs[k]), fabs(X[k])), p.atol);
        sum = fma(w, w, sum);
      }
      err = sqrt(sum * (1.0 / NSP));
    }
    if (!isfinite(err)) {
#pragma unroll
      for (int k = 0; k < NSP; ++k) X[k] = Xs[k];
      ++nrej;
      h *= 0.2;
      continue;
    }
    const double fac = (err == 0.0) ? 5.0 : fmin(5.0, fmax(0.2, 0.9 / sqrt(sqrt(err))));
    if (err <= 1.0) {
      t += h;
      ++nacc;
    } else {
#pragma unroll
      for (int k = 0; k < NSP; ++k) X[k] = Xs[k];
      ++nrej;
    }
    h *= fac;
  }
  if (status != CHEM_CELL_NONFINITE) {
    double yw[NSP];
#pragma unroll
    for (int k = 0; k < NSP; ++k) yw[k] = X[k] * mt.invW[k];
    if (!solve_T(mt, yw, eR, T)) {
      if (status == CHEM_CELL_OK) status = CHEM_CELL_NEWTON_FAIL;
      T = CUDART_NAN;
    }
  }
  return status;
}

template <int V>
__global__ void __launch_bounds__(128) k_lsrk(const __grid_constant__ MechTables mt,
                                              const CellArgs a, const StepParams p) {
  load_math_tables();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = i < a.n;
  int nacc = 0, nrej = 0, nrhs = 0, status = 0;
  if (live) {
    double X[NSP];
#pragma unroll
    for (int k = 0; k < NSP; ++k) X[k] = a.Y[k * a.ld + i];
    double T = a.T[i];
    double h = p.dt;
    if (a.h) {
      const double h0 = a.h[i];
      if (isfinite(h0) && h0 > 0.0) h = h0;
    }
    status = integrate_cell<V>(mt, a.rho[i], a.e[i], X, T, h, p, nacc, nrej, nrhs);
#pragma unroll
    for (int k = 0; k < NSP; ++k) a.Y[k * a.ld + i] = X[k];
    a.T[i] = T;
    if (a.h) a.h[i] = h;
    if (a.status) a.status[i] = status;
    if (a.nsteps) a.nsteps[i] = nacc + nrej;
  }
  if (a.stats) accumulate_stats(a.stats, live, nacc, nrej, nrhs, status);
}

__global__ void k_state_from_TPY(const __grid_constant__ MechTables mt, int64_t n,
                                 const double *__restrict__ T, const double *__restrict__ p,
                                 const double *__restrict__ Y, int64_t ld, double *__restrict__ rho,
                                 double *__restrict__ e) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double Ti = T[i];
  double yw[NSP], inv_w = 0.0;
#pragma unroll
  for (int k = 0; k < NSP; ++k) {
    yw[k] = Y[k * ld + i] * mt.invW[k];
    inv_w += yw[k];
  }
  double m[6];
  mix_ecoef(mt, Ti >= mt.T_mid, yw, m);
  rho[i] = p[i] / (R_U * Ti * inv_w);
  e[i] = R_U * e_over_R(m, Ti);
}

cudaError_t launch_lsrk(int variant, const MechTables &mt, const CellArgs &a, const StepParams &p,
                        int block, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  if (block != 128) block = 128;  // the kernel's launch bounds
  const int64_t grid = (a.n + block - 1) / block;
  if (variant == CHEM_VARIANT_MIXED)
    k_lsrk<CHEM_VARIANT_MIXED><<<(unsigned)grid, block, 0, s>>>(mt, a, p);
  else
    k_lsrk<CHEM_VARIANT_FP64><<<(unsigned)grid, block, 0, s>>>(mt, a, p);
  return cudaGetLastError();
}

cudaError_t launch_state_from_TPY(const MechTables &mt, int64_t n, const double *T,
                                  const double *p, const double *Y, int64_t ld, double *rho,
                                  double *e, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int block = 256;
  const int64_t grid = (n + block - 1) / block;
  k_state_from_TPY<<<(unsigned)grid, block, 0, s>>>(mt, n, T, p, Y, ld, rho, e);
  return cudaGetLastError();
}

}  // namespace chem
