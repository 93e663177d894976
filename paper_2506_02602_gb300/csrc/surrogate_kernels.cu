// surrogate_kernels.cu -- device kernels of the learned surrogate around the MLP:
// featurisation, column statistics, the inference epilogue (inverse transform,
// element-conservation projection, temperature solve, gate, fallback compaction) and
// the one-box batch of the fallback integration.
//
// Features of a cell (12, padded to 16): T, ln p, log10 dt and the Box-Cox transforms
// BC(Y_k) = (max(Y_k, 1e-30)^lam - 1) / lam of the 9 mass fractions; targets (9, padded
// to 16): (BC(Y_k(t + dt)) - BC(Y_k(t))) (1e-8 s / dt)^dt_power.  Both are z-scored with
// training statistics.
// The temperature is always solved from (e, Y) in fp64, so energy is conserved exactly
// by construction; the projection restores the element (H, O, N) mass fractions, hence
// sum Y too, in fp64.
//
// A-posteriori error test: the integrator's own right-hand side checks each candidate result.  With
// F0 = f(Y0), F1 = f(Y1) and Fm = f(Ym) at the cubic Hermite midpoint
// Ym = (Y0 + Y1) / 2 + dt/8 (F0 - F1), Simpson's rule Yc = Y0 + dt/6 (F0 + 4 Fm + F1)
// differs from the exact solution by O(dt^5) where the cell is smooth over dt, so the
// defect D = Y1 - Yc estimates the error of Y1.  At constant e the temperature moves by
// -sum_k (u_k - e) dY_k / c_v for a change dY with sum_k dY_k = 0, so the test takes
//   est = sum_k |u_k(T1) - e| |D_k| / c_v(T1)
// (no cancellation between species counted) and sends a cell with est > err_tol * T1
// to the integrator.  Stiff cells (dt beyond the fast time scales), where the
// quadrature itself is not accurate, fail the check too.  Linearised, an error d of Y1
// shows in the defect as (I - z/2 + z^2/12) d, z = dt J; the factor has no real root
// (its minimum is 1/4, at z = 3) but shrinks along growing modes, so the test also
// bounds the cell's reactivity over the step,
//   rate = dt * max_k max(|F0_k| / (|Y0_k| + 1e-6), |F1_k| / (|Y1_k| + 1e-6)) <= rate_max,
// and divides the estimate by the factor at z = rate, 1 - rate/2 + rate^2/12, before
// comparing it with err_tol * T (1e-6: the mass fraction below which a species'
// share of the mixture energy is under ~1 K).  A trapezoidal check (two right-hand
// sides) was tried first: its O(dt^3) truncation can cancel a surrogate error of the
// same size, which let a few cells through with twice the tolerated error.
#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "cell.cuh"
#include "internal.cuh"
#include "surrogate.cuh"

namespace chem {

__device__ __forceinline__ double boxcox_d(double y, double lam) {
  return (pow(fmax(y, 1e-30), lam) - 1.0) / lam;
}

// The features' transform in fp32 (they are fp32 network inputs).
__device__ __forceinline__ float boxcox_f(double y, float lam) {
  return (powf(fmaxf(d2f(y), 1e-30f), lam) - 1.0f) / lam;
}

// max(x, c) for c > 0 on the integer pipe (a negative x, whose bit pattern is a negative
// integer, gives c)
__device__ __forceinline__ double max_pos(double x, double c) {
  return __double_as_longlong(x) > __double_as_longlong(c) ? x : c;
}

// Y1 from Y0, its fp32 feature bc0 = BC(Y0) and the predicted increment d, as an
// increment on Y0: with y = max(Y0, 1e-30) (the transform's floor) and 1 + lam bc0
// standing for y^lam, the Box-Cox inverse of bc0 + d is y r with
// r = (1 + lam d / (1 + lam bc0))^(1/lam), and Y1 = Y0 + y (r - 1).  The feature's
// rounding cancels, d = 0 returns Y0 exactly, and a species absent from Y0 can form.
// A base at or below zero (r = 0) gives Y1 = Y0 - y.
__device__ __forceinline__ double boxcox_step(double y0, float bc0, float d, float lam) {
  const double y = max_pos(y0, 1e-30);
  const float s = lam * d / fmaf(lam, bc0, 1.0f);
  if (!(s > -1.0f)) return y0 - y;
  return fma(y, f2d(expm1f(log1pf(s) / lam)), y0);
}

// Raw (un-normalised) features and, when Y1 is given, targets of n cells.
// X[i, 0:12] = T, ln p, log10 dt, BC(Y0); Tg[i, 0:9] = BC(Y1) - BC(Y0).  Padding zero.
// ok (nullable) 1 where T solved.  The features are fp32 network inputs (rounded to BF16
// in the first layer), so T is solved in fp32 (Newton to 2e-6 T from the cell's T), the
// same way for training and inference.
__global__ void k_features(const __grid_constant__ MechTables mt, int64_t n, const double *rho,
                           const double *e, const double *Y0, int64_t ld0, const double *Tg0,
                           const double *dt_cell, double dt_scalar, const double *Y1, int64_t ld1,
                           double lam, double dt_power, float *X, float *Tg, uint8_t *ok) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double y[NSP];
  float yw[NSP];
  float inv_w = 0.0f;
#pragma unroll
  for (int k = 0; k < NSP; ++k) {
    y[k] = Y0[k * ld0 + i];
    yw[k] = d2f(y[k]) * mt.f.invW[k];
    inv_w += yw[k];
  }
  float T = Tg0 ? d2f(Tg0[i]) : CUDART_NAN_F;
  const bool good = isfinite(rho[i]) && rho[i] > 0.0 && isfinite(e[i]) &&
                    solve_T_f32(mt, yw, d2f(e[i] * (1.0 / R_U)), T);
  if (!good) T = 1500.0f;
  const float p = d2f(rho[i]) * (float)R_U * T * inv_w;
  const double dt = dt_cell ? dt_cell[i] : dt_scalar;
  float *x = X + i * kSurIn;
  x[0] = T;
  x[1] = logf(fmaxf(p, 1e-30f));
  x[2] = log10f(d2f(dt));
#pragma unroll
  for (int k = 0; k < NSP; ++k) x[3 + k] = boxcox_f(y[k], (float)lam);
#pragma unroll
  for (int c = 12; c < kSurIn; ++c) x[c] = 0.0f;
  if (Y1) {  // training targets: the fp64 increment (no cancellation of two fp32 values)
    float *t = Tg + i * kSurOut;
    const double sc = dt_power == 0.0 ? 1.0 : pow(kSurDtRef / dt, dt_power);
#pragma unroll
    for (int k = 0; k < NSP; ++k)
      t[k] = (float)((boxcox_d(Y1[k * ld1 + i], lam) - boxcox_d(y[k], lam)) * sc);
#pragma unroll
    for (int c = NSP; c < kSurOut; ++c) t[c] = 0.0f;
  }
  if (ok) ok[i] = good;
}

// Column sums, sums of squares, minima and maxima of the first ncol columns of a
// row-major [n x ld] float matrix (double sums; minima and maxima as order-preserving
// integer keys of the float bits, which the host initialises to INT_MAX / INT_MIN and
// decodes with float_key_decode).
__device__ __forceinline__ int float_key(float f) {
  const int b = __float_as_int(f);
  return b >= 0 ? b : b ^ 0x7fffffff;
}

__global__ void k_colstats(int64_t n, int ncol, int ld, const float *__restrict__ A, double *sum,
                           double *sumsq, int *mnkey, int *mxkey) {
  __shared__ double s1[32][9], s2[32][9];
  __shared__ float smin[32][9], smax[32][9];
  const int lane = threadIdx.x & 31, row = threadIdx.x >> 5;  // blockDim 256: 8 row groups
  double a = 0.0, b = 0.0;
  float lo = 3.0e38f, hi = -3.0e38f;
  if (lane < ncol) {
    for (int64_t i = (int64_t)blockIdx.x * 8 + row; i < n; i += (int64_t)gridDim.x * 8) {
      const float v = A[i * ld + lane];
      a += v;
      b += (double)v * v;
      lo = fminf(lo, v);
      hi = fmaxf(hi, v);
    }
  }
  s1[lane][row] = a;
  s2[lane][row] = b;
  smin[lane][row] = lo;
  smax[lane][row] = hi;
  __syncthreads();
  if (threadIdx.x < ncol) {
    double ta = 0.0, tb = 0.0;
    float tl = 3.0e38f, th = -3.0e38f;
    for (int r = 0; r < 8; ++r) {
      ta += s1[threadIdx.x][r];
      tb += s2[threadIdx.x][r];
      tl = fminf(tl, smin[threadIdx.x][r]);
      th = fmaxf(th, smax[threadIdx.x][r]);
    }
    atomicAdd(&sum[threadIdx.x], ta);
    atomicAdd(&sumsq[threadIdx.x], tb);
    atomicMin(&mnkey[threadIdx.x], float_key(tl));
    atomicMax(&mxkey[threadIdx.x], float_key(th));
  }
}

// In place: A[i, c] = (A[i, c] - mean[c]) * inv_std[c] for c < ncol, and a bf16 copy.
__global__ void k_normalize(int64_t n, int ncol, int ld, float *A, const float *mean,
                            const float *inv_std, __nv_bfloat16 *Abf) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * ld) return;
  const int c = (int)(t % ld);
  float v = A[t];
  if (c < ncol) v = (v - mean[c]) * inv_std[c];
  else v = 0.0f;
  A[t] = v;
  if (Abf) Abf[t] = __float2bfloat16(v);
}

// Temperature-error estimate of a surrogate result y1 (see the file comment): returns
// false if a right-hand side fails, else sets dT = est (K) and rate = dt * the largest
// relative rate of change at either end.  All in fp32 with the fast intrinsics
// (cell_rhs_f32), whatever the context's variant: an estimate compared with a tolerance
// of ~5e-4 T needs nothing finer; y1 - y0 is formed in fp64 first, so the defect does not
// lose it to rounding.
__device__ __forceinline__ bool posterior_error(const MechTables &mt, const double (&y0)[NSP],
                                             const double (&y1)[NSP], float rho_f, float eR,
                                             float T0, float T1f, float dtf, float &dT, float &rate) {
  float u0[NSP], u1[NSP], F0[NSP], F1[NSP];
#pragma unroll
  for (int k = 0; k < NSP; ++k) {
    u0[k] = d2f(y0[k]);
    u1[k] = d2f(y1[k]);
  }
  const float invRho_f = __fdividef(1.0f, rho_f);
  float Ta = T0, Tb = T1f;
  if (!cell_rhs_f32(mt, u0, rho_f, invRho_f, eR, Ta, F0) || !cell_rhs_f32(mt, u1, rho_f, invRho_f, eR, Tb, F1))
    return false;
  float um[NSP], Fm[NSP];
#pragma unroll
  for (int k = 0; k < NSP; ++k) um[k] = 0.5f * (u0[k] + u1[k]) + 0.125f * dtf * (F0[k] - F1[k]);
  float Tm = 0.5f * (Ta + Tb);
  if (!cell_rhs_f32(mt, um, rho_f, invRho_f, eR, Tm, Fm)) return false;
  const float sdt = dtf * (1.0f / 6.0f);
  const int range = T1f >= mt.f.T_mid;
  float m[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int k = 0; k < NSP; ++k) {
    const float yw = u1[k] * mt.f.invW[k];
#pragma unroll
    for (int i = 0; i < 5; ++i) m[i] = fmaf(yw, mt.f.ec[range][k][i], m[i]);
  }
  const float cvR = fmaf(T1f, fmaf(T1f, fmaf(T1f, fmaf(T1f, 5.0f * m[4], 4.0f * m[3]), 3.0f * m[2]), 2.0f * m[1]), m[0]);
  float r = 0.0f, sum = 0.0f;
#pragma unroll
  for (int k = 0; k < NSP; ++k) {
    const float *c = mt.f.ec[range][k];
    const float ukR =
        fmaf(T1f, fmaf(T1f, fmaf(T1f, fmaf(T1f, fmaf(T1f, c[4], c[3]), c[2]), c[1]), c[0]), c[5]) * mt.f.invW[k];
    const float defect = d2f(y1[k] - y0[k]) - sdt * (F0[k] + 4.0f * Fm[k] + F1[k]);
    sum = fmaf(fabsf(ukR - eR), fabsf(defect), sum);
    r = fmaxf(r, fmaxf(__fdividef(fabsf(F0[k]), fabsf(u0[k]) + 1e-6f), __fdividef(fabsf(F1[k]), fabsf(u1[k]) + 1e-6f)));
  }
  rate = dtf * r;
  dT = __fdividef(sum, cvR);
  return isfinite(dT) && cvR > 0.0f;
}

// The inference epilogue, one thread per cell.  Takes the network output O [n x 16]
// (z-scored BC increments), the raw features X (un-normalised: T, ln p, log10 dt,
// BC(Y0)) and the state; writes accepted cells (Y'', T'', status OK, nsteps 0) and
// appends rejected ones to the fallback list.
// Weighted least-squares projection of the prediction y1 onto the element (H, O, N) mass
// fractions of y0: Y'' = Y' - W E^T (E W E^T)^-1 r with W = diag(max(Y'_k, 1e-12)) and
// r = E (Y' - Y0), in fp64 (terms with a zero element fraction skipped: uniform branches
// on the masks).  rn and zn receive |r|^2 and |E Y0|^2 of the raw prediction (the
// residual gate's inputs).  Returns false, with y1 unchanged, when the 3x3 system is
// singular or not finite.
__device__ __forceinline__ bool project_elements(const SurrogateConsts &sc, const double (&y0)[NSP],
                                                 double (&y1)[NSP], double &rn, double &zn) {
  double z0[3] = {0.0, 0.0, 0.0}, r[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int el = 0; el < 3; ++el)
#pragma unroll
    for (int k = 0; k < NSP; ++k)
      if ((sc.emask[el] >> k) & 1) {
        z0[el] = fma(sc.E[el][k], y0[k], z0[el]);
        r[el] = fma(sc.E[el][k], y1[k] - y0[k], r[el]);
      }
  rn = 0.0;
  zn = 0.0;
#pragma unroll
  for (int el = 0; el < 3; ++el) {
    rn = fma(r[el], r[el], rn);
    zn = fma(z0[el], z0[el], zn);
  }
  double w[NSP], M[3][3];
#pragma unroll
  for (int k = 0; k < NSP; ++k) w[k] = max_pos(y1[k], 1e-12);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = a; b < 3; ++b) {
      double s = 0.0;
#pragma unroll
      for (int k = 0; k < NSP; ++k)
        if (((sc.emask[a] & sc.emask[b]) >> k) & 1) s = fma(sc.E[a][k] * w[k], sc.E[b][k], s);
      M[a][b] = s;
      M[b][a] = s;
    }
  // 3x3 solve by Cramer's rule (M is symmetric positive definite for the H, O, N rows)
  const double det = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
                     M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                     M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
  if (!(det != 0.0 && isfinite(det))) return false;
  const double id = rcp2(det);
  double lamv[3];
  lamv[0] = (r[0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) - M[0][1] * (r[1] * M[2][2] - M[1][2] * r[2]) +
             M[0][2] * (r[1] * M[2][1] - M[1][1] * r[2])) * id;
  lamv[1] = (M[0][0] * (r[1] * M[2][2] - M[1][2] * r[2]) - r[0] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
             M[0][2] * (M[1][0] * r[2] - r[1] * M[2][0])) * id;
  lamv[2] = (M[0][0] * (M[1][1] * r[2] - r[1] * M[2][1]) - M[0][1] * (M[1][0] * r[2] - r[1] * M[2][0]) +
             r[0] * (M[1][0] * M[2][1] - M[1][1] * M[2][0])) * id;
#pragma unroll
  for (int k = 0; k < NSP; ++k) {
    double corr = 0.0;
#pragma unroll
    for (int el = 0; el < 3; ++el)
      if ((sc.emask[el] >> k) & 1) corr = fma(sc.E[el][k], lamv[el], corr);
    y1[k] = fma(-w[k], corr, y1[k]);
  }
  return true;
}

// The projection alone on given predictions (a check entry; see project_elements).
__global__ void k_project_check(const __grid_constant__ SurrogateConsts sc, int64_t n,
                                const double *__restrict__ Y0, const double *__restrict__ Yp,
                                int64_t ld, double *__restrict__ Yout) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double y0[NSP], y1[NSP];
#pragma unroll
  for (int k = 0; k < NSP; ++k) {
    y0[k] = Y0[k * ld + i];
    y1[k] = Yp[k * ld + i];
  }
  double rn, zn;
  project_elements(sc, y0, y1, rn, zn);
#pragma unroll
  for (int k = 0; k < NSP; ++k) Yout[k * ld + i] = y1[k];
}

// 4 blocks of 128 per SM (16 warps): the register cap of 128 costs 4 bytes of spill
// stores, against 8 warps at the uncapped 255 registers.  The error test is inlined: as a
// called function it took its state arrays by reference through a ~580-byte local
// stack frame, and the kernel ran 10-14 % slower.
template <int V>
__global__ void __launch_bounds__(128, 4)
    k_surrogate_finish(const __grid_constant__ MechTables mt, const __grid_constant__ SurrogateConsts sc,
                       int64_t n, double dt, const float *__restrict__ O,
                       const float *__restrict__ Xraw, const uint8_t *__restrict__ Tok,
                       const double *__restrict__ rho, const double *__restrict__ e, double *Y,
                       int64_t ld, double *T, int32_t *status, int32_t *nsteps, uint8_t *mask,
                       int32_t *fb_idx, unsigned int *fb_count, int64_t base) {
  load_math_tables();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float *x = Xraw + i * kSurIn;
  const float *o = O + i * kSurOut;
  // reason of a rejection (the first gate that fails), reported in the fallback mask
  int reason = Tok[i] != 0 ? 0 : kFbTemperature;
  // out-of-distribution: every feature within the training box widened by the margin
  bool inbox = true;
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    const float w = sc.margin * (sc.fmax[c] - sc.fmin[c]);
    inbox &= x[c] >= sc.fmin[c] - w && x[c] <= sc.fmax[c] + w;
  }
  if (!reason && !inbox) reason = kFbRange;
  double y0[NSP], y1[NSP];
  const float unscale =
      sc.dt_power == 0.0 ? 1.0f : powf(d2f(dt) * (float)(1.0 / kSurDtRef), d2f(sc.dt_power));
#pragma unroll
  for (int k = 0; k < NSP; ++k) {
    y0[k] = Y[k * ld + i];
    const float d = fmaf(o[k], sc.tstd[k], sc.tmean[k]) * unscale;
    y1[k] = boxcox_step(y0[k], x[3 + k], d, (float)sc.lam);
  }
  double rn = 0.0, zn = 0.0;
  const bool solved = project_elements(sc, y0, y1, rn, zn);
  if (!reason && !(rn <= (double)sc.resid_max * sc.resid_max * zn)) reason = kFbResidual;
  if (!reason && !solved) reason = kFbResidual;
  // the negativity test on the fp32-rounded result (a NaN fails it)
  bool neg = false;
#pragma unroll
  for (int k = 0; k < NSP; ++k) neg |= !(d2f(y1[k]) >= -sc.neg_tol);
  if (!reason && neg) reason = kFbNegative;
  // temperature of the projected state (fp64 Newton from the input temperature)
  const double eR = e[i] * (1.0 / R_U);
  double T1 = f2d(x[0]);
  const bool tok = solve_T(mt, y1, eR, T1);
  const float T1f = d2f(T1);
  if (!reason && !(tok && fabsf(T1f - x[0]) <= sc.max_dT)) reason = kFbTemperature;
  if (!reason && sc.err_tol > 0.0f) {
    float dT = 0.0f, rate = 0.0f;
    const bool jok = posterior_error(mt, y0, y1, d2f(rho[i]), d2f(eR), x[0], T1f, d2f(dt), dT, rate);
    if (!jok || !(sc.rate_max < 0.0f || rate <= sc.rate_max)) reason = kFbReactive;
    else if (!(dT <= sc.err_tol * T1f * (1.0f - 0.5f * rate + rate * rate * (1.0f / 12.0f)))) reason = kFbError;
  }
  if (!reason) {
#pragma unroll
    for (int k = 0; k < NSP; ++k) Y[k * ld + i] = y1[k];
    T[i] = T1;
    if (status) status[i] = CHEM_CELL_OK;
    if (nsteps) nsteps[i] = 0;
    if (mask) mask[i] = 0;
  } else {
    if (mask) mask[i] = (uint8_t)reason;
    // one atomic per group of rejecting lanes, each lane at its rank after the group's base
    const cooperative_groups::coalesced_group grp = cooperative_groups::coalesced_threads();
    unsigned slot = 0;
    if (grp.thread_rank() == 0) slot = atomicAdd(fb_count, grp.size());
    slot = grp.shfl(slot, 0) + grp.thread_rank();
    fb_idx[slot] = (int32_t)(base + i);
  }
}

// The one-box batch of the fallback integration: all n cells, step dt, one substep.
__global__ void k_one_box(int64_t *box_off, double *box_dt, int32_t *box_nsub, int64_t n, double dt) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    box_off[0] = 0;
    box_off[1] = n;
    box_dt[0] = dt;
    box_nsub[0] = 1;
  }
}

// Surrogate-call totals, launched after the fallback kernel on the same stream: every
// cell counted once (cells = n overrides the fallback kernel's count of its own cells),
// accepted cells as CHEM_CELL_OK (the fallback kernel counted the rejected ones by status).
__global__ void k_surrogate_stats(chem_stats *st, int64_t n, const unsigned int *fb_count) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    st->cells = n;
    st->status_count[CHEM_CELL_OK] += n - (int64_t)*fb_count;
  }
}

// One substep round of chem_surrogate_infer_batched: the `active` cells of the round not
// in the fallback list were accepted (the fallback launch counts its own cells).
__global__ void k_surrogate_stats_add(chem_stats *st, int64_t active, const unsigned int *fb_count) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const int64_t acc = active - (int64_t)*fb_count;
    st->cells += acc;
    st->status_count[CHEM_CELL_OK] += acc;
  }
}

__global__ void k_fill_i32(int32_t *a, int64_t n, int32_t v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = v;
}

static unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

cudaError_t launch_surrogate_stats_add(chem_stats *st, int64_t active, const unsigned int *fb_count,
                                       cudaStream_t s) {
  k_surrogate_stats_add<<<1, 32, 0, s>>>(st, active, fb_count);
  return cudaGetLastError();
}

cudaError_t launch_fill_i32(int32_t *a, int64_t n, int32_t v, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_fill_i32<<<nblk(n, 256), 256, 0, s>>>(a, n, v);
  return cudaGetLastError();
}

cudaError_t launch_surrogate_stats(chem_stats *st, int64_t n, const unsigned int *fb_count,
                                   cudaStream_t s) {
  k_surrogate_stats<<<1, 32, 0, s>>>(st, n, fb_count);
  return cudaGetLastError();
}

cudaError_t launch_features(const MechTables &mt, int64_t n, const double *rho, const double *e,
                            const double *Y0, int64_t ld0, const double *T0, const double *dt_cell,
                            double dt, const double *Y1, int64_t ld1, double lam, double dt_power,
                            float *X, float *Tg, uint8_t *ok, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_features<<<nblk(n, 128), 128, 0, s>>>(mt, n, rho, e, Y0, ld0, T0, dt_cell, dt, Y1, ld1, lam, dt_power, X, Tg,
                                          ok);
  return cudaGetLastError();
}

cudaError_t launch_colstats(int64_t n, int ncol, int ld, const float *A, double *sum, double *sumsq,
                            int *mnkey, int *mxkey, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int64_t want = (n + 7) / 8;
  const unsigned grid = (unsigned)(want < 1024 ? want : 1024);
  k_colstats<<<grid, 256, 0, s>>>(n, ncol, ld, A, sum, sumsq, mnkey, mxkey);
  return cudaGetLastError();
}

cudaError_t launch_normalize(int64_t n, int ncol, int ld, float *A, const float *mean,
                             const float *inv_std, __nv_bfloat16 *Abf, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_normalize<<<nblk(n * ld, 256), 256, 0, s>>>(n, ncol, ld, A, mean, inv_std, Abf);
  return cudaGetLastError();
}

cudaError_t launch_surrogate_finish(int variant, const MechTables &mt, const SurrogateConsts &sc,
                                    int64_t n, double dt, const float *O, const float *Xraw,
                                    const uint8_t *Tok, const double *rho, const double *e, double *Y,
                                    int64_t ld, double *T, int32_t *status, int32_t *nsteps,
                                    uint8_t *mask, int32_t *fb_idx, unsigned int *fb_count,
                                    int64_t base, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (variant == CHEM_VARIANT_MIXED)
    k_surrogate_finish<CHEM_VARIANT_MIXED><<<nblk(n, 128), 128, 0, s>>>(
        mt, sc, n, dt, O, Xraw, Tok, rho, e, Y, ld, T, status, nsteps, mask, fb_idx, fb_count, base);
  else
    k_surrogate_finish<CHEM_VARIANT_FP64><<<nblk(n, 128), 128, 0, s>>>(
        mt, sc, n, dt, O, Xraw, Tok, rho, e, Y, ld, T, status, nsteps, mask, fb_idx, fb_count, base);
  return cudaGetLastError();
}

cudaError_t launch_one_box(int64_t *box_off, double *box_dt, int32_t *box_nsub, int64_t n, double dt,
                           cudaStream_t s) {
  k_one_box<<<1, 32, 0, s>>>(box_off, box_dt, box_nsub, n, dt);
  return cudaGetLastError();
}

cudaError_t launch_project_check(const SurrogateConsts &sc, int64_t n, const double *Y0,
                                 const double *Yp, int64_t ld, double *Yout, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_project_check<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(sc, n, Y0, Yp, ld, Yout);
  return cudaGetLastError();
}

}  // namespace chem
