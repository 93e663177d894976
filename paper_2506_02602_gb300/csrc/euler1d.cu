// euler1d.cu -- the operator either side of the chemistry: a minimal 1D reactive Euler
// step and the Strang-split step that couples it to the integrator (Sec. 2.2.1: Strang
// splitting of the reactive Euler equations, Eq. 14 without transport).
//
// State: the conserved planes rho, rho u, rho E, rho Y_k of n cells of width dx (SoA fp64,
// plane k of rho Y at rhoY + k ldY) and the temperature (Newton start in, temperature of
// the new state out).  The step: primitive variables (rho, u, p, Y_k) per cell (T from
// e = E - u^2/2 by the integrator's Newton solve, p = rho R_u T sum_k Y_k / W_k);
// minmod-limited MUSCL slopes and face states (T from p, rho, Y), the cell averages where
// a face state's density or pressure is not positive; the HLL flux with Davis wave speeds
// (sound speed from gamma = c_p / c_v of the mixture at T); the two-stage SSP Runge-Kutta
// (Heun) update.  Boundaries: transmissive (zero gradient) or reflecting walls.
//
// One thread per cell (primitives, update) or per face (fluxes); every access is a
// coalesced plane read.  The work per cell is a few hundred fp64 operations against the
// chemistry's thousands per step, so these kernels are not the hot path; they exist to
// run the split scheme end to end on the GPU.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>

#include "internal.cuh"
#include "rhs.cuh"

namespace chem {

namespace {

constexpr int NV = 3 + NSP;  // conserved components

struct Flow {
  const double *U;  // NV planes of n (the state the primitives are taken from)
  int64_t ldU;
  double *W;        // primitive planes: rho, u, p, Y_k (3 + NSP planes of n)
  double *Tw;       // working temperature (n)
  int32_t *status;  // nullable: 3 where no temperature root exists
  int64_t n;
};

// e / R_u and c_v / R_u of a mixture (per unit mass) at T.
__device__ __forceinline__ void mix_e_cv(const MechTables &mt, const double (&Y)[NSP], double T,
                                         double &eR, double &cvR) {
  double m[6], d[5];
  mix_ecoef(mt, ge_nonneg(T, mt.T_mid), Y, 0.0, m);
  cv_coef(m, d);
  eR = e_over_R(m, T);
  cvR = cv_over_R(d, T);
}

__device__ __forceinline__ double inv_w(const MechTables &mt, const double (&Y)[NSP]) {
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < NSP; ++k) s = fma(Y[k], mt.invW[k], s);
  return s;
}

__global__ void k_prim(const __grid_constant__ MechTables mt, const Flow f) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= f.n) return;
  const double rho = f.U[i], u = f.U[f.ldU + i] / rho;
  double Y[NSP];
#pragma unroll
  for (int k = 0; k < NSP; ++k) Y[k] = f.U[(3 + k) * f.ldU + i] / rho;
  const double e = f.U[2 * f.ldU + i] / rho - 0.5 * u * u;
  double T = f.Tw[i];
  if (!solve_T(mt, Y, e * (1.0 / R_U), T)) {
    if (f.status) f.status[i] = CHEM_CELL_NEWTON_FAIL;
    T = f.Tw[i];
  }
  f.Tw[i] = T;
  f.W[i] = rho;
  f.W[f.n + i] = u;
  f.W[2 * f.n + i] = rho * R_U * T * inv_w(mt, Y);
#pragma unroll
  for (int k = 0; k < NSP; ++k) f.W[(3 + k) * f.n + i] = Y[k];
}

struct Prim {
  double rho, u, p, T;
  double Y[NSP];
};

// Cell j in [-2, n+1] of the primitive planes, with the boundary ghosts.
__device__ __forceinline__ void load_cell(const Flow &f, int64_t j, int bcl, int bcr, Prim &w) {
  const int64_t n = f.n;
  int64_t src = j;
  bool flip = false;
  if (j < 0) {
    src = bcl == 0 ? 0 : -j - 1;
    flip = bcl != 0;
  } else if (j >= n) {
    src = bcr == 0 ? n - 1 : 2 * n - 1 - j;
    flip = bcr != 0;
  }
  w.rho = f.W[src];
  w.u = flip ? -f.W[n + src] : f.W[n + src];
  w.p = f.W[2 * n + src];
  w.T = f.Tw[src];
#pragma unroll
  for (int k = 0; k < NSP; ++k) w.Y[k] = f.W[(3 + k) * n + src];
}

__device__ __forceinline__ double minmod(double a, double b) {
  if (a * b <= 0.0) return 0.0;
  return fabs(a) < fabs(b) ? a : b;
}

// Face state from cell b with the slope of (a, b, c), offset `half` (+1/2 or -1/2).
__device__ __forceinline__ void face(const MechTables &mt, const Prim &a, const Prim &b, const Prim &c,
                                     double half, Prim &out) {
  out.rho = b.rho + half * minmod(b.rho - a.rho, c.rho - b.rho);
  out.u = b.u + half * minmod(b.u - a.u, c.u - b.u);
  out.p = b.p + half * minmod(b.p - a.p, c.p - b.p);
#pragma unroll
  for (int k = 0; k < NSP; ++k) out.Y[k] = b.Y[k] + half * minmod(b.Y[k] - a.Y[k], c.Y[k] - b.Y[k]);
  out.T = out.p / (out.rho * R_U * inv_w(mt, out.Y));
}

// Physical flux and conserved vector of a primitive state, and its sound speed.
__device__ __forceinline__ void flux_state(const MechTables &mt, const Prim &w, double (&F)[NV],
                                           double (&U)[NV], double &c) {
  double eR, cvR;
  mix_e_cv(mt, w.Y, w.T, eR, cvR);
  const double E = R_U * eR + 0.5 * w.u * w.u;
  const double cpR = cvR + inv_w(mt, w.Y);
  c = sqrt(cpR / cvR * w.p / w.rho);
  U[0] = w.rho;
  U[1] = w.rho * w.u;
  U[2] = w.rho * E;
  F[0] = w.rho * w.u;
  F[1] = w.rho * w.u * w.u + w.p;
  F[2] = (w.rho * E + w.p) * w.u;
#pragma unroll
  for (int k = 0; k < NSP; ++k) {
    U[3 + k] = w.rho * w.Y[k];
    F[3 + k] = w.rho * w.Y[k] * w.u;
  }
}

// HLL flux at every face f in [0, n] (between cells f-1 and f): Fl planes NV x (n + 1).
__global__ void k_flux(const __grid_constant__ MechTables mt, const Flow f, int bcl, int bcr, double *Fl) {
  const int64_t fc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (fc > f.n) return;
  Prim a, b, c, d, L, R;
  load_cell(f, fc - 2, bcl, bcr, a);
  load_cell(f, fc - 1, bcl, bcr, b);
  load_cell(f, fc, bcl, bcr, c);
  load_cell(f, fc + 1, bcl, bcr, d);
  face(mt, a, b, c, 0.5, L);
  face(mt, b, c, d, -0.5, R);
  if (!(L.rho > 0.0 && L.p > 0.0 && R.rho > 0.0 && R.p > 0.0)) {
    L = b;
    R = c;
  }
  double FL[NV], FR[NV], UL[NV], UR[NV], cL, cR;
  flux_state(mt, L, FL, UL, cL);
  flux_state(mt, R, FR, UR, cR);
  const double SL = fmin(L.u - cL, R.u - cR), SR = fmax(L.u + cL, R.u + cR);
  const int64_t ld = f.n + 1;
  if (SL >= 0.0) {
#pragma unroll
    for (int v = 0; v < NV; ++v) Fl[v * ld + fc] = FL[v];
  } else if (SR <= 0.0) {
#pragma unroll
    for (int v = 0; v < NV; ++v) Fl[v * ld + fc] = FR[v];
  } else {
    const double inv = 1.0 / (SR - SL);
#pragma unroll
    for (int v = 0; v < NV; ++v) Fl[v * ld + fc] = (SR * FL[v] - SL * FR[v] + SL * SR * (UR[v] - UL[v])) * inv;
  }
}

// Stage update: stage 0, U1 = U0 + dt dU(U0); stage 1, out = (U0 + U1 + dt dU(U1)) / 2.
// dU_i = (F_i - F_(i+1)) / dx.  The result goes to the planes rho, rhou, rhoE and the
// species planes rhoY + k ldY (stage 0: the U1 planes themselves, so Uc may alias them).
__global__ void k_update(int64_t n, const double *__restrict__ U0, const double *Uc,
                         const double *__restrict__ Fl, double dtdx, int stage, double *rho, double *rhou,
                         double *rhoE, double *rhoY, int64_t ldY) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t ld = n + 1;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const double du = dtdx * (Fl[v * ld + i] - Fl[v * ld + i + 1]);
    const double u0 = U0[v * n + i];
    const double r = stage == 0 ? u0 + du : 0.5 * (u0 + (Uc[v * n + i] + du));
    double *dst = v == 0 ? rho + i : v == 1 ? rhou + i : v == 2 ? rhoE + i : rhoY + (v - 3) * ldY + i;
    *dst = r;
  }
}

// U0 <- the state planes; Tw <- T.
__global__ void k_load(int64_t n, const double *rho, const double *rhou, const double *rhoE,
                       const double *rhoY, int64_t ldY, const double *T, double *U0, double *Tw) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  U0[i] = rho[i];
  U0[n + i] = rhou[i];
  U0[2 * n + i] = rhoE[i];
#pragma unroll
  for (int k = 0; k < NSP; ++k) U0[(3 + k) * n + i] = rhoY[k * ldY + i];
  Tw[i] = T[i];
}

__global__ void k_copy(int64_t n, const double *src, double *dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[i];
}

// Largest |u| + c over the cells, as the bit pattern of a non-negative double (which
// orders like the value) in *smax.
__global__ void k_speed(const __grid_constant__ MechTables mt, const Flow f, unsigned long long *smax) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double s = 0.0;
  if (i < f.n) {
    Prim w;
    load_cell(f, i, 0, 0, w);
    double eR, cvR;
    mix_e_cv(mt, w.Y, w.T, eR, cvR);
    s = fabs(w.u) + sqrt((cvR + inv_w(mt, w.Y)) / cvR * w.p / w.rho);
    if (!(s >= 0.0)) s = INFINITY;  // a NaN state stops the caller's time step choice
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
  if ((threadIdx.x & 31) == 0) atomicMax(smax, (unsigned long long)__double_as_longlong(s));
}

// Chemistry half-step staging: e = E - u^2/2 and Y = rho Y / rho (planes of n), and back.
__global__ void k_to_chem(int64_t n, const double *rho, const double *rhou, const double *rhoE,
                          const double *rhoY, int64_t ldY, double *e, double *Y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double r = rho[i], u = rhou[i] / r;
  e[i] = rhoE[i] / r - 0.5 * u * u;
#pragma unroll
  for (int k = 0; k < NSP; ++k) Y[k * n + i] = rhoY[k * ldY + i] / r;
}

__global__ void k_from_chem(int64_t n, const double *rho, const double *Y, double *rhoY, int64_t ldY) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
#pragma unroll
  for (int k = 0; k < NSP; ++k) rhoY[k * ldY + i] = rho[i] * Y[k * n + i];
}

inline unsigned blocks(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// Scratch: U0, U1 (NV x n each), W (NV x n), Tw (n), F (NV x (n + 1)), e and Y of the
// chemistry staging ((1 + NSP) x n), the speed word.
struct Scratch {
  double *U0, *U1, *W, *Tw, *F, *ce, *cY;
  unsigned long long *smax;
};

size_t scratch_bytes(int64_t n) {
  return sizeof(double) * ((size_t)NV * n * 3 + (size_t)n + (size_t)NV * (n + 1) + (size_t)(1 + NSP) * n) + 64;
}

Scratch carve(void *base, int64_t n) {
  double *p = static_cast<double *>(base);
  Scratch s;
  s.U0 = p; p += NV * n;
  s.U1 = p; p += NV * n;
  s.W = p; p += NV * n;
  s.Tw = p; p += n;
  s.F = p; p += NV * (n + 1);
  s.ce = p; p += n;
  s.cY = p; p += NSP * n;
  s.smax = reinterpret_cast<unsigned long long *>(p);
  return s;
}

cudaError_t euler_step(const MechTables &mt, const chem_flow1d &st, int64_t n, double dx, double dt, int bcl,
                       int bcr, const Scratch &sc, cudaStream_t s) {
  const int B = 128;
  k_load<<<blocks(n, B), B, 0, s>>>(n, st.d_rho, st.d_rhou, st.d_rhoE, st.d_rhoY, st.ldY, st.d_T, sc.U0, sc.Tw);
  for (int stage = 0; stage < 2; ++stage) {
    const Flow f{stage == 0 ? sc.U0 : sc.U1, n, sc.W, sc.Tw, st.d_status, n};
    k_prim<<<blocks(n, B), B, 0, s>>>(mt, f);
    k_flux<<<blocks(n + 1, B), B, 0, s>>>(mt, f, bcl, bcr, sc.F);
    if (stage == 0)
      k_update<<<blocks(n, B), B, 0, s>>>(n, sc.U0, sc.U1, sc.F, dt / dx, 0, sc.U1, sc.U1 + n, sc.U1 + 2 * n,
                                          sc.U1 + 3 * n, n);
    else
      k_update<<<blocks(n, B), B, 0, s>>>(n, sc.U0, sc.U1, sc.F, dt / dx, 1, st.d_rho, st.d_rhou, st.d_rhoE,
                                          st.d_rhoY, st.ldY);
  }
  // temperature of the new state (the Newton start is the last stage's)
  k_load<<<blocks(n, B), B, 0, s>>>(n, st.d_rho, st.d_rhou, st.d_rhoE, st.d_rhoY, st.ldY, sc.Tw, sc.U1, sc.ce);
  const Flow f{sc.U1, n, sc.W, sc.ce, st.d_status, n};
  k_prim<<<blocks(n, B), B, 0, s>>>(mt, f);
  k_copy<<<blocks(n, B), B, 0, s>>>(n, sc.ce, st.d_T);
  return cudaGetLastError();
}

}  // namespace

}  // namespace chem

using namespace chem;

static int flow_checks(chem_ctx *ctx, const chem_flow1d *st, int64_t n, double dx) {
  if (!ctx) return CHEM_ERR_INVALID;
  std::string &err = chem_ctx_error(ctx);
  if (!st || !st->d_rho || !st->d_rhou || !st->d_rhoE || !st->d_rhoY || !st->d_T) {
    err = "the flow state needs rho, rho u, rho E, rho Y and T";
    return CHEM_ERR_INVALID;
  }
  if (n < 2 || st->ldY < n) {
    err = "the flow needs n >= 2 cells and ldY >= n";
    return CHEM_ERR_INVALID;
  }
  if (!(dx > 0.0) || !std::isfinite(dx)) {
    err = "dx must be > 0";
    return CHEM_ERR_INVALID;
  }
  return CHEM_OK;
}

extern "C" int chem_euler1d_step(chem_ctx *ctx, const chem_flow1d *st, int64_t n, double dx, double dt,
                                 int32_t bc_left, int32_t bc_right, void *stream) {
  int rc = flow_checks(ctx, st, n, dx);
  if (rc) return rc;
  std::string &err = chem_ctx_error(ctx);
  if (!(dt > 0.0) || !std::isfinite(dt) || (bc_left != 0 && bc_left != 1) || (bc_right != 0 && bc_right != 1)) {
    err = "dt must be > 0 and boundaries 0 (transmissive) or 1 (wall)";
    return CHEM_ERR_INVALID;
  }
  void *base = nullptr;
  cudaError_t e = chem_ctx_flow_scratch(ctx, scratch_bytes(n), &base);
  if (e != cudaSuccess) {
    err = std::string("flow scratch: ") + cudaGetErrorString(e);
    return CHEM_ERR_NOMEM;
  }
  e = euler_step(chem_ctx_tables(ctx), *st, n, dx, dt, bc_left, bc_right, carve(base, n), (cudaStream_t)stream);
  if (e != cudaSuccess) {
    err = std::string("Euler step: ") + cudaGetErrorString(e);
    return CHEM_ERR_CUDA;
  }
  return CHEM_OK;
}

extern "C" int chem_euler1d_max_speed(chem_ctx *ctx, const chem_flow1d *st, int64_t n, double *h_smax,
                                      void *stream) {
  int rc = flow_checks(ctx, st, n, 1.0);
  if (rc) return rc;
  if (!h_smax) return CHEM_ERR_INVALID;
  std::string &err = chem_ctx_error(ctx);
  void *base = nullptr;
  cudaError_t e = chem_ctx_flow_scratch(ctx, scratch_bytes(n), &base);
  if (e != cudaSuccess) {
    err = std::string("flow scratch: ") + cudaGetErrorString(e);
    return CHEM_ERR_NOMEM;
  }
  const Scratch sc = carve(base, n);
  cudaStream_t s = (cudaStream_t)stream;
  const int B = 128;
  const MechTables &mt = chem_ctx_tables(ctx);
  k_load<<<blocks(n, B), B, 0, s>>>(n, st->d_rho, st->d_rhou, st->d_rhoE, st->d_rhoY, st->ldY, st->d_T, sc.U0,
                                    sc.Tw);
  const Flow f{sc.U0, n, sc.W, sc.Tw, nullptr, n};
  k_prim<<<blocks(n, B), B, 0, s>>>(mt, f);
  e = cudaMemsetAsync(sc.smax, 0, sizeof(unsigned long long), s);
  if (e == cudaSuccess) {
    k_speed<<<blocks(n, B), B, 0, s>>>(mt, f, sc.smax);
    e = cudaGetLastError();
  }
  unsigned long long bits = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, sc.smax, sizeof bits, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    err = std::string("max speed: ") + cudaGetErrorString(e);
    return CHEM_ERR_CUDA;
  }
  double v = 0.0;
  std::memcpy(&v, &bits, sizeof v);  // the bit pattern the device's atomicMax kept
  *h_smax = v;
  return CHEM_OK;
}

extern "C" int chem_strang_step(chem_ctx *ctx, const chem_flow1d *st, int64_t n, double dx, double dt,
                                int32_t bc_left, int32_t bc_right, double rtol, double atol, void *stream,
                                chem_stats *d_stats) {
  int rc = flow_checks(ctx, st, n, dx);
  if (rc) return rc;
  std::string &err = chem_ctx_error(ctx);
  if (!(dt > 0.0) || !std::isfinite(dt) || (bc_left != 0 && bc_left != 1) || (bc_right != 0 && bc_right != 1) ||
      !(rtol > 0.0) || !(atol >= 0.0)) {
    err = "dt, rtol must be > 0, atol >= 0 and boundaries 0 (transmissive) or 1 (wall)";
    return CHEM_ERR_INVALID;
  }
  void *base = nullptr;
  cudaError_t e = chem_ctx_flow_scratch(ctx, scratch_bytes(n), &base);
  if (e != cudaSuccess) {
    err = std::string("flow scratch: ") + cudaGetErrorString(e);
    return CHEM_ERR_NOMEM;
  }
  const Scratch sc = carve(base, n);
  cudaStream_t s = (cudaStream_t)stream;
  const MechTables &mt = chem_ctx_tables(ctx);
  const int B = 128;
  if (d_stats) e = cudaMemsetAsync(d_stats, 0, sizeof(chem_stats), s);
  const StepParams p{0.5 * dt, rtol, atol, chem_ctx_max_steps(ctx)};
  for (int half = 0; half < 2 && e == cudaSuccess; ++half) {
    if (half == 1) e = euler_step(mt, *st, n, dx, dt, bc_left, bc_right, sc, s);
    if (e != cudaSuccess) break;
    k_to_chem<<<blocks(n, B), B, 0, s>>>(n, st->d_rho, st->d_rhou, st->d_rhoE, st->d_rhoY, st->ldY, sc.ce, sc.cY);
    const CellArgs a{st->d_rho, sc.ce, sc.cY, n, st->d_T, nullptr, st->d_status, nullptr, n, d_stats};
    e = launch_lsrk(chem_ctx_variant(ctx), chem_ctx_scheme(ctx), mt, a, p, chem_ctx_block(ctx), s);
    if (e == cudaSuccess) {
      k_from_chem<<<blocks(n, B), B, 0, s>>>(n, st->d_rho, sc.cY, st->d_rhoY, st->ldY);
      e = cudaGetLastError();
    }
  }
  if (e != cudaSuccess) {
    err = std::string("Strang step: ") + cudaGetErrorString(e);
    return CHEM_ERR_CUDA;
  }
  return CHEM_OK;
}
