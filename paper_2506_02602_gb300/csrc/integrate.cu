// integrate.cu -- the one-pass integration kernel (one thread per cell, Sec. 4.1.2) and
// the (rho, e) from (T, p, Y) kernel.  The per-cell arithmetic is in cell.cuh.
#include <cuda_runtime.h>

#include "cell.cuh"
#include "internal.cuh"

namespace chem {

template <int V>
__global__ void __launch_bounds__(128) k_lsrk(const __grid_constant__ MechTables mt,
                                              const CellArgs a, const StepParams p) {
  load_math_tables();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = i < a.n;
  CellState c;
  c.nacc = c.nrej = c.nrhs = 0;
  c.status = CHEM_CELL_OK;
  if (live) {
#pragma unroll
    for (int k = 0; k < NSP; ++k) c.X[k] = a.Y[k * a.ld + i];
    c.T = a.T[i];
    c.h = a.h ? a.h[i] : CUDART_NAN;
    cell_begin(c, a.rho[i], a.e[i], p.dt);
    while (!c.done) cell_attempt<V>(mt, c, p);
    cell_finish(mt, c);
#pragma unroll
    for (int k = 0; k < NSP; ++k) a.Y[k * a.ld + i] = c.X[k];
    a.T[i] = c.T;
    if (a.h) a.h[i] = c.h;
    if (a.status) a.status[i] = c.status;
    if (a.nsteps) a.nsteps[i] = c.nacc + c.nrej;
  }
  if (a.stats) {
    int hist[6];
#pragma unroll
    for (int s = 0; s < 6; ++s) hist[s] = live && c.status == s;
    accumulate_stats(a.stats, live ? 1 : 0, c.nacc, c.nrej, c.nrhs, c.nacc + c.nrej, hist);
  }
}

__global__ void k_state_from_TPY(const __grid_constant__ MechTables mt, int64_t n,
                                 const double *__restrict__ T, const double *__restrict__ p,
                                 const double *__restrict__ Y, int64_t ld, double *__restrict__ rho,
                                 double *__restrict__ e) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double Ti = T[i];
  double y[NSP], inv_w = 0.0;
#pragma unroll
  for (int k = 0; k < NSP; ++k) {
    y[k] = Y[k * ld + i];
    inv_w += y[k] * mt.invW[k];
  }
  double m[6];
  mix_ecoef(mt, Ti >= mt.T_mid, y, 0.0, m);
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
