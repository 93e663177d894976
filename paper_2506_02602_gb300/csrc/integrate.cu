// integrate.cu -- the one-pass integration kernel (one thread per cell, Sec. 4.1.2) and
// the (rho, e) from (T, p, Y) kernel.  The per-cell arithmetic is in cell.cuh.
#include <cuda_runtime.h>

#include "cell.cuh"
#include "internal.cuh"

namespace chem {

// BLOCK threads per block, MINB resident blocks per SM.  The register file is split
// between the SM's four sub-partitions, so 12 warps per SM allow 170 registers a thread
// (128 x 3), 16 warps 128 (64 x 8, 32 x 16) and 32 warps 64 (64 x 16, 32 x 32); anything
// between rounds down; 8 warps (256 x 1) leave the 255-register maximum.
// SCH: CHEM_SCHEME_LSRK (the two-register scheme of Eq. 21) or one of the full-storage
// comparators (cell_attempt_full).
template <int V, int BLOCK, int MINB, int SCH = CHEM_SCHEME_LSRK>
__global__ void __launch_bounds__(BLOCK, MINB) k_lsrk(const __grid_constant__ MechTables mt,
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
    if constexpr (SCH == CHEM_SCHEME_LSRK) {
      while (!c.done) cell_attempt<V>(mt, c, p);
    } else {
      while (!c.done) cell_attempt_full<V, SCH>(mt, c, p);
    }
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

// Blocks per SM of the 32- and 64-thread shapes.  The mixed two-register kernel runs them
// at 32 warps per SM (64 registers, spilling to L1 and L2): the FP64 pipe's latency is
// hidden by more warps rather than by registers, and the 1M-cell detonation slice ran
// 3.8 % faster than at 16 warps (128 registers) with the 9-species structure, 4.3 % with
// the 13-species one.  The fp64 variant (fp64 state and rates) and the full-storage
// comparators keep 16 warps: the fp64 kernel measured 7 % slower at 32.
template <int V, int SCH>
constexpr int kDense = (V == CHEM_VARIANT_MIXED && SCH == CHEM_SCHEME_LSRK) ? 2 : 1;

template <int V, int SCH>
static void launch_shape(const MechTables &mt, const CellArgs &a, const StepParams &p, int block,
                         cudaStream_t s) {
  const unsigned grid = (unsigned)((a.n + block - 1) / block);
  if (block == 32) k_lsrk<V, 32, 16 * kDense<V, SCH>, SCH><<<grid, 32, 0, s>>>(mt, a, p);
  else if (block == 64) k_lsrk<V, 64, 8 * kDense<V, SCH>, SCH><<<grid, 64, 0, s>>>(mt, a, p);
  else if (block == 256) k_lsrk<V, 256, 1, SCH><<<grid, 256, 0, s>>>(mt, a, p);
  else k_lsrk<V, 128, 3, SCH><<<grid, 128, 0, s>>>(mt, a, p);
}

template <int SCH>
static void launch_variant(int variant, const MechTables &mt, const CellArgs &a,
                           const StepParams &p, int block, cudaStream_t s) {
  if (variant == CHEM_VARIANT_MIXED) launch_shape<CHEM_VARIANT_MIXED, SCH>(mt, a, p, block, s);
  else launch_shape<CHEM_VARIANT_FP64, SCH>(mt, a, p, block, s);
}

cudaError_t launch_lsrk(int variant, int scheme, const MechTables &mt, const CellArgs &a,
                        const StepParams &p, int block, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  if (block != 32 && block != 64 && block != 256) block = 128;  // the compiled shapes
  if (scheme == CHEM_SCHEME_FULL_STORAGE)
    launch_variant<CHEM_SCHEME_FULL_STORAGE>(variant, mt, a, p, block, s);
  else if (scheme == CHEM_SCHEME_RKF45)
    launch_variant<CHEM_SCHEME_RKF45>(variant, mt, a, p, block, s);
  else
    launch_variant<CHEM_SCHEME_LSRK>(variant, mt, a, p, block, s);
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
