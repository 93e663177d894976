// surrogate.cuh -- shapes and constants of the learned surrogate.
//
// Network: 12 -> 256 -> 256 -> 256 -> 9, GELU between layers, BF16 weights and
// activations with FP32 accumulation and FP32 master weights.  Input width is padded to
// 16 and output width to 16 (zero columns) so every GEMM tile is a whole number of
// 16-wide MMA fragments.  Parameters are stored per layer as W [N x K] (row-major,
// output unit n, input k contiguous) and b [N]; the flat layout concatenates
// W0, b0, W1, b1, W2, b2, W3, b3.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.cuh"

namespace chem {

constexpr int kSurIn = 16;       // 12 features, padded
constexpr int kSurFeat = 12;
constexpr int kSurOut = 16;      // 9 outputs, padded
constexpr int kSurHidden = 256;
constexpr int kSurLayers = 4;
constexpr double kSurDtRef = 1e-8;  // s, reference step of the target scaling
constexpr int kSurN[kSurLayers] = {kSurHidden, kSurHidden, kSurHidden, kSurOut};
constexpr int kSurK[kSurLayers] = {kSurIn, kSurHidden, kSurHidden, kSurHidden};
constexpr int64_t kSurParams = (int64_t)kSurHidden * kSurIn + kSurHidden +
                               2 * ((int64_t)kSurHidden * kSurHidden + kSurHidden) +
                               (int64_t)kSurOut * kSurHidden + kSurOut;

// Why a cell was sent to the integrator (the fallback mask's values; 0 = accepted).
enum {
  kFbRange = 1,        // a feature outside the training box (with the margin)
  kFbResidual = 2,     // element residual of the raw prediction too large
  kFbNegative = 3,     // a mass fraction below -neg_tol after the projection
  kFbTemperature = 4,  // no temperature root, or |T' - T0| > max_dT
  kFbReactive = 5,     // error test: the step is not slow for the cell (rate_max)
  kFbError = 6,        // error test: error estimate above err_tol
};

// Everything the inference epilogue needs besides the mechanism (passed by value).
struct SurrogateConsts {
  float tmean[NSP], tstd[NSP];          // target normalisation
  float fmin[kSurFeat], fmax[kSurFeat]; // training range of the raw features
  float margin;                         // OOD margin, fraction of the range
  float resid_max;                      // max relative element residual before projection
  float neg_tol;                        // most negative mass fraction allowed after projection
  float max_dT;                         // largest accepted |T' - T0| (K)
  float err_tol;                      // largest estimated relative T error (<= 0: no test)
  float rate_max;                     // largest dt * relative rate of change (< 0: no bound)
  double lam;                           // Box-Cox lambda
  double dt_power;                      // targets scaled by (kSurDtRef / dt)^dt_power
  double E[3][NSP];                     // element mass fraction per unit species mass fraction
  int32_t emask[3];                     // bit k set where E[el][k] != 0 (the sums skip the rest)
};

cudaError_t launch_features(const MechTables &mt, int64_t n, const double *rho, const double *e,
                            const double *Y0, int64_t ld0, const double *T0, const double *dt_cell,
                            double dt, const double *Y1, int64_t ld1, double lam, double dt_power,
                            float *X, float *Tg, uint8_t *ok, cudaStream_t s);
cudaError_t launch_colstats(int64_t n, int ncol, int ld, const float *A, double *sum, double *sumsq,
                            int *mnkey, int *mxkey, cudaStream_t s);
cudaError_t launch_normalize(int64_t n, int ncol, int ld, float *A, const float *mean,
                             const float *inv_std, __nv_bfloat16 *Abf, cudaStream_t s);
cudaError_t launch_surrogate_finish(int variant, const MechTables &mt, const SurrogateConsts &sc,
                                    int64_t n, double dt, const float *O, const float *Xraw,
                                    const uint8_t *Tok, const double *rho, const double *e, double *Y,
                                    int64_t ld, double *T, int32_t *status, int32_t *nsteps,
                                    uint8_t *mask, int32_t *fb_idx, unsigned int *fb_count,
                                    int64_t base, cudaStream_t s);
cudaError_t launch_surrogate_stats(chem_stats *st, int64_t n, const unsigned int *fb_count,
                                   cudaStream_t s);
// The whole network on n rows in one kernel (mlp_fused.cu): X [n x 16] raw features
// normalised with norm = {fmean[16], fistd[16]} (or already normalised when norm is
// NULL), W / b the BF16 weights and FP32 biases per layer, O [n x 16] the outputs.
cudaError_t launch_mlp_fused(int64_t n, const float *X, const float *norm,
                             const __nv_bfloat16 *const (&W)[kSurLayers],
                             const float *const (&b)[kSurLayers], float *O, cudaStream_t s);
// The network on the 5th-generation tensor cores (mlp_tc.cu): weights repacked into the
// kernel's operand layout by launch_pack_weights (packed_weight_bytes() bytes); err is
// a device word set to 1 if one of the kernel's bounded waits ran out.
cudaError_t launch_pack_weights(const __nv_bfloat16 *const (&W)[kSurLayers], unsigned char *Wpk, cudaStream_t s);
size_t packed_weight_bytes();
cudaError_t launch_mlp_tc(int64_t n, const float *X, const float *norm, const unsigned char *Wpk,
                          const float *const (&b)[kSurLayers], float *O, int *err, cudaStream_t s);
// The fp64 element projection of the inference epilogue alone (only sc.E and sc.emask are
// read): Yout = projection of Yp onto the element mass fractions of Y0 (planes, stride ld).
cudaError_t launch_project_check(const SurrogateConsts &sc, int64_t n, const double *Y0,
                                 const double *Yp, int64_t ld, double *Yout, cudaStream_t s);
// Statistics of one substep round of the batched inference (cells and accepted counts).
cudaError_t launch_surrogate_stats_add(chem_stats *st, int64_t active, const unsigned int *fb_count,
                                       cudaStream_t s);
cudaError_t launch_fill_i32(int32_t *a, int64_t n, int32_t v, cudaStream_t s);
// box_off = {0, n}, box_dt = {dt}, box_nsub = {1}: the fallback's one-box batch.
cudaError_t launch_one_box(int64_t *box_off, double *box_dt, int32_t *box_nsub, int64_t n, double dt,
                           cudaStream_t s);

}  // namespace chem
