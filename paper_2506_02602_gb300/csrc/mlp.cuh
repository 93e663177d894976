// mlp.cuh -- declarations of the surrogate's GEMM and elementwise kernels (mlp.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace chem {

// C[m, n] = alpha * sum_k A(m, k) B(n, k) (+ bias[n]) (+ Cf[m, n] if accumulate), on the
// 5th-generation tensor cores (mlp_gemm_tc.cu);
// A(m, k) = A[m*sam + k*sak], B(n, k) = B[n*sbn + k*sbk].  Outputs: Cf (fp32, ldc) and/or
// Cb (bf16, ldcb) holding the value, or GELU(value) when gelu is set.
// Split-K (split > 1): the K range is cut into `split` slices of whole 32-wide steps and
// slice z writes its partial sum (alpha applied, no bias, no bf16 output) to
// Cf + z * split_ld; launch_reduce_splits adds the slices in a fixed order.
struct GemmArgs {
  int64_t M, N, K;
  const __nv_bfloat16 *A;
  int64_t sam, sak;
  const __nv_bfloat16 *B;
  int64_t sbn, sbk;
  float alpha;
  const float *bias;
  float *Cf;
  int64_t ldc;
  __nv_bfloat16 *Cb;
  int64_t ldcb;
  int gelu;
  int accumulate;
  int split;
  int64_t split_ld;
  int *err;  // nullable device word: set to 1 if a bounded wait of the kernel ran out
  // nullable: Cb receives bf16(x * GELU'(dgelu_z[m * ldz + n])) instead of bf16(x) or
  // bf16(GELU(x)) (the backward pass's dZ = dH * GELU'(Z), fused into the dH GEMM)
  const float *dgelu_z;
  int64_t ldz;
};

cudaError_t launch_gemm(const GemmArgs &g, cudaStream_t s);
cudaError_t launch_mse(int64_t M, int nout, int ldy, const float *Y, const float *Tg, int ldt,
                       __nv_bfloat16 *dY, int lddy, float *loss, cudaStream_t s);
cudaError_t launch_reduce_splits(int64_t n, int nsplit, const float *part, int64_t split_ld,
                                 float *out, cudaStream_t s);
// db[n] = sum_m dZ[m, n], through nsplit row slices written to part [nsplit x N], then
// reduced in a fixed order (deterministic).
cudaError_t launch_bias_grad(int64_t M, int N, const __nv_bfloat16 *dZ, int ld, float *part,
                             int nsplit, float *db, cudaStream_t s);
cudaError_t launch_adam(int64_t n, float *w, const float *g, float *m, float *v, float lr, float b1,
                        float b2, float eps, int step, __nv_bfloat16 *w_bf, __nv_bfloat16 *wT_bf,
                        int rows, int cols, cudaStream_t s);
cudaError_t launch_to_bf16(int64_t n, const float *in, __nv_bfloat16 *out, cudaStream_t s);
// The device-scheduled pieces of a graph-captured training step: Adam with {lr, 1 - b1^t,
// 1 - b2^t} read from sched[3 * (*step)], the batch gather of step *step, the counter.
// One Adam launch over every parameter of the network: segment j covers
// [end[j - 1], end[j]) of w, g, m, v (end[-1] = 0); a weight segment also writes its bf16
// copy w_bf (rows x cols, k contiguous) and transpose wT_bf (null for the biases).
constexpr int kAdamSegs = 8;  // a weight and a bias segment per layer
struct AdamSegs {
  int64_t end[kAdamSegs];
  __nv_bfloat16 *w_bf[kAdamSegs];
  __nv_bfloat16 *wT_bf[kAdamSegs];
  int rows[kAdamSegs], cols[kAdamSegs];
};
cudaError_t launch_adam_sched_all(int64_t n, float *w, const float *g, float *m, float *v, const float *sched,
                                  const int64_t *step, float b1, float b2, float eps, const AdamSegs &segs,
                                  cudaStream_t s);
cudaError_t launch_gather_rows_step(int64_t nrows, int ncol, const int32_t *idx, const int64_t *step,
                                    int64_t nbatch, const float *in, int ldin, float *out, int ldout,
                                    cudaStream_t s);
cudaError_t launch_step_inc(int64_t *step, cudaStream_t s);
// Sets the tensor-core GEMM's shared-memory attribute on the current device (once), so
// that GEMM launches can be captured in a CUDA graph.
cudaError_t gemm_prepare();

}  // namespace chem
