// mlp.cu -- the elementwise kernels of the learned surrogate's training: GELU backward,
// MSE gradient, split-K and bias-gradient reductions, Adam with FP32 master weights and
// BF16 shadows, row gather, BF16 conversion.  The GEMMs run on the tensor cores
// (mlp_gemm_tc.cu).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.cuh"
#include "mlp.cuh"
#include "mma.cuh"

namespace chem {

// MSE over the first `nout` columns: loss += sum (y - t)^2 / (M nout); dY = 2 (y - t) / (M nout)
// (bf16, padded columns zero).  loss is accumulated with one atomic per block.
__global__ void k_mse(int64_t M, int nout, int ldy, const float *__restrict__ Y,
                      const float *__restrict__ Tg, int ldt, __nv_bfloat16 *__restrict__ dY,
                      int lddy, float *loss) {
  __shared__ float red[256];
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.0f;
  if (idx < M * lddy) {
    const int64_t m = idx / lddy;
    const int n = (int)(idx % lddy);
    float d = 0.0f;
    if (n < nout) {
      d = Y[m * ldy + n] - Tg[m * ldt + n];
      l = d * d;
    }
    dY[m * lddy + n] = __float2bfloat16(2.0f * d / (float)(M * nout));
  }
  red[threadIdx.x] = l;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, red[0] / (float)(M * nout));
}

// db[n] = sum_m dZ[m, n] (one block per 32 columns, fp32 accumulation)
// Partial column sums: CTA (x, y) sums rows y, y + nsplit, ... of columns 32x .. 32x+31
// into part[y * N + n] (8 row groups per CTA, combined in a fixed order).
__global__ void k_bias_grad(int64_t M, int N, const __nv_bfloat16 *__restrict__ dZ, int ld,
                            float *__restrict__ part) {
  __shared__ float red[8][33];
  const int n = blockIdx.x * 32 + (threadIdx.x & 31);
  const int row = threadIdx.x >> 5;  // 8 row groups
  const int64_t stride = 8 * (int64_t)gridDim.y;
  float s = 0.0f;
  if (n < N)
    for (int64_t m = (int64_t)blockIdx.y * 8 + row; m < M; m += stride) s += __bfloat162float(dZ[m * ld + n]);
  red[row][threadIdx.x & 31] = s;
  __syncthreads();
  if (threadIdx.x < 32 && n < N) {
    float t = 0.0f;
#pragma unroll
    for (int r = 0; r < 8; ++r) t += red[r][threadIdx.x];
    part[(int64_t)blockIdx.y * N + n] = t;
  }
}

// out[i] = sum_{s < nsplit} part[s * split_ld + i], in order of s
__global__ void k_reduce_splits(int64_t n, int nsplit, const float *__restrict__ part, int64_t split_ld,
                                float *__restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float t = 0.0f;
  for (int z = 0; z < nsplit; ++z) t += part[z * split_ld + i];
  out[i] = t;
}

// Adam on fp32 master weights; refreshes the bf16 shadows (both orientations for W).
__global__ void k_adam(int64_t n, float *__restrict__ w, const float *__restrict__ g,
                       float *__restrict__ m, float *__restrict__ v, float lr, float b1, float b2,
                       float eps, float bc1, float bc2, __nv_bfloat16 *__restrict__ w_bf,
                       __nv_bfloat16 *__restrict__ wT_bf, int rows, int cols) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float wi = w[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  w[i] = wi;
  if (w_bf) w_bf[i] = __float2bfloat16(wi);
  if (wT_bf) {  // w is [rows x cols] row-major; the transpose is [cols x rows]
    const int64_t r = i / cols, c = i % cols;
    wT_bf[c * rows + r] = __float2bfloat16(wi);
  }
}

// Adam on every parameter (the segments of AdamSegs) with the step's learning rate and
// bias corrections read from a device schedule: sched[3 t .. 3 t + 2] = {lr, 1 - b1^(t+1),
// 1 - b2^(t+1)} at t = *step (a CUDA graph of one training step replays with the counter
// advancing on the device).
__global__ void k_adam_sched_all(int64_t n, float *__restrict__ w, const float *__restrict__ g,
                                 float *__restrict__ m, float *__restrict__ v, const float *__restrict__ sched,
                                 const int64_t *__restrict__ step, float b1, float b2, float eps,
                                 const __grid_constant__ AdamSegs sg) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int j = 0;
  while (j < kAdamSegs - 1 && i >= sg.end[j]) ++j;
  const int64_t li = i - (j ? sg.end[j - 1] : 0);
  const float *sc = sched + 3 * *step;
  const float lr = sc[0], bc1 = sc[1], bc2 = sc[2];
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float wi = w[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  w[i] = wi;
  if (sg.w_bf[j]) sg.w_bf[j][li] = __float2bfloat16(wi);
  if (sg.wT_bf[j]) {
    const int64_t r = li / sg.cols[j], c = li % sg.cols[j];
    sg.wT_bf[j][c * sg.rows[j] + r] = __float2bfloat16(wi);
  }
}

// out[r, :] = in[idx[base + r], :] with base = (*step mod nbatch) * nrows: the batch of
// the current step of an epoch's permutation
__global__ void k_gather_rows_step(int64_t nrows, int ncol, const int32_t *__restrict__ idx,
                                   const int64_t *__restrict__ step, int64_t nbatch, const float *__restrict__ in,
                                   int ldin, float *__restrict__ out, int ldout) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nrows * ncol) return;
  const int64_t r = t / ncol;
  const int c = (int)(t % ncol);
  const int64_t base = (*step % nbatch) * nrows;
  out[r * ldout + c] = in[(int64_t)idx[base + r] * ldin + c];
}

__global__ void k_step_inc(int64_t *step) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *step += 1;
}

// bf16 copy of a float matrix (for the gathered input features)
__global__ void k_to_bf16(int64_t n, const float *__restrict__ in, __nv_bfloat16 *__restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = __float2bfloat16(in[i]);
}

static unsigned blocks(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

cudaError_t launch_mse(int64_t M, int nout, int ldy, const float *Y, const float *Tg, int ldt,
                       __nv_bfloat16 *dY, int lddy, float *loss, cudaStream_t s) {
  k_mse<<<blocks(M * lddy, 256), 256, 0, s>>>(M, nout, ldy, Y, Tg, ldt, dY, lddy, loss);
  return cudaGetLastError();
}
cudaError_t launch_reduce_splits(int64_t n, int nsplit, const float *part, int64_t split_ld, float *out,
                                 cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_reduce_splits<<<blocks(n, 256), 256, 0, s>>>(n, nsplit, part, split_ld, out);
  return cudaGetLastError();
}
cudaError_t launch_bias_grad(int64_t M, int N, const __nv_bfloat16 *dZ, int ld, float *part, int nsplit,
                             float *db, cudaStream_t s) {
  k_bias_grad<<<dim3(blocks(N, 32), (unsigned)nsplit), 256, 0, s>>>(M, N, dZ, ld, part);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? launch_reduce_splits(N, nsplit, part, N, db, s) : e;
}
cudaError_t launch_adam(int64_t n, float *w, const float *g, float *m, float *v, float lr, float b1,
                        float b2, float eps, int step, __nv_bfloat16 *w_bf, __nv_bfloat16 *wT_bf,
                        int rows, int cols, cudaStream_t s) {
  const float bc1 = 1.0f - powf(b1, (float)step), bc2 = 1.0f - powf(b2, (float)step);
  k_adam<<<blocks(n, 256), 256, 0, s>>>(n, w, g, m, v, lr, b1, b2, eps, bc1, bc2, w_bf, wT_bf, rows, cols);
  return cudaGetLastError();
}
cudaError_t launch_adam_sched_all(int64_t n, float *w, const float *g, float *m, float *v, const float *sched,
                                  const int64_t *step, float b1, float b2, float eps, const AdamSegs &segs,
                                  cudaStream_t s) {
  k_adam_sched_all<<<blocks(n, 256), 256, 0, s>>>(n, w, g, m, v, sched, step, b1, b2, eps, segs);
  return cudaGetLastError();
}
cudaError_t launch_gather_rows_step(int64_t nrows, int ncol, const int32_t *idx, const int64_t *step,
                                    int64_t nbatch, const float *in, int ldin, float *out, int ldout,
                                    cudaStream_t s) {
  k_gather_rows_step<<<blocks(nrows * ncol, 256), 256, 0, s>>>(nrows, ncol, idx, step, nbatch, in, ldin, out,
                                                               ldout);
  return cudaGetLastError();
}
cudaError_t launch_step_inc(int64_t *step, cudaStream_t s) {
  k_step_inc<<<1, 32, 0, s>>>(step);
  return cudaGetLastError();
}
cudaError_t launch_to_bf16(int64_t n, const float *in, __nv_bfloat16 *out, cudaStream_t s) {
  k_to_bf16<<<blocks(n, 256), 256, 0, s>>>(n, in, out);
  return cudaGetLastError();
}

}  // namespace chem
