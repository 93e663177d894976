// diag.cu -- diagnostics: chem_diag_math (the kernels' device math routines on caller
// arrays, for accuracy tests against the CUDA library and the IEEE-754 definitions),
// chem_diag_fma_peak (an FMA-throughput probe of the fp64 and fp32 pipes, the
// denominators of the integrators' compute roofline) and chem_diag_ln_inv_kc (the
// equilibrium exponents as the mixed-precision right-hand sides form them).
#include <cuda_runtime.h>

#include <string>
#include <utility>

#include "fastmath.cuh"
#include "internal.cuh"
#include "mma.cuh"
#include "rhs_mixed.cuh"

namespace chem {

__global__ void k_diag_math(int op, int64_t n, const double *__restrict__ x, double *__restrict__ y) {
  load_math_tables();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = x[i];
  double r;
  float h, l;
  switch (op) {
    case 0: r = exp_t(v); break;
    case 1: r = log_t(v); break;
    case 2: r = exp(v); break;
    case 3: r = log(v); break;
    case 4: r = rcp1(v); break;
    case 5: r = rcp2(v); break;
    case 6: r = rcp_approx(v); break;
    case 7: r = (double)d2f(v); break;          // widened exactly by the hardware
    case 8: r = f2d(__double2float_rn(v)); break;
    case 9: split_hilo(v, h, l); r = (double)h; break;
    case 10: split_hilo(v, h, l); r = (double)l; break;
    case 11: r = (double)gelu_f((float)v); break;
    case 12: r = (double)gelu_grad_f((float)v); break;
    case 13: {  // the same with the CUDA library's erff and expf
      const float x = (float)v;
      r = (double)(0.5f * x * (1.0f + erff(x * 0.70710678118654752f)));
      break;
    }
    default: {
      const float x = (float)v;
      r = (double)(0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x));
      break;
    }
  }
  y[i] = r;
}

// FMA-pipe throughput probe: 8 independent dependent chains per thread, x <- x a + b,
// iters rounds; one store per thread keeps the chains live.  2 flops per FMA.  a and b
// are read from device memory into registers: measured on GB300, an FMA whose operand
// comes straight from the constant bank (a kernel parameter) issues at ~0.84 of the rate
// of the all-register form, which reaches 2 fp64 FMAs per clock per SM.
template <typename R>
__global__ void k_fma_peak(int64_t iters, const R *__restrict__ ab, R *__restrict__ sink) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const R a = ab[0], b = ab[1];
  R x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = (R)(threadIdx.x & 15) + (R)j;
#pragma unroll 1
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int j = 0; j < 8; ++j) x[j] = fma(x[j], a, b);
  }
  R s = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += x[j];
  sink[t] = s;
}

template <typename R>
__global__ void k_fma_coefs(R *ab, R a, R b) {
  ab[0] = a;
  ab[1] = b;
}

template <typename Gibbs, int... J>
__device__ __forceinline__ void store_ln_inv_kc(const Gibbs &g, double *o, std::integer_sequence<int, J...>) {
  ((o[J] = (double)ln_inv_kc<J>(g)), ...);
}

// ln(1 / K_c,j) of every reaction at T[i] into out[i * NRX + j], through the same
// helpers the right-hand sides call: form 0 the mixed variant's (fp64 Gibbs functions
// summed as fp32 hi/lo pairs, after the fp64 ln T and 1 / T it takes from the
// temperature solve), form 1 the error test's all-fp32 one.
__global__ void k_ln_inv_kc(const __grid_constant__ MechTables mt, int form, int64_t n,
                            const double *__restrict__ T, double *__restrict__ out) {
  load_math_tables();  // log_t reads the per-block tables
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double t = T[i];
  double *o = out + i * NRX;
  if (form == 0) {
    GibbsHL g;
    gibbs_hl(mt, t, log_t(t), rcp1(t), g);
    store_ln_inv_kc(g, o, std::make_integer_sequence<int, NRX>{});
  } else {
    const float tf = (float)t;
    GibbsF g;
    gibbs_f(mt, tf, logf(tf), 1.0f / tf, g);
    store_ln_inv_kc(g, o, std::make_integer_sequence<int, NRX>{});
  }
}

}  // namespace chem

extern "C" int chem_diag_fma_peak(int op, int32_t blocks, int32_t threads, int64_t iters,
                                  void *d_sink, void *stream) {
  if ((op != 0 && op != 1) || blocks < 1 || threads < 32 || threads > 1024 || (threads & 31) ||
      iters < 1 || !d_sink)
    return CHEM_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  // the chains' two coefficients are written to the two elements past the threads'
  // outputs by a one-thread launch before the probe
  const int64_t nt = (int64_t)blocks * threads;
  if (op == 0) {
    double *sink = static_cast<double *>(d_sink);
    chem::k_fma_coefs<double><<<1, 1, 0, s>>>(sink + nt, 0.9999999, 1e-7);
    chem::k_fma_peak<double><<<(unsigned)blocks, threads, 0, s>>>(iters, sink + nt, sink);
  } else {
    float *sink = static_cast<float *>(d_sink);
    chem::k_fma_coefs<float><<<1, 1, 0, s>>>(sink + nt, 0.9999f, 1e-4f);
    chem::k_fma_peak<float><<<(unsigned)blocks, threads, 0, s>>>(iters, sink + nt, sink);
  }
  return cudaGetLastError() == cudaSuccess ? CHEM_OK : CHEM_ERR_CUDA;
}

extern "C" int chem_diag_math(int op, int64_t n, const double *d_x, double *d_y, void *stream) {
  if (op < 0 || op > 14 || n < 0) return CHEM_ERR_INVALID;
  if (n == 0) return CHEM_OK;
  if (!d_x || !d_y) return CHEM_ERR_INVALID;
  const int block = 256;
  chem::k_diag_math<<<(unsigned)((n + block - 1) / block), block, 0, (cudaStream_t)stream>>>(op, n, d_x, d_y);
  return cudaGetLastError() == cudaSuccess ? CHEM_OK : CHEM_ERR_CUDA;
}

extern "C" int chem_diag_ln_inv_kc(chem_ctx *ctx, int form, int64_t n, const double *d_T, double *d_out,
                                   void *stream) {
  if (!ctx) return CHEM_ERR_INVALID;
  std::string &err = chem::chem_ctx_error(ctx);
  if ((form != 0 && form != 1) || n < 0 || n > (int64_t(1) << 30)) {
    err = "chem_diag_ln_inv_kc: form must be 0 or 1 and n in [0, 2^30], got form " + std::to_string(form) +
          ", n " + std::to_string(n);
    return CHEM_ERR_INVALID;
  }
  if (n == 0) return CHEM_OK;
  if (!d_T || !d_out) {
    err = "chem_diag_ln_inv_kc: NULL d_T or d_out";
    return CHEM_ERR_INVALID;
  }
  const int block = 128;
  chem::k_ln_inv_kc<<<(unsigned)((n + block - 1) / block), block, 0, (cudaStream_t)stream>>>(
      chem::chem_ctx_tables(ctx), form, n, d_T, d_out);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    err = std::string("chem_diag_ln_inv_kc: ") + cudaGetErrorString(e);
    return CHEM_ERR_CUDA;
  }
  return CHEM_OK;
}
