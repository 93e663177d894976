// diag.cu -- chem_diag_math: the kernels' device math routines on caller arrays, for
// accuracy tests against the CUDA library and the IEEE-754 definitions.
#include <cuda_runtime.h>

#include "fastmath.cuh"
#include "internal.cuh"

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
    default: split_hilo(v, h, l); r = (double)l; break;
  }
  y[i] = r;
}

}  // namespace chem

extern "C" int chem_diag_math(int op, int64_t n, const double *d_x, double *d_y, void *stream) {
  if (op < 0 || op > 10 || n < 0) return CHEM_ERR_INVALID;
  if (n == 0) return CHEM_OK;
  if (!d_x || !d_y) return CHEM_ERR_INVALID;
  const int block = 256;
  chem::k_diag_math<<<(unsigned)((n + block - 1) / block), block, 0, (cudaStream_t)stream>>>(op, n, d_x, d_y);
  return cudaGetLastError() == cudaSuccess ? CHEM_OK : CHEM_ERR_CUDA;
}
