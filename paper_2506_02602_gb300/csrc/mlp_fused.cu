// mlp_fused.cu -- the surrogate network's whole forward pass in one kernel (inference).
//
// A CTA takes 128 rows (cells).  Their activations stay in shared memory for all four
// layers (128 x 256 BF16), so HBM sees only the 16 input features and the 16 outputs of
// a cell; the layer-by-layer path would write and re-read 3 x 256 BF16 activations per
// cell.  Weights (BF16, [N x K], k contiguous, 272 KB in all and resident in L2) are
// streamed through a two-stage cp.async buffer in 32-wide K chunks.  Each layer is
// 8 warps of mma.sync m16n8k16 (BF16 in, FP32 accumulate) with the same fragment code,
// K order and epilogue (bias, GELU, BF16 rounding) as the layer-by-layer GEMM, so both
// paths give the same numbers.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "mma.cuh"
#include "surrogate.cuh"

namespace chem {

constexpr int FBM = 128;                // rows per CTA
constexpr int FTHREADS = 256;           // 8 warps
constexpr int HPITCH = kSurHidden + 8;  // bf16 per activation row in shared memory
constexpr int WKC = 32;                 // K chunk of staged weights
constexpr int WPITCH = WKC + 8;         // bf16 per staged weight row
constexpr int WSTAGE = kSurHidden * WPITCH;
constexpr size_t kFusedSmem = ((size_t)FBM * HPITCH + 2 * (size_t)WSTAGE) * sizeof(__nv_bfloat16);

// Stage K chunk c of W ([N x K], k contiguous) into Ws[N][WPITCH] (16-byte cp.async).
template <int N, int K>
__device__ __forceinline__ void stage_w(__nv_bfloat16 *Ws, const __nv_bfloat16 *__restrict__ W, int c) {
  constexpr int KC = K < WKC ? K : WKC;
  constexpr int PIECES = KC / 8;
  for (int p = threadIdx.x; p < N * PIECES; p += FTHREADS) {
    const int n = p / PIECES, q = p % PIECES;
    cp_async16(Ws + n * WPITCH + q * 8, W + (int64_t)n * K + c * KC + q * 8);
  }
  cp_async_commit();
}

// One layer on the CTA's rows: Hs <- GELU(Hs W^T + b) (hidden), or O = Hs W^T + b (last).
// Warp grid WGM x WGN over the 128 x N output; warp tile (TM * 16) x (TN * 8).
template <int K, int N, int WGM, int WGN, int TM, int TN, bool kLast>
__device__ __forceinline__ void fused_layer(__nv_bfloat16 *Hs, __nv_bfloat16 *Ws,
                                            const __nv_bfloat16 *__restrict__ W,
                                            const float *__restrict__ bias, float *__restrict__ O,
                                            int64_t row0, int64_t n) {
  static_assert(WGM * WGN == FTHREADS / 32 && WGM * TM * 16 == FBM && WGN * TN * 8 == N, "tiling");
  constexpr int KC = K < WKC ? K : WKC;
  constexpr int NCH = K / KC;
  static_assert(NCH * KC == K && KC % 16 == 0, "K chunks");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wm = (warp % WGM) * TM * 16, wn = (warp / WGM) * TN * 8;
  float acc[TM][TN][4];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.0f;
  stage_w<N, K>(Ws, W, 0);
  for (int c = 0; c < NCH; ++c) {
    const __nv_bfloat16 *cur = Ws + (c & 1) * WSTAGE;
    if (c + 1 < NCH) {
      stage_w<N, K>(Ws + ((c + 1) & 1) * WSTAGE, W, c + 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KC; kk += 16) {
      uint32_t af[TM][4];
#pragma unroll
      for (int i = 0; i < TM; ++i) {
        const int q = lane >> 3, rr = lane & 7;
        ldmatrix_x4(af[i], Hs + (wm + i * 16 + (q & 1) * 8 + rr) * HPITCH + c * KC + kk + (q >> 1) * 8);
      }
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        uint32_t bfr[2];
        const int q = (lane >> 3) & 1, rr = lane & 7;
        ldmatrix_x2(bfr, cur + (wn + j * 8 + rr) * WPITCH + kk + q * 8);
#pragma unroll
        for (int i = 0; i < TM; ++i) mma_bf16(acc[i][j], af[i], bfr);
      }
    }
    __syncthreads();  // every warp is done with Hs and this weight stage
  }
  // epilogue: fragment (i, j) holds rows wm + 16i + {g, g + 8}, columns wn + 8j + 2t + {0, 1}
  const int gq = lane >> 2, tq = lane & 3;
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int r = wm + i * 16 + gq + h * 8;
        const int col = wn + j * 8 + tq * 2;
        const float v0 = acc[i][j][2 * h] + bias[col];
        const float v1 = acc[i][j][2 * h + 1] + bias[col + 1];
        if constexpr (kLast) {
          if (row0 + r < n) *reinterpret_cast<float2 *>(O + (row0 + r) * kSurOut + col) = make_float2(v0, v1);
        } else {
          __nv_bfloat162 o;
          o.x = __float2bfloat16(gelu_f(v0));
          o.y = __float2bfloat16(gelu_f(v1));
          *reinterpret_cast<__nv_bfloat162 *>(Hs + r * HPITCH + col) = o;
        }
      }
  if constexpr (!kLast) __syncthreads();
}

struct FusedArgs {
  int64_t n;
  const float *X;     // [n x 16] features: raw when norm is set, else already normalised
  const float *norm;  // fmean[16], fistd[16] (nullable)
  const __nv_bfloat16 *W[kSurLayers];
  const float *b[kSurLayers];
  float *O;           // [n x 16] network outputs
};

__global__ void __launch_bounds__(FTHREADS, 1) k_mlp_fused(const __grid_constant__ FusedArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __nv_bfloat16 *Hs = reinterpret_cast<__nv_bfloat16 *>(smem_raw);
  __nv_bfloat16 *Ws = Hs + FBM * HPITCH;
  const int64_t row0 = (int64_t)blockIdx.x * FBM;
  {  // input features: thread t fills row t / 2, columns 8 (t % 2) .. + 7
    const int r = threadIdx.x >> 1, c0 = (threadIdx.x & 1) * 8;
    float v[8];
    if (row0 + r < a.n) {
      const float4 *src = reinterpret_cast<const float4 *>(a.X + (row0 + r) * kSurIn + c0);
      const float4 p = src[0], q = src[1];
      v[0] = p.x; v[1] = p.y; v[2] = p.z; v[3] = p.w; v[4] = q.x; v[5] = q.y; v[6] = q.z; v[7] = q.w;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int c = c0 + u;
        if (a.norm) v[u] = c < kSurFeat ? (v[u] - a.norm[c]) * a.norm[16 + c] : 0.0f;
      }
    } else {
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = 0.0f;
    }
    __align__(16) __nv_bfloat16 hb[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) hb[u] = __float2bfloat16(v[u]);
    *reinterpret_cast<uint4 *>(Hs + r * HPITCH + c0) = *reinterpret_cast<const uint4 *>(hb);
  }
  __syncthreads();
  fused_layer<kSurIn, kSurHidden, 2, 4, 4, 8, false>(Hs, Ws, a.W[0], a.b[0], nullptr, row0, a.n);
  fused_layer<kSurHidden, kSurHidden, 2, 4, 4, 8, false>(Hs, Ws, a.W[1], a.b[1], nullptr, row0, a.n);
  fused_layer<kSurHidden, kSurHidden, 2, 4, 4, 8, false>(Hs, Ws, a.W[2], a.b[2], nullptr, row0, a.n);
  fused_layer<kSurHidden, kSurOut, 8, 1, 1, 2, true>(Hs, Ws, a.W[3], a.b[3], a.O, row0, a.n);
}

cudaError_t launch_mlp_fused(int64_t n, const float *X, const float *norm,
                             const __nv_bfloat16 *const (&W)[kSurLayers],
                             const float *const (&b)[kSurLayers], float *O, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  // the shared-memory opt-in is a per-device attribute of the kernel (setting it twice
  // from racing threads is harmless)
  static bool attr_set[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64 || !attr_set[dev]) {
    e = cudaFuncSetAttribute(k_mlp_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFusedSmem);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) attr_set[dev] = true;
  }
  FusedArgs a{};
  a.n = n;
  a.X = X;
  a.norm = norm;
  for (int l = 0; l < kSurLayers; ++l) {
    a.W[l] = W[l];
    a.b[l] = b[l];
  }
  a.O = O;
  k_mlp_fused<<<(unsigned)((n + FBM - 1) / FBM), FTHREADS, kFusedSmem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace chem
