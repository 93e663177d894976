// mlp_gemm_tc.cu -- the surrogate's training GEMM on the 5th-generation tensor cores:
// C[m, n] = alpha * sum_k A(m, k) B(n, k) (+ bias[n]) with A(m, k) = A[m*sam + k*sak] and
// B(n, k) = B[n*sbn + k*sbk] in BF16, FP32 accumulation in tensor memory (GemmArgs,
// mlp.cuh).  One kernel serves the forward layer (H W^T), the input gradient (G W) and
// the weight gradient (G^T H, split over the batch) through the strides.
//
// A CTA computes a 128 x Nt tile (Nt = 16, or 64 for wider outputs, which run as several
// tiles so a batch of 4096 rows spreads over 128 CTAs): 16 warps, one elected thread
// issues tcgen05.mma (M = 128, N = Nt, K = 16) into a 128-lane x Nt-column
// FP32 accumulator in tensor memory.  K runs in chunks of 64 through two shared-memory
// stages: all threads stage chunk c + 1 into the canonical K-major core-matrix layout of
// tc.cuh (operands whose unit stride runs along k by 16-byte cp.async copies, those whose
// unit stride runs along m or n by batched 16-byte loads transposed on the way) while the
// tensor cores work on chunk c; a stage is refilled once the commit of the MMAs that read
// it has arrived.  Epilogue: each warp reads 32 accumulator lanes (its lane quarter,
// tcgen05.ld 32x32b) for a quarter of the columns and applies alpha, bias, accumulation
// into Cf, GELU (or the product with GELU' of a given Z) and the FP32 / BF16 stores.
//
// Every mbarrier wait is bounded; a wait that runs out sets *err (when given), the CTA
// issues nothing more, and still frees its tensor memory.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.cuh"
#include "mlp.cuh"
#include "mma.cuh"
#include "tc.cuh"

namespace chem {

namespace {

constexpr int GM = 128;      // rows per CTA tile (MMA M)
constexpr int GKC = 64;      // K chunk per stage
constexpr int GNMAX = 64;    // widest N tile (MMA N): 256-wide outputs run as 4 tiles, 4x the CTAs
constexpr int GTHR = 512;    // 16 warps: 4 per accumulator lane quarter, each a quarter of the columns
constexpr uint32_t kStageA = GM * GKC * 2;            // 16 KB
constexpr uint32_t kStageB = GNMAX * GKC * 2;         // 8 KB
constexpr uint32_t kStage = kStageA + kStageB;
constexpr uint32_t SMG_BAR = 2 * kStage;              // two mbarriers
constexpr uint32_t SMG_MISC = SMG_BAR + 16;           // tmem address, abort flag
constexpr uint32_t kGemmSmem = SMG_MISC + 16 + 1024;  // + alignment slack

// Operand staging modes (uniform per launch): 0 unit stride along k (16-byte rows of 8
// k), 1 unit stride along the row index (16-byte runs of 8 rows, transposed), 2 scalar.
__host__ inline int stage_mode(const __nv_bfloat16 *p, int64_t srow, int64_t sk) {
  const bool al = (reinterpret_cast<uintptr_t>(p) & 15u) == 0;
  if (sk == 1 && srow % 8 == 0 && al) return 0;
  if (srow == 1 && sk % 8 == 0 && al) return 1;
  return 2;
}

// 16-byte asynchronous copy global -> shared; src_bytes 0 fills the 16 bytes with zeros
// (the address is then not read).
__device__ __forceinline__ void cp_async16_zfill(uint32_t dst, const void *src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(src_bytes)
               : "memory");
}

// Stage rows [r0, r0 + ROWS) x k [k0, k0 + 64) of an operand into the core-matrix tile at
// `tile` (zeros outside [0, rmax) x [k0, kend)).  Mode 0 issues 16-byte asynchronous
// copies (completed by the caller's cp.async.wait_all); the transposing modes load
// their ROWS / 16 16-byte runs per thread into registers first, then store.
template <int ROWS>
__device__ __forceinline__ void stage_tile(unsigned char *tile, const __nv_bfloat16 *G, int64_t r0,
                                           int64_t rmax, int64_t sr, int64_t k0, int64_t kend, int64_t sk,
                                           int mode) {
  constexpr int UNITS = ROWS * (GKC / 8);              // 16-byte units of the tile
  constexpr int NU = (UNITS + GTHR - 1) / GTHR;        // per thread
  const int tid = threadIdx.x;
  const __nv_bfloat16 z = __float2bfloat16(0.0f);
  if (mode == 0) {
#pragma unroll
    for (int q = 0; q < NU; ++q) {
      const int u = tid + q * GTHR;
      if (UNITS % GTHR != 0 && u >= UNITS) break;
      const int r = u / (GKC / 8), j = u % (GKC / 8);
      const int64_t row = r0 + r, k = k0 + 8 * j;
      const uint32_t dst = smem_u32(tile + core_off(r, 8 * j, GKC));
      if (row < rmax && k + 8 <= kend) {
        cp_async16_zfill(dst, G + row * sr + k, 16u);
      } else if (row < rmax && k < kend) {
        __align__(16) __nv_bfloat16 h[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) h[i] = (k + i < kend) ? G[row * sr + k + i] : z;
        *reinterpret_cast<uint4 *>(tile + core_off(r, 8 * j, GKC)) = *reinterpret_cast<const uint4 *>(h);
      } else {
        cp_async16_zfill(dst, G, 0u);
      }
    }
  } else {
    uint4 h[NU];
#pragma unroll
    for (int q = 0; q < NU; ++q) {
      const int u = tid + q * GTHR;
      if (UNITS % GTHR != 0 && u >= UNITS) break;
      const int kk = u / (ROWS / 8), rg = u % (ROWS / 8);
      const int64_t row = r0 + 8 * rg, k = k0 + kk;
      if (k < kend && mode == 1 && row + 8 <= rmax) {
        h[q] = *reinterpret_cast<const uint4 *>(G + k * sk + row);
      } else {
        __align__(16) __nv_bfloat16 t[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) t[i] = (k < kend && row + i < rmax) ? G[(row + i) * sr + k * sk] : z;
        h[q] = *reinterpret_cast<const uint4 *>(t);
      }
    }
#pragma unroll
    for (int q = 0; q < NU; ++q) {
      const int u = tid + q * GTHR;
      if (UNITS % GTHR != 0 && u >= UNITS) break;
      const int kk = u / (ROWS / 8), rg = u % (ROWS / 8);
      const __nv_bfloat16 *t = reinterpret_cast<const __nv_bfloat16 *>(&h[q]);
#pragma unroll
      for (int i = 0; i < 8; ++i)
        *reinterpret_cast<__nv_bfloat16 *>(tile + core_off(8 * rg + i, kk, GKC)) = t[i];
    }
  }
}

struct GemmTc {
  GemmArgs g;
  int mode_a, mode_b;
  int nt;         // N tile width (multiple of 16, <= 256)
  uint32_t cols;  // tensor-memory columns allocated (power of two >= 32, >= nt)
  int *err;
};

template <int NT>
__device__ __forceinline__ void gemm_body(const GemmTc &p, unsigned char *sm, uint32_t sbase) {
  const GemmArgs &g = p.g;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  volatile uint32_t *s_tmem = reinterpret_cast<volatile uint32_t *>(sm + SMG_MISC);
  volatile int *s_abort = reinterpret_cast<volatile int *>(sm + SMG_MISC + 4);
  const uint32_t bar0 = sbase + SMG_BAR;
  if (tid == 0) {
    *s_abort = 0;
    mbar_init(bar0, 1);
    mbar_init(bar0 + 8, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(sbase + SMG_MISC),
                 "r"(p.cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;

  const int64_t m0 = (int64_t)blockIdx.y * GM, n0 = (int64_t)blockIdx.x * NT;
  int64_t kbeg = 0, kend = g.K;
  if (g.split > 1) {
    const int64_t steps = (g.K + GKC - 1) / GKC, per = (steps + g.split - 1) / g.split;
    kbeg = (int64_t)blockIdx.z * per * GKC;
    kend = kbeg + per * GKC < g.K ? kbeg + per * GKC : g.K;
  }
  const int nch = kend > kbeg ? (int)((kend - kbeg + GKC - 1) / GKC) : 0;
  const uint32_t idesc = idesc_bf16(GM, NT);
  bool fail = false;
  for (int c = 0; c < nch; ++c) {
    const int st = c & 1;
    if (c >= 2 && !fail) {  // the MMAs of chunk c - 2 read this stage
      if (!mbar_wait(bar0 + 8u * st, (uint32_t)(((c - 2) >> 1) & 1))) fail = true;
    }
    if (fail) *s_abort = 1;
    unsigned char *sa = sm + (uint32_t)st * kStage, *sb = sa + kStageA;
    const int64_t k0 = kbeg + (int64_t)c * GKC;
    if (!*s_abort) {
      stage_tile<GM>(sa, g.A, m0, g.M, g.sam, k0, kend, g.sak, p.mode_a);
      stage_tile<NT>(sb, g.B, n0, g.N, g.sbn, k0, kend, g.sbk, p.mode_b);
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (*s_abort) break;
    if (tid == 0) {
      tc_fence_after();
      const int nk = (int)((kend - k0 + 15) / 16) < GKC / 16 ? (int)((kend - k0 + 15) / 16) : GKC / 16;
      const uint32_t a0 = sbase + (uint32_t)st * kStage, b0 = a0 + kStageA;
      for (int kk = 0; kk < nk; ++kk)
        mma_bf16_tc(tmem, smem_desc(a0 + (uint32_t)(kk * 2) * 128, 128, (GKC / 8) * 128),
                    smem_desc(b0 + (uint32_t)(kk * 2) * 128, 128, (GKC / 8) * 128), idesc,
                    (c > 0 || kk > 0) ? 1u : 0u);
      mma_commit(bar0 + 8u * st);
    }
  }
  // the last commit covers every MMA of the tile
  bool have = nch > 0 && !*s_abort;
  if (have && !mbar_wait(bar0 + 8u * ((nch - 1) & 1), (uint32_t)(((nch - 1) >> 1) & 1))) {
    have = false;
    *s_abort = 1;
  }
  tc_fence_after();
  __syncthreads();
  if (*s_abort) {
    if (p.err && tid == 0) atomicExch(p.err, 1);
  } else {
    // epilogue: warp w reads accumulator lanes (rows) m0 + 32 (w % 4) .. + 31, the lane
    // quarter tcgen05.ld lets it reach, and a quarter of the columns (w / 4; the 16-wide
    // tile has one group); each 32-column chunk goes through a padded 32 x 33 shared-memory
    // tile (the stages are idle: the last commit covered every MMA), so the global stores
    // run along rows, coalesced
    const int q = warp & 3, grp = warp >> 2;
    constexpr int NG = NT >= 32 ? NT / 32 : 1;  // column groups (at most 4 with 16 warps)
    static_assert(NG <= 4, "four column groups at most");
    constexpr int GW = NT / NG;                 // columns per group
    constexpr int CW = GW < 32 ? GW : 32;       // columns per tensor-memory load
    if (grp < NG) {
      float *tp = reinterpret_cast<float *>(sm) + warp * (32 * 33);
      const uint32_t t_lane = tmem + ((uint32_t)(32 * q) << 16);
      for (int cb = grp * GW; cb < (grp + 1) * GW; cb += CW) {
        if constexpr (CW == 32) {
          uint32_t r[32];
          tmem_ld32_async(t_lane + (uint32_t)cb, r);
          tmem_wait32(r);
#pragma unroll
          for (int i = 0; i < 32; ++i) tp[lane * 33 + i] = have ? __uint_as_float(r[i]) : 0.0f;
        } else {
          float w[16];
          tmem_ld16(t_lane + (uint32_t)cb, w);
#pragma unroll
          for (int i = 0; i < 16; ++i) tp[lane * 33 + i] = have ? w[i] : 0.0f;
        }
        __syncwarp();
        const int64_t n = n0 + cb + lane;
        if (lane < CW && n < g.N) {
          const float bn = (g.bias && g.split <= 1) ? g.bias[n] : 0.0f;
          const int64_t mq = m0 + 32 * q;
          if (g.split > 1) {
            for (int rr = 0; rr < 32 && mq + rr < g.M; ++rr)
              g.Cf[(int64_t)blockIdx.z * g.split_ld + (mq + rr) * g.ldc + n] = tp[rr * 33 + lane] * g.alpha;
          } else if (g.dgelu_z) {
            // the 32 rows' Z first, all loads in flight together, then the products
            float z[32];
#pragma unroll
            for (int rr = 0; rr < 32; ++rr)
              z[rr] = mq + rr < g.M ? __ldg(g.dgelu_z + (mq + rr) * g.ldz + n) : 0.0f;
#pragma unroll
            for (int rr = 0; rr < 32; ++rr) {
              if (mq + rr < g.M) {
                const int64_t m = mq + rr;
                float x = tp[rr * 33 + lane] * g.alpha;
                x += bn;
                if (g.accumulate) x += g.Cf[m * g.ldc + n];
                if (g.Cf) g.Cf[m * g.ldc + n] = x;
                if (g.Cb) g.Cb[m * g.ldcb + n] = __float2bfloat16(x * gelu_grad_f(z[rr]));
              }
            }
          } else {
            for (int rr = 0; rr < 32; ++rr) {
              const int64_t m = mq + rr;
              if (m >= g.M) break;
              float x = tp[rr * 33 + lane] * g.alpha;
              x += bn;
              if (g.accumulate) x += g.Cf[m * g.ldc + n];
              if (g.Cf) g.Cf[m * g.ldc + n] = x;
              if (g.Cb) g.Cb[m * g.ldcb + n] = __float2bfloat16(g.gelu ? gelu_f(x) : x);
            }
          }
        }
        __syncwarp();
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(p.cols) : "memory");
}

__global__ void __launch_bounds__(GTHR) k_gemm_tc(const __grid_constant__ GemmTc p) {
  extern __shared__ __align__(1024) unsigned char gsm_raw[];
  unsigned char *sm = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(gsm_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const uint32_t sbase = smem_u32(sm);
  // the tile widths: 16 (the padded input and output layers) and 64 (the hidden layers'
  // 256 outputs as four tiles); a column beyond N is zero-filled and not stored
  if (p.nt == 16) gemm_body<16>(p, sm, sbase);
  else gemm_body<GNMAX>(p, sm, sbase);
}

}  // namespace

cudaError_t gemm_prepare() {
  static bool attr_set[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64 || !attr_set[dev]) {
    e = cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGemmSmem);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) attr_set[dev] = true;
  }
  return cudaSuccess;
}

cudaError_t launch_gemm(const GemmArgs &g, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0) return cudaSuccess;
  if (g.split > 1 && (!g.Cf || g.Cb || g.bias || g.accumulate)) return cudaErrorInvalidValue;
  cudaError_t e = gemm_prepare();
  if (e != cudaSuccess) return e;
  GemmTc p{};
  p.g = g;
  p.mode_a = stage_mode(g.A, g.sam, g.sak);
  p.mode_b = stage_mode(g.B, g.sbn, g.sbk);
  p.nt = g.N <= 16 ? 16 : GNMAX;
  p.cols = p.nt <= 32 ? 32u : (uint32_t)GNMAX;
  p.err = g.err;
  dim3 grid((unsigned)((g.N + p.nt - 1) / p.nt), (unsigned)((g.M + GM - 1) / GM),
            (unsigned)(g.split > 1 ? g.split : 1));
  k_gemm_tc<<<grid, GTHR, kGemmSmem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace chem
