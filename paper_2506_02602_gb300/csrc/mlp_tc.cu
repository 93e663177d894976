// mlp_tc.cu -- the surrogate network's forward pass on the 5th-generation tensor cores
// (tcgen05): one persistent CTA per SM, 128 cells (rows) per tile.
//
// Per tile the CTA keeps the activations in shared memory (128 x 256 BF16, the MMA's A
// operand) and the FP32 accumulator in tensor memory (128 lanes x 256 columns); one
// thread issues every tcgen05.mma (M = 128, N = 256 or 16, K = 16, BF16 x BF16 -> FP32)
// and the bulk copies of the weights; all 512 threads run the epilogues (tcgen05.ld of
// the accumulator, bias, GELU, BF16 rounding, store as the next layer's A operand):
// warp w reads accumulator lanes 32 (w % 4) .. + 31 (the lane quarter tcgen05.ld lets it
// reach) and 64 of the 256 columns.
//
// Operands use the canonical K-major layout without swizzle: "core matrices" of 8 rows
// x 16 bytes (8 BF16) stored as 128 contiguous bytes; the core matrix holding rows
// 8i..8i+7 and k = 8j..8j+7 of a tile sits at i * SBO + j * LBO.  Here LBO = 128 (core
// matrices adjacent along k are adjacent in memory) and SBO = 128 * (k extent / 8).
// The weights are repacked once into that layout (k_pack_weights), the hidden layers in
// K chunks of 64 (256 x 64 BF16 = 32 KB each), so every weight transfer is one
// contiguous cp.async.bulk into a two-stage ring; the first and last layers' weights
// stay resident.
//
// Every mbarrier wait is bounded; a wait that runs out sets an error word, and the CTA
// stops issuing work, waits (bounded) for what it issued, frees its tensor memory and
// returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "mma.cuh"
#include "surrogate.cuh"
#include "tc.cuh"

namespace chem {

namespace {

constexpr int TM = 128;                   // rows per tile (MMA M)
constexpr int TTHREADS = 512;             // 16 warps: 4 per accumulator lane quarter
constexpr int COLS_PER_WARP = kSurHidden / (TTHREADS / 128);  // hidden columns per warp
constexpr int KC = 64;                    // K chunk of a streamed hidden-layer weight
constexpr int NCHUNK = kSurHidden / KC;   // 4 chunks per hidden layer
constexpr uint32_t kChunkBytes = kSurHidden * KC * 2;            // 32 KB
constexpr uint32_t kW0Bytes = kSurHidden * kSurIn * 2;           // 8 KB
constexpr uint32_t kW3Bytes = kSurOut * kSurHidden * 2;          // 8 KB
constexpr uint32_t kHiddenBytes = kSurHidden * kSurHidden * 2;   // 128 KB
// packed weights: W0 | W1 (4 chunks) | W2 (4 chunks) | W3
constexpr uint32_t kPackOffW1 = kW0Bytes;
constexpr uint32_t kPackOffW2 = kW0Bytes + kHiddenBytes;
constexpr uint32_t kPackOffW3 = kW0Bytes + 2 * kHiddenBytes;
constexpr uint32_t kPackBytes = kPackOffW3 + kW3Bytes;

// shared memory map (bytes from a 1024-aligned base)
constexpr uint32_t SM_X = 0;                              // 128 x 16 bf16: 4 KB
constexpr uint32_t SM_H = SM_X + TM * kSurIn * 2;         // 128 x 256 bf16: 64 KB
constexpr uint32_t SM_W0 = SM_H + TM * kSurHidden * 2;    // 8 KB
constexpr uint32_t SM_W3 = SM_W0 + kW0Bytes;              // 8 KB
constexpr uint32_t SM_WB = SM_W3 + kW3Bytes;              // 2 x 32 KB ring
constexpr uint32_t SM_BIAS = SM_WB + 2 * kChunkBytes;     // 3 x 256 + 16 floats
constexpr uint32_t SM_BAR = SM_BIAS + (3 * kSurHidden + kSurOut) * 4;  // mbarriers
constexpr uint32_t SM_MISC = SM_BAR + 8 * 8;              // tmem address, abort flag
constexpr uint32_t kTcSmem = SM_MISC + 16 + 1024;         // + alignment slack
constexpr int BAR_FULL0 = 0, BAR_EMPTY0 = 2, BAR_MMA = 4, BAR_WRES = 5;

constexpr uint32_t kTmemCols = 256;

struct TcArgs {
  int64_t n;
  const float *X;      // [n x 16] features: raw when norm is set, else normalised
  const float *norm;   // fmean[16], fistd[16] (nullable)
  const unsigned char *Wpk;  // packed weights (kPackBytes)
  const float *b[kSurLayers];
  float *O;            // [n x 16]
  int *err;            // error word (nonzero: a wait ran out)
};

}  // namespace

// Pack the BF16 weights (W_l [N x K], k contiguous) into the core-matrix layout above.
__global__ void k_pack_weights(const __nv_bfloat16 *W0, const __nv_bfloat16 *W1, const __nv_bfloat16 *W2,
                               const __nv_bfloat16 *W3, unsigned char *Wpk) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int n0 = kSurHidden * kSurIn, nh = kSurHidden * kSurHidden, n3 = kSurOut * kSurHidden;
  if (t >= n0 + 2 * nh + n3) return;
  __nv_bfloat16 v;
  uint32_t off;
  if (t < n0) {
    const int n = t / kSurIn, k = t % kSurIn;
    v = W0[t];
    off = core_off(n, k, kSurIn);
  } else if (t < n0 + 2 * nh) {
    const int l = (t - n0) / nh, u = (t - n0) % nh;
    const int n = u / kSurHidden, k = u % kSurHidden;
    v = (l ? W2 : W1)[u];
    off = (l ? kPackOffW2 : kPackOffW1) + (uint32_t)(k / KC) * kChunkBytes + core_off(n, k % KC, KC);
  } else {
    const int u = t - n0 - 2 * nh;
    const int n = u / kSurHidden, k = u % kSurHidden;
    v = W3[u];
    off = kPackOffW3 + core_off(n, k, kSurHidden);
  }
  *reinterpret_cast<__nv_bfloat16 *>(Wpk + off) = v;
}

__global__ void __launch_bounds__(TTHREADS, 1) k_mlp_tc(const __grid_constant__ TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *sm = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const uint32_t sbase = smem_u32(sm);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  float *sbias = reinterpret_cast<float *>(sm + SM_BIAS);
  volatile uint32_t *s_tmem = reinterpret_cast<volatile uint32_t *>(sm + SM_MISC);
  volatile int *s_abort = reinterpret_cast<volatile int *>(sm + SM_MISC + 4);
  const uint32_t bar = sbase + SM_BAR;
  auto barrier_addr = [&](int i) { return bar + 8u * (uint32_t)i; };

  // biases to shared memory
  for (int i = tid; i < 3 * kSurHidden + kSurOut; i += TTHREADS)
    sbias[i] = i < 3 * kSurHidden ? a.b[i / kSurHidden][i % kSurHidden] : a.b[3][i - 3 * kSurHidden];
  if (tid == 0) {
    *s_abort = 0;
    for (int i = 0; i < 6; ++i) mbar_init(barrier_addr(i), 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {  // tensor memory for the 128 x 256 FP32 accumulator
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(sbase + SM_MISC),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;

  // issuer state (thread 0): phases of the ring's full / empty barriers and the chunk
  // sequence number of the weight stream (W1 chunks 0..3, W2 chunks 0..3, next tile ...)
  uint32_t full_ph[2] = {0, 0}, empty_ph[2] = {0, 0};
  uint32_t mma_ph = 0;  // every thread tracks the MMA-done barrier
  const int64_t ntiles = (a.n + TM - 1) / TM;
  bool fail = false;

  // weight stream: stream index s = 0 .. 7 per tile (W1 chunk s, then W2 chunk s - 4);
  // chunk s goes to ring slot s % 2
  auto issue_chunk = [&](int s) {
    const int slot = s & 1;
    const uint32_t dst = sbase + SM_WB + (uint32_t)slot * kChunkBytes;
    const unsigned char *src = a.Wpk + (s < NCHUNK ? kPackOffW1 : kPackOffW2) + (uint32_t)(s % NCHUNK) * kChunkBytes;
    mbar_expect_tx(barrier_addr(BAR_FULL0 + slot), kChunkBytes);
    bulk_g2s(dst, src, kChunkBytes, barrier_addr(BAR_FULL0 + slot));
  };

  if (tid == 0 && blockIdx.x < ntiles) {
    mbar_expect_tx(barrier_addr(BAR_WRES), kW0Bytes + kW3Bytes);
    bulk_g2s(sbase + SM_W0, a.Wpk, kW0Bytes, barrier_addr(BAR_WRES));
    bulk_g2s(sbase + SM_W3, a.Wpk + kPackOffW3, kW3Bytes, barrier_addr(BAR_WRES));
    issue_chunk(0);
    issue_chunk(1);
  }
  bool wres_ready = false;

  const uint32_t id_h = idesc_bf16(TM, kSurHidden), id_o = idesc_bf16(TM, kSurOut);
  const int q = warp & 3, cblk = warp >> 2;
  const int row = q * 32 + lane;                     // this thread's accumulator lane
  const uint32_t t_lane = tmem + ((uint32_t)(q * 32) << 16);

  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t row0 = tile * TM;
    // 1. features -> sX (row t / 2, 8 columns (t % 2) * 8 ..): one 16-byte core row
    if (tid < 2 * TM) {
      const int r = tid >> 1, c0 = (tid & 1) * 8;
      float v[8];
      if (row0 + r < a.n) {
        const float4 *src = reinterpret_cast<const float4 *>(a.X + (row0 + r) * kSurIn + c0);
        const float4 p = src[0], u = src[1];
        v[0] = p.x; v[1] = p.y; v[2] = p.z; v[3] = p.w; v[4] = u.x; v[5] = u.y; v[6] = u.z; v[7] = u.w;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int c = c0 + i;
          if (a.norm) v[i] = c < kSurFeat ? (v[i] - a.norm[c]) * a.norm[16 + c] : 0.0f;
        }
      } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = 0.0f;
      }
      __align__(16) __nv_bfloat16 hb[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) hb[i] = __float2bfloat16(v[i]);
      *reinterpret_cast<uint4 *>(sm + SM_X + core_off(r, c0, kSurIn)) = *reinterpret_cast<const uint4 *>(hb);
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (*s_abort) break;

    for (int layer = 0; layer < kSurLayers; ++layer) {
      // 2. the issuing thread: this layer's MMAs, then a commit to the MMA barrier
      if (tid == 0 && !fail) {
        tc_fence_after();
        if (layer == 0) {
          if (!wres_ready) {
            fail = !mbar_wait(barrier_addr(BAR_WRES), 0);
            wres_ready = true;
          }
          if (!fail)
            mma_bf16_tc(tmem, smem_desc(sbase + SM_X, 128, 2 * 128), smem_desc(sbase + SM_W0, 128, 2 * 128),
                        id_h, 0);
        } else if (layer < 3) {
          for (int c = 0; c < NCHUNK && !fail; ++c) {
            const int s = (layer - 1) * NCHUNK + c, slot = s & 1;
            fail = !mbar_wait(barrier_addr(BAR_FULL0 + slot), full_ph[slot]);
            full_ph[slot] ^= 1u;
            if (fail) break;
            const uint32_t wb = sbase + SM_WB + (uint32_t)slot * kChunkBytes;
#pragma unroll
            for (int kk = 0; kk < KC / 16; ++kk) {
              const uint32_t koff = (uint32_t)((c * KC + kk * 16) / 8) * 128;
              mma_bf16_tc(tmem, smem_desc(sbase + SM_H + koff, 128, (kSurHidden / 8) * 128),
                          smem_desc(wb + (uint32_t)(kk * 2) * 128, 128, (KC / 8) * 128), id_h,
                          (c > 0 || kk > 0) ? 1u : 0u);
            }
            mma_commit(barrier_addr(BAR_EMPTY0 + slot));
            // refill the other slot with stream chunk s + 1 once the MMAs that read it
            // (chunk s - 1) are done; chunks 0 and 1 of a tile were issued ahead
            const int nxt = s + 1;
            if (s >= 1 && nxt < 2 * NCHUNK) {
              const int ps = nxt & 1;
              fail = !mbar_wait(barrier_addr(BAR_EMPTY0 + ps), empty_ph[ps]);
              empty_ph[ps] ^= 1u;
              if (!fail) issue_chunk(nxt);
            }
          }
        } else {
#pragma unroll 1
          for (int kk = 0; kk < kSurHidden / 16; ++kk)
            mma_bf16_tc(tmem, smem_desc(sbase + SM_H + (uint32_t)(kk * 2) * 128, 128, (kSurHidden / 8) * 128),
                        smem_desc(sbase + SM_W3 + (uint32_t)(kk * 2) * 128, 128, (kSurHidden / 8) * 128), id_o,
                        kk > 0 ? 1u : 0u);
        }
        if (!fail) mma_commit(barrier_addr(BAR_MMA));
        if (fail) *s_abort = 1;
      }
      // 3. everyone: wait for the accumulator
      if (!mbar_wait(barrier_addr(BAR_MMA), mma_ph)) {
        *s_abort = 1;
        if (a.err) atomicExch(a.err, 1);
      }
      mma_ph ^= 1u;
      tc_fence_after();
      if (tid == 0 && layer == 2 && !fail) {
        // the ring's last two chunks of this tile are consumed: stream the next tile's
        // first two W1 chunks (their MMAs are complete, the MMA barrier said so)
        for (int ps = 0; ps < 2 && !fail; ++ps) {
          fail = !mbar_wait(barrier_addr(BAR_EMPTY0 + ps), empty_ph[ps]);
          empty_ph[ps] ^= 1u;
        }
        if (!fail && tile + gridDim.x < ntiles) {
          issue_chunk(0);
          issue_chunk(1);
        }
        if (fail) *s_abort = 1;
      }
      // 4. epilogue
      if (layer < 3) {
        const float *bl = sbias + layer * kSurHidden;
        static_assert(COLS_PER_WARP == 64, "two 32-column chunks per warp");
        uint32_t ra[32], rb[32];
        const int colA = cblk * COLS_PER_WARP, colB = colA + 32;
        tmem_ld32_async(t_lane + (uint32_t)colA, ra);
        tmem_wait32(ra);
        tmem_ld32_async(t_lane + (uint32_t)colB, rb);  // overlaps the first chunk's math
        auto emit = [&](const uint32_t(&r)[32], int col0) {
#pragma unroll
          for (int g = 0; g < 4; ++g) {
            __align__(16) __nv_bfloat16 hb[8];
#pragma unroll
            for (int i = 0; i < 8; ++i)
              hb[i] = __float2bfloat16(gelu_f(__uint_as_float(r[g * 8 + i]) + bl[col0 + g * 8 + i]));
            *reinterpret_cast<uint4 *>(sm + SM_H + core_off(row, col0 + g * 8, kSurHidden)) =
                *reinterpret_cast<const uint4 *>(hb);
          }
        };
        emit(ra, colA);
        tmem_wait32(rb);
        emit(rb, colB);
      } else if (cblk == 0) {
        float v[16];
        tmem_ld16(t_lane, v);
        if (row0 + row < a.n) {
          float4 *dst = reinterpret_cast<float4 *>(a.O + (row0 + row) * kSurOut);
          const float *bl = sbias + 3 * kSurHidden;
#pragma unroll
          for (int g = 0; g < 4; ++g)
            dst[g] = make_float4(v[4 * g] + bl[4 * g], v[4 * g + 1] + bl[4 * g + 1], v[4 * g + 2] + bl[4 * g + 2],
                                 v[4 * g + 3] + bl[4 * g + 3]);
        }
      }
      fence_async_smem();
      tc_fence_before();
      __syncthreads();
      if (*s_abort) break;
    }
    if (*s_abort) break;
  }
  if (*s_abort && a.err) atomicExch(a.err, 1);
  // drain: the issuer waits (bounded) for the MMAs it committed; then free the tensor
  // memory (the allocating warp)
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

cudaError_t launch_pack_weights(const __nv_bfloat16 *const (&W)[kSurLayers], unsigned char *Wpk, cudaStream_t s) {
  const int total = kSurHidden * kSurIn + 2 * kSurHidden * kSurHidden + kSurOut * kSurHidden;
  k_pack_weights<<<(total + 255) / 256, 256, 0, s>>>(W[0], W[1], W[2], W[3], Wpk);
  return cudaGetLastError();
}

size_t packed_weight_bytes() { return kPackBytes; }

cudaError_t launch_mlp_tc(int64_t n, const float *X, const float *norm, const unsigned char *Wpk,
                          const float *const (&b)[kSurLayers], float *O, int *err, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  static bool attr_set[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64 || !attr_set[dev]) {
    e = cudaFuncSetAttribute(k_mlp_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) attr_set[dev] = true;
  }
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int64_t ntiles = (n + TM - 1) / TM;
  const unsigned grid = (unsigned)(ntiles < sms ? ntiles : sms);
  TcArgs a{};
  a.n = n;
  a.X = X;
  a.norm = norm;
  a.Wpk = Wpk;
  for (int l = 0; l < kSurLayers; ++l) a.b[l] = b[l];
  a.O = O;
  a.err = err;
  k_mlp_tc<<<grid, TTHREADS, kTcSmem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace chem
