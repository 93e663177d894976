// mlp_tc.cu -- the surrogate network's forward pass on the 5th-generation tensor cores
// (tcgen05): one persistent CTA per SM, 128 cells (rows) per tile, two tiles in flight.
//
// Each tile in flight has its own activations in shared memory (128 x 256 BF16, the
// MMA's A operand), its own FP32 accumulator in tensor memory (128 lanes x 256 of the 512
// columns) and its own epilogue group of 8 warps (tcgen05.ld of the accumulator, bias,
// GELU, BF16 rounding, store as the next layer's A operand): warp w of a group reads
// accumulator lanes 32 (w % 4) .. + 31 (the lane quarter tcgen05.ld lets it reach) and
// 128 of the 256 columns, in chunks of 32 whose loads overlap the previous chunk's
// arithmetic.  A 17th warp issues every tcgen05.mma (M = 128, N = 256 or 16, K = 16,
// BF16 x BF16 -> FP32) and the bulk copies of the weights.  The issuing thread takes the
// layers of the two tiles in turn (layer l of tile 0, layer l of tile 1, layer l + 1 of
// tile 0, ...), so one tile's MMAs run while the other tile's epilogue runs; a group
// tells it through a per-tile mbarrier when the next A operand is in shared memory and
// the accumulator has been read.
//
// Operands use the canonical K-major layout without swizzle: "core matrices" of 8 rows
// x 16 bytes (8 BF16) stored as 128 contiguous bytes; the core matrix holding rows
// 8i..8i+7 and k = 8j..8j+7 of a tile sits at i * SBO + j * LBO.  Here LBO = 128 (core
// matrices adjacent along k are adjacent in memory) and SBO = 128 * (k extent / 8).
// The weights are repacked once into that layout (k_pack_weights), the hidden layers in
// K chunks of 32 (256 x 32 BF16 = 16 KB each), so every weight transfer is one
// contiguous cp.async.bulk into a four-slot ring, which the issuing thread refills
// whenever a slot's MMAs are done (also while it waits for an epilogue group); the
// first and last layers' weights stay resident.
//
// Every mbarrier wait is bounded; a wait that runs out sets an error word and a shared
// abort flag, every warp then stops issuing work, the issuing thread waits (bounded) for
// the copies and MMAs it issued, and the tensor memory is freed before the CTA returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "mma.cuh"
#include "surrogate.cuh"
#include "tc.cuh"

namespace chem {

namespace {

constexpr int TM = 128;                   // rows per tile (MMA M)
constexpr int NGRP = 2;                   // tiles in flight, one epilogue group each
constexpr int GWARPS = 8;                 // warps per epilogue group (2 per lane quarter)
constexpr int ISSUER_WARP = NGRP * GWARPS;           // warp 16
constexpr int TTHREADS = (ISSUER_WARP + 1) * 32;     // 544
constexpr int COLS_PER_WARP = kSurHidden / (GWARPS / 4);  // 128 hidden columns per warp
constexpr int KC = 32;                    // K chunk of a streamed hidden-layer weight
constexpr int NCHUNK = kSurHidden / KC;   // 8 chunks per hidden layer
constexpr int NSLOT = 4;                  // weight ring slots
constexpr uint32_t kChunkBytes = kSurHidden * KC * 2;            // 16 KB
constexpr uint32_t kW0Bytes = kSurHidden * kSurIn * 2;           // 8 KB
constexpr uint32_t kW3Bytes = kSurOut * kSurHidden * 2;          // 8 KB
constexpr uint32_t kHiddenBytes = kSurHidden * kSurHidden * 2;   // 128 KB
// packed weights: W0 | W1 (8 chunks) | W2 (8 chunks) | W3
constexpr uint32_t kPackOffW1 = kW0Bytes;
constexpr uint32_t kPackOffW2 = kW0Bytes + kHiddenBytes;
constexpr uint32_t kPackOffW3 = kW0Bytes + 2 * kHiddenBytes;
constexpr uint32_t kPackBytes = kPackOffW3 + kW3Bytes;

// shared memory map (bytes from a 1024-aligned base)
constexpr uint32_t kXBytes = TM * kSurIn * 2;                 // 4 KB per tile
constexpr uint32_t kHBytes = TM * kSurHidden * 2;             // 64 KB per tile
constexpr uint32_t SM_X = 0;                                  // 2 x 128 x 16 bf16
constexpr uint32_t SM_H = SM_X + NGRP * kXBytes;              // 2 x 128 x 256 bf16
constexpr uint32_t SM_W0 = SM_H + NGRP * kHBytes;             // 8 KB
constexpr uint32_t SM_W3 = SM_W0 + kW0Bytes;                  // 8 KB
constexpr uint32_t SM_WB = SM_W3 + kW3Bytes;                  // 4 x 16 KB ring
constexpr uint32_t SM_BIAS = SM_WB + NSLOT * kChunkBytes;     // 3 x 256 + 16 floats
constexpr uint32_t SM_BAR = SM_BIAS + (3 * kSurHidden + kSurOut) * 4;  // mbarriers
constexpr int BAR_FULL0 = 0, BAR_EMPTY0 = NSLOT, BAR_MMA0 = 2 * NSLOT, BAR_HREADY0 = BAR_MMA0 + NGRP,
              BAR_WRES = BAR_HREADY0 + NGRP, BAR_DRAIN = BAR_WRES + 1, NBAR = BAR_DRAIN + 1;
constexpr uint32_t SM_MISC = SM_BAR + NBAR * 8;               // tmem address, abort flag
constexpr uint32_t kTcSmem = SM_MISC + 16 + 1024;             // + alignment slack
static_assert(kTcSmem <= 232448, "over the per-CTA shared memory limit");
static_assert(SM_WB + NSLOT * kChunkBytes <= (1u << 18), "descriptor start addresses are 18-bit");

constexpr uint32_t kTmemCols = NGRP * kSurHidden;  // 512: one accumulator per tile in flight
constexpr uint32_t kSpinLimit = 1u << 22;          // bounded waits (each try suspends ~0.2-1 us)

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
    for (int i = 0; i < NBAR; ++i)
      mbar_init(barrier_addr(i), (i >= BAR_HREADY0 && i < BAR_HREADY0 + NGRP) ? GWARPS : 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == ISSUER_WARP) {  // tensor memory for the two 128 x 256 FP32 accumulators
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(sbase + SM_MISC),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;

  // this CTA's tiles: blockIdx.x + k gridDim.x, k = 0 .. my - 1; tile k belongs to
  // epilogue group k % 2, and tiles 2p, 2p + 1 form pair p
  const int64_t ntiles = (a.n + TM - 1) / TM;
  const int64_t my = blockIdx.x < ntiles ? (ntiles - 1 - (int64_t)blockIdx.x) / gridDim.x + 1 : 0;

  if (warp == ISSUER_WARP) {
    if (lane == 0 && my > 0) {
      // weight stream: per pair, W1 for each of its tiles, then W2 for each, NCHUNK
      // chunks per tile and layer; chunk s sits in ring slot s % NSLOT
      const int64_t npairs = (my + 1) / 2;
      const int nt_last = (my & 1) ? 1 : 2;
      const int64_t full_chunks = (npairs - 1) * (4 * NCHUNK);
      const int64_t total = 2 * NCHUNK * my;
      auto chunk_src = [&](int64_t s) {
        const int nt = s < full_chunks ? 2 : nt_last;
        const int64_t u = s < full_chunks ? s % (4 * NCHUNK) : s - full_chunks;
        const int layer = (int)(u / (nt * NCHUNK));
        return a.Wpk + (layer ? kPackOffW2 : kPackOffW1) + (uint32_t)(u % NCHUNK) * kChunkBytes;
      };
      int64_t loaded = 0, used = 0;
      // issue every chunk whose slot is free (its previous chunk's MMAs are done)
      auto service = [&]() {
        while (loaded < total && loaded - used < NSLOT) {
          const int slot = (int)(loaded % NSLOT);
          if (loaded >= NSLOT && !mbar_test(barrier_addr(BAR_EMPTY0 + slot), (uint32_t)(((loaded - NSLOT) / NSLOT) & 1)))
            break;
          mbar_expect_tx(barrier_addr(BAR_FULL0 + slot), kChunkBytes);
          bulk_g2s(sbase + SM_WB + (uint32_t)slot * kChunkBytes, chunk_src(loaded), kChunkBytes,
                   barrier_addr(BAR_FULL0 + slot));
          ++loaded;
        }
      };
      // bounded wait that keeps the ring full meanwhile
      auto wait_serving = [&](int b, uint32_t parity) {
        for (uint32_t it = 0; it < kSpinLimit; ++it) {
          if (mbar_try(barrier_addr(b), parity, 200)) return true;
          service();
          if (*s_abort) return false;
        }
        return false;
      };
      mbar_expect_tx(barrier_addr(BAR_WRES), kW0Bytes + kW3Bytes);
      bulk_g2s(sbase + SM_W0, a.Wpk, kW0Bytes, barrier_addr(BAR_WRES));
      bulk_g2s(sbase + SM_W3, a.Wpk + kPackOffW3, kW3Bytes, barrier_addr(BAR_WRES));
      service();
      const uint32_t id_h = idesc_bf16(TM, kSurHidden), id_o = idesc_bf16(TM, kSurOut);
      uint32_t hr_ph[NGRP] = {0, 0};
      bool fail = false, wres = false, issued = false;
      for (int64_t p = 0; p < npairs && !fail; ++p) {
        const int nt = (2 * p + 1 < my) ? 2 : 1;
        for (int layer = 0; layer < kSurLayers && !fail; ++layer) {
          for (int x = 0; x < nt && !fail; ++x) {
            // the group's A operand is written and its accumulator read
            fail = !wait_serving(BAR_HREADY0 + x, hr_ph[x]);
            hr_ph[x] ^= 1u;
            if (fail) break;
            tc_fence_after();
            const uint32_t acc = tmem + (uint32_t)(x * kSurHidden);
            const uint32_t hA = sbase + SM_H + (uint32_t)x * kHBytes;
            if (layer == 0) {
              if (!wres) {
                fail = !wait_serving(BAR_WRES, 0);
                wres = true;
                if (fail) break;
              }
              mma_bf16_tc(acc, smem_desc(sbase + SM_X + (uint32_t)x * kXBytes, 128, 2 * 128),
                          smem_desc(sbase + SM_W0, 128, 2 * 128), id_h, 0);
            } else if (layer < 3) {
              for (int c = 0; c < NCHUNK; ++c) {
                const int slot = (int)(used % NSLOT);
                fail = !wait_serving(BAR_FULL0 + slot, (uint32_t)((used / NSLOT) & 1));
                if (fail) break;
                const uint32_t wb = sbase + SM_WB + (uint32_t)slot * kChunkBytes;
#pragma unroll
                for (int kk = 0; kk < KC / 16; ++kk) {
                  const uint32_t koff = (uint32_t)((c * KC + kk * 16) / 8) * 128;
                  mma_bf16_tc(acc, smem_desc(hA + koff, 128, (kSurHidden / 8) * 128),
                              smem_desc(wb + (uint32_t)(kk * 2) * 128, 128, (KC / 8) * 128), id_h,
                              (c > 0 || kk > 0) ? 1u : 0u);
                }
                mma_commit(barrier_addr(BAR_EMPTY0 + slot));
                ++used;
                service();
              }
              if (fail) break;
            } else {
#pragma unroll 1
              for (int kk = 0; kk < kSurHidden / 16; ++kk)
                mma_bf16_tc(acc, smem_desc(hA + (uint32_t)(kk * 2) * 128, 128, (kSurHidden / 8) * 128),
                            smem_desc(sbase + SM_W3 + (uint32_t)(kk * 2) * 128, 128, (kSurHidden / 8) * 128),
                            id_o, kk > 0 ? 1u : 0u);
            }
            mma_commit(barrier_addr(BAR_MMA0 + x));
            issued = true;
          }
        }
      }
      if (fail) {
        *s_abort = 1;
        if (a.err) atomicExch(a.err, 1);
      }
      // drain (bounded): the MMAs and copies this thread issued complete before the
      // tensor memory is freed and the CTA exits
      bool ok = true;
      if (issued) {
        mma_commit(barrier_addr(BAR_DRAIN));
        ok = mbar_wait(barrier_addr(BAR_DRAIN), 0);
      }
      for (int64_t s = used; s < loaded; ++s)
        ok = mbar_wait(barrier_addr(BAR_FULL0 + (int)(s % NSLOT)), (uint32_t)((s / NSLOT) & 1)) && ok;
      if (!wres) ok = mbar_wait(barrier_addr(BAR_WRES), 0) && ok;
      if (!ok && a.err) atomicExch(a.err, 1);
    }
  } else {
    // epilogue group g: tiles k = g, g + 2, ... of this CTA
    const int g = warp / GWARPS, q = warp & 3, ch = (warp % GWARPS) >> 2;
    const int gtid = tid - g * GWARPS * 32;
    const int row = q * 32 + lane;  // this thread's accumulator lane
    const uint32_t t_lane = tmem + (uint32_t)(g * kSurHidden) + ((uint32_t)(q * 32) << 16);
    const uint32_t sX32 = sbase + SM_X + (uint32_t)g * kXBytes;
    const uint32_t sH32 = sbase + SM_H + (uint32_t)g * kHBytes;
    const uint32_t b_mma = barrier_addr(BAR_MMA0 + g), b_ready = barrier_addr(BAR_HREADY0 + g);
    uint32_t mma_ph = 0;
    auto ready = [&]() {  // this warp's part of the next A operand is written
      fence_async_smem();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(b_ready);
    };
    auto wait_mma = [&]() {
      for (uint32_t it = 0; it < kSpinLimit; ++it) {
        if (mbar_try(b_mma, mma_ph, 1000)) {
          mma_ph ^= 1u;
          tc_fence_after();
          return true;
        }
        if (*s_abort) return false;
      }
      *s_abort = 1;
      if (a.err) atomicExch(a.err, 1);
      return false;
    };
    bool stop = false;
    for (int64_t k = g; k < my && !stop; k += NGRP) {
      const int64_t row0 = ((int64_t)blockIdx.x + k * gridDim.x) * TM;
      {  // features -> sX: thread t of the group writes row t / 2, columns (t % 2) * 8 ..
        const int r = gtid >> 1, c0 = (gtid & 1) * 8;
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
        uint32_t pk[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
          pk[i] = *reinterpret_cast<const uint32_t *>(&h2);
        }
        sts128(sX32 + core_off(r, c0, kSurIn), pk[0], pk[1], pk[2], pk[3]);
      }
      ready();
      for (int layer = 0; layer < kSurLayers; ++layer) {
        if (!wait_mma()) {
          stop = true;
          break;
        }
        if (layer < 3) {
          const uint32_t sB = sbase + SM_BIAS + (uint32_t)((layer * kSurHidden + ch * COLS_PER_WARP) * 4);
          const uint32_t tc = t_lane + (uint32_t)(ch * COLS_PER_WARP);
          auto emit = [&](const uint32_t(&r)[32], int c32) {
#pragma unroll
            for (int g4 = 0; g4 < 4; ++g4) {
              const float4 b0 = lds128(sB + (uint32_t)(c32 + g4 * 8) * 4);
              const float4 b1 = lds128(sB + (uint32_t)(c32 + g4 * 8 + 4) * 4);
              const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
              uint32_t pk[4];
#pragma unroll
              for (int i = 0; i < 4; ++i) {
                const int j = g4 * 8 + 2 * i;
                const __nv_bfloat162 h2 = __floats2bfloat162_rn(gelu_f(__uint_as_float(r[j]) + bv[2 * i]),
                                                                gelu_f(__uint_as_float(r[j + 1]) + bv[2 * i + 1]));
                pk[i] = *reinterpret_cast<const uint32_t *>(&h2);
              }
              sts128(sH32 + core_off(row, ch * COLS_PER_WARP + c32 + g4 * 8, kSurHidden), pk[0], pk[1], pk[2],
                     pk[3]);
            }
          };
          static_assert(COLS_PER_WARP == 128, "four 32-column chunks per warp");
          // each chunk's tensor-memory load overlaps the previous chunk's arithmetic
          uint32_t ra[32], rb[32];
          tmem_ld32_async(tc, ra);
          tmem_wait32(ra);
          tmem_ld32_async(tc + 32, rb);
          emit(ra, 0);
          tmem_wait32(rb);
          tmem_ld32_async(tc + 64, ra);
          emit(rb, 32);
          tmem_wait32(ra);
          tmem_ld32_async(tc + 96, rb);
          emit(ra, 64);
          tmem_wait32(rb);
          emit(rb, 96);
          ready();
        } else if (ch == 0) {
          float v[16];
          tmem_ld16(t_lane, v);
          if (row0 + row < a.n) {
            float4 *dst = reinterpret_cast<float4 *>(a.O + (row0 + row) * kSurOut);
            const float *bl = sbias + 3 * kSurHidden;
#pragma unroll
            for (int g4 = 0; g4 < 4; ++g4)
              dst[g4] = make_float4(v[4 * g4] + bl[4 * g4], v[4 * g4 + 1] + bl[4 * g4 + 1],
                                    v[4 * g4 + 2] + bl[4 * g4 + 2], v[4 * g4 + 3] + bl[4 * g4 + 3]);
          }
        }
      }
    }
  }
  // teardown: every MMA has completed (the groups waited for each one, or the issuing
  // thread drained them); the allocating warp frees the tensor memory
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == ISSUER_WARP) {
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
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
