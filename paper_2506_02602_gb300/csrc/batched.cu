// batched.cu -- ragged AMR-like batches in one persistent launch with work stealing.
//
// A batch is a set of boxes; box b owns the contiguous cells [off[b], off[b+1]) of the
// state and advances them through nsub[b] successive substeps of dt[b] (a subcycled
// level of Alg. 1 takes 2^l substeps of dt/2^l).  Per-cell cost is heavy-tailed: an
// ignition front needs ~100x the steps of inert gas.  The paper fills the GPU with large
// boxes and one stream per box (Sec. 4.1); here the whole batch is one launch:
//
//   1. k_probe: a stiffness key per cell -- the caller's cost hint (for example the
//      attempted steps of the previous call), or one right-hand side giving an
//      accuracy estimate (dt max|F| / tol)^(1/4) and a stability estimate
//      dt max_k (consumption rate of k / c_k) / 3 -- times the box's substeps, binned
//      into half-octave buckets with a block histogram;
//   2. k_scan + k_scatter: a counting sort of the cell indices into descending-cost
//      order (warp-aggregated atomics per bucket);
//   3. k_lsrk_persistent: one CTA set sized to the resident capacity; every iteration of
//      its loop is one attempted RK step for each lane's current cell, so lanes stay
//      converged inside the right-hand side; a lane whose cell finishes (all substeps)
//      stores it and takes the next cell from the queue through one warp-aggregated
//      atomicAdd on a global cursor.  Expensive cells start first, so the tail is short.
//
// The per-cell arithmetic is cell.cuh, identical to the one-pass kernel, so results
// do not depend on the processing order.  No CTA ever waits on another: a CTA that finds
// the queue empty exits.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "cell.cuh"
#include "internal.cuh"

namespace chem {

__device__ __forceinline__ int find_box(const int64_t *off, int nb, int64_t i) {
  int lo = 0, hi = nb;  // off[lo] <= i < off[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= i) lo = mid; else hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(128) k_probe(const __grid_constant__ MechTables mt,
                                               const BatchArgs a, double rtol, double atol,
                                               uint8_t *__restrict__ bucket,
                                               int32_t *__restrict__ hist) {
  __shared__ int sh[kBatchBuckets];
  load_math_tables();
  for (int t = threadIdx.x; t < kBatchBuckets; t += blockDim.x) sh[t] = 0;
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < a.n) {
    const int b = find_box(a.box_off, a.nboxes, i);
    const double dt = a.box_dt[b];
    double key = 1.0;
    if (a.cost_hint) {
      key = (double)max(a.cost_hint[i], 1);
    } else {
      const double rho = a.rho[i];
      double Y[NSP], yw[NSP], T = a.T[i];
#pragma unroll
      for (int k = 0; k < NSP; ++k) {
        Y[k] = a.Y[k * a.ld + i];
        yw[k] = Y[k] * mt.invW[k];
      }
      if (isfinite(rho) && rho > 0.0 && solve_T(mt, Y, a.e[i] / R_U, T)) {
        double c[NSP], wdot[NSP], dflux[NSP];
#pragma unroll
        for (int k = 0; k < NSP; ++k) c[k] = fmax(rho * yw[k], 0.0);
        production_rates<true>(mt, T, c, wdot, dflux);
        double acc = 0.0, stab = 0.0;
#pragma unroll
        for (int k = 0; k < NSP; ++k) {
          const double F = wdot[k] * mt.W[k] / rho;
          acc = fmax(acc, fabs(F) * dt / (rtol * fabs(Y[k]) + atol));
          if (c[k] > 1e-30) stab = fmax(stab, dflux[k] / c[k] * dt);
        }
        key = fmax(1.0, fmax(sqrt(sqrt(acc)), stab * (1.0 / 3.0)));
        if (!isfinite(key)) key = 1.0;
      }
      key *= (double)a.box_nsub[b];
    }
    const int bk = min(kBatchBuckets - 1, max(0, (int)(2.0f * log2f((float)key))));
    bucket[i] = (uint8_t)bk;
    atomicAdd(&sh[bk], 1);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < kBatchBuckets; t += blockDim.x)
    if (sh[t]) atomicAdd(&hist[t], sh[t]);
}

// Exclusive scan of the bucket counts in descending-cost order; resets the cursor.
__global__ void k_scan(int32_t *hist, unsigned long long *cursor) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    int run = 0;
    for (int b = kBatchBuckets - 1; b >= 0; --b) {
      const int cnt = hist[b];
      hist[b] = run;
      run += cnt;
    }
    *cursor = 0ull;
  }
}

__global__ void k_scatter(int64_t n, const uint8_t *__restrict__ bucket, int32_t *offs,
                          int32_t *__restrict__ order) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = i < n;
  const int bk = live ? bucket[i] : -1;
  const unsigned mask = __ballot_sync(0xffffffffu, live);
  if (!live) return;
  // lanes with the same bucket share one atomicAdd
  const unsigned peers = __match_any_sync(mask, bk);
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(peers) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(&offs[bk], __popc(peers));
  base = __shfl_sync(peers, base, leader);
  order[base + __popc(peers & ((1u << lane) - 1u))] = (int32_t)i;
}

// The persistent kernel is compiled in several shapes (threads per CTA, minimum
// resident CTAs per SM); the second number caps the registers per thread at
// 65536 / (block * minb), trading registers (and spills) against resident warps.  The
// autotuner picks among them.  Every shape runs the same algorithm, but the compiler
// contracts multiply-adds per compiled kernel, so shapes agree to rounding, not bit for
// bit; shape 0 (no register cap) compiles like the one-pass kernel.
template <int V, int BLOCK, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB) k_lsrk_persistent(const __grid_constant__ MechTables mt,
                                                                 const BatchArgs a, const StepParams p,
                                                                 const int32_t *__restrict__ order,
                                                                 unsigned long long *cursor) {
  load_math_tables();
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  CellState c;
  c.done = true;
  c.nacc = c.nrej = c.nrhs = 0;
  c.status = CHEM_CELL_OK;
  int64_t cell = -1;
  int sub_left = 0;
  bool need = true;
  int done_cells = 0, tot_acc = 0, tot_rej = 0, tot_rhs = 0, max_steps = 0;
  int hist[6] = {0, 0, 0, 0, 0, 0};
  const unsigned long long nq = a.nq_dev ? (unsigned long long)*a.nq_dev : (unsigned long long)a.n;
  for (;;) {
    const unsigned needmask = __ballot_sync(FULL, need);
    if (needmask) {
      const int leader = __ffs(needmask) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(cursor, (unsigned long long)__popc(needmask));
      base = __shfl_sync(FULL, base, leader);
      if (need) {
        need = false;
        const unsigned long long slot = base + __popc(needmask & ((1u << lane) - 1u));
        if (slot < nq) {
          cell = order ? (int64_t)order[slot] : (int64_t)slot;
          const int b = find_box(a.box_off, a.nboxes, cell);
          sub_left = a.box_nsub[b];
#pragma unroll
          for (int k = 0; k < NSP; ++k) c.X[k] = a.Y[k * a.ld + cell];
          c.T = a.T[cell];
          c.h = a.h ? a.h[cell] : CUDART_NAN;
          c.nacc = c.nrej = c.nrhs = 0;
          cell_begin(c, a.rho[cell], a.e[cell], a.box_dt[b]);
        } else {
          cell = -1;
        }
      }
    }
    if (__ballot_sync(FULL, cell >= 0) == 0) break;
    if (cell >= 0) {
      if (!c.done) cell_attempt<V>(mt, c, p);
      if (c.done) {
        if (c.status == CHEM_CELL_OK && --sub_left > 0) {
          c.t = 0.0;  // next substep from the current state; h and the T guess carry
          c.done = false;
        } else {
          cell_finish(mt, c);
#pragma unroll
          for (int k = 0; k < NSP; ++k) a.Y[k * a.ld + cell] = c.X[k];
          a.T[cell] = c.T;
          if (a.h) a.h[cell] = c.h;
          if (a.status) a.status[cell] = c.status == CHEM_CELL_OK ? a.ok_status : c.status;
          if (a.nsteps) a.nsteps[cell] = c.nacc + c.nrej;
          ++done_cells;
          tot_acc += c.nacc;
          tot_rej += c.nrej;
          tot_rhs += c.nrhs;
          max_steps = max(max_steps, c.nacc + c.nrej);
          const int hs = c.status == CHEM_CELL_OK ? a.ok_status : c.status;
          if (hs >= 0 && hs < 6) ++hist[hs];
          cell = -1;
          need = true;
        }
      }
    }
  }
  if (a.stats) accumulate_stats(a.stats, done_cells, tot_acc, tot_rej, tot_rhs, max_steps, hist);
}

// Threads per CTA of each shape; shape 0 is the default.  Resident CTAs per SM: 2, 3, 4,
// 6, 8 (16 for the mixed variant of the 9-species structure: 32 warps at 64 registers,
// spilling to L1, which hides the FP64 pipe's latency by warps rather than registers),
// 2.
static constexpr int kShapeBlock[CHEM_BATCH_SHAPES] = {128, 128, 128, 64, 64, 256};
template <int V>
constexpr int kMinB4 = (V == CHEM_VARIANT_MIXED && NSP <= 9) ? 16 : 8;

template <int V>
static const void *persistent_fn(int shape) {
  switch (shape) {
    case 1: return reinterpret_cast<const void *>(k_lsrk_persistent<V, 128, 3>);
    case 2: return reinterpret_cast<const void *>(k_lsrk_persistent<V, 128, 4>);
    case 3: return reinterpret_cast<const void *>(k_lsrk_persistent<V, 64, 6>);
    case 4: return reinterpret_cast<const void *>(k_lsrk_persistent<V, 64, kMinB4<V>>);
    case 5: return reinterpret_cast<const void *>(k_lsrk_persistent<V, 256, 2>);
    default: return reinterpret_cast<const void *>(k_lsrk_persistent<V, 128, 2>);
  }
}
static_assert(CHEM_BATCH_SHAPES == 6, "persistent_fn lists every shape");

static const void *persistent_kernel(int variant, int shape) {
  return variant == CHEM_VARIANT_MIXED ? persistent_fn<CHEM_VARIANT_MIXED>(shape)
                                       : persistent_fn<CHEM_VARIANT_FP64>(shape);
}

// Resident CTAs per SM and registers per thread of every (variant, shape), per device
// ordinal (looked up once; 0 = not yet).
static int g_persist_ctas[16][2][CHEM_BATCH_SHAPES];
static int g_persist_regs[16][2][CHEM_BATCH_SHAPES];

cudaError_t persistent_shape(int variant, int shape, int *block, int *ctas_per_sm, int *regs, int *num_sms) {
  if (shape < 0 || shape >= CHEM_BATCH_SHAPES) return cudaErrorInvalidValue;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int v = variant == CHEM_VARIANT_MIXED ? 1 : 0;
  const int d = dev >= 0 && dev < 16 ? dev : -1;
  if (d < 0 || g_persist_ctas[d][v][shape] == 0) {
    const void *fn = persistent_kernel(variant, shape);
    int per = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kShapeBlock[shape], 0);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa{};
    e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return e;
    if (d < 0) {
      *ctas_per_sm = per > 0 ? per : 1;
      *regs = fa.numRegs;
      *block = kShapeBlock[shape];
      return cudaSuccess;
    }
    g_persist_regs[d][v][shape] = fa.numRegs;
    g_persist_ctas[d][v][shape] = per > 0 ? per : 1;
  }
  *ctas_per_sm = g_persist_ctas[d][v][shape];
  *regs = g_persist_regs[d][v][shape];
  *block = kShapeBlock[shape];
  return cudaSuccess;
}

template <int V, int B, int M>
static void launch_persistent_t(unsigned grid, cudaStream_t st, const MechTables &mt, const BatchArgs &a,
                                const StepParams &p, const int32_t *order, unsigned long long *cursor) {
  k_lsrk_persistent<V, B, M><<<grid, B, 0, st>>>(mt, a, p, order, cursor);
}

template <int V>
static void launch_persistent(int shape, unsigned grid, cudaStream_t st, const MechTables &mt,
                              const BatchArgs &a, const StepParams &p, const int32_t *order,
                              unsigned long long *cursor) {
  switch (shape) {
    case 1: launch_persistent_t<V, 128, 3>(grid, st, mt, a, p, order, cursor); break;
    case 2: launch_persistent_t<V, 128, 4>(grid, st, mt, a, p, order, cursor); break;
    case 3: launch_persistent_t<V, 64, 6>(grid, st, mt, a, p, order, cursor); break;
    case 4: launch_persistent_t<V, 64, kMinB4<V>>(grid, st, mt, a, p, order, cursor); break;
    case 5: launch_persistent_t<V, 256, 2>(grid, st, mt, a, p, order, cursor); break;
    default: launch_persistent_t<V, 128, 2>(grid, st, mt, a, p, order, cursor); break;
  }
}

cudaError_t launch_persistent_queue(int variant, const MechTables &mt, const BatchArgs &a,
                                    const StepParams &p, const int32_t *order,
                                    unsigned long long *cursor, cudaStream_t st) {
  if (a.n <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(cursor, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  // the fastest shape of each variant on the ragged AMR batch: the default for fp64, the
  // 32-warp shape 4 for mixed (127 ms against 137.5 for the default)
  const int shape = variant == CHEM_VARIANT_MIXED ? 4 : 0;
  int sms = 0, pblock = 0, per = 0, regs = 0;
  e = persistent_shape(variant, shape, &pblock, &per, &regs, &sms);
  if (e != cudaSuccess) return e;
  const int64_t cap_ctas = (int64_t)sms * per, need = (a.n + pblock - 1) / pblock;
  const unsigned grid = (unsigned)(cap_ctas < need ? cap_ctas : need);
  if (variant == CHEM_VARIANT_MIXED)
    launch_persistent<CHEM_VARIANT_MIXED>(shape, grid, st, mt, a, p, order, cursor);
  else
    launch_persistent<CHEM_VARIANT_FP64>(shape, grid, st, mt, a, p, order, cursor);
  return cudaGetLastError();
}

cudaError_t launch_batched(int variant, const MechTables &mt, const BatchArgs &a,
                           const StepParams &p, const BatchScratch &s, int order_mode,
                           int ctas_per_sm, int shape, cudaStream_t st) {
  if (a.n <= 0) return cudaSuccess;
  const int block = 128;  // of the probe and scatter kernels
  const unsigned grid_cells = (unsigned)((a.n + block - 1) / block);
  cudaError_t e;
  const int32_t *order = nullptr;
  if (order_mode == CHEM_ORDER_STIFFNESS) {
    e = cudaMemsetAsync(s.hist, 0, kBatchBuckets * sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    k_probe<<<grid_cells, block, 0, st>>>(mt, a, p.rtol, p.atol, s.bucket, s.hist);
    k_scan<<<1, 32, 0, st>>>(s.hist, s.cursor);
    k_scatter<<<grid_cells, block, 0, st>>>(a.n, s.bucket, s.hist, s.order);
    order = s.order;
  } else {
    e = cudaMemsetAsync(s.cursor, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
  }
  int sms = 0, pblock = 0, cap = 0, regs = 0;
  e = persistent_shape(variant, shape, &pblock, &cap, &regs, &sms);
  if (e != cudaSuccess) return e;
  const int per = (ctas_per_sm > 0 && ctas_per_sm < cap) ? ctas_per_sm : cap;
  const int64_t cap_ctas = (int64_t)sms * per;
  const int64_t need = (a.n + pblock - 1) / pblock;
  const unsigned grid = (unsigned)(cap_ctas < need ? cap_ctas : need);
  if (variant == CHEM_VARIANT_MIXED)
    launch_persistent<CHEM_VARIANT_MIXED>(shape, grid, st, mt, a, p, order, s.cursor);
  else
    launch_persistent<CHEM_VARIANT_FP64>(shape, grid, st, mt, a, p, order, s.cursor);
  return cudaGetLastError();
}

}  // namespace chem

// ------------------------------------------------------------------------------------
// Allocation-free variant of chem_integrate_batched.
//
// Some callers cannot allocate device memory at the moment they integrate: host solvers
// whose memory arena has already claimed the GPU's memory and forbids allocations made
// behind its back, and time-critical loops that cannot afford cudaMalloc's latency and
// implicit synchronisation.  For them the queue scratch of the batched path lives in the
// fixed array below, which every GPU that loads this library keeps until the process
// exits.  Only host code needs its device address, taken with cudaGetSymbolAddress with
// the caller's device current: the array's name in host code is a stand-in, not an
// address a kernel can use.
namespace chem {

constexpr int64_t kNoAllocMaxCells = 1 << 20;  // 1,048,576 cells: 5 MiB + 512 B of scratch
// layout: cursor at 0, bucket counts at 256, queue order at 512, buckets after the order
static __device__ __align__(256) unsigned char g_noalloc_scratch[512 + kNoAllocMaxCells * 5];

// Device address of the fixed scratch in the current device's context.  It is looked up
// on every call rather than cached: a device reset or a re-created primary context loads
// the module again at another address, and a cached pointer would then be stale.  The
// first lookup in a context loads the module (allocating nothing the caller sees); later
// ones are a table lookup in the runtime.
static cudaError_t noalloc_scratch(void **addr) {
  *addr = nullptr;
  return cudaGetSymbolAddress(addr, g_noalloc_scratch);
}

}  // namespace chem

extern "C" int chem_integrate_batched_noalloc(chem_ctx *ctx, const chem_state *state,
                                              int64_t ncells, const chem_batch *batch,
                                              double rtol, double atol,
                                              const chem_batch_options *opt, void *stream,
                                              chem_stats *d_stats) {
  using namespace chem;
  // the same argument rules and messages as chem_integrate_batched, then the size limit
  chem_batch_options o{};
  int rc = check_batched_call(ctx, state, ncells, batch, rtol, atol, opt, &o);
  if (rc) return rc;
  std::string &err = chem_ctx_error(ctx);
  if (ncells > kNoAllocMaxCells) {
    err = "chem_integrate_batched_noalloc holds at most 1048576 cells (fixed scratch); got " +
          std::to_string(ncells) + ": split the batch or use chem_integrate_batched";
    return CHEM_ERR_INVALID;
  }
  void *base = nullptr;
  cudaError_t e = noalloc_scratch(&base);
  if (e != cudaSuccess || !base) {
    err = std::string("looking up the fixed scratch: ") + cudaGetErrorString(e);
    return CHEM_ERR_CUDA;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (d_stats) {
    e = cudaMemsetAsync(d_stats, 0, sizeof(chem_stats), s);
    if (e != cudaSuccess) {
      err = std::string("clearing stats: ") + cudaGetErrorString(e);
      return CHEM_ERR_CUDA;
    }
  }
  if (ncells == 0) return CHEM_OK;
  char *b = static_cast<char *>(base);
  BatchScratch sc;
  sc.cursor = reinterpret_cast<unsigned long long *>(b);
  sc.hist = reinterpret_cast<int32_t *>(b + 256);
  sc.order = reinterpret_cast<int32_t *>(b + 512);
  sc.bucket = reinterpret_cast<uint8_t *>(b + 512 + kNoAllocMaxCells * sizeof(int32_t));
  BatchArgs a{state->d_rho, state->d_e, state->d_Y, state->ldY, state->d_T, state->d_h,
              state->d_status, state->d_nsteps, ncells, batch->d_box_offset, batch->d_box_dt,
              batch->d_box_nsub, batch->nboxes, o.d_cost_hint, d_stats,
              /*nq_dev=*/nullptr, /*ok_status=*/CHEM_CELL_OK};
  StepParams p{0.0, rtol, atol, chem_ctx_max_steps(ctx)};
  // launch_batched clears the bucket counts (cudaMemsetAsync) and resets the cursor
  // (k_scan, or cudaMemsetAsync in natural order) before the kernels read them
  e = launch_batched(chem_ctx_variant(ctx), chem_ctx_tables(ctx), a, p, sc, o.order,
                     o.ctas_per_sm, o.shape, s);
  if (e != cudaSuccess) {
    err = std::string("batched launch: ") + cudaGetErrorString(e);
    return CHEM_ERR_CUDA;
  }
  return CHEM_OK;
}
