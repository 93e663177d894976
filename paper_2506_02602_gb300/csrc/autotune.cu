// autotune.cu -- launch-shape information and the autotuner of chem_integrate_batched.
//
// The tuner times candidate options on the caller's own batch, integrating private
// copies of the mutable state so that the caller's buffers stay as they were, and walks
// the option space by coordinate descent: kernel shape (threads per CTA and register
// cap), queue order, resident CTAs per SM, CUDA-graph replay.  Results can be kept in a
// plain-text cache keyed by the device and the problem's size class, so a production run
// tunes once per (device, variant, tolerances, size class).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "internal.cuh"

namespace chem {
namespace {

int tune_fail(chem_ctx *ctx, int code, const std::string &msg) {
  chem_ctx_error(ctx) = msg;
  return code;
}

int floor_log2(int64_t v) {
  int l = 0;
  while (v > 1) {
    v >>= 1;
    ++l;
  }
  return l;
}

// Cache key: device name (spaces as '_'), SM count, variant, max_steps, rtol, atol,
// floor(log2 ncells), floor(log2 nboxes).
std::string tune_key(chem_ctx *ctx, double rtol, double atol, int64_t ncells, int64_t nboxes) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop{};
  cudaGetDeviceProperties(&prop, dev);
  std::string name = prop.name;
  for (char &c : name)
    if (c == ' ' || c == '\t') c = '_';
  char buf[512];
  std::snprintf(buf, sizeof buf, "%s %d %d %d %.6e %.6e %d %d", name.c_str(), prop.multiProcessorCount,
                chem_ctx_variant(ctx), (int)chem_ctx_max_steps(ctx), rtol, atol, floor_log2(ncells),
                floor_log2(nboxes));
  return buf;
}

// Looks the key up; a line is "<key> | <order> <ctas_per_sm> <use_graph> <shape>".
bool cache_lookup(const char *path, const std::string &key, chem_batch_options *o) {
  FILE *f = std::fopen(path, "r");
  if (!f) return false;
  char line[1024];
  bool hit = false;
  while (std::fgets(line, sizeof line, f)) {
    const char *bar = std::strstr(line, " | ");
    if (!bar || (size_t)(bar - line) != key.size() || std::strncmp(line, key.c_str(), key.size()) != 0) continue;
    int order, ctas, graph, shape;
    if (std::sscanf(bar + 3, "%d %d %d %d", &order, &ctas, &graph, &shape) != 4) continue;
    if ((order != CHEM_ORDER_STIFFNESS && order != CHEM_ORDER_NATURAL) || ctas < 0 || shape < 0 ||
        shape >= CHEM_BATCH_SHAPES)
      continue;
    o->order = order;
    o->ctas_per_sm = ctas;
    o->use_graph = graph != 0;
    o->shape = shape;
    hit = true;  // the last valid line for the key wins
  }
  std::fclose(f);
  return hit;
}

bool cache_append(const char *path, const std::string &key, const chem_batch_options &o) {
  FILE *f = std::fopen(path, "a");
  if (!f) return false;
  const bool ok = std::fprintf(f, "%s | %d %d %d %d\n", key.c_str(), o.order, o.ctas_per_sm, o.use_graph,
                               o.shape) > 0;
  return std::fclose(f) == 0 && ok;
}

}  // namespace
}  // namespace chem

using namespace chem;

extern "C" {

int chem_batch_shape_info(chem_ctx *ctx, int32_t shape, int32_t *block, int32_t *regs, int32_t *ctas_per_sm) {
  if (!ctx) return CHEM_ERR_INVALID;
  if (shape < 0 || shape >= CHEM_BATCH_SHAPES)
    return tune_fail(ctx, CHEM_ERR_INVALID, "shape out of range");
  int b = 0, per = 0, r = 0, sms = 0;
  const cudaError_t e = persistent_shape(chem_ctx_variant(ctx), shape, &b, &per, &r, &sms);
  if (e != cudaSuccess) return tune_fail(ctx, CHEM_ERR_CUDA, std::string("shape query: ") + cudaGetErrorString(e));
  if (block) *block = b;
  if (regs) *regs = r;
  if (ctas_per_sm) *ctas_per_sm = per;
  return CHEM_OK;
}

int chem_autotune_batched(chem_ctx *ctx, const chem_state *state, int64_t ncells, const chem_batch *batch,
                          double rtol, double atol, const chem_batch_options *base, const char *cache_path,
                          void *stream, chem_batch_options *best, chem_tune_result *h_results,
                          int32_t max_results, int32_t *n_results) {
  if (!ctx) return CHEM_ERR_INVALID;
  if (n_results) *n_results = 0;
  if (!best || !state || ncells <= 0 || !batch || batch->nboxes < 1)
    return tune_fail(ctx, CHEM_ERR_INVALID, "autotune needs best, a state, ncells > 0 and a batch");
  if (!state->d_rho || !state->d_e || !state->d_Y || !state->d_T || state->ldY < ncells)
    return tune_fail(ctx, CHEM_ERR_INVALID, "rho, e, Y and T are required and ldY >= ncells");
  if (max_results < 0 || (max_results > 0 && !h_results))
    return tune_fail(ctx, CHEM_ERR_INVALID, "h_results is required when max_results > 0");
  if (chem_ctx_scheme(ctx) != CHEM_SCHEME_LSRK)
    return tune_fail(ctx, CHEM_ERR_UNSUPPORTED, "the batched integrator runs the two-register scheme only");
  chem_batch_options b0{};
  if (base) b0 = *base;
  const std::string key = tune_key(ctx, rtol, atol, ncells, batch->nboxes);
  if (cache_path) {
    chem_batch_options o = b0;
    if (cache_lookup(cache_path, key, &o)) {
      *best = o;
      return CHEM_OK;
    }
  }
  cudaStream_t st = (cudaStream_t)stream;
  // private copies of the state the integration modifies
  double *Y = nullptr, *T = nullptr, *h = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  auto release = [&]() {
    cudaFree(Y);
    cudaFree(T);
    cudaFree(h);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
  };
  cudaError_t e = cudaMalloc(&Y, (size_t)NSP * ncells * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&T, (size_t)ncells * sizeof(double));
  if (e == cudaSuccess && state->d_h) e = cudaMalloc(&h, (size_t)ncells * sizeof(double));
  if (e == cudaSuccess) e = cudaEventCreate(&ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&ev1);
  if (e != cudaSuccess) {
    release();
    return tune_fail(ctx, CHEM_ERR_NOMEM, std::string("autotune copies: ") + cudaGetErrorString(e));
  }
  chem_state trial = *state;
  trial.d_Y = Y;
  trial.ldY = ncells;
  trial.d_T = T;
  trial.d_h = h;
  trial.d_status = nullptr;
  trial.d_nsteps = nullptr;
  auto restore = [&]() -> cudaError_t {
    cudaError_t r = cudaMemcpy2DAsync(Y, ncells * sizeof(double), state->d_Y, state->ldY * sizeof(double),
                                      ncells * sizeof(double), NSP, cudaMemcpyDeviceToDevice, st);
    if (r == cudaSuccess) r = cudaMemcpyAsync(T, state->d_T, ncells * sizeof(double), cudaMemcpyDeviceToDevice, st);
    if (r == cudaSuccess && h) r = cudaMemcpyAsync(h, state->d_h, ncells * sizeof(double), cudaMemcpyDeviceToDevice, st);
    return r;
  };
  std::vector<chem_tune_result> all;
  int rc = CHEM_OK;
  // best of two timed launches after one untimed one; < 0 on failure (rc set)
  auto run = [&](const chem_batch_options &o) -> float {
    float bestms = -1.0f;
    for (int rep = 0; rep < 3; ++rep) {
      cudaError_t r = restore();
      if (r == cudaSuccess) r = cudaEventRecord(ev0, st);
      if (r != cudaSuccess) {
        rc = tune_fail(ctx, CHEM_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(r));
        return -1.0f;
      }
      const int c = chem_integrate_batched(ctx, &trial, ncells, batch, rtol, atol, &o, stream, nullptr);
      if (c != CHEM_OK) {
        rc = c;
        return -1.0f;
      }
      r = cudaEventRecord(ev1, st);
      if (r == cudaSuccess) r = cudaEventSynchronize(ev1);
      float ms = 0.0f;
      if (r == cudaSuccess) r = cudaEventElapsedTime(&ms, ev0, ev1);
      if (r != cudaSuccess) {
        rc = tune_fail(ctx, CHEM_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(r));
        return -1.0f;
      }
      if (rep > 0 && (bestms < 0.0f || ms < bestms)) bestms = ms;
    }
    chem_tune_result t{};
    t.opt = o;
    t.ms = bestms;
    int blk = 0, per = 0, regs = 0, sms = 0;
    if (persistent_shape(chem_ctx_variant(ctx), o.shape, &blk, &per, &regs, &sms) == cudaSuccess) {
      t.block = blk;
      t.regs = regs;
      t.ctas_per_sm = (o.ctas_per_sm > 0 && o.ctas_per_sm < per) ? o.ctas_per_sm : per;
    }
    all.push_back(t);
    return bestms;
  };
  chem_batch_options cur = b0;
  cur.order = CHEM_ORDER_STIFFNESS;
  cur.ctas_per_sm = 0;
  cur.use_graph = 0;
  float cur_ms = -1.0f;
  // 1. shape
  for (int s = 0; s < CHEM_BATCH_SHAPES && rc == CHEM_OK; ++s) {
    chem_batch_options o = cur;
    o.shape = s;
    const float ms = run(o);
    if (ms >= 0.0f && (cur_ms < 0.0f || ms < cur_ms)) {
      cur_ms = ms;
      cur = o;
    }
  }
  // 2. queue order
  if (rc == CHEM_OK) {
    chem_batch_options o = cur;
    o.order = CHEM_ORDER_NATURAL;
    const float ms = run(o);
    if (ms >= 0.0f && ms < cur_ms) {
      cur_ms = ms;
      cur = o;
    }
  }
  // 3. fewer resident CTAs per SM than fit
  if (rc == CHEM_OK) {
    int blk = 0, per = 0, regs = 0, sms = 0;
    if (persistent_shape(chem_ctx_variant(ctx), cur.shape, &blk, &per, &regs, &sms) == cudaSuccess) {
      const chem_batch_options fixed = cur;
      for (int c = 1; c < per && rc == CHEM_OK; ++c) {
        chem_batch_options o = fixed;
        o.ctas_per_sm = c;
        const float ms = run(o);
        if (ms >= 0.0f && ms < cur_ms) {
          cur_ms = ms;
          cur = o;
        }
      }
    }
  }
  // 4. graph replay
  if (rc == CHEM_OK) {
    chem_batch_options o = cur;
    o.use_graph = 1;
    const float ms = run(o);
    if (ms >= 0.0f && ms < cur_ms) {
      cur_ms = ms;
      cur = o;
    }
  }
  cudaStreamSynchronize(st);
  release();
  if (rc != CHEM_OK) return rc;
  *best = cur;
  const int32_t nres = (int32_t)all.size() < max_results ? (int32_t)all.size() : max_results;
  for (int32_t i = 0; i < nres; ++i) h_results[i] = all[(size_t)i];
  if (n_results) *n_results = (int32_t)all.size();
  if (cache_path && !cache_append(cache_path, key, cur))
    return tune_fail(ctx, CHEM_ERR_INVALID, std::string("cannot append to the tuning cache ") + cache_path);
  return CHEM_OK;
}

}  // extern "C"
