// surrogate.cu -- the learned surrogate's host side: parameters and Adam state, the
// training loop (featurise -> statistics -> per-epoch shuffled batches -> forward ->
// MSE -> backward -> Adam), chunked inference (featurise -> four GEMM layers -> the
// epilogue with projection, temperature solve and gate -> integrator fallback of the
// rejected cells through an index list), save/load, and the entry points of chem.h.
//
// All arithmetic runs in the kernels of mlp.cu and surrogate_kernels.cu; this file
// allocates, sequences launches on the caller's stream and keeps the host copies of
// the normalisation constants.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "internal.cuh"
#include "mlp.cuh"
#include "surrogate.cuh"

namespace chem {

struct Surrogate {
  // parameters (fp32 master, flat), gradients, Adam moments
  float *param = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
  // bf16 shadows per layer: W [N x K] and its transpose [K x N]
  __nv_bfloat16 *W[kSurLayers] = {}, *WT[kSurLayers] = {};
  int64_t off_W[kSurLayers], off_b[kSurLayers];
  bool ready = false;
  int64_t step = 0;
  // normalisation (host copies; device copies in dev_norm)
  float fmean[kSurIn], fistd[kSurIn], fmin[kSurFeat], fmax[kSurFeat];
  float tmean[kSurOut], tistd[kSurOut];
  float *dev_norm = nullptr;  // fmean[16], fistd[16], tmean[16], tistd[16]
  double lam = 0.1;
  double dt_power = 0.0;
  // inference scratch
  int64_t chunk_cap = 0;
  float *Xraw = nullptr, *O = nullptr;
  uint8_t *Tok = nullptr;
  int64_t fb_cap = 0;
  int32_t *fb_idx = nullptr;
  unsigned int *fb_count = nullptr;
  // the weights in the tensor-core kernel's layout (repacked when the weights change)
  unsigned char *Wpk = nullptr;
  bool packed = false;
  // the fallback's one-box batch and queue cursor (persistent work-stealing kernel)
  int64_t *box_off = nullptr;
  double *box_dt = nullptr;
  int32_t *box_nsub = nullptr;
  unsigned long long *cursor = nullptr;
  int *tc_err = nullptr;  // error word of the tensor-core kernel (a wait ran out)
  // per-box substep counts of one round of the batched inference (all 1)
  int32_t *ones = nullptr;
  int64_t ones_cap = 0;
};

static void free_surrogate(Surrogate *s) {
  if (!s) return;
  cudaFree(s->param);
  cudaFree(s->grad);
  cudaFree(s->m);
  cudaFree(s->v);
  for (int l = 0; l < kSurLayers; ++l) {
    cudaFree(s->W[l]);
    cudaFree(s->WT[l]);
  }
  cudaFree(s->dev_norm);
  cudaFree(s->Xraw);
  cudaFree(s->O);
  cudaFree(s->Tok);
  cudaFree(s->fb_idx);
  cudaFree(s->fb_count);
  cudaFree(s->Wpk);
  cudaFree(s->tc_err);
  cudaFree(s->box_off);
  cudaFree(s->box_dt);
  cudaFree(s->box_nsub);
  cudaFree(s->cursor);
  cudaFree(s->ones);
  delete s;
}

void surrogate_destroy(void *p) { free_surrogate(static_cast<Surrogate *>(p)); }

// splitmix64: seeded, platform-independent random numbers for init and shuffling
struct Rng {
  uint64_t s;
  uint64_t next() {
    uint64_t z = (s += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
  }
  double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
  double normal() {  // Box-Muller
    const double u1 = uniform() + 1e-300, u2 = uniform();
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
  }
};

#define SCHK(call)                                  \
  do {                                              \
    cudaError_t e_ = (call);                        \
    if (e_ != cudaSuccess) return e_;               \
  } while (0)

static cudaError_t alloc_params(Surrogate *s) {
  int64_t o = 0;
  for (int l = 0; l < kSurLayers; ++l) {
    s->off_W[l] = o;
    o += (int64_t)kSurN[l] * kSurK[l];
    s->off_b[l] = o;
    o += kSurN[l];
  }
  const size_t bytes = (size_t)kSurParams * sizeof(float);
  SCHK(cudaMalloc(&s->param, bytes));
  SCHK(cudaMalloc(&s->grad, bytes));
  SCHK(cudaMalloc(&s->m, bytes));
  SCHK(cudaMalloc(&s->v, bytes));
  for (int l = 0; l < kSurLayers; ++l) {
    SCHK(cudaMalloc(&s->W[l], (size_t)kSurN[l] * kSurK[l] * sizeof(__nv_bfloat16)));
    SCHK(cudaMalloc(&s->WT[l], (size_t)kSurN[l] * kSurK[l] * sizeof(__nv_bfloat16)));
  }
  SCHK(cudaMalloc(&s->dev_norm, 4 * 16 * sizeof(float)));
  SCHK(cudaMalloc(&s->fb_count, sizeof(unsigned int)));
  SCHK(cudaMalloc(&s->Wpk, packed_weight_bytes()));
  SCHK(cudaMalloc(&s->tc_err, sizeof(int)));
  SCHK(cudaMalloc(&s->box_off, 2 * sizeof(int64_t)));
  SCHK(cudaMalloc(&s->box_dt, sizeof(double)));
  SCHK(cudaMalloc(&s->box_nsub, sizeof(int32_t)));
  SCHK(cudaMalloc(&s->cursor, sizeof(unsigned long long)));
  SCHK(cudaMemset(s->tc_err, 0, sizeof(int)));
  return cudaSuccess;
}

// Upload host parameters, reset Adam, refresh the bf16 shadows (an Adam step with zero
// learning rate and zero gradient writes them).
static cudaError_t set_params(Surrogate *s, const float *h, cudaStream_t st) {
  const size_t bytes = (size_t)kSurParams * sizeof(float);
  SCHK(cudaMemcpyAsync(s->param, h, bytes, cudaMemcpyHostToDevice, st));
  SCHK(cudaMemsetAsync(s->m, 0, bytes, st));
  SCHK(cudaMemsetAsync(s->v, 0, bytes, st));
  SCHK(cudaMemsetAsync(s->grad, 0, bytes, st));
  for (int l = 0; l < kSurLayers; ++l)
    SCHK(launch_adam((int64_t)kSurN[l] * kSurK[l], s->param + s->off_W[l], s->grad + s->off_W[l],
                     s->m + s->off_W[l], s->v + s->off_W[l], 0.0f, 0.9f, 0.999f, 1e-8f, 1, s->W[l],
                     s->WT[l], kSurN[l], kSurK[l], st));
  s->step = 0;
  s->packed = false;
  return cudaSuccess;
}

static void init_params(Surrogate *s, uint64_t seed, std::vector<float> &h) {
  h.assign((size_t)kSurParams, 0.0f);
  Rng r{seed * 0x2545F4914F6CDD1Dull + 1};
  const int fan_in[kSurLayers] = {kSurFeat, kSurHidden, kSurHidden, kSurHidden};
  const int nout[kSurLayers] = {kSurHidden, kSurHidden, kSurHidden, NSP};
  for (int l = 0; l < kSurLayers; ++l) {
    const double sd = std::sqrt(2.0 / fan_in[l]);
    for (int n = 0; n < kSurN[l]; ++n)
      for (int k = 0; k < kSurK[l]; ++k) {
        const bool live = n < nout[l] && k < fan_in[l];
        h[(size_t)(s->off_W[l] + (int64_t)n * kSurK[l] + k)] = live ? (float)(sd * r.normal()) : 0.0f;
      }
  }
}

static cudaError_t upload_norm(Surrogate *s, cudaStream_t st) {
  float h[64] = {0};
  for (int c = 0; c < kSurIn; ++c) {
    h[c] = s->fmean[c];
    h[16 + c] = s->fistd[c];
  }
  for (int c = 0; c < kSurOut; ++c) {
    h[32 + c] = s->tmean[c];
    h[48 + c] = s->tistd[c];
  }
  SCHK(cudaMemcpyAsync(s->dev_norm, h, sizeof h, cudaMemcpyHostToDevice, st));
  return cudaStreamSynchronize(st);
}

static float key_decode(int k) {
  const int b = k >= 0 ? k : k ^ 0x7fffffff;
  float f;
  std::memcpy(&f, &b, sizeof f);
  return f;
}

// One layer forward: Z (fp32, nullable) = H W^T + b; Hout (bf16) = GELU(Z) (or Z for the
// last layer into Of fp32).
static cudaError_t layer_forward(Surrogate *s, int l, int64_t M, const __nv_bfloat16 *H, float *Z,
                                 __nv_bfloat16 *Hout, float *Of, cudaStream_t st) {
  GemmArgs g{};
  g.M = M;
  g.N = kSurN[l];
  g.K = kSurK[l];
  g.A = H;
  g.sam = kSurK[l];
  g.sak = 1;
  g.B = s->W[l];
  g.sbn = kSurK[l];
  g.sbk = 1;
  g.alpha = 1.0f;
  g.bias = s->param + s->off_b[l];
  const bool last = l == kSurLayers - 1;
  g.Cf = last ? Of : Z;
  g.ldc = kSurN[l];
  g.Cb = last ? nullptr : Hout;
  g.ldcb = kSurN[l];
  g.gelu = !last;
  g.err = s->tc_err;
  return launch_gemm(g, st);
}

// Training buffers for a batch of B rows.
// Split-K factor of the weight-gradient GEMMs (the batch is their reduction dimension)
// and the row slices of the bias-gradient sums.
constexpr int kGradSplit = 16;
// Training steps per replayed CUDA graph (the host launches one graph per this many steps).
constexpr int kGraphSteps = 8;

struct TrainBufs {
  float *Xb = nullptr, *Tb = nullptr, *Y = nullptr, *loss = nullptr, *part = nullptr;
  float *Z[3] = {}, *dH = nullptr;
  __nv_bfloat16 *Xbf = nullptr, *H[3] = {}, *dY = nullptr, *dZ = nullptr;
  void release() {
    cudaFree(Xb); cudaFree(Tb); cudaFree(Y); cudaFree(loss); cudaFree(part); cudaFree(dH); cudaFree(Xbf);
    cudaFree(dY); cudaFree(dZ);
    for (int i = 0; i < 3; ++i) { cudaFree(Z[i]); cudaFree(H[i]); }
  }
  cudaError_t alloc(int64_t B) {
    SCHK(cudaMalloc(&Xb, B * kSurIn * sizeof(float)));
    SCHK(cudaMalloc(&Tb, B * kSurOut * sizeof(float)));
    SCHK(cudaMalloc(&Y, B * kSurOut * sizeof(float)));
    SCHK(cudaMalloc(&loss, sizeof(float)));
    SCHK(cudaMalloc(&part, (size_t)kGradSplit * kSurHidden * kSurHidden * sizeof(float)));
    SCHK(cudaMalloc(&dH, B * kSurHidden * sizeof(float)));
    SCHK(cudaMalloc(&Xbf, B * kSurIn * sizeof(__nv_bfloat16)));
    SCHK(cudaMalloc(&dY, B * kSurOut * sizeof(__nv_bfloat16)));
    SCHK(cudaMalloc(&dZ, B * kSurHidden * sizeof(__nv_bfloat16)));
    for (int i = 0; i < 3; ++i) {
      SCHK(cudaMalloc(&Z[i], B * kSurHidden * sizeof(float)));
      SCHK(cudaMalloc(&H[i], B * kSurHidden * sizeof(__nv_bfloat16)));
    }
    return cudaSuccess;
  }
};

// Optional copies of a pass's intermediates (chem_surrogate_trace; every field nullable).
struct Trace {
  float *Z;                // [3][B][256] hidden pre-activations
  __nv_bfloat16 *H;        // [3][B][256] hidden activations
  __nv_bfloat16 *G;        // [4][B][256] output gradient per layer (layer 3: B x 16, stride 16)
  float *dH;               // [3][B][256] gradient w.r.t. hidden activation l
};

static cudaError_t trace_copy(void *dst, const void *src, size_t bytes, cudaStream_t st) {
  return dst ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, st) : cudaSuccess;
}

// Forward with saved activations, MSE over the 9 outputs, backward into s->grad.
// X: normalised features [B x 16] (fp32, also converted to bf16), T: normalised targets.
// tr (nullable) receives copies of the intermediates.
static cudaError_t forward_backward(Surrogate *s, TrainBufs &b, int64_t B, cudaStream_t st,
                                    const Trace *tr = nullptr) {
  SCHK(launch_to_bf16(B * kSurIn, b.Xb, b.Xbf, st));
  SCHK(layer_forward(s, 0, B, b.Xbf, b.Z[0], b.H[0], nullptr, st));
  SCHK(layer_forward(s, 1, B, b.H[0], b.Z[1], b.H[1], nullptr, st));
  SCHK(layer_forward(s, 2, B, b.H[1], b.Z[2], b.H[2], nullptr, st));
  SCHK(layer_forward(s, 3, B, b.H[2], nullptr, nullptr, b.Y, st));
  SCHK(launch_mse(B, NSP, kSurOut, b.Y, b.Tb, kSurOut, b.dY, kSurOut, b.loss, st));
  const size_t slab = (size_t)B * kSurHidden;
  if (tr) {
    for (int l = 0; l < 3; ++l) {
      SCHK(trace_copy(tr->Z ? tr->Z + l * slab : nullptr, b.Z[l], slab * sizeof(float), st));
      SCHK(trace_copy(tr->H ? tr->H + l * slab : nullptr, b.H[l], slab * sizeof(__nv_bfloat16), st));
    }
    SCHK(trace_copy(tr->G ? tr->G + 3 * slab : nullptr, b.dY, (size_t)B * kSurOut * sizeof(__nv_bfloat16), st));
  }
  // layer l: input Hin [B x K], output gradient G [B x N] (bf16)
  const __nv_bfloat16 *Hin[kSurLayers] = {b.Xbf, b.H[0], b.H[1], b.H[2]};
  const __nv_bfloat16 *G = b.dY;
  for (int l = kSurLayers - 1; l >= 0; --l) {
    const int N = kSurN[l], K = kSurK[l];
    // dW[n, k] = sum_m G[m, n] Hin[m, k]
    // (split-K over the batch into b.part, then a fixed-order reduction)
    GemmArgs gw{};
    gw.M = N; gw.N = K; gw.K = B;
    gw.A = G; gw.sam = 1; gw.sak = N;
    gw.B = Hin[l]; gw.sbn = 1; gw.sbk = K;
    gw.alpha = 1.0f;
    gw.Cf = b.part; gw.ldc = K;
    gw.split = kGradSplit;
    gw.split_ld = (int64_t)N * K;
    gw.err = s->tc_err;
    SCHK(launch_gemm(gw, st));
    SCHK(launch_reduce_splits((int64_t)N * K, kGradSplit, b.part, (int64_t)N * K, s->grad + s->off_W[l], st));
    SCHK(launch_bias_grad(B, N, G, N, b.part, kGradSplit, s->grad + s->off_b[l], st));
    if (l == 0) break;
    // dHin[m, k] = sum_n G[m, n] W[n, k] (W^T stored [K x N])
    // and in the same epilogue G for layer l-1: dZ = dHin * GELU'(Z_{l-1}) (bf16); the fp32
    // dHin itself is stored only for a trace
    GemmArgs gx{};
    gx.M = B; gx.N = K; gx.K = N;
    gx.A = G; gx.sam = N; gx.sak = 1;
    gx.B = s->WT[l]; gx.sbn = N; gx.sbk = 1;
    gx.alpha = 1.0f;
    gx.Cf = (tr && tr->dH) ? b.dH : nullptr; gx.ldc = K;
    gx.Cb = b.dZ; gx.ldcb = K;
    gx.dgelu_z = b.Z[l - 1]; gx.ldz = K;
    gx.err = s->tc_err;
    SCHK(launch_gemm(gx, st));
    if (tr) {
      SCHK(trace_copy(tr->dH ? tr->dH + (l - 1) * slab : nullptr, b.dH, slab * sizeof(float), st));
      SCHK(trace_copy(tr->G ? tr->G + (l - 1) * slab : nullptr, b.dZ, slab * sizeof(__nv_bfloat16), st));
    }
    G = b.dZ;
  }
  return cudaSuccess;
}

static cudaError_t adam_all(Surrogate *s, float lr, cudaStream_t st) {
  ++s->step;
  s->packed = false;
  for (int l = 0; l < kSurLayers; ++l) {
    const int64_t nw = (int64_t)kSurN[l] * kSurK[l];
    SCHK(launch_adam(nw, s->param + s->off_W[l], s->grad + s->off_W[l], s->m + s->off_W[l],
                     s->v + s->off_W[l], lr, 0.9f, 0.999f, 1e-8f, (int)s->step, s->W[l], s->WT[l],
                     kSurN[l], kSurK[l], st));
    SCHK(launch_adam(kSurN[l], s->param + s->off_b[l], s->grad + s->off_b[l], s->m + s->off_b[l],
                     s->v + s->off_b[l], lr, 0.9f, 0.999f, 1e-8f, (int)s->step, nullptr, nullptr,
                     1, kSurN[l], st));
  }
  return cudaSuccess;
}

static SurrogateConsts make_consts(const Surrogate *s, const chem_surrogate_gate &g,
                                   const MechTables &mt) {
  SurrogateConsts c{};
  for (int k = 0; k < NSP; ++k) {
    c.tmean[k] = s->tmean[k];
    c.tstd[k] = 1.0f / s->tistd[k];
  }
  for (int f = 0; f < kSurFeat; ++f) {
    c.fmin[f] = s->fmin[f];
    c.fmax[f] = s->fmax[f];
  }
  c.margin = g.ood_margin;
  c.resid_max = g.resid_max;
  c.neg_tol = g.neg_tol;
  c.max_dT = g.max_dT;
  c.err_tol = g.err_tol;
  c.rate_max = g.rate_max;
  c.lam = s->lam;
  c.dt_power = s->dt_power;
  for (int el = 0; el < 3; ++el) {
    c.emask[el] = 0;
    for (int k = 0; k < NSP; ++k) {
      c.E[el][k] = mt.Emat[el][k];
      c.emask[el] |= (mt.Emat[el][k] != 0.0) << k;
    }
  }
  return c;
}

}  // namespace chem

namespace chem {

static int sur_fail(chem_ctx *ctx, int code, const std::string &msg) {
  chem_ctx_error(ctx) = msg;
  return code;
}

static int sur_cuda(chem_ctx *ctx, cudaError_t e, const char *what) {
  return sur_fail(ctx, e == cudaErrorMemoryAllocation ? CHEM_ERR_NOMEM : CHEM_ERR_CUDA,
                  std::string(what) + ": " + cudaGetErrorString(e));
}

static Surrogate *ensure_surrogate(chem_ctx *ctx, cudaError_t *err) {
  void *&slot = chem_ctx_sur(ctx);
  *err = cudaSuccess;
  if (!slot) {
    Surrogate *s = new Surrogate;
    *err = alloc_params(s);
    if (*err != cudaSuccess) {
      cudaGetLastError();
      free_surrogate(s);
      return nullptr;
    }
    slot = s;
  }
  return static_cast<Surrogate *>(slot);
}

// Cells per inference chunk (features and outputs, 132 B a cell, are staged per chunk).
constexpr int64_t kInferChunk = 1 << 22;

// Forward kernels of the network: the tcgen05 one (inference), the mma.sync one-kernel
// version and the layer-by-layer GEMMs of training (checks).
enum { kFwdTc = 0, kFwdFused = 1, kFwdLayers = 2 };

// The network over n rows of features X (raw with norm, else normalised), in one kernel.
static cudaError_t mlp_forward(Surrogate *s, int64_t n, const float *X, const float *norm, float *O,
                               cudaStream_t st, int impl = kFwdTc) {
  const __nv_bfloat16 *W[kSurLayers];
  const float *b[kSurLayers];
  for (int l = 0; l < kSurLayers; ++l) {
    W[l] = s->W[l];
    b[l] = s->param + s->off_b[l];
  }
  if (impl == kFwdFused) return launch_mlp_fused(n, X, norm, W, b, O, st);
  if (!s->packed) {
    SCHK(launch_pack_weights(W, s->Wpk, st));
    s->packed = true;
  }
  return launch_mlp_tc(n, X, norm, s->Wpk, b, O, s->tc_err, st);
}

static cudaError_t ensure_infer_buffers(Surrogate *s, int64_t chunk, int64_t n) {
  if (chunk > s->chunk_cap) {
    cudaFree(s->Xraw); cudaFree(s->O); cudaFree(s->Tok);
    s->Xraw = s->O = nullptr; s->Tok = nullptr;
    s->chunk_cap = 0;
    SCHK(cudaMalloc(&s->Xraw, chunk * kSurIn * sizeof(float)));
    SCHK(cudaMalloc(&s->O, chunk * kSurOut * sizeof(float)));
    SCHK(cudaMalloc(&s->Tok, chunk));
    s->chunk_cap = chunk;
  }
  if (n > s->fb_cap) {
    cudaFree(s->fb_idx);
    s->fb_idx = nullptr;
    s->fb_cap = 0;
    SCHK(cudaMalloc(&s->fb_idx, n * sizeof(int32_t)));
    s->fb_cap = n;
  }
  return cudaSuccess;
}

}  // namespace chem

using namespace chem;

extern "C" {

int64_t chem_surrogate_param_count(void) { return kSurParams; }

int chem_surrogate_params(chem_ctx *ctx, float *h_out, const float *h_in, int64_t n) {
  if (!ctx) return CHEM_ERR_INVALID;
  if (n != kSurParams) return sur_fail(ctx, CHEM_ERR_INVALID, "parameter count mismatch");
  cudaError_t e;
  Surrogate *s = ensure_surrogate(ctx, &e);
  if (!s) return sur_cuda(ctx, e, "allocating the surrogate");
  if (h_in) {
    e = set_params(s, h_in, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(0);
    if (e != cudaSuccess) return sur_cuda(ctx, e, "setting parameters");
  }
  if (h_out) {
    e = cudaMemcpy(h_out, s->param, (size_t)kSurParams * sizeof(float), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return sur_cuda(ctx, e, "reading parameters");
  }
  return CHEM_OK;
}

static int surrogate_pass(chem_ctx *ctx, const float *d_X, const float *d_T, int64_t B, float *d_Y,
                          float *h_grad, float *h_loss, void *stream, const Trace *tr) {
  if (!ctx) return CHEM_ERR_INVALID;
  if (B <= 0 || !d_X || !d_T) return sur_fail(ctx, CHEM_ERR_INVALID, "B > 0, X and T required");
  cudaError_t e;
  Surrogate *s = ensure_surrogate(ctx, &e);
  if (!s) return sur_cuda(ctx, e, "allocating the surrogate");
  cudaStream_t st = (cudaStream_t)stream;
  TrainBufs b;
  e = b.alloc(B);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->tc_err, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b.Xb, d_X, B * kSurIn * sizeof(float), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b.Tb, d_T, B * kSurOut * sizeof(float), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(b.loss, 0, sizeof(float), st);
  if (e == cudaSuccess) e = forward_backward(s, b, B, st, tr);
  if (e == cudaSuccess && d_Y) e = cudaMemcpyAsync(d_Y, b.Y, B * kSurOut * sizeof(float), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && h_grad)
    e = cudaMemcpyAsync(h_grad, s->grad, (size_t)kSurParams * sizeof(float), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && h_loss) e = cudaMemcpyAsync(h_loss, b.loss, sizeof(float), cudaMemcpyDeviceToHost, st);
  int terr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&terr, s->tc_err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  b.release();
  if (e == cudaSuccess && terr) return sur_fail(ctx, CHEM_ERR_TIMEOUT, "a bounded wait of the tensor-core GEMM ran out");
  return e == cudaSuccess ? CHEM_OK : sur_cuda(ctx, e, "surrogate forward/backward");
}

int chem_surrogate_grad(chem_ctx *ctx, const float *d_X, const float *d_T, int64_t B, float *d_Y,
                        float *h_grad, float *h_loss, void *stream) {
  return surrogate_pass(ctx, d_X, d_T, B, d_Y, h_grad, h_loss, stream, nullptr);
}

int chem_surrogate_trace(chem_ctx *ctx, const float *d_X, const float *d_T, int64_t B, float *d_Y,
                         float *d_Z, uint16_t *d_H, uint16_t *d_G, float *d_dH, float *h_grad,
                         float *h_loss, void *stream) {
  const Trace tr{d_Z, reinterpret_cast<__nv_bfloat16 *>(d_H), reinterpret_cast<__nv_bfloat16 *>(d_G), d_dH};
  return surrogate_pass(ctx, d_X, d_T, B, d_Y, h_grad, h_loss, stream, &tr);
}

int chem_surrogate_adam(chem_ctx *ctx, const float *h_grad, int64_t n, float lr) {
  if (!ctx) return CHEM_ERR_INVALID;
  if (n != kSurParams || !h_grad) return sur_fail(ctx, CHEM_ERR_INVALID, "n must equal the parameter count");
  if (!(lr >= 0.0f) || !std::isfinite(lr)) return sur_fail(ctx, CHEM_ERR_INVALID, "lr must be >= 0");
  cudaError_t e;
  Surrogate *s = ensure_surrogate(ctx, &e);
  if (!s) return sur_cuda(ctx, e, "allocating the surrogate");
  e = cudaMemcpyAsync(s->grad, h_grad, (size_t)kSurParams * sizeof(float), cudaMemcpyHostToDevice, 0);
  if (e == cudaSuccess) e = adam_all(s, lr, 0);
  if (e == cudaSuccess) e = cudaStreamSynchronize(0);
  return e == cudaSuccess ? CHEM_OK : sur_cuda(ctx, e, "Adam step");
}

int chem_surrogate_project(chem_ctx *ctx, int64_t n, const double *d_Y0, const double *d_Yp,
                           int64_t ldY, double *d_Yout, void *stream) {
  if (!ctx) return CHEM_ERR_INVALID;
  if (n < 0) return sur_fail(ctx, CHEM_ERR_INVALID, "n < 0");
  if (n == 0) return CHEM_OK;
  if (!d_Y0 || !d_Yp || !d_Yout) return sur_fail(ctx, CHEM_ERR_INVALID, "Y0, Yp and Yout are required");
  if (ldY < n) return sur_fail(ctx, CHEM_ERR_INVALID, "ldY < n");
  const MechTables &mt = chem_ctx_tables(ctx);
  SurrogateConsts c{};
  for (int el = 0; el < 3; ++el)
    for (int k = 0; k < NSP; ++k) {
      c.E[el][k] = mt.Emat[el][k];
      c.emask[el] |= (mt.Emat[el][k] != 0.0) << k;
    }
  const cudaError_t e = launch_project_check(c, n, d_Y0, d_Yp, ldY, d_Yout, (cudaStream_t)stream);
  return e == cudaSuccess ? CHEM_OK : sur_cuda(ctx, e, "projection");
}

int chem_surrogate_forward(chem_ctx *ctx, const float *d_X, int64_t B, float *d_Y, int32_t impl,
                           void *stream, int32_t *h_err) {
  if (!ctx) return CHEM_ERR_INVALID;
  if (B < 0 || (B > 0 && (!d_X || !d_Y))) return sur_fail(ctx, CHEM_ERR_INVALID, "B >= 0, X and Y required");
  if (impl < kFwdTc || impl > kFwdLayers) return sur_fail(ctx, CHEM_ERR_INVALID, "unknown forward kernel");
  cudaError_t e;
  Surrogate *s = ensure_surrogate(ctx, &e);
  if (!s) return sur_cuda(ctx, e, "allocating the surrogate");
  cudaStream_t st = (cudaStream_t)stream;
  if (impl == kFwdLayers) {
    if (B == 0) return CHEM_OK;
    TrainBufs b;
    e = b.alloc(B);
    if (e == cudaSuccess) e = launch_to_bf16(B * kSurIn, d_X, b.Xbf, st);
    if (e == cudaSuccess) e = layer_forward(s, 0, B, b.Xbf, nullptr, b.H[0], nullptr, st);
    if (e == cudaSuccess) e = layer_forward(s, 1, B, b.H[0], nullptr, b.H[1], nullptr, st);
    if (e == cudaSuccess) e = layer_forward(s, 2, B, b.H[1], nullptr, b.H[2], nullptr, st);
    if (e == cudaSuccess) e = layer_forward(s, 3, B, b.H[2], nullptr, nullptr, d_Y, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    b.release();
  } else {
    if (h_err && impl == kFwdTc) e = cudaMemsetAsync(s->tc_err, 0, sizeof(int), st);
    if (e == cudaSuccess) e = mlp_forward(s, B, d_X, nullptr, d_Y, st, impl);
  }
  if (e == cudaSuccess && h_err) {
    int v = 0;
    if (impl == kFwdTc) e = cudaMemcpyAsync(&v, s->tc_err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    *h_err = v;
  }
  return e == cudaSuccess ? CHEM_OK : sur_cuda(ctx, e, "surrogate forward");
}

int chem_surrogate_train(chem_ctx *ctx, const chem_pairs *pairs, int64_t npairs,
                         const chem_train_cfg *cfg_in, void *stream, float *h_epoch_loss) {
  if (!ctx) return CHEM_ERR_INVALID;
  chem_train_cfg cfg{};
  if (cfg_in) cfg = *cfg_in;
  if (cfg.epochs == 0) cfg.epochs = 20;
  if (cfg.batch == 0) cfg.batch = 4096;
  if (cfg.lr == 0.0f) cfg.lr = 1e-3f;
  if (cfg.lr_final == 0.0f) cfg.lr_final = cfg.lr / 20.0f;
  if (cfg.boxcox_lambda == 0.0f) cfg.boxcox_lambda = 0.1f;
  if (cfg.epochs < 0 || cfg.batch < 1 || !(cfg.lr > 0.0f) || !(cfg.boxcox_lambda > 0.0f) ||
      !std::isfinite(cfg.dt_power))
    return sur_fail(ctx, CHEM_ERR_INVALID, "invalid training configuration");
  if (!pairs || !pairs->d_rho || !pairs->d_e || !pairs->d_Y0 || !pairs->d_dt || !pairs->d_Y1)
    return sur_fail(ctx, CHEM_ERR_INVALID, "pairs need rho, e, Y0, dt and Y1");
  if (npairs < cfg.batch || npairs > INT32_MAX)
    return sur_fail(ctx, CHEM_ERR_INVALID, "npairs must be at least one batch and below 2^31");
  if (pairs->ldY0 < npairs || pairs->ldY1 < npairs)
    return sur_fail(ctx, CHEM_ERR_INVALID, "ldY0 / ldY1 < npairs");
  cudaError_t e;
  Surrogate *s = ensure_surrogate(ctx, &e);
  if (!s) return sur_cuda(ctx, e, "allocating the surrogate");
  cudaStream_t st = (cudaStream_t)stream;
  const MechTables &mt = chem_ctx_tables(ctx);
  s->lam = cfg.boxcox_lambda;
  s->dt_power = cfg.dt_power;
  s->ready = false;
  std::vector<float> h;
  init_params(s, cfg.seed, h);
  e = set_params(s, h.data(), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->tc_err, 0, sizeof(int), st);
  if (e != cudaSuccess) return sur_cuda(ctx, e, "initialising parameters");
  const int64_t n = npairs, B = cfg.batch;
  float *X = nullptr, *Tg = nullptr;
  double *sums = nullptr;
  int *keys = nullptr;
  int32_t *idx = nullptr;
  TrainBufs b;
  auto cleanup = [&]() {
    cudaFree(X); cudaFree(Tg); cudaFree(sums); cudaFree(keys); cudaFree(idx);
    b.release();
  };
  e = cudaMalloc(&X, n * kSurIn * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&Tg, n * kSurOut * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&sums, 4 * 32 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&keys, 4 * 32 * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&idx, n * sizeof(int32_t));
  if (e == cudaSuccess) e = b.alloc(B);
  if (e != cudaSuccess) { cleanup(); return sur_cuda(ctx, e, "allocating training buffers"); }
  // features and targets of every pair, then their statistics
  e = launch_features(mt, n, pairs->d_rho, pairs->d_e, pairs->d_Y0, pairs->ldY0, pairs->d_T0,
                      pairs->d_dt, 0.0, pairs->d_Y1, pairs->ldY1, s->lam, s->dt_power, X, Tg, nullptr, st);
  int hkeys[4 * 32];
  for (int i = 0; i < 32; ++i) {
    hkeys[i] = INT_MAX; hkeys[32 + i] = INT_MIN; hkeys[64 + i] = INT_MAX; hkeys[96 + i] = INT_MIN;
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(sums, 0, 4 * 32 * sizeof(double), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(keys, hkeys, sizeof hkeys, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = launch_colstats(n, kSurFeat, kSurIn, X, sums, sums + 32, keys, keys + 32, st);
  if (e == cudaSuccess) e = launch_colstats(n, NSP, kSurOut, Tg, sums + 64, sums + 96, keys + 64, keys + 96, st);
  double hs[4 * 32];
  if (e == cudaSuccess) e = cudaMemcpyAsync(hs, sums, sizeof hs, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hkeys, keys, sizeof hkeys, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) { cleanup(); return sur_cuda(ctx, e, "featurising the pairs"); }
  for (int c = 0; c < kSurIn; ++c) {
    if (c < kSurFeat) {
      const double mean = hs[c] / n, var = std::fmax(hs[32 + c] / n - mean * mean, 0.0);
      s->fmean[c] = (float)mean;
      s->fistd[c] = (float)(1.0 / std::fmax(std::sqrt(var), 1e-6));
      s->fmin[c] = key_decode(hkeys[c]);
      s->fmax[c] = key_decode(hkeys[32 + c]);
    } else {
      s->fmean[c] = 0.0f;
      s->fistd[c] = 0.0f;
    }
  }
  for (int c = 0; c < kSurOut; ++c) {
    if (c < NSP) {
      const double mean = hs[64 + c] / n, var = std::fmax(hs[96 + c] / n - mean * mean, 0.0);
      s->tmean[c] = (float)mean;
      s->tistd[c] = (float)(1.0 / std::fmax(std::sqrt(var), 1e-6));
    } else {
      s->tmean[c] = 0.0f;
      s->tistd[c] = 0.0f;
    }
  }
  e = upload_norm(s, st);
  if (e == cudaSuccess) e = launch_normalize(n, kSurFeat, kSurIn, X, s->dev_norm, s->dev_norm + 16, nullptr, st);
  if (e == cudaSuccess) e = launch_normalize(n, NSP, kSurOut, Tg, s->dev_norm + 32, s->dev_norm + 48, nullptr, st);
  if (e != cudaSuccess) { cleanup(); return sur_cuda(ctx, e, "normalising"); }
  // epochs of shuffled batches.  The training step (the batch gather, forward, loss,
  // backward, Adam) is captured as CUDA graphs on a private stream, of one step and of
  // kGraphSteps steps, and replayed for every batch: the batch offset, the learning rate
  // of the cosine schedule and Adam's bias corrections come from a step counter on the
  // device and a schedule table computed here, so the replays need no host arguments.
  const int64_t nb = n / B;
  const int64_t total = nb * cfg.epochs;
  std::vector<float> hsched((size_t)(3 * (total > 0 ? total : 1)));
  for (int64_t it = 0; it < total; ++it) {
    const double frac = total > 1 ? (double)it / (double)(total - 1) : 1.0;
    hsched[(size_t)(3 * it)] =
        (float)(cfg.lr_final + 0.5 * (cfg.lr - cfg.lr_final) * (1.0 + std::cos(3.141592653589793 * frac)));
    hsched[(size_t)(3 * it + 1)] = 1.0f - powf(0.9f, (float)(it + 1));
    hsched[(size_t)(3 * it + 2)] = 1.0f - powf(0.999f, (float)(it + 1));
  }
  float *dsched = nullptr;
  int64_t *dstep = nullptr;
  int32_t *idx2 = nullptr;   // the second permutation buffer (epochs alternate)
  int32_t *hperm = nullptr;  // pinned staging of the permutations, two slots
  float *hloss = nullptr;    // pinned per-epoch loss sums
  cudaStream_t ps = nullptr;
  cudaGraph_t graph[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaGraphExec_t exec[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t up_done[2] = {nullptr, nullptr};
  auto release_graph = [&]() {
    for (int i = 0; i < 4; ++i) {
      if (exec[i]) cudaGraphExecDestroy(exec[i]);
      if (graph[i]) cudaGraphDestroy(graph[i]);
    }
    for (int i = 0; i < 2; ++i)
      if (up_done[i]) cudaEventDestroy(up_done[i]);
    if (ps) cudaStreamDestroy(ps);
    cudaFree(dsched);
    cudaFree(dstep);
    cudaFree(idx2);
    cudaFreeHost(hperm);
    cudaFreeHost(hloss);
  };
  e = cudaMalloc(&dsched, hsched.size() * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&dstep, sizeof(int64_t));
  if (e == cudaSuccess) e = cudaMalloc(&idx2, n * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMallocHost(&hperm, 2 * n * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMallocHost(&hloss, (size_t)(cfg.epochs > 0 ? cfg.epochs : 1) * sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpy(dsched, hsched.data(), hsched.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(dstep, 0, sizeof(int64_t));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&up_done[i], cudaEventDisableTiming);
  if (e == cudaSuccess) e = gemm_prepare();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // features and statistics are done
  int32_t *idxs[2] = {idx, idx2};
  static_assert(kAdamSegs == 2 * kSurLayers, "one weight and one bias segment per layer");
  AdamSegs sg{};  // Adam on every parameter in one launch (the layout W0 b0 W1 b1 ...)
  for (int l = 0; l < kSurLayers; ++l) {
    sg.end[2 * l] = s->off_b[l];
    sg.end[2 * l + 1] = s->off_b[l] + kSurN[l];
    sg.w_bf[2 * l] = s->W[l];
    sg.wT_bf[2 * l] = s->WT[l];
    sg.rows[2 * l] = kSurN[l];
    sg.cols[2 * l] = kSurK[l];
    sg.rows[2 * l + 1] = 1;
    sg.cols[2 * l + 1] = kSurN[l];
  }
  auto capture_step = [&](int gi) {
    cudaError_t ce = launch_gather_rows_step(B, kSurIn, idxs[gi], dstep, nb, X, kSurIn, b.Xb, kSurIn, ps);
    if (ce == cudaSuccess) ce = launch_gather_rows_step(B, kSurOut, idxs[gi], dstep, nb, Tg, kSurOut, b.Tb, kSurOut, ps);
    if (ce == cudaSuccess) ce = forward_backward(s, b, B, ps);
    if (ce == cudaSuccess)
      ce = launch_adam_sched_all(kSurParams, s->param, s->grad, s->m, s->v, dsched, dstep, 0.9f, 0.999f, 1e-8f, sg,
                                 ps);
    if (ce == cudaSuccess) ce = launch_step_inc(dstep, ps);
    return ce;
  };
  // graph g = gi (one step) and g = 2 + gi (kGraphSteps steps) for permutation buffer gi:
  // an epoch replays the long graph nb / kGraphSteps times and the short one for the rest,
  // so the host launches a graph per kGraphSteps steps, not per step
  for (int g = 0; g < 4 && e == cudaSuccess && total > 0; ++g) {
    e = cudaStreamBeginCapture(ps, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) break;
    cudaError_t ce = cudaSuccess;
    for (int k = 0; k < (g < 2 ? 1 : kGraphSteps) && ce == cudaSuccess; ++k) ce = capture_step(g & 1);
    e = cudaStreamEndCapture(ps, &graph[g]);
    if (e == cudaSuccess) e = ce;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec[g], graph[g], 0);
  }
  // the host shuffles epoch ep + 1 while the GPU replays epoch ep: permutations alternate
  // between two device buffers (one graph each) and two pinned staging slots
  Rng r{cfg.seed ^ 0x5bd1e995ull};
  auto shuffle_into = [&](int32_t *dst) {
    for (int64_t i = 0; i < n; ++i) dst[i] = (int32_t)i;
    for (int64_t i = n - 1; i > 0; --i) std::swap(dst[i], dst[(size_t)(r.next() % (uint64_t)(i + 1))]);
  };
  if (e == cudaSuccess && cfg.epochs > 0) {
    shuffle_into(hperm);
    e = cudaMemcpyAsync(idx, hperm, n * sizeof(int32_t), cudaMemcpyHostToDevice, ps);
    if (e == cudaSuccess) e = cudaEventRecord(up_done[0], ps);
  }
  for (int ep = 0; ep < cfg.epochs && e == cudaSuccess; ++ep) {
    const int cur = ep & 1, nxt = cur ^ 1;
    e = cudaMemsetAsync(b.loss, 0, sizeof(float), ps);
    for (int64_t bi = 0; bi + kGraphSteps <= nb && e == cudaSuccess; bi += kGraphSteps)
      e = cudaGraphLaunch(exec[2 + cur], ps);
    for (int64_t bi = nb - nb % kGraphSteps; bi < nb && e == cudaSuccess; ++bi) e = cudaGraphLaunch(exec[cur], ps);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hloss + ep, b.loss, sizeof(float), cudaMemcpyDeviceToHost, ps);
    if (e == cudaSuccess && ep + 1 < cfg.epochs) {
      // the staging slot of epoch ep + 1 was last copied for epoch ep - 1
      if (ep >= 1) e = cudaEventSynchronize(up_done[nxt]);
      if (e == cudaSuccess) {
        shuffle_into(hperm + (size_t)nxt * n);
        e = cudaMemcpyAsync(idxs[nxt], hperm + (size_t)nxt * n, n * sizeof(int32_t), cudaMemcpyHostToDevice, ps);
      }
      if (e == cudaSuccess) e = cudaEventRecord(up_done[nxt], ps);
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(ps);
  if (e == cudaSuccess && h_epoch_loss)
    for (int ep = 0; ep < cfg.epochs; ++ep) h_epoch_loss[ep] = hloss[ep] / (float)nb;
  s->step = total;
  s->packed = false;
  release_graph();
  cleanup();
  if (e != cudaSuccess) return sur_cuda(ctx, e, "training");
  int terr = 0;
  e = cudaMemcpy(&terr, s->tc_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return sur_cuda(ctx, e, "training");
  if (terr) return sur_fail(ctx, CHEM_ERR_TIMEOUT, "a bounded wait of the tensor-core GEMM ran out in training");
  s->ready = true;
  return CHEM_OK;
}

// Gate defaults of chem_surrogate_gate (zero fields take them).
static chem_surrogate_gate gate_defaults(const chem_surrogate_gate *gate_in) {
  chem_surrogate_gate g{};
  if (gate_in) g = *gate_in;
  if (g.ood_margin == 0.0f) g.ood_margin = 0.05f;
  if (g.resid_max == 0.0f) g.resid_max = 0.02f;
  if (g.neg_tol == 0.0f) g.neg_tol = 1e-6f;
  if (g.max_dT == 0.0f) g.max_dT = 200.0f;
  if (g.err_tol == 0.0f) g.err_tol = 6e-4f;
  if (g.rate_max == 0.0f) g.rate_max = 1.5f;
  return g;
}

// Network, projection, temperature, gate and error test on the cells [first, first + n)
// of the state over dt, in chunks; accepted cells are written, rejected ones appended to
// the fallback list (global indices) without resetting its count.
static cudaError_t infer_range(chem_ctx *ctx, Surrogate *s, const SurrogateConsts &sc,
                               const chem_state *state, int64_t first, int64_t n, double dt,
                               uint8_t *d_mask, cudaStream_t st) {
  const MechTables &mt = chem_ctx_tables(ctx);
  const int64_t chunk = s->chunk_cap;
  cudaError_t e = cudaSuccess;
  for (int64_t off = 0; off < n && e == cudaSuccess; off += chunk) {
    const int64_t base = first + off;
    const int64_t m = (n - off) < chunk ? (n - off) : chunk;
    e = launch_features(mt, m, state->d_rho + base, state->d_e + base, state->d_Y + base, state->ldY,
                        state->d_T + base, nullptr, dt, nullptr, 0, s->lam, s->dt_power, s->Xraw, nullptr,
                        s->Tok, st);
    if (e == cudaSuccess) e = mlp_forward(s, m, s->Xraw, s->dev_norm, s->O, st);
    if (e == cudaSuccess)
      e = launch_surrogate_finish(chem_ctx_variant(ctx), mt, sc, m, dt, s->O, s->Xraw, s->Tok,
                                  state->d_rho + base, state->d_e + base,
                                  state->d_Y + base, state->ldY, state->d_T + base,
                                  state->d_status ? state->d_status + base : nullptr,
                                  state->d_nsteps ? state->d_nsteps + base : nullptr,
                                  d_mask ? d_mask + base : nullptr, s->fb_idx, s->fb_count, base, st);
  }
  return e;
}

// Checks shared by the inference entry points; on CHEM_OK *sp is the trained surrogate.
static int infer_checks(chem_ctx *ctx, const chem_state *state, int64_t n, double rtol, double atol,
                        Surrogate **sp) {
  Surrogate *s = static_cast<Surrogate *>(chem_ctx_sur(ctx));
  if (!s || !s->ready) return sur_fail(ctx, CHEM_ERR_STATE, "no trained or loaded surrogate");
  if (chem_ctx_scheme(ctx) != CHEM_SCHEME_LSRK)
    return sur_fail(ctx, CHEM_ERR_UNSUPPORTED, "the surrogate's fallback runs the two-register scheme only");
  if (!state || n < 0) return sur_fail(ctx, CHEM_ERR_INVALID, "state is NULL or ncells < 0");
  if (!(rtol > 0.0) || !std::isfinite(rtol) || !(atol >= 0.0) || !std::isfinite(atol))
    return sur_fail(ctx, CHEM_ERR_INVALID, "rtol must be > 0 and atol >= 0");
  if (n > INT32_MAX) return sur_fail(ctx, CHEM_ERR_INVALID, "at most 2^31-1 cells per call");
  if (n > 0 && (!state->d_rho || !state->d_e || !state->d_Y || !state->d_T || state->ldY < n))
    return sur_fail(ctx, CHEM_ERR_INVALID, "rho, e, Y, T required and ldY >= ncells");
  *sp = s;
  return CHEM_OK;
}

int chem_surrogate_infer(chem_ctx *ctx, const chem_state *state, int64_t n, double dt, double rtol,
                         double atol, const chem_surrogate_gate *gate_in, void *stream,
                         uint8_t *d_mask, chem_stats *d_stats) {
  if (!ctx) return CHEM_ERR_INVALID;
  Surrogate *s = nullptr;
  int rc = infer_checks(ctx, state, n, rtol, atol, &s);
  if (rc) return rc;
  if (!(dt > 0.0) || !std::isfinite(dt)) return sur_fail(ctx, CHEM_ERR_INVALID, "dt must be > 0");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (d_stats) e = cudaMemsetAsync(d_stats, 0, sizeof(chem_stats), st);
  if (e != cudaSuccess) return sur_cuda(ctx, e, "clearing stats");
  if (n == 0) return CHEM_OK;
  const chem_surrogate_gate g = gate_defaults(gate_in);
  const int64_t chunk = n < kInferChunk ? n : kInferChunk;
  e = ensure_infer_buffers(s, chunk, n);
  if (e != cudaSuccess) return sur_cuda(ctx, e, "allocating inference buffers");
  const MechTables &mt = chem_ctx_tables(ctx);
  const SurrogateConsts sc = make_consts(s, g, mt);
  e = cudaMemsetAsync(s->fb_count, 0, sizeof(unsigned int), st);
  if (e == cudaSuccess) e = infer_range(ctx, s, sc, state, 0, n, dt, d_mask, st);
  if (e == cudaSuccess) e = launch_one_box(s->box_off, s->box_dt, s->box_nsub, n, dt, st);
  if (e == cudaSuccess) {
    // the rejected cells: a queue (the fallback list, its length on the device) for the
    // persistent work-stealing integrator, every cell one box of one step dt
    BatchArgs a{state->d_rho, state->d_e, state->d_Y, state->ldY, state->d_T, nullptr,
                state->d_status, state->d_nsteps, n, s->box_off, s->box_dt, s->box_nsub, 1,
                nullptr, d_stats, s->fb_count, CHEM_CELL_SURROGATE};
    StepParams p{0.0, rtol, atol, chem_ctx_max_steps(ctx)};
    e = launch_persistent_queue(chem_ctx_variant(ctx), mt, a, p, s->fb_idx, s->cursor, st);
  }
  if (e == cudaSuccess && d_stats) e = launch_surrogate_stats(d_stats, n, s->fb_count, st);
  return e == cudaSuccess ? CHEM_OK : sur_cuda(ctx, e, "surrogate inference");
}

int chem_surrogate_infer_batched(chem_ctx *ctx, const chem_state *state, int64_t n,
                                 const chem_batch *batch, double rtol, double atol,
                                 const chem_surrogate_gate *gate_in, void *stream, uint8_t *d_mask,
                                 chem_stats *d_stats) {
  if (!ctx) return CHEM_ERR_INVALID;
  Surrogate *s = nullptr;
  int rc = infer_checks(ctx, state, n, rtol, atol, &s);
  if (rc) return rc;
  if (!batch || batch->nboxes < 1 || !batch->d_box_offset || !batch->d_box_dt || !batch->d_box_nsub)
    return sur_fail(ctx, CHEM_ERR_INVALID, "batch needs nboxes >= 1 and its three device arrays");
  cudaStream_t st = (cudaStream_t)stream;
  const int nb = batch->nboxes;
  // the box table on the host: the rounds and their cell ranges are sequenced here
  std::vector<int64_t> off((size_t)nb + 1);
  std::vector<double> bdt((size_t)nb);
  std::vector<int32_t> nsub((size_t)nb);
  cudaError_t e = cudaMemcpyAsync(off.data(), batch->d_box_offset, off.size() * sizeof(int64_t),
                                  cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(bdt.data(), batch->d_box_dt, bdt.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(nsub.data(), batch->d_box_nsub, nsub.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return sur_cuda(ctx, e, "reading the box table");
  if (off[0] != 0 || off[(size_t)nb] != n)
    return sur_fail(ctx, CHEM_ERR_INVALID, "box offsets must start at 0 and end at ncells");
  int32_t rounds = 0;
  for (int b = 0; b < nb; ++b) {
    if (off[(size_t)b + 1] < off[(size_t)b]) return sur_fail(ctx, CHEM_ERR_INVALID, "box offsets must not decrease");
    if (!(bdt[(size_t)b] > 0.0) || !std::isfinite(bdt[(size_t)b]) || nsub[(size_t)b] < 1)
      return sur_fail(ctx, CHEM_ERR_INVALID, "box dt must be > 0 and substeps >= 1");
    rounds = std::max(rounds, nsub[(size_t)b]);
  }
  if (d_stats) e = cudaMemsetAsync(d_stats, 0, sizeof(chem_stats), st);
  if (e != cudaSuccess) return sur_cuda(ctx, e, "clearing stats");
  if (n == 0) return CHEM_OK;
  const chem_surrogate_gate g = gate_defaults(gate_in);
  const int64_t chunk = n < kInferChunk ? n : kInferChunk;
  e = ensure_infer_buffers(s, chunk, n);
  if (e == cudaSuccess && nb > s->ones_cap) {
    cudaFree(s->ones);
    s->ones = nullptr;
    s->ones_cap = 0;
    e = cudaMalloc(&s->ones, (size_t)nb * sizeof(int32_t));
    if (e == cudaSuccess) s->ones_cap = nb;
  }
  if (e == cudaSuccess) e = launch_fill_i32(s->ones, nb, 1, st);
  if (e != cudaSuccess) return sur_cuda(ctx, e, "allocating inference buffers");
  const MechTables &mt = chem_ctx_tables(ctx);
  const SurrogateConsts sc = make_consts(s, g, mt);
  StepParams p{0.0, rtol, atol, chem_ctx_max_steps(ctx)};
  for (int32_t r = 0; r < rounds && e == cudaSuccess; ++r) {
    // round r: every box with more than r substeps advances one substep of its dt; the
    // cells the gate rejects, from all boxes, form one queue for one persistent launch
    e = cudaMemsetAsync(s->fb_count, 0, sizeof(unsigned int), st);
    int64_t active = 0;
    for (int b = 0; b < nb && e == cudaSuccess; ++b) {
      const int64_t a0 = off[(size_t)b], m = off[(size_t)b + 1] - a0;
      if (nsub[(size_t)b] <= r || m == 0) continue;
      e = infer_range(ctx, s, sc, state, a0, m, bdt[(size_t)b], d_mask, st);
      active += m;
    }
    if (e == cudaSuccess) {
      BatchArgs a{state->d_rho, state->d_e, state->d_Y, state->ldY, state->d_T, nullptr,
                  state->d_status, state->d_nsteps, n, batch->d_box_offset, batch->d_box_dt, s->ones, nb,
                  nullptr, d_stats, s->fb_count, CHEM_CELL_SURROGATE};
      e = launch_persistent_queue(chem_ctx_variant(ctx), mt, a, p, s->fb_idx, s->cursor, st);
    }
    if (e == cudaSuccess && d_stats) e = launch_surrogate_stats_add(d_stats, active, s->fb_count, st);
  }
  return e == cudaSuccess ? CHEM_OK : sur_cuda(ctx, e, "batched surrogate inference");
}

static const char kSurMagic[8] = {'C', 'H', 'E', 'M', 'S', 'U', 'R', '2'};

int chem_surrogate_save(chem_ctx *ctx, const char *path) {
  if (!ctx || !path) return CHEM_ERR_INVALID;
  Surrogate *s = static_cast<Surrogate *>(chem_ctx_sur(ctx));
  if (!s || !s->ready) return sur_fail(ctx, CHEM_ERR_STATE, "no trained or loaded surrogate");
  std::vector<float> h((size_t)kSurParams);
  cudaError_t e = cudaMemcpy(h.data(), s->param, h.size() * sizeof(float), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return sur_cuda(ctx, e, "reading parameters");
  FILE *f = std::fopen(path, "wb");
  if (!f) return sur_fail(ctx, CHEM_ERR_INVALID, std::string("cannot open ") + path);
  const int64_t np = kSurParams;
  bool ok = std::fwrite(kSurMagic, 1, 8, f) == 8 && std::fwrite(&np, sizeof np, 1, f) == 1 &&
            std::fwrite(&s->lam, sizeof s->lam, 1, f) == 1 &&
            std::fwrite(&s->dt_power, sizeof s->dt_power, 1, f) == 1 &&
            std::fwrite(s->fmean, sizeof s->fmean, 1, f) == 1 && std::fwrite(s->fistd, sizeof s->fistd, 1, f) == 1 &&
            std::fwrite(s->fmin, sizeof s->fmin, 1, f) == 1 && std::fwrite(s->fmax, sizeof s->fmax, 1, f) == 1 &&
            std::fwrite(s->tmean, sizeof s->tmean, 1, f) == 1 && std::fwrite(s->tistd, sizeof s->tistd, 1, f) == 1 &&
            std::fwrite(h.data(), sizeof(float), h.size(), f) == h.size();
  ok = (std::fclose(f) == 0) && ok;
  return ok ? CHEM_OK : sur_fail(ctx, CHEM_ERR_INVALID, std::string("write failed: ") + path);
}

int chem_surrogate_load(chem_ctx *ctx, const char *path) {
  if (!ctx || !path) return CHEM_ERR_INVALID;
  FILE *f = std::fopen(path, "rb");
  if (!f) return sur_fail(ctx, CHEM_ERR_INVALID, std::string("cannot open ") + path);
  char magic[8];
  int64_t np = 0;
  double lam = 0.0, dt_power = 0.0;
  float fmean[kSurIn], fistd[kSurIn], fmin[kSurFeat], fmax[kSurFeat], tmean[kSurOut], tistd[kSurOut];
  std::vector<float> h((size_t)kSurParams);
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kSurMagic, 8) == 0 &&
            std::fread(&np, sizeof np, 1, f) == 1 && np == kSurParams &&
            std::fread(&lam, sizeof lam, 1, f) == 1 && std::fread(&dt_power, sizeof dt_power, 1, f) == 1 &&
            std::fread(fmean, sizeof fmean, 1, f) == 1 &&
            std::fread(fistd, sizeof fistd, 1, f) == 1 && std::fread(fmin, sizeof fmin, 1, f) == 1 &&
            std::fread(fmax, sizeof fmax, 1, f) == 1 && std::fread(tmean, sizeof tmean, 1, f) == 1 &&
            std::fread(tistd, sizeof tistd, 1, f) == 1 &&
            std::fread(h.data(), sizeof(float), h.size(), f) == h.size();
  std::fclose(f);
  if (!ok) return sur_fail(ctx, CHEM_ERR_INVALID, std::string("not a surrogate file: ") + path);
  cudaError_t e;
  Surrogate *s = ensure_surrogate(ctx, &e);
  if (!s) return sur_cuda(ctx, e, "allocating the surrogate");
  s->lam = lam;
  s->dt_power = dt_power;
  std::memcpy(s->fmean, fmean, sizeof fmean);
  std::memcpy(s->fistd, fistd, sizeof fistd);
  std::memcpy(s->fmin, fmin, sizeof fmin);
  std::memcpy(s->fmax, fmax, sizeof fmax);
  std::memcpy(s->tmean, tmean, sizeof tmean);
  std::memcpy(s->tistd, tistd, sizeof tistd);
  e = set_params(s, h.data(), 0);
  if (e == cudaSuccess) e = upload_norm(s, 0);
  if (e != cudaSuccess) return sur_cuda(ctx, e, "loading the surrogate");
  s->ready = true;
  return CHEM_OK;
}

}  // extern "C"
