// api.cu -- the extern "C" entry points of libchem.so (declared in include/chem.h):
// context set-up with mechanism validation and table packing, argument checking,
// launches on the caller's stream, the host-buffer convenience path, error strings.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <cstdint>
#include <string>

#include "internal.cuh"

using namespace chem;

struct chem_ctx {
  MechTables tables;
  chem_options opt;
  int device = 0;
  std::string err;
  // device scratch of chem_integrate_host (grown on demand, freed at teardown)
  void *host_scratch = nullptr;
  size_t host_scratch_bytes = 0;
  // queue scratch of chem_integrate_batched (grown on demand)
  void *batch_scratch = nullptr;
  int64_t batch_cap = 0;
  // cached CUDA graph of the last batched call and the arguments it was captured with
  cudaGraphExec_t graph = nullptr;
  cudaStream_t cap_stream = nullptr;  // private stream the graph is captured on
  unsigned char graph_key[512];
  size_t graph_key_len = 0;
  // learned surrogate (surrogate.cu), created by training or loading
  void *sur = nullptr;
  // copy pipeline of chem_integrate_host: copy-in, copy-out and a second compute stream,
  // and per-chunk events (created on first use)
  cudaStream_t io[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t ev[3 * 8 + 2] = {};
  // device scratch of the 1D flow operators (euler1d.cu; grown on demand)
  void *flow_scratch = nullptr;
  size_t flow_bytes = 0;
};

namespace {

thread_local std::string g_setup_err;

int fail(chem_ctx *ctx, int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (ctx) ctx->err = buf; else g_setup_err = buf;
  return code;
}

int cuda_fail(chem_ctx *ctx, cudaError_t e, const char *what) {
  return fail(ctx, CHEM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// NASA-7 helpers for validation (host side).
double nasa_cp(const double *a, double T) {
  return a[0] + T * (a[1] + T * (a[2] + T * (a[3] + T * a[4])));
}
double nasa_h(const double *a, double T) {  // h / R
  return T * (a[0] + T * (a[1] / 2 + T * (a[2] / 3 + T * (a[3] / 4 + T * a[4] / 5)))) + a[5];
}
double nasa_s(const double *a, double T) {  // s / R
  return a[0] * std::log(T) + T * (a[1] + T * (a[2] / 2 + T * (a[3] / 3 + T * a[4] / 4))) + a[6];
}

bool close_rel(double x, double y, double tol) {
  return std::fabs(x - y) <= tol * std::fmax(1.0, std::fmax(std::fabs(x), std::fabs(y)));
}

// Validate *m and pack it into *t.  Returns CHEM_OK or an error code (message set).
int build_tables(const chem_mechanism *m, MechTables *t) {
  if (m->n_species != NSP || m->n_reactions != NRX)
    return fail(nullptr, CHEM_ERR_UNSUPPORTED,
                "the library is compiled for %d species / %d reactions (got %d / %d)", NSP, NRX,
                m->n_species, m->n_reactions);
  std::memset(t, 0, sizeof *t);
  const double Tmid = m->T_mid[0];
  for (int k = 0; k < NSP; ++k) {
    if (!(m->W[k] > 0.0) || !std::isfinite(m->W[k]))
      return fail(nullptr, CHEM_ERR_INVALID, "species %d: molar mass must be positive", k);
    if (m->T_mid[k] != Tmid)
      return fail(nullptr, CHEM_ERR_UNSUPPORTED, "species %d: NASA-7 T_mid differs from species 0", k);
    for (int i = 0; i < 7; ++i)
      if (!std::isfinite(m->nasa_lo[k][i]) || !std::isfinite(m->nasa_hi[k][i]))
        return fail(nullptr, CHEM_ERR_INVALID, "species %d: non-finite NASA-7 coefficient", k);
    const double *lo = m->nasa_lo[k], *hi = m->nasa_hi[k];
    if (!close_rel(nasa_cp(lo, Tmid), nasa_cp(hi, Tmid), 1e-6) ||
        !close_rel(nasa_h(lo, Tmid), nasa_h(hi, Tmid), 1e-6) ||
        !close_rel(nasa_s(lo, Tmid), nasa_s(hi, Tmid), 1e-6))
      return fail(nullptr, CHEM_ERR_INVALID, "species %d: NASA-7 tables discontinuous at T_mid", k);
  }
  if (!(Tmid > 0.0)) return fail(nullptr, CHEM_ERR_INVALID, "T_mid must be positive");
  for (int j = 0; j < NRX; ++j) {
    // element balance (integers)
    for (int el = 0; el < CHEM_NUM_ELEMENTS; ++el) {
      long bal = 0;
      for (int k = 0; k < NSP; ++k) bal += (long)(m->nu_r[j][k] - m->nu_f[j][k]) * m->ncomp[k][el];
      if (bal != 0)
        return fail(nullptr, CHEM_ERR_INVALID, "reaction %d does not balance element %d", j, el);
    }
    // stoichiometry and type must match the compiled structure
    int want_f[NSP] = {0}, want_r[NSP] = {0};
    const RxStruct &R = kRx[j];
    if (R.r0 >= 0) want_f[R.r0]++;
    if (R.r1 >= 0) want_f[R.r1]++;
    if (R.p0 >= 0) want_r[R.p0]++;
    if (R.p1 >= 0) want_r[R.p1]++;
    for (int k = 0; k < NSP; ++k)
      if (m->nu_f[j][k] != want_f[k] || m->nu_r[j][k] != want_r[k])
        return fail(nullptr, CHEM_ERR_UNSUPPORTED,
                    "reaction %d: stoichiometry differs from the compiled structure %s", j, kMechStructure);
    for (int k = NSP; k < CHEM_MAX_SPECIES; ++k)
      if (m->nu_f[j][k] || m->nu_r[j][k])
        return fail(nullptr, CHEM_ERR_INVALID, "reaction %d uses a species beyond n_species", j);
    if (m->rtype[j] != R.type)
      return fail(nullptr, CHEM_ERR_UNSUPPORTED, "reaction %d: type %d, compiled type %d", j,
                  m->rtype[j], R.type);
    if (R.type == FALLOFF && m->troe_n[j] != R.troe_n)
      return fail(nullptr, CHEM_ERR_UNSUPPORTED, "reaction %d: %d Troe parameters, compiled %d", j,
                  m->troe_n[j], R.troe_n);
    if (!(m->A[j] > 0.0) || !std::isfinite(m->b[j]) || !std::isfinite(m->Ea[j]))
      return fail(nullptr, CHEM_ERR_INVALID, "reaction %d: Arrhenius parameters invalid", j);
    if (R.type == FALLOFF && (!(m->A0[j] > 0.0) || !std::isfinite(m->b0[j]) ||
                              !std::isfinite(m->Ea0[j])))
      return fail(nullptr, CHEM_ERR_INVALID, "reaction %d: low-pressure parameters invalid", j);
    if (R.type == FALLOFF && R.troe_n > 0 &&
        (!(m->troe[j][1] > 0.0) || !(m->troe[j][2] > 0.0) ||
         (R.troe_n == 4 && !std::isfinite(m->troe[j][3]))))
      return fail(nullptr, CHEM_ERR_INVALID, "reaction %d: Troe temperatures invalid", j);
  }

  t->T_mid = Tmid;
  for (int k = 0; k < NSP; ++k) {
    t->W[k] = m->W[k];
    t->invW[k] = 1.0 / m->W[k];
    for (int r = 0; r < 2; ++r) {
      const double *a = r ? m->nasa_hi[k] : m->nasa_lo[k];
      t->ec[r][k][0] = a[0] - 1.0;
      t->ec[r][k][1] = a[1] / 2.0;
      t->ec[r][k][2] = a[2] / 3.0;
      t->ec[r][k][3] = a[3] / 4.0;
      t->ec[r][k][4] = a[4] / 5.0;
      t->ec[r][k][5] = a[5];
      t->gc[r][k][0] = a[0];
      t->gc[r][k][1] = -a[1] / 2.0;
      t->gc[r][k][2] = -a[2] / 6.0;
      t->gc[r][k][3] = -a[3] / 12.0;
      t->gc[r][k][4] = -a[4] / 20.0;
      t->gc[r][k][5] = a[5];
      t->gc[r][k][6] = -a[6];
      for (int i = 0; i < 6; ++i) t->ecw[r][k][i] = t->ec[r][k][i] / m->W[k];
    }
  }
  {  // the largest |c_v' / c_v| of the tables on [200, 6000] K (1 K sampling)
    double C = 0.0;
    for (int k = 0; k < NSP; ++k)
      for (int r = 0; r < 2; ++r) {
        const double *a = r ? m->nasa_hi[k] : m->nasa_lo[k];
        const double T0 = r ? Tmid : 200.0, T1 = r ? 6000.0 : Tmid;
        for (double T = T0; T <= T1; T += 1.0) {
          const double cv = a[0] - 1.0 + T * (a[1] + T * (a[2] + T * (a[3] + T * a[4])));
          const double dcv = a[1] + T * (2.0 * a[2] + T * (3.0 * a[3] + T * 4.0 * a[4]));
          if (cv > 0.1) C = std::fmax(C, std::fabs(dcv / cv));
        }
      }
    t->newton_sq = C > 1e-6 ? 1e-12 / C : 1e-6;
  }
  for (int j = 0; j < NRX; ++j) {
    t->A[j] = m->A[j];
    t->lnA[j] = std::log(m->A[j]);
    t->beta[j] = m->b[j];
    t->Ta[j] = m->Ea[j] / R_U;
    t->kconst[j] = m->Ea[j] != 0.0 ? 0 : m->b[j] == 0.0 ? 1 : m->b[j] == -1.0 ? 2 : m->b[j] == -2.0 ? 3 : 0;
    t->reversible[j] = m->reversible[j] != 0;
    if (kRx[j].type == FALLOFF) {
      t->lnA0[j] = std::log(m->A0[j]);
      t->beta0[j] = m->b0[j];
      t->Ta0[j] = m->Ea0[j] / R_U;
      t->troe_a[j] = m->troe[j][0];
      t->troe_i3[j] = kRx[j].troe_n ? 1.0 / m->troe[j][1] : 0.0;
      t->troe_i1[j] = kRx[j].troe_n ? 1.0 / m->troe[j][2] : 0.0;
      t->troe_T2[j] = m->troe[j][3];
    }
    int any = 0, mask = 0;
    for (int k = 0; k < NSP; ++k) {
      t->effm1[j][k] = kRx[j].type == ELEM ? 0.0 : m->eff[j][k] - 1.0;
      any |= t->effm1[j][k] != 0.0;
      mask |= (t->effm1[j][k] != 0.0) << k;
    }
    t->has_eff[j] = any;
    t->eff_mask[j] = mask;
  }
  // element matrix (standard atomic masses of H, O, N)
  const double amass[CHEM_NUM_ELEMENTS] = {1.008e-3, 15.999e-3, 14.007e-3};
  for (int k = 0; k < NSP; ++k) {
    double wk = 0.0;
    for (int el = 0; el < CHEM_NUM_ELEMENTS; ++el) wk += m->ncomp[k][el] * amass[el];
    for (int el = 0; el < CHEM_NUM_ELEMENTS; ++el)
      t->Emat[el][k] = wk > 0.0 ? m->ncomp[k][el] * amass[el] / wk : 0.0;
  }
  // fp32 copies for the mixed-precision kernel
  t->ln_R_over_Pref = std::log(R_U / P_REF);
  for (int k = 0; k < NSP; ++k) {
    t->f.W[k] = (float)t->W[k];
    t->f.invW[k] = (float)t->invW[k];
  }
  for (int j = 0; j < NRX; ++j) {
    t->f.A[j] = (float)t->A[j];
    t->f.lnA[j] = (float)t->lnA[j];
    t->f.beta[j] = (float)t->beta[j];
    t->f.Ta[j] = (float)t->Ta[j];
    t->f.lnA0[j] = (float)t->lnA0[j];
    t->f.beta0[j] = (float)t->beta0[j];
    t->f.Ta0[j] = (float)t->Ta0[j];
    t->f.troe_a[j] = (float)t->troe_a[j];
    t->f.troe_i3[j] = (float)t->troe_i3[j];
    t->f.troe_i1[j] = (float)t->troe_i1[j];
    t->f.troe_T2[j] = (float)t->troe_T2[j];
    for (int k = 0; k < NSP; ++k) t->f.effm1[j][k] = (float)t->effm1[j][k];
  }
  for (int r = 0; r < 2; ++r)
    for (int k = 0; k < NSP; ++k) {
      for (int i = 0; i < 6; ++i) t->f.ec[r][k][i] = (float)t->ec[r][k][i];
      for (int i = 0; i < 7; ++i) t->f.gc[r][k][i] = (float)t->gc[r][k][i];
    }
  t->f.T_mid = (float)t->T_mid;
  t->f.ln_R_over_Pref = (float)t->ln_R_over_Pref;
  t->f.newton_sq = (float)t->newton_sq;
  return CHEM_OK;
}

bool aligned8(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 7u) == 0; }

int check_state(chem_ctx *ctx, const chem_state *s, int64_t n) {
  if (!s) return fail(ctx, CHEM_ERR_INVALID, "state is NULL");
  if (n < 0) return fail(ctx, CHEM_ERR_INVALID, "ncells < 0");
  if (n == 0) return CHEM_OK;
  if (!s->d_rho || !s->d_e || !s->d_Y || !s->d_T)
    return fail(ctx, CHEM_ERR_INVALID, "rho, e, Y and T are required");
  if (s->ldY < n) return fail(ctx, CHEM_ERR_INVALID, "ldY (%lld) < ncells (%lld)",
                              (long long)s->ldY, (long long)n);
  if (!aligned8(s->d_rho) || !aligned8(s->d_e) || !aligned8(s->d_Y) || !aligned8(s->d_T) ||
      !aligned8(s->d_h))
    return fail(ctx, CHEM_ERR_INVALID, "state pointers must be 8-byte aligned");
  return CHEM_OK;
}

int check_step(chem_ctx *ctx, double dt, double rtol, double atol) {
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(ctx, CHEM_ERR_INVALID, "dt must be > 0");
  if (!(rtol > 0.0) || !std::isfinite(rtol)) return fail(ctx, CHEM_ERR_INVALID, "rtol must be > 0");
  if (!(atol >= 0.0) || !std::isfinite(atol)) return fail(ctx, CHEM_ERR_INVALID, "atol must be >= 0");
  return CHEM_OK;
}

}  // namespace

namespace chem {

int check_batched_call(chem_ctx *ctx, const chem_state *state, int64_t ncells,
                       const chem_batch *batch, double rtol, double atol,
                       const chem_batch_options *opt, chem_batch_options *o) {
  if (!ctx) return fail(nullptr, CHEM_ERR_INVALID, "ctx is NULL");
  int rc = check_state(ctx, state, ncells);
  if (rc) return rc;
  rc = check_step(ctx, 1.0, rtol, atol);
  if (rc) return rc;
  if (ncells > INT32_MAX) return fail(ctx, CHEM_ERR_INVALID, "batched calls hold at most 2^31-1 cells");
  if (ctx->opt.scheme != CHEM_SCHEME_LSRK)
    return fail(ctx, CHEM_ERR_UNSUPPORTED, "the batched integrator runs the two-register scheme only");
  *o = chem_batch_options{};
  if (opt) *o = *opt;
  if (o->order != CHEM_ORDER_STIFFNESS && o->order != CHEM_ORDER_NATURAL)
    return fail(ctx, CHEM_ERR_INVALID, "unknown queue order %d", o->order);
  if (o->shape < 0 || o->shape >= CHEM_BATCH_SHAPES || o->ctas_per_sm < 0)
    return fail(ctx, CHEM_ERR_INVALID, "invalid batch options (shape %d, ctas_per_sm %d)", o->shape,
                o->ctas_per_sm);
  if (!batch || batch->nboxes < 1 || !batch->d_box_offset || !batch->d_box_dt || !batch->d_box_nsub)
    return fail(ctx, CHEM_ERR_INVALID, "batch needs nboxes >= 1 and its three device arrays");
  return CHEM_OK;
}

}  // namespace chem

extern "C" {

int chem_version(void) { return 10000; }

const char *chem_last_error(const chem_ctx *ctx) {
  return ctx ? ctx->err.c_str() : g_setup_err.c_str();
}

int chem_setup(const chem_mechanism *mech, const chem_options *opt, chem_ctx **out) {
  g_setup_err.clear();
  if (!mech || !out) return fail(nullptr, CHEM_ERR_INVALID, "mech and out are required");
  *out = nullptr;
  chem_options o{};
  if (opt) o = *opt;
  if (o.variant != CHEM_VARIANT_FP64 && o.variant != CHEM_VARIANT_MIXED)
    return fail(nullptr, CHEM_ERR_INVALID, "unknown variant %d", o.variant);
  if (o.max_steps < 0) return fail(nullptr, CHEM_ERR_INVALID, "max_steps < 0");
  if (o.max_steps == 0) o.max_steps = 100000;
  // default shape of the one-pass kernel: the 64-thread blocks for the mixed variant
  // (32 warps per SM at 64 registers, measured 3.8 % faster than 16 warps at 128), 12
  // warps at 170 registers for fp64 (whose 128-register build spills)
  if (o.block_size == 0) o.block_size = o.variant == CHEM_VARIANT_MIXED ? 64 : 128;
  if (o.scheme != CHEM_SCHEME_LSRK && o.scheme != CHEM_SCHEME_FULL_STORAGE && o.scheme != CHEM_SCHEME_RKF45)
    return fail(nullptr, CHEM_ERR_INVALID, "unknown scheme %d", o.scheme);
  for (int i = 0; i < 4; ++i)
    if (o.reserved[i]) return fail(nullptr, CHEM_ERR_INVALID, "reserved options must be zero");
  MechTables t;
  int rc = build_tables(mech, &t);
  if (rc != CHEM_OK) return rc;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return fail(nullptr, CHEM_ERR_CUDA, "no CUDA device available (%s)", cudaGetErrorString(e));
  }
  chem_ctx *ctx = new chem_ctx;
  ctx->tables = t;
  ctx->opt = o;
  cudaGetDevice(&ctx->device);
  *out = ctx;
  return CHEM_OK;
}

int chem_teardown(chem_ctx *ctx) {
  if (!ctx) return CHEM_OK;
  cudaDeviceSynchronize();
  if (ctx->host_scratch) cudaFree(ctx->host_scratch);
  for (cudaStream_t &q : ctx->io)
    if (q) cudaStreamDestroy(q);
  for (cudaEvent_t &v : ctx->ev)
    if (v) cudaEventDestroy(v);
  if (ctx->batch_scratch) cudaFree(ctx->batch_scratch);
  if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  if (ctx->sur) surrogate_destroy(ctx->sur);
  if (ctx->flow_scratch) cudaFree(ctx->flow_scratch);
  delete ctx;
  return CHEM_OK;
}

int chem_state_from_TPY(chem_ctx *ctx, int64_t n, const double *d_T, const double *d_p,
                        const double *d_Y, int64_t ldY, double *d_rho, double *d_e, void *stream) {
  if (!ctx) return fail(nullptr, CHEM_ERR_INVALID, "ctx is NULL");
  if (n < 0) return fail(ctx, CHEM_ERR_INVALID, "n < 0");
  if (n == 0) return CHEM_OK;
  if (!d_T || !d_p || !d_Y || !d_rho || !d_e) return fail(ctx, CHEM_ERR_INVALID, "NULL pointer");
  if (ldY < n) return fail(ctx, CHEM_ERR_INVALID, "ldY < n");
  cudaError_t e = launch_state_from_TPY(ctx->tables, n, d_T, d_p, d_Y, ldY, d_rho, d_e,
                                        (cudaStream_t)stream);
  return e == cudaSuccess ? CHEM_OK : cuda_fail(ctx, e, "state_from_TPY launch");
}

int chem_integrate(chem_ctx *ctx, const chem_state *state, int64_t ncells, double dt, double rtol,
                   double atol, void *stream, chem_stats *d_stats) {
  if (!ctx) return fail(nullptr, CHEM_ERR_INVALID, "ctx is NULL");
  int rc = check_state(ctx, state, ncells);
  if (rc) return rc;
  rc = check_step(ctx, dt, rtol, atol);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if (d_stats) {
    cudaError_t e = cudaMemsetAsync(d_stats, 0, sizeof(chem_stats), s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "clearing stats");
  }
  if (ncells == 0) return CHEM_OK;
  CellArgs a{state->d_rho, state->d_e, state->d_Y, state->ldY, state->d_T, state->d_h,
             state->d_status, state->d_nsteps, ncells, d_stats};
  StepParams p{dt, rtol, atol, ctx->opt.max_steps};
  cudaError_t e = launch_lsrk(ctx->opt.variant, ctx->opt.scheme, ctx->tables, a, p, ctx->opt.block_size, s);
  return e == cudaSuccess ? CHEM_OK : cuda_fail(ctx, e, "integration launch");
}

// Grow the batched path's queue scratch to hold n cells.
static int batch_scratch(chem_ctx *ctx, int64_t n, BatchScratch *out) {
  if (n > ctx->batch_cap) {
    if (ctx->batch_scratch) {
      cudaDeviceSynchronize();
      cudaFree(ctx->batch_scratch);
      ctx->batch_scratch = nullptr;
      ctx->batch_cap = 0;
    }
    if (ctx->graph) {  // the cached graph points into the old scratch
      cudaGraphExecDestroy(ctx->graph);
      ctx->graph = nullptr;
      ctx->graph_key_len = 0;
    }
    const size_t bytes = 256 + kBatchBuckets * sizeof(int32_t) + (size_t)n * 5 + 256;
    cudaError_t e = cudaMalloc(&ctx->batch_scratch, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      ctx->batch_scratch = nullptr;
      return fail(ctx, CHEM_ERR_NOMEM, "batch scratch of %zu bytes: %s", bytes, cudaGetErrorString(e));
    }
    ctx->batch_cap = n;
  }
  char *base = static_cast<char *>(ctx->batch_scratch);
  out->cursor = reinterpret_cast<unsigned long long *>(base);
  out->hist = reinterpret_cast<int32_t *>(base + 256);
  out->order = reinterpret_cast<int32_t *>(base + 256 + kBatchBuckets * sizeof(int32_t));
  out->bucket = reinterpret_cast<uint8_t *>(out->order + ctx->batch_cap);
  return CHEM_OK;
}

int chem_integrate_batched(chem_ctx *ctx, const chem_state *state, int64_t ncells,
                           const chem_batch *batch, double rtol, double atol,
                           const chem_batch_options *opt, void *stream, chem_stats *d_stats) {
  chem_batch_options o{};
  int rc = check_batched_call(ctx, state, ncells, batch, rtol, atol, opt, &o);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if (ncells == 0) {
    if (d_stats) {
      cudaError_t e = cudaMemsetAsync(d_stats, 0, sizeof(chem_stats), s);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "clearing stats");
    }
    return CHEM_OK;
  }
  BatchScratch sc;
  rc = batch_scratch(ctx, ncells, &sc);
  if (rc) return rc;
  BatchArgs a{state->d_rho, state->d_e, state->d_Y, state->ldY, state->d_T, state->d_h,
              state->d_status, state->d_nsteps, ncells, batch->d_box_offset, batch->d_box_dt,
              batch->d_box_nsub, batch->nboxes, o.d_cost_hint, d_stats,
              /*nq_dev=*/nullptr, /*ok_status=*/CHEM_CELL_OK};
  StepParams p{0.0, rtol, atol, ctx->opt.max_steps};
  auto issue = [&](cudaStream_t st) -> cudaError_t {
    if (d_stats) {
      cudaError_t e = cudaMemsetAsync(d_stats, 0, sizeof(chem_stats), st);
      if (e != cudaSuccess) return e;
    }
    return launch_batched(ctx->opt.variant, ctx->tables, a, p, sc, o.order, o.ctas_per_sm, o.shape, st);
  };
  if (!o.use_graph) {
    cudaError_t e = issue(s);
    return e == cudaSuccess ? CHEM_OK : cuda_fail(ctx, e, "batched launch");
  }
  // graph path: replay the cached graph when every argument is unchanged
  unsigned char key[512];
  size_t kl = 0;
  auto put = [&](const void *v, size_t nbytes) {
    std::memcpy(key + kl, v, nbytes);
    kl += nbytes;
  };
  put(&a, sizeof a);
  put(&p, sizeof p);
  put(&sc, sizeof sc);
  put(&o, sizeof o);
  cudaError_t e;
  if (!(ctx->graph && kl == ctx->graph_key_len && std::memcmp(key, ctx->graph_key, kl) == 0)) {
    cudaStreamCaptureStatus cap;
    e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "querying capture");
    if (cap != cudaStreamCaptureStatusNone) {  // already inside the caller's capture
      e = issue(s);
      return e == cudaSuccess ? CHEM_OK : cuda_fail(ctx, e, "batched launch");
    }
    if (ctx->graph) {
      cudaGraphExecDestroy(ctx->graph);
      ctx->graph = nullptr;
      ctx->graph_key_len = 0;
    }
    // capture on a private stream (the caller's may be the legacy default stream,
    // which cannot be captured); the graph then runs on the caller's stream
    if (!ctx->cap_stream) {
      e = cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "creating the capture stream");
    }
    e = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "beginning capture");
    cudaError_t le = issue(ctx->cap_stream);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(ctx->cap_stream, &g);
    if (le != cudaSuccess || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return cuda_fail(ctx, le != cudaSuccess ? le : e, "capturing the batched launch");
    }
    e = cudaGraphInstantiate(&ctx->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      ctx->graph = nullptr;
      return cuda_fail(ctx, e, "instantiating the batched graph");
    }
    std::memcpy(ctx->graph_key, key, kl);
    ctx->graph_key_len = kl;
  }
  e = cudaGraphLaunch(ctx->graph, s);
  return e == cudaSuccess ? CHEM_OK : cuda_fail(ctx, e, "graph launch");
}

int chem_integrate_host(chem_ctx *ctx, int64_t n, const double *h_rho, const double *h_e,
                        double *h_Y, int64_t ldY, double *h_T, double *h_h, int32_t *h_status,
                        int32_t *h_nsteps, double dt, double rtol, double atol, void *stream) {
  if (!ctx) return fail(nullptr, CHEM_ERR_INVALID, "ctx is NULL");
  if (n < 0) return fail(ctx, CHEM_ERR_INVALID, "ncells < 0");
  int rc = check_step(ctx, dt, rtol, atol);
  if (rc) return rc;
  if (n == 0) return CHEM_OK;
  if (!h_rho || !h_e || !h_Y || !h_T) return fail(ctx, CHEM_ERR_INVALID, "rho, e, Y, T required");
  if (ldY < n) return fail(ctx, CHEM_ERR_INVALID, "ldY < ncells");
  // device layout: rho, e, T, h [n] + Y [NSP * n] doubles, then status, nsteps [n] int32
  const size_t nd = (size_t)n;
  const size_t need = (4 + NSP) * nd * sizeof(double) + 2 * nd * sizeof(int32_t);
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if (need > ctx->host_scratch_bytes) {
    if (ctx->host_scratch) {
      cudaStreamSynchronize(s);
      cudaFree(ctx->host_scratch);
      ctx->host_scratch = nullptr;
      ctx->host_scratch_bytes = 0;
    }
    e = cudaMalloc(&ctx->host_scratch, need);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, CHEM_ERR_NOMEM, "device scratch of %zu bytes: %s", need,
                  cudaGetErrorString(e));
    }
    ctx->host_scratch_bytes = need;
  }
  double *d = static_cast<double *>(ctx->host_scratch);
  double *d_rho = d, *d_e = d + nd, *d_T = d + 2 * nd, *d_h = d + 3 * nd, *d_Y = d + 4 * nd;
  int32_t *d_status = reinterpret_cast<int32_t *>(d + (4 + NSP) * nd);
  int32_t *d_nsteps = d_status + nd;
  const size_t bytes = nd * sizeof(double);
#define CK(call, what)                                   \
  do {                                                   \
    e = (call);                                          \
    if (e != cudaSuccess) return cuda_fail(ctx, e, what); \
  } while (0)
  // Large calls: a chunked pipeline that overlaps the copies with the integration.
  // Chunk c's cells go in on a copy-in stream, are integrated on one of two compute
  // streams (the caller's and a private one, alternating, so one chunk's tail overlaps
  // the next chunk's start), and come back on a copy-out stream; events order the
  // three, and the caller's stream waits for the whole pipeline.
  constexpr int kChunks = 4;
  if (n >= (1 << 18)) {
    for (cudaStream_t &q : ctx->io)
      if (!q) CK(cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking), "creating copy streams");
    for (cudaEvent_t &v : ctx->ev)
      if (!v) CK(cudaEventCreateWithFlags(&v, cudaEventDisableTiming), "creating events");
    cudaStream_t in = ctx->io[0], out = ctx->io[1], comp2 = ctx->io[2];
    cudaEvent_t ev_start = ctx->ev[3 * 8], ev_done = ctx->ev[3 * 8 + 1];
    CK(cudaEventRecord(ev_start, s), "event");
    CK(cudaStreamWaitEvent(in, ev_start, 0), "event wait");
    CK(cudaStreamWaitEvent(comp2, ev_start, 0), "event wait");
    const int64_t per = (n + kChunks - 1) / kChunks;
    for (int c = 0; c < kChunks; ++c) {
      const int64_t c0 = c * per, c1 = c0 + per < n ? c0 + per : n;
      if (c1 <= c0) break;
      const size_t m = (size_t)(c1 - c0), mb = m * sizeof(double);
      cudaEvent_t ev_in = ctx->ev[3 * c], ev_comp = ctx->ev[3 * c + 1];
      CK(cudaMemcpyAsync(d_rho + c0, h_rho + c0, mb, cudaMemcpyHostToDevice, in), "copy rho");
      CK(cudaMemcpyAsync(d_e + c0, h_e + c0, mb, cudaMemcpyHostToDevice, in), "copy e");
      CK(cudaMemcpyAsync(d_T + c0, h_T + c0, mb, cudaMemcpyHostToDevice, in), "copy T");
      if (h_h) CK(cudaMemcpyAsync(d_h + c0, h_h + c0, mb, cudaMemcpyHostToDevice, in), "copy h");
      CK(cudaMemcpy2DAsync(d_Y + c0, bytes, h_Y + c0, (size_t)ldY * sizeof(double), mb, NSP,
                           cudaMemcpyHostToDevice, in), "copy Y");
      CK(cudaEventRecord(ev_in, in), "event");
      cudaStream_t cs = (c & 1) ? comp2 : s;
      CK(cudaStreamWaitEvent(cs, ev_in, 0), "event wait");
      CellArgs a{d_rho + c0, d_e + c0, d_Y + c0, (int64_t)nd, d_T + c0, h_h ? d_h + c0 : nullptr,
                 d_status + c0, d_nsteps + c0, (int64_t)m, nullptr};
      StepParams p{dt, rtol, atol, ctx->opt.max_steps};
      CK(launch_lsrk(ctx->opt.variant, ctx->opt.scheme, ctx->tables, a, p, ctx->opt.block_size, cs), "integration launch");
      CK(cudaEventRecord(ev_comp, cs), "event");
      CK(cudaStreamWaitEvent(out, ev_comp, 0), "event wait");
      CK(cudaMemcpy2DAsync(h_Y + c0, (size_t)ldY * sizeof(double), d_Y + c0, bytes, mb, NSP,
                           cudaMemcpyDeviceToHost, out), "copy Y back");
      CK(cudaMemcpyAsync(h_T + c0, d_T + c0, mb, cudaMemcpyDeviceToHost, out), "copy T back");
      if (h_h) CK(cudaMemcpyAsync(h_h + c0, d_h + c0, mb, cudaMemcpyDeviceToHost, out), "copy h back");
      if (h_status)
        CK(cudaMemcpyAsync(h_status + c0, d_status + c0, m * sizeof(int32_t), cudaMemcpyDeviceToHost, out),
           "copy status back");
      if (h_nsteps)
        CK(cudaMemcpyAsync(h_nsteps + c0, d_nsteps + c0, m * sizeof(int32_t), cudaMemcpyDeviceToHost, out),
           "copy nsteps back");
    }
    CK(cudaEventRecord(ev_done, out), "event");
    CK(cudaStreamWaitEvent(s, ev_done, 0), "event wait");
    CK(cudaStreamSynchronize(s), "synchronising");
    return CHEM_OK;
  }
  CK(cudaMemcpyAsync(d_rho, h_rho, bytes, cudaMemcpyHostToDevice, s), "copy rho");
  CK(cudaMemcpyAsync(d_e, h_e, bytes, cudaMemcpyHostToDevice, s), "copy e");
  CK(cudaMemcpyAsync(d_T, h_T, bytes, cudaMemcpyHostToDevice, s), "copy T");
  if (h_h) CK(cudaMemcpyAsync(d_h, h_h, bytes, cudaMemcpyHostToDevice, s), "copy h");
  CK(cudaMemcpy2DAsync(d_Y, bytes, h_Y, (size_t)ldY * sizeof(double), bytes, NSP,
                       cudaMemcpyHostToDevice, s), "copy Y");
  CellArgs a{d_rho, d_e, d_Y, (int64_t)nd, d_T, h_h ? d_h : nullptr, d_status, d_nsteps, n, nullptr};
  StepParams p{dt, rtol, atol, ctx->opt.max_steps};
  CK(launch_lsrk(ctx->opt.variant, ctx->opt.scheme, ctx->tables, a, p, ctx->opt.block_size, s), "integration launch");
  CK(cudaMemcpy2DAsync(h_Y, (size_t)ldY * sizeof(double), d_Y, bytes, bytes, NSP,
                       cudaMemcpyDeviceToHost, s), "copy Y back");
  CK(cudaMemcpyAsync(h_T, d_T, bytes, cudaMemcpyDeviceToHost, s), "copy T back");
  if (h_h) CK(cudaMemcpyAsync(h_h, d_h, bytes, cudaMemcpyDeviceToHost, s), "copy h back");
  if (h_status)
    CK(cudaMemcpyAsync(h_status, d_status, nd * sizeof(int32_t), cudaMemcpyDeviceToHost, s),
       "copy status back");
  if (h_nsteps)
    CK(cudaMemcpyAsync(h_nsteps, d_nsteps, nd * sizeof(int32_t), cudaMemcpyDeviceToHost, s),
       "copy nsteps back");
  CK(cudaStreamSynchronize(s), "synchronising");
#undef CK
  return CHEM_OK;
}

}  // extern "C"

// Accessors for the allocation-free batched entry point (batched.cu).
namespace chem {
std::string &chem_ctx_error(chem_ctx *ctx) { return ctx->err; }
const MechTables &chem_ctx_tables(const chem_ctx *ctx) { return ctx->tables; }
int chem_ctx_variant(const chem_ctx *ctx) { return ctx->opt.variant; }
int chem_ctx_scheme(const chem_ctx *ctx) { return ctx->opt.scheme; }
int chem_ctx_block(const chem_ctx *ctx) { return ctx->opt.block_size; }
cudaError_t chem_ctx_flow_scratch(chem_ctx *ctx, size_t bytes, void **out) {
  if (bytes > ctx->flow_bytes) {
    if (ctx->flow_scratch) cudaFree(ctx->flow_scratch);
    ctx->flow_scratch = nullptr;
    ctx->flow_bytes = 0;
    cudaError_t e = cudaMalloc(&ctx->flow_scratch, bytes);
    if (e != cudaSuccess) return e;
    ctx->flow_bytes = bytes;
  }
  *out = ctx->flow_scratch;
  return cudaSuccess;
}
int32_t chem_ctx_max_steps(const chem_ctx *ctx) { return ctx->opt.max_steps; }
void *&chem_ctx_sur(chem_ctx *ctx) { return ctx->sur; }
}  // namespace chem
