// surrogate_stub.cu -- the chem_surrogate_* entry points of a library compiled for a
// mechanism structure other than the 9-species one.  The learned surrogate's network
// shape (12 features -> 9 outputs) and its element projection are those of the
// 9-species mechanism, so these builds carry no surrogate: every call returns
// CHEM_ERR_UNSUPPORTED with a message, and chem_surrogate_param_count returns 0.
#include <cuda_runtime.h>

#include <string>

#include "internal.cuh"

namespace chem {

void surrogate_destroy(void *) {}

static int no_surrogate(chem_ctx *ctx) {
  if (ctx) chem_ctx_error(ctx) = std::string("the learned surrogate is built for the 9-species mechanism only; "
                                             "this library is compiled for ") + kMechStructure;
  return CHEM_ERR_UNSUPPORTED;
}

}  // namespace chem

using chem::no_surrogate;

extern "C" {

int64_t chem_surrogate_param_count(void) { return 0; }
int chem_surrogate_params(chem_ctx *ctx, float *, const float *, int64_t) { return no_surrogate(ctx); }
int chem_surrogate_grad(chem_ctx *ctx, const float *, const float *, int64_t, float *, float *, float *,
                        void *) {
  return no_surrogate(ctx);
}
int chem_surrogate_trace(chem_ctx *ctx, const float *, const float *, int64_t, float *, float *, uint16_t *,
                         uint16_t *, float *, float *, float *, void *) {
  return no_surrogate(ctx);
}
int chem_surrogate_adam(chem_ctx *ctx, const float *, int64_t, float) { return no_surrogate(ctx); }
int chem_surrogate_project(chem_ctx *ctx, int64_t, const double *, const double *, int64_t, double *,
                           void *) {
  return no_surrogate(ctx);
}
int chem_surrogate_forward(chem_ctx *ctx, const float *, int64_t, float *, int32_t, void *, int32_t *) {
  return no_surrogate(ctx);
}
int chem_surrogate_train(chem_ctx *ctx, const chem_pairs *, int64_t, const chem_train_cfg *, void *,
                         float *) {
  return no_surrogate(ctx);
}
int chem_surrogate_infer(chem_ctx *ctx, const chem_state *, int64_t, double, double, double,
                         const chem_surrogate_gate *, void *, uint8_t *, chem_stats *) {
  return no_surrogate(ctx);
}
int chem_surrogate_infer_batched(chem_ctx *ctx, const chem_state *, int64_t, const chem_batch *, double,
                                 double, const chem_surrogate_gate *, void *, uint8_t *, chem_stats *) {
  return no_surrogate(ctx);
}
int chem_surrogate_save(chem_ctx *ctx, const char *) { return no_surrogate(ctx); }
int chem_surrogate_load(chem_ctx *ctx, const char *) { return no_surrogate(ctx); }

}  // extern "C"
