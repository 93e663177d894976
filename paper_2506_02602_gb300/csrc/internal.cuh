// internal.cuh -- declarations shared by the library's translation units (not part of
// the public ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "chem.h"
#include "mech.cuh"

namespace chem {

// Pointers and sizes of one integration call (device pointers).
struct CellArgs {
  const double *rho;
  const double *e;
  double *Y;
  int64_t ld;
  double *T;
  double *h;
  int32_t *status;
  int32_t *nsteps;
  int64_t n;
  chem_stats *stats;
};

struct StepParams {
  double dt, rtol, atol;
  int32_t max_steps;
};

constexpr int kBatchBuckets = 64;

// A ragged batch (device pointers).
struct BatchArgs {
  const double *rho;
  const double *e;
  double *Y;
  int64_t ld;
  double *T;
  double *h;
  int32_t *status;
  int32_t *nsteps;
  int64_t n;
  const int64_t *box_off;
  const double *box_dt;
  const int32_t *box_nsub;
  int32_t nboxes;
  const int32_t *cost_hint;
  chem_stats *stats;
  // queue length read on the device (nullable: the queue holds n cells); lets a queue
  // built on the device (the surrogate's fallback list) run without a host round trip
  const unsigned int *nq_dev;
  int32_t ok_status;  // status written for cells that finish OK (CHEM_CELL_OK unless set)
};

// Context-owned queue scratch of the batched path.
struct BatchScratch {
  int32_t *order;                // [n] cell indices in queue order
  uint8_t *bucket;               // [n] stiffness bucket per cell
  int32_t *hist;                 // [kBatchBuckets] counts, then running offsets
  unsigned long long *cursor;    // [1] next queue slot
};

// Launchers (integrate.cu).  Return the cudaError_t of the launch.
cudaError_t launch_lsrk(int variant, int scheme, const MechTables &mt, const CellArgs &a,
                        const StepParams &p, int block, cudaStream_t s);
// Context accessors (api.cu) for entry points defined in other translation units.
std::string &chem_ctx_error(chem_ctx *ctx);
const MechTables &chem_ctx_tables(const chem_ctx *ctx);
int chem_ctx_variant(const chem_ctx *ctx);
int chem_ctx_scheme(const chem_ctx *ctx);
int chem_ctx_block(const chem_ctx *ctx);
// Device scratch of the 1D flow operators, grown to at least `bytes` (freed at teardown).
cudaError_t chem_ctx_flow_scratch(chem_ctx *ctx, size_t bytes, void **out);
int32_t chem_ctx_max_steps(const chem_ctx *ctx);
void *&chem_ctx_sur(chem_ctx *ctx);
void surrogate_destroy(void *sur);

// Argument checks of chem_integrate_batched and chem_integrate_batched_noalloc (api.cu):
// state, tolerances, batch arrays and options; on CHEM_OK *o holds the options with the
// defaults applied (opt may be NULL).  The message of a failure is set on ctx.
int check_batched_call(chem_ctx *ctx, const chem_state *state, int64_t ncells,
                       const chem_batch *batch, double rtol, double atol,
                       const chem_batch_options *opt, chem_batch_options *o);

cudaError_t launch_batched(int variant, const MechTables &mt, const BatchArgs &a,
                           const StepParams &p, const BatchScratch &s, int order_mode,
                           int ctas_per_sm, int shape, cudaStream_t st);
// The persistent kernel over a given queue of cell indices (order[0 .. queue length))
// with the variant's fastest shape (0 for fp64, the 32-warp shape 4 for mixed) and all
// resident CTAs; resets the cursor first.
cudaError_t launch_persistent_queue(int variant, const MechTables &mt, const BatchArgs &a,
                                    const StepParams &p, const int32_t *order,
                                    unsigned long long *cursor, cudaStream_t st);
// Threads per CTA, resident CTAs per SM, registers per thread of a persistent-kernel
// shape, and the device's SM count.
cudaError_t persistent_shape(int variant, int shape, int *block, int *ctas_per_sm, int *regs, int *num_sms);
cudaError_t launch_state_from_TPY(const MechTables &mt, int64_t n, const double *T,
                                  const double *p, const double *Y, int64_t ld, double *rho,
                                  double *e, cudaStream_t s);

}  // namespace chem
