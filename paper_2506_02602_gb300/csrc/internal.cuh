// internal.cuh -- declarations shared by the library's translation units (not part of
// the public ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

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

// Launchers (integrate.cu).  Return the cudaError_t of the launch.
cudaError_t launch_lsrk(int variant, const MechTables &mt, const CellArgs &a, const StepParams &p,
                        int block, cudaStream_t s);
cudaError_t launch_state_from_TPY(const MechTables &mt, int64_t n, const double *T,
                                  const double *p, const double *Y, int64_t ld, double *rho,
                                  double *e, cudaStream_t s);

}  // namespace chem
