/*
 * chem.h -- C ABI of the GB300 per-cell chemistry integrator (libchem.so).
 *
 * The library advances every cell of a reacting-flow field through one hydrodynamic
 * time step of the chemical source term.  Each cell is an independent
 * constant-density, constant-internal-energy adiabatic reactor: the source term of
 * Eq. 14 changes only the species partial densities, so (rho, e) stay fixed while the
 * mass fractions Y_k evolve under the law of mass action (Eq. 15-16) with Arrhenius
 * forward rates and reverse rates from equilibrium constants (Sec. 2.1.2).  The
 * temperature is recovered from e by Newton iteration on NASA-7 polynomials (Eq. 10;
 * calculate_T of Table 1) at every right-hand-side evaluation.  The integrator is the
 * five-stage fourth-order low-storage embedded Runge-Kutta scheme of Eq. 21 with the
 * WRMS step-size controller of Eq. 22 (Sec. 2.2.3), one GPU thread per cell
 * (Sec. 4.1.2).
 *
 * Conventions for every entry point:
 *   - Return value: CHEM_OK (0) or a negative chem_error code.  Arguments are checked
 *     before anything is launched; chem_last_error() describes the last failure of a
 *     context.  Per-cell outcomes never fail a call: they go to status[].
 *   - Pointers named d_* are device pointers (cudaMalloc'd, or any memory the
 *     device can address); h_* are host pointers.  The caller owns all of them; the
 *     library never frees a caller pointer.  The library owns its context and the
 *     scratch it allocates.
 *   - stream is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *     Calls that take a stream are asynchronous with respect to the host unless they
 *     say otherwise; results are ready once the stream has been synchronised.
 *   - Cell arrays are structure-of-arrays fp64: plane k of Y starts at Y + k * ldY
 *     (ldY >= ncells), and every plane pointer must be 8-byte aligned.
 *   - Units are SI: kg/m^3, J/kg, K, Pa, s, kg/mol, J/mol.
 *   - There is no CPU fallback: without a CUDA device every compute call returns
 *     CHEM_ERR_CUDA.
 */
#ifndef CHEM_H
#define CHEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CHEM_MAX_SPECIES 16
#define CHEM_MAX_REACTIONS 32
#define CHEM_NUM_ELEMENTS 3 /* H, O, N */

typedef enum {
  CHEM_OK = 0,
  CHEM_ERR_INVALID = -1,     /* bad argument; nothing was launched */
  CHEM_ERR_CUDA = -2,        /* a CUDA call or launch failed */
  CHEM_ERR_UNSUPPORTED = -3, /* valid input the compiled library has no kernel for */
  CHEM_ERR_NOMEM = -4,       /* a device allocation failed */
  CHEM_ERR_TIMEOUT = -5,     /* a bounded device-side wait gave up */
  CHEM_ERR_STATE = -6        /* call out of order (e.g. inference before training) */
} chem_error;

/* Per-cell outcome codes written to status[]. */
typedef enum {
  CHEM_CELL_OK = 0,
  CHEM_CELL_MAX_STEPS = 1,   /* attempted-step limit reached; state = last accepted */
  CHEM_CELL_H_UNDERFLOW = 2, /* step fell below 1e-15 dt; state = last accepted */
  CHEM_CELL_NEWTON_FAIL = 3, /* no temperature root for the accepted state */
  CHEM_CELL_NONFINITE = 4,   /* non-finite or non-positive input */
  CHEM_CELL_SURROGATE = 5    /* informational: the surrogate's answer was rejected and
                                the cell was integrated instead */
} chem_cell_status;

typedef enum {
  CHEM_VARIANT_FP64 = 0,  /* every value in fp64 (reciprocals by Newton-Raphson refinement
                             of the hardware approximation, within 2 ulp except in the
                             temperature solve's step, 2^-40; that solve's stop test
                             compares the fp32-rounded step and temperature) */
  CHEM_VARIANT_MIXED = 1  /* rates and RK stage derivatives in fp32; temperature solve,
                             Gibbs functions, solution and error registers and step
                             control in fp64; ln(1/K_c) is the fp64 sum of the Gibbs
                             terms rounded once to fp32 for the fp32 reverse rate */
} chem_variant;

/*
 * Reaction mechanism (Eq. 15-16; thermo of Eq. 10).  Species k has molar mass W[k],
 * element counts ncomp[k][H, O, N] and NASA-7 tables nasa_lo[k] (T < T_mid[k]) and
 * nasa_hi[k]: cp/R = a1 + a2 T + a3 T^2 + a4 T^3 + a5 T^4, h/RT adds a6/T, s/R adds a7.
 * Reaction j has stoichiometric coefficients nu_f[j][k] (reactants) and nu_r[j][k]
 * (products), type rtype[j] (0 elementary, 1 third body: rate times
 * [M] = sum_k eff[j][k] c_k, 2 fall-off: k = k_inf Pr / (1 + Pr) F with
 * Pr = k0 [M] / k_inf), Arrhenius k = A T^b exp(-Ea / (R_u T)) (high-pressure limit for
 * fall-off; low-pressure limit A0, b0, Ea0), Troe parameters troe[j] = {alpha, T***,
 * T*, T**} with troe_n[j] in {0 (Lindemann), 3, 4}, and reversible[j].  Reverse rates
 * are k_f / K_c with K_c = exp(-sum_k nu_jk g_k / (R_u T)) (101325 Pa / (R_u T))^sum nu.
 */
typedef struct {
  int32_t n_species;
  int32_t n_reactions;
  double W[CHEM_MAX_SPECIES];
  int32_t ncomp[CHEM_MAX_SPECIES][CHEM_NUM_ELEMENTS];
  double T_mid[CHEM_MAX_SPECIES];
  double nasa_lo[CHEM_MAX_SPECIES][7];
  double nasa_hi[CHEM_MAX_SPECIES][7];
  int32_t rtype[CHEM_MAX_REACTIONS];
  int32_t nu_f[CHEM_MAX_REACTIONS][CHEM_MAX_SPECIES];
  int32_t nu_r[CHEM_MAX_REACTIONS][CHEM_MAX_SPECIES];
  double A[CHEM_MAX_REACTIONS], b[CHEM_MAX_REACTIONS], Ea[CHEM_MAX_REACTIONS];
  double A0[CHEM_MAX_REACTIONS], b0[CHEM_MAX_REACTIONS], Ea0[CHEM_MAX_REACTIONS];
  double troe[CHEM_MAX_REACTIONS][4];
  int32_t troe_n[CHEM_MAX_REACTIONS];
  double eff[CHEM_MAX_REACTIONS][CHEM_MAX_SPECIES];
  int32_t reversible[CHEM_MAX_REACTIONS];
} chem_mechanism;

/*
 * Integration scheme.  The paper's method is the two-register low-storage scheme of
 * Eq. 21; the others are the conventional explicit comparators the paper measures it
 * against (Sec. 2.2.3, Sec. 4.2.2), keeping every stage derivative: the same RK4(3)5
 * tableau in Butcher form, and Fehlberg's RKF45 (six stages, fourth-order solution,
 * fifth-order error estimate, controller exponent 1/5).  Only chem_integrate and
 * chem_integrate_host run the comparators.
 */
typedef enum {
  CHEM_SCHEME_LSRK = 0,          /* RK4(3)5[2R+]C, two registers plus the error register */
  CHEM_SCHEME_FULL_STORAGE = 1,  /* the same tableau with all five k_i kept */
  CHEM_SCHEME_RKF45 = 2          /* Fehlberg 4(5), all six k_i kept */
} chem_scheme;

/* Options fixed at setup.  Zero-initialised fields take the defaults in brackets. */
typedef struct {
  int32_t variant;     /* chem_variant [CHEM_VARIANT_FP64] */
  int32_t max_steps;   /* attempted-step limit per cell and call [100000] */
  int32_t block_size;  /* threads per block of the one-pass integration kernel: 32 or 64
                          (16 warps per SM, 128 registers a thread; 32 warps at 64
                          registers for the mixed two-register scheme), 128 (12 warps,
                          170 registers) or 256 (8 warps, 255 registers); other values
                          take 128 [0: 64 for the mixed variant, 128 for fp64] */
  int32_t scheme;      /* chem_scheme [CHEM_SCHEME_LSRK]; the comparators serve
                          chem_integrate and chem_integrate_host only: the batched and
                          surrogate calls of a context with another scheme return
                          CHEM_ERR_UNSUPPORTED */
  int32_t reserved[4]; /* must be zero */
} chem_options;

/*
 * State of ncells cells, all device pointers, structure of arrays.
 *   d_rho[n], d_e[n]      in: density, specific internal energy (constant over dt)
 *   d_Y[k * ldY + i]      in/out: mass fractions, advanced in place
 *   d_T[n]                in: Newton starting guess (NaN or <= 0 -> 1500 K);
 *                         out: temperature of the final state
 *   d_h[n]  (nullable)    in: initial step per cell (<= 0 or NaN -> dt);
 *                         out: the controller's next step, to carry into the next call
 *   d_status[n] (nullable) out: chem_cell_status
 *   d_nsteps[n] (nullable) out: attempted steps (accepted + rejected)
 */
typedef struct {
  const double *d_rho;
  const double *d_e;
  double *d_Y;
  int64_t ldY;
  double *d_T;
  double *d_h;
  int32_t *d_status;
  int32_t *d_nsteps;
} chem_state;

/* Aggregate counters of one call (filled by warp reductions, one atomic per warp). */
typedef struct {
  int64_t cells;
  int64_t accepted;
  int64_t rejected;
  int64_t rhs_evals;
  int64_t max_steps_cell; /* largest attempted-step count of any cell */
  int64_t status_count[8];
} chem_stats;

typedef struct chem_ctx chem_ctx;

/*
 * Create a context for mechanism *mech (copied; the caller keeps ownership).
 * Validates the mechanism: element balance of every reaction (integers), NASA-7
 * continuity of cp, h and s at T_mid (relative 1e-6), a common T_mid, positive molar
 * masses.  The library's kernels are specialised at compile time to the structure of
 * the 9-species / 21-reaction H2-O2-N2 mechanism (species H2, O2, H2O, H, O, OH, HO2,
 * H2O2, N2 in that order; the reaction list of chem_inputs.mechanism): a mechanism
 * with other stoichiometry or reaction types returns CHEM_ERR_UNSUPPORTED.  Its
 * coefficients (rates, efficiencies, Troe, thermo) are free.  Needs a CUDA device.
 * On success *out owns device scratch until chem_teardown.  opt may be NULL.
 */
int chem_setup(const chem_mechanism *mech, const chem_options *opt, chem_ctx **out);

/* Free a context and everything it owns.  NULL is accepted.  Synchronises the device. */
int chem_teardown(chem_ctx *ctx);

/* Message of the last failed call on ctx (or of the last failed chem_setup when ctx
 * is NULL).  The string stays valid until the next call on the same context. */
const char *chem_last_error(const chem_ctx *ctx);

/*
 * Conserved state from (T, p, Y) (Eq. 6 and Eq. 10): rho = p Wbar / (R_u T),
 * e = sum_k Y_k (h_k(T) - R_u T) / W_k.  d_T, d_p: [n]; d_Y: planes with stride ldY;
 * outputs d_rho, d_e: [n].  Asynchronous on stream.
 */
int chem_state_from_TPY(chem_ctx *ctx, int64_t n, const double *d_T, const double *d_p,
                        const double *d_Y, int64_t ldY, double *d_rho, double *d_e,
                        void *stream);

/*
 * Integrate every cell of *state over [0, dt] (Eq. 20-22), one thread per cell, in the
 * precision variant chosen at setup.  rtol, atol: the WRMS tolerances of Eq. 22
 * (the paper uses 1e-6 and 1e-10); the norm runs over the species mass fractions with
 * |u_i| = max(|y_n,i|, |y_n+1,i|).  Step controller: safety 0.9, exponent 1/4,
 * growth and shrink factors clamped to [1/5, 5]; accept iff ||e|| <= 1; the step is
 * clipped to land on dt.  A trial stage without a temperature root rejects the
 * attempt with factor 1/5.
 * d_stats (nullable): a device pointer to a chem_stats that the call zeroes and fills.
 * Errors: ncells < 0, dt <= 0, rtol <= 0, atol < 0, a NULL required pointer or
 * ldY < ncells -> CHEM_ERR_INVALID.  ncells == 0 is a no-op.  Asynchronous on stream.
 */
int chem_integrate(chem_ctx *ctx, const chem_state *state, int64_t ncells, double dt,
                   double rtol, double atol, void *stream, chem_stats *d_stats);

/*
 * The same integration with the cells' host copies: copies h_rho, h_e, h_Y (ldY),
 * h_T (and h_h if given) to device scratch owned by the context, integrates, and
 * copies Y, T, status, nsteps (and h) back into the host arrays.  Synchronous: it
 * returns after the results are in host memory.  Pinned host memory gives the
 * fastest copies.  Same argument rules as chem_integrate; h_status/h_nsteps/h_h are
 * nullable.
 */
int chem_integrate_host(chem_ctx *ctx, int64_t ncells, const double *h_rho,
                        const double *h_e, double *h_Y, int64_t ldY, double *h_T,
                        double *h_h, int32_t *h_status, int32_t *h_nsteps, double dt,
                        double rtol, double atol, void *stream);

/* Queue order of the batched integrator. */
typedef enum {
  CHEM_ORDER_STIFFNESS = 0, /* cells sorted by a stiffness key, most expensive first */
  CHEM_ORDER_NATURAL = 1    /* cells taken in index order */
} chem_queue_order;

/*
 * A ragged batch of boxes (the boxes of an AMR hierarchy, Sec. 3.1).  Box b owns the
 * contiguous cells [d_box_offset[b], d_box_offset[b+1]) of the state and advances them
 * by d_box_nsub[b] successive substeps of d_box_dt[b] seconds each (a level subcycled
 * per Alg. 1 takes 2^l substeps of dt / 2^l).  All three arrays are device memory:
 * d_box_offset[nboxes + 1] (int64, nondecreasing, d_box_offset[0] = 0,
 * d_box_offset[nboxes] = ncells), d_box_dt[nboxes] (> 0), d_box_nsub[nboxes] (>= 1).
 * Offsets that break these rules assign cells to the wrong box but never address memory
 * outside the state.
 */
typedef struct {
  int32_t nboxes;
  const int64_t *d_box_offset;
  const double *d_box_dt;
  const int32_t *d_box_nsub;
} chem_batch;

/* Compiled shapes of the persistent kernel: (threads per CTA, minimum resident CTAs
 * per SM, hence a register cap of min(255, 65536 / (threads * CTAs))):
 * 0 = (128, 2) [default, no cap in effect], 1 = (128, 3), 2 = (128, 4), 3 = (64, 6),
 * 4 = (64, 8) [(64, 16) for the mixed variant of the 9-species library], 5 = (256, 2).
 * All run the same algorithm; the compiler contracts
 * multiply-adds per compiled kernel, so results of different shapes agree to rounding
 * (to the integration tolerance in ill-conditioned cells), not bit for bit.  Shape 0
 * gives the results of chem_integrate. */
#define CHEM_BATCH_SHAPES 6

/* Options of chem_integrate_batched.  Zero-initialised = the defaults. */
typedef struct {
  int32_t order;               /* chem_queue_order [CHEM_ORDER_STIFFNESS] */
  int32_t ctas_per_sm;         /* persistent CTAs per SM; 0 = all that fit [0] */
  int32_t use_graph;           /* 1: capture the call's launches in a CUDA graph and
                                  replay it while the arguments are unchanged [0] */
  int32_t shape;               /* persistent-kernel shape, 0 .. CHEM_BATCH_SHAPES-1 [0] */
  const int32_t *d_cost_hint;  /* nullable device [ncells]: per-cell cost used as the
                                  stiffness key instead of the probe (e.g. d_nsteps of
                                  the previous call) */
} chem_batch_options;

/*
 * Integrate a ragged batch in one persistent launch with work stealing (Eq. 21-22 per
 * cell, as chem_integrate).  The state covers all ncells cells of all boxes.  Steps:
 * a stiffness key per cell (the cost hint, or one right-hand side giving accuracy and
 * stability step estimates, times the box's substeps), a counting sort of the cells
 * into descending-cost order, then a persistent kernel whose lanes take cells from the
 * sorted queue through an atomic cursor and integrate all their substeps; a lane that
 * finishes takes the next cell.  d_h carries the step across substeps; d_nsteps counts
 * attempts over all substeps; max_steps applies per cell and call.  Results do not
 * depend on the queue order.  The context owns the queue scratch (5 bytes per cell plus
 * 520 bytes), allocated on the first call that needs more: make one uncaptured call of
 * the largest size before capturing calls in a CUDA graph.  opt may be NULL.
 * Errors: as chem_integrate, plus nboxes < 1, NULL box arrays, unknown order, shape out
 * of range, ctas_per_sm < 0 -> CHEM_ERR_INVALID; allocation failure -> CHEM_ERR_NOMEM.
 * Asynchronous.
 */
int chem_integrate_batched(chem_ctx *ctx, const chem_state *state, int64_t ncells,
                           const chem_batch *batch, double rtol, double atol,
                           const chem_batch_options *opt, void *stream, chem_stats *d_stats);

/* Threads per CTA, registers per thread and resident CTAs per SM of a persistent-kernel
 * shape in the context's variant (outputs nullable).  Errors: shape out of range ->
 * CHEM_ERR_INVALID; CUDA -> CHEM_ERR_CUDA. */
int chem_batch_shape_info(chem_ctx *ctx, int32_t shape, int32_t *block, int32_t *regs,
                          int32_t *ctas_per_sm);

/* One timed candidate of chem_autotune_batched. */
typedef struct {
  chem_batch_options opt;  /* the candidate */
  float ms;                /* best of two timed launches (after one untimed), ms */
  int32_t block;           /* threads per CTA of its shape */
  int32_t regs;            /* registers per thread of its shape */
  int32_t ctas_per_sm;     /* resident CTAs per SM it ran with */
} chem_tune_result;

/*
 * Autotuner of chem_integrate_batched (no counterpart in the paper, which sizes boxes
 * and streams by hand, Sec. 4.1.2).  Times candidate options on the caller's own batch,
 * integrating private copies of Y, T (and h): the caller's state is not modified.
 * Coordinate descent: every shape (stiffness order, all resident CTAs), then the
 * natural order, then fewer CTAs per SM, then graph replay, each step keeping the
 * fastest.  *best receives the fastest options (base's d_cost_hint kept; base may be
 * NULL).  h_results (nullable, host [max_results]) receives the timed candidates and
 * *n_results their count.
 * cache_path (nullable): a text file of earlier results, one line per key (device name,
 * SM count, variant, max_steps, rtol, atol, floor(log2 ncells), floor(log2 nboxes));
 * on a hit *best comes from the file, nothing is launched and *n_results = 0; on a miss
 * the result is appended.  Synchronous; allocates the copies for the duration of the
 * call.  Errors: as chem_integrate_batched; unreadable cache lines are skipped; a cache
 * file that cannot be written -> CHEM_ERR_INVALID after *best is set.
 */
int chem_autotune_batched(chem_ctx *ctx, const chem_state *state, int64_t ncells,
                          const chem_batch *batch, double rtol, double atol,
                          const chem_batch_options *base, const char *cache_path, void *stream,
                          chem_batch_options *best, chem_tune_result *h_results,
                          int32_t max_results, int32_t *n_results);

/* ---------------------------------------------------------------- learned surrogate
 *
 * A multilayer perceptron 12 -> 256 -> 256 -> 256 -> 9 (GELU, BF16 weights and
 * activations, FP32 accumulation and master weights) that maps a cell's state and step
 * to the change of its Box-Cox-transformed mass fractions over the step.  The paper
 * names learning the chemical source term as future work (Sec. 7).  Inputs (z-scored
 * with training statistics): T, ln p, log10 dt, BC(Y_k) = (max(Y_k, 1e-30)^lam - 1) / lam;
 * outputs: BC(Y_k(t + dt)) - BC(Y_k(t)), times (1e-8 s / dt)^dt_power (training option,
 * stored with the network).  After inference the predicted mass fractions
 * are projected in fp64 onto the element (H, O, N) mass fractions of the input (weighted
 * least squares), the temperature is solved from (e, Y) in fp64, and a gate decides per
 * cell whether the answer stands; rejected cells are integrated by the cell's precision
 * variant of chem_integrate instead.
 */

/* Training pairs, all device arrays of n entries (Y planes with stride ld). */
typedef struct {
  const double *d_rho;
  const double *d_e;
  const double *d_Y0;  /* mass fractions at t (planes, stride ldY0) */
  int64_t ldY0;
  const double *d_T0;  /* nullable: temperature guess at t */
  const double *d_dt;  /* step of each pair, s */
  const double *d_Y1;  /* mass fractions at t + dt (planes, stride ldY1) */
  int64_t ldY1;
} chem_pairs;

/* Training configuration.  Zero-initialised fields take the defaults in brackets. */
typedef struct {
  int32_t epochs;       /* [20] */
  int32_t batch;        /* [4096] rows per Adam step */
  float lr;             /* [1e-3] Adam learning rate, cosine-decayed to lr_final */
  float lr_final;       /* [lr / 20] */
  float boxcox_lambda;  /* [0.1] */
  float dt_power;       /* [0] targets are the BC increments times (1e-8 s / dt)^dt_power,
                           so a target is near a rate of change where dt_power = 1 */
  uint64_t seed;        /* weight initialisation and shuffling [0] */
} chem_train_cfg;

/* Inference gate.  Zero-initialised fields take the defaults in brackets. */
typedef struct {
  float ood_margin;  /* [0.05] accepted feature range: training range widened by this fraction */
  float resid_max;   /* [0.02] largest relative element-mass residual before projection */
  float neg_tol;     /* [1e-6] most negative mass fraction allowed after projection */
  float max_dT;      /* [200] largest accepted |T(t + dt) - T(t)|, K */
  float err_tol;   /* [6e-4] largest accepted error estimate relative to T (the
                        quadrature error test of chem_surrogate_infer); negative: no test */
  float rate_max;  /* [1.5] largest dt * max_k |dY_k/dt| / (|Y_k| + 1e-6) at either end of
                        the step for the test to accept; negative: no bound */
} chem_surrogate_gate;

/* Number of float parameters of the network (flat layout W0 [256x16], b0 [256], W1
 * [256x256], b1, W2 [256x256], b2, W3 [16x256], b3 [16]; input columns 12..15 and output
 * rows 9..15 are padding and stay zero). */
int64_t chem_surrogate_param_count(void);

/*
 * Train the surrogate on npairs pairs (fresh weights from cfg->seed): featurise all
 * pairs, take the normalisation statistics and feature ranges, then per epoch a seeded
 * shuffle and floor(npairs / batch) Adam steps of forward, mean-squared error over the
 * 9 outputs, and backward, all on the GPU.  h_epoch_loss (nullable, host [epochs])
 * receives the mean loss of each epoch.  Synchronous (returns when training is done).
 * Errors: npairs < batch or NULL arrays -> CHEM_ERR_INVALID; allocation -> CHEM_ERR_NOMEM.
 */
int chem_surrogate_train(chem_ctx *ctx, const chem_pairs *pairs, int64_t npairs,
                         const chem_train_cfg *cfg, void *stream, float *h_epoch_loss);

/*
 * Advance the state over dt with the surrogate (chem_state as in chem_integrate).  Per
 * cell: features -> network -> inverse transform -> fp64 projection -> fp64 temperature
 * -> gate (feature range, element residual, negativity, temperature solve, |dT|) ->
 * error test: with the integrator's right-hand side (evaluated in fp32: an estimator)
 * at Y0, Y1 and the Hermite midpoint
 * Ym = (Y0 + Y1)/2 + dt/8 (F0 - F1), Simpson's defect D = Y1 - Y0 - dt/6 (F0 + 4 Fm + F1)
 * gives the temperature-error estimate sum_k |u_k(T1) - e| |D_k| / c_v(T1), which must
 * not exceed err_tol * T1 (u_k the species internal energies per mass) times
 * 1 - rate/2 + rate^2/12 (the defect's shrink factor along a growing mode); and the
 * step must be slow for the cell (rate <= rate_max, below).
 * Accepted cells get the projected Y, its T, status CHEM_CELL_OK and nsteps 0; rejected
 * cells are integrated with rtol, atol by the persistent work-stealing kernel of
 * chem_integrate_batched (the fallback list is its queue; the context's variant) and
 * get status CHEM_CELL_SURROGATE, or the integrator's failure code, and their attempted
 * steps.  d_fallback_mask (nullable, device uint8 [ncells]) receives 0 for accepted
 * cells and, for rejected ones, the first gate that failed: 1 feature outside the
 * training range, 2 element residual, 3 negative mass fraction, 4 temperature (no
 * root or |dT| > max_dT), 5 error test: the step is not slow for the cell, 6 error test: error
 * estimate above err_tol.  d_stats (nullable): status_count[CHEM_CELL_SURROGATE] counts fallbacks.
 * gate may be NULL.  Errors: no trained or loaded network -> CHEM_ERR_STATE; arguments
 * as chem_integrate.  Asynchronous on stream.
 */
int chem_surrogate_infer(chem_ctx *ctx, const chem_state *state, int64_t ncells, double dt,
                         double rtol, double atol, const chem_surrogate_gate *gate, void *stream,
                         uint8_t *d_fallback_mask, chem_stats *d_stats);

/*
 * The surrogate on a ragged batch of boxes (chem_batch as in chem_integrate_batched:
 * box b owns cells [offset[b], offset[b+1]) and advances them by nsub[b] substeps of
 * dt[b]; an AMR hierarchy's levels subcycled per Alg. 1), in one call: substep round r
 * runs the network, projection, temperature, gate and error test of chem_surrogate_infer
 * on every box with more than r substeps (at its own dt), and all the cells the gate
 * rejects in that round, from every box, form one queue that one persistent
 * work-stealing launch integrates (each cell over its box's dt, the context's variant).
 * Each cell's result equals what per-box, per-substep chem_surrogate_infer calls give.
 * The call reads the box table to the host once (a synchronisation of stream); the
 * rounds are then issued asynchronously.  status, nsteps and d_fallback_mask
 * (nullable, as chem_surrogate_infer) hold each cell's last substep; d_stats
 * (nullable) counts cell-substeps: cells, status_count[CHEM_CELL_OK] for accepted ones
 * and the integrator's codes (CHEM_CELL_SURROGATE for its successes) for the rest.
 * Errors: as chem_surrogate_infer; a box table whose offsets do not run from 0 to
 * ncells without decreasing, or with dt <= 0 or nsub < 1 -> CHEM_ERR_INVALID.
 */
int chem_surrogate_infer_batched(chem_ctx *ctx, const chem_state *state, int64_t ncells,
                                 const chem_batch *batch, double rtol, double atol,
                                 const chem_surrogate_gate *gate, void *stream,
                                 uint8_t *d_fallback_mask, chem_stats *d_stats);

/* Write / read the trained network (parameters, Box-Cox lambda, normalisation and
 * feature ranges) to / from a binary file.  Synchronous.  Errors: I/O -> CHEM_ERR_INVALID;
 * save without a network -> CHEM_ERR_STATE. */
int chem_surrogate_save(chem_ctx *ctx, const char *path);
int chem_surrogate_load(chem_ctx *ctx, const char *path);

/* Copy the flat fp32 parameters out (h_out) and / or in (h_in, resets Adam); n must equal
 * chem_surrogate_param_count().  Synchronous. */
int chem_surrogate_params(chem_ctx *ctx, float *h_out, const float *h_in, int64_t n);

/*
 * One forward and backward pass on a given batch without updating the weights, for
 * checks: d_X [B x 16] normalised features, d_T [B x 16] normalised targets (fp32 device),
 * d_Y [B x 16] (fp32 device, out) network output, h_grad (host, flat like the parameters,
 * out) gradient of the mean squared error over the 9 outputs, h_loss (host, out).
 * Synchronous.
 */
int chem_surrogate_grad(chem_ctx *ctx, const float *d_X, const float *d_T, int64_t B, float *d_Y,
                        float *h_grad, float *h_loss, void *stream);

/*
 * chem_surrogate_grad keeping every intermediate of the pass, for layer-by-layer checks
 * of the GEMMs and elementwise kernels (not a call of the paper's method).  With
 * H_-1 = bf16(X), hidden layers l = 0, 1, 2 and the output layer 3 (W_l [N x K] of the
 * flat parameters, G_l the loss gradient with respect to layer l's output), the device
 * outputs (each nullable) are:
 *   d_Z  fp32 [3][B][256]: Z_l = H_{l-1} W_l^T + b_l (FP32 accumulation);
 *   d_H  bf16 bit patterns [3][B][256]: H_l = bf16(GELU(Z_l));
 *   d_G  bf16 bit patterns [4][B][256]: G_3 = bf16(2 (Y - T) / (9 B)) over the 9 live
 *        outputs as B x 16 (stride 16) at the start of slab 3; G_l = bf16(dH_l GELU'(Z_l))
 *        for l < 3;
 *   d_dH fp32 [3][B][256]: dH_l = G_{l+1} W_{l+1}, the gradient with respect to H_l.
 * The weight gradients (h_grad) are G_l^T H_{l-1} and the bias gradients the column sums
 * of G_l.  Other arguments, results and errors as chem_surrogate_grad.  Synchronous.
 */
int chem_surrogate_trace(chem_ctx *ctx, const float *d_X, const float *d_T, int64_t B, float *d_Y,
                         float *d_Z, uint16_t *d_H, uint16_t *d_G, float *d_dH, float *h_grad,
                         float *h_loss, void *stream);

/*
 * One Adam step of the network's parameters with a given gradient, for checks of the
 * optimizer kernel that training runs (not a call of the paper's method): h_grad (host,
 * flat like the parameters, n = chem_surrogate_param_count()), learning rate lr >= 0,
 * b1 = 0.9, b2 = 0.999, eps = 1e-8 (Kingma & Ba 2015, with bias correction; the step
 * count starts at 1 after chem_surrogate_params uploads parameters and advances by one
 * per call).  The bf16 copies of the weights are refreshed.  Synchronous.  Errors:
 * wrong n, NULL h_grad or invalid lr -> CHEM_ERR_INVALID.
 */
int chem_surrogate_adam(chem_ctx *ctx, const float *h_grad, int64_t n, float lr);

/*
 * The fp64 element projection of chem_surrogate_infer alone, for checks (not a call of
 * the paper's method): for n cells (device planes with stride ldY), d_Yout receives the
 * weighted least-squares projection of the prediction d_Yp onto the element (H, O, N)
 * mass fractions of d_Y0: Y'' = Y' - W E^T (E W E^T)^-1 E (Y' - Y0), W = diag(max(Y'_k,
 * 1e-12)), E the element mass fraction per unit species mass fraction.  A cell whose
 * 3x3 system is singular gets d_Yp unchanged.  Needs no trained network.  Asynchronous
 * on stream.  Errors: n < 0, NULL arrays with n > 0, ldY < n -> CHEM_ERR_INVALID.
 */
int chem_surrogate_project(chem_ctx *ctx, int64_t n, const double *d_Y0, const double *d_Yp,
                           int64_t ldY, double *d_Yout, void *stream);

/*
 * The network alone on B rows (a check of the kernels; not a call of the paper's
 * method): d_X [B x 16] normalised features (fp32 device), d_Y [B x 16] outputs (fp32
 * device, out; columns 9..15 zero).  impl: 0 = the kernel inference uses (tcgen05
 * tensor cores, tensor-memory accumulators, weights streamed by bulk copies), 1 = the
 * one-kernel mma.sync version (same numbers as 2), 2 = the layer-by-layer GEMMs of
 * training.  h_err (nullable, host): when given, the call synchronises and receives
 * 1 if a bounded wait of the tensor-core kernel ran out (its outputs are then invalid),
 * else 0.  Asynchronous on stream otherwise (impl 2 is synchronous).  Errors: B < 0,
 * NULL arrays with B > 0, unknown impl -> CHEM_ERR_INVALID.
 */
int chem_surrogate_forward(chem_ctx *ctx, const float *d_X, int64_t B, float *d_Y, int32_t impl,
                           void *stream, int32_t *h_err);

/*
 * chem_integrate_batched for callers that cannot allocate device memory during the call.
 * The paper has no counterpart.
 *
 * Some callers cannot allocate at that moment:
 *   - host solvers whose memory arena has already taken the GPU's memory and forbids
 *     allocations made outside it;
 *   - time-critical loops that cannot afford cudaMalloc's latency and the implicit
 *     synchronisation that cudaMalloc and cudaFree bring.
 *
 * This entry point integrates exactly like chem_integrate_batched, with the same
 * arguments, argument checks, error codes and results. It calls no cudaMalloc, cudaFree
 * or other allocating routine. The queue scratch comes from a fixed array compiled into
 * the library: about 5 MiB, which every GPU that loads the library keeps until the
 * process exits.
 *
 * Limits and rules:
 *   - At most 1,048,576 cells per call. Larger ncells returns CHEM_ERR_INVALID with a
 *     message, before anything is launched.
 *   - opt->use_graph is ignored: the launches go straight to the stream; opt->shape is
 *     honoured.
 *   - Set-up: every call looks up the array's device address in the current device's
 *     context (so a device reset never leaves a stale address). The first call in a
 *     context also loads the library's device code there: make that first call on each
 *     device before any stream capture.
 *   - Every call on a device shares the one array, and the array keeps the last call's
 *     contents. Each call clears the parts that must start at zero, but two calls whose
 *     work overlaps on the GPU race on it, even from different contexts or streams. Order
 *     such calls on one stream, or synchronise between them.
 */
int chem_integrate_batched_noalloc(chem_ctx *ctx, const chem_state *state, int64_t ncells,
                                   const chem_batch *batch, double rtol, double atol,
                                   const chem_batch_options *opt, void *stream,
                                   chem_stats *d_stats);

/* ------------------------------------------------------------- the split scheme
 *
 * The operator on either side of the chemistry in the paper's split solver (Sec. 2.2.1:
 * Strang splitting of the reactive Euler equations): a minimal 1D finite-volume Euler
 * step and the Strang step that couples it to the integrator.  It exists to run the
 * split scheme end to end (a 1D detonation); the paper's multi-dimensional AMR hydro
 * solver is not part of this library.
 *
 * A 1D flow of n cells of width dx, all device arrays, structure of arrays:
 *   d_rho[n], d_rhou[n], d_rhoE[n]   in/out: density, momentum, total energy per volume
 *                                    (E = e + u^2 / 2, e as in chem_state_from_TPY)
 *   d_rhoY[k * ldY + i]              in/out: partial densities rho Y_k
 *   d_T[n]                           in: Newton start (NaN or <= 0 -> 1500 K); out: the
 *                                    temperature of the new state
 *   d_status[n] (nullable)           out: the last operator's per-cell outcome
 *                                    (chem_cell_status; the Euler step writes
 *                                    CHEM_CELL_NEWTON_FAIL where a cell has no
 *                                    temperature root)
 */
typedef struct {
  double *d_rho;
  double *d_rhou;
  double *d_rhoE;
  double *d_rhoY;
  int64_t ldY;
  double *d_T;
  int32_t *d_status;
} chem_flow1d;

/*
 * One step dt of the 1D Euler equations for a reacting mixture (no source term):
 * second-order MUSCL reconstruction of (rho, u, p, Y_k) with minmod-limited slopes (a face
 * whose reconstructed density or pressure is not positive takes the cell averages), the
 * HLL flux with Davis wave speeds (sound speed from gamma = c_p / c_v of the mixture's
 * NASA-7 thermo), and the two-stage SSP Runge-Kutta (Heun) update; p = rho R_u T
 * sum_k Y_k / W_k with T from e by the integrator's Newton solve.  bc_left, bc_right:
 * 0 transmissive (zero gradient), 1 reflecting wall.  The caller keeps dt within the
 * CFL limit (chem_euler1d_max_speed).  The context owns the scratch (~(4 (3 + S) + S + 3)
 * n doubles, grown on demand).  Errors: NULL arrays, n < 2, ldY < n, dx or dt <= 0, an
 * unknown boundary -> CHEM_ERR_INVALID; allocation -> CHEM_ERR_NOMEM.  Asynchronous.
 */
int chem_euler1d_step(chem_ctx *ctx, const chem_flow1d *flow, int64_t n, double dx, double dt,
                      int32_t bc_left, int32_t bc_right, void *stream);

/* Largest |u| + c over the cells (for the CFL step dt = CFL dx / max), into *h_smax
 * (host).  Synchronous.  The flow's temperatures are Newton starts and are not changed.
 * Errors as chem_euler1d_step. */
int chem_euler1d_max_speed(chem_ctx *ctx, const chem_flow1d *flow, int64_t n, double *h_smax,
                           void *stream);

/*
 * One Strang-split step (Sec. 2.2.1): the chemistry over dt / 2 (chem_integrate on
 * Y = rho Y / rho at fixed rho and e = E - u^2 / 2, in the context's variant and scheme;
 * rho, rho u and rho E do not change), chem_euler1d_step over dt, the chemistry over
 * dt / 2 again.  rtol, atol as chem_integrate; d_stats (nullable, device) counts both
 * chemistry half-steps.  Errors as chem_euler1d_step, plus rtol <= 0 or atol < 0 ->
 * CHEM_ERR_INVALID.  Asynchronous.
 */
int chem_strang_step(chem_ctx *ctx, const chem_flow1d *flow, int64_t n, double dx, double dt,
                     int32_t bc_left, int32_t bc_right, double rtol, double atol, void *stream,
                     chem_stats *d_stats);

/*
 * Diagnostic: evaluate one of the device math routines the integration kernels use on
 * n fp64 arguments (device pointers d_x -> d_y), so tests can check them against the
 * CUDA library and the IEEE-754 definitions.  op: 0 table-driven exp, 1 table-driven
 * log (Tang's methods, used by the kernels), 2 library exp, 3 library log,
 * 4 reciprocal with one Newton-Raphson step, 5 with two, 6 the hardware reciprocal
 * approximation alone, 7 the integer-pipe fp64 -> fp32 rounding (widened back exactly),
 * 8 the integer-pipe fp32 -> fp64 widening of the hardware-rounded fp32 of x,
 * 9 / 10 the hi / lo fp32 parts of the 2^-12-grid split of x, 11 / 12 the network's fp32
 * GELU and GELU' of (float)x (erf by Abramowitz & Stegun 7.1.26), 13 / 14 the same with
 * the CUDA library's erff and expf.  Not part of the integration path; the paper has no
 * counterpart.  Errors: unknown op or n < 0 -> CHEM_ERR_INVALID.  Asynchronous on stream.
 */
int chem_diag_math(int op, int64_t n, const double *d_x, double *d_y, void *stream);

/*
 * Diagnostic: a throughput probe of the FMA pipe the integration kernels are bound by
 * (the denominator of their compute roofline; the paper has no counterpart).  op 0:
 * fp64, 1: fp32.  Launches blocks x threads threads; each runs iters rounds of 32 FMAs
 * (8 independent dependent chains, 4 FMAs each per round, all operands in registers),
 * i.e. 64 flops per round, and writes one value to d_sink (device, blocks * threads + 2
 * elements of 8 bytes for op 0, 4 for op 1; the last two hold the chains' coefficients,
 * written by a one-thread launch first).  The caller times the call (CUDA events around
 * it) to get flop/s.  Errors: unknown
 * op, blocks < 1, threads not a multiple of 32 in [32, 1024], iters < 1 or NULL d_sink
 * -> CHEM_ERR_INVALID.  Asynchronous on stream.
 */
int chem_diag_fma_peak(int op, int32_t blocks, int32_t threads, int64_t iters, void *d_sink,
                       void *stream);

/*
 * Diagnostic: the equilibrium exponents ln(1 / K_c,j) = sum_k nu_jk g_k / (R_u T)
 * + (sum_k nu_jk) ln(R_u T / p_ref) (Sec. 2.2.3: the reverse rates k_r = k_f / K_c of the
 * law of mass action) of every reaction of the context's mechanism at n temperatures
 * d_T (device, fp64, kelvin, > 0; non-positive values give NaN), written to d_out
 * (device, n * n_reactions fp64, row i = temperature i, the fp32 results widened
 * exactly), as the mixed-precision right-hand sides form them: form 0 the mixed
 * variant's (fp64 Gibbs functions summed as fp32 hi/lo pairs), form 1 the all-fp32 one of
 * the surrogate's error test.  The plain fp64 variant never forms ln K_c (it multiplies
 * exp(-g_k / (R_u T)) factors) and has no form here.  Errors: NULL ctx, form not 0 or 1,
 * n outside [0, 2^30] or NULL pointers with n > 0 -> CHEM_ERR_INVALID; a failed launch ->
 * CHEM_ERR_CUDA.  Asynchronous on stream.
 */
int chem_diag_ln_inv_kc(chem_ctx *ctx, int form, int64_t n, const double *d_T, double *d_out,
                        void *stream);

/* Library version, as major * 10000 + minor * 100 + patch. */
int chem_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CHEM_H */
