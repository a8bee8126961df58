/*
 * nb.h -- C ABI of libnb, a direct N-body block-step Hermite integrator whose
 * hot path runs as hand-written CUDA kernels on one B300 (sm_103a).
 *
 * The method is the one the paper benchmarks (Berczik, Spurzem et al., "Up to
 * 700k GPU cores, Kepler, and the Exascale future for simulations of star
 * clusters around black holes"): direct summation of the Newtonian forces
 * between all particles, individual hierarchical block time-steps, and Hermite
 * integration of 4th, 6th and 8th order (abstract; "Codes description"), with
 * the force evaluated either all in FP64 or in mixed FP32 + FP64 precision
 * (captions of the speed figures for the K20 and C2050 cards).
 *
 * Units: G = 1.  Pair softening: eps_ij^2 = max(eps_i^2, eps_j^2).
 *
 * Conventions for every call:
 *   - returns NB_OK (0) or a negative NB_ERR_* code; no C++ exception crosses
 *     the ABI; nb_last_error(ctx) describes the last failure on that context;
 *   - host arrays are float64, row-major [n][3] for vectors; they are copied,
 *     never retained: the caller keeps ownership;
 *   - device work is ordered on the context's stream (nb_set_stream); calls
 *     that return values to the host synchronise that stream;
 *   - a context belongs to the device that was current at nb_create and is
 *     not thread safe: use one context per host thread.
 */
#ifndef NB_H
#define NB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ codes */
#define NB_OK 0
#define NB_ERR_ARG (-1)          /* invalid argument or call order                 */
#define NB_ERR_CUDA (-2)         /* a CUDA runtime call or kernel launch failed    */
#define NB_ERR_NOT_SYNC (-3)     /* nb_energy with particles at different times    */
#define NB_ERR_DT_UNDERFLOW (-4) /* a particle's time step fell below dt_min       */
#define NB_ERR_TIMEOUT (-5)      /* a bounded device-side wait ran out             */
#define NB_ERR_NAN (-6)          /* non-finite input or state                      */
#define NB_ERR_NOMEM (-7)        /* device allocation failed                       */

#define NB_FP64 0  /* every force operation in FP64                              */
#define NB_MIXED 1 /* positions as double-single pairs, FP32 force chain,        */
                   /* compensated (double-single) accumulation, FP64 outside    */

typedef struct nb_ctx nb_ctx;

/* -------------------------------------------------------------- lifetime */

/* Route every device allocation of contexts created afterwards through
 * alloc/free_ (for example a framework's caching allocator).  alloc must return
 * device memory aligned to at least 256 bytes, or NULL on failure; free_ is
 * called with the pointers alloc returned.  Pass NULL, NULL to restore
 * cudaMalloc/cudaFree.  Process-wide; call before nb_create.                */
int nb_set_allocator(void* (*alloc)(size_t bytes, void* user), void (*free_)(void* ptr, void* user),
                     void* user);

/* Create a context for n >= 1 particles integrated with the Hermite scheme of
 * the given order (4, 6 or 8; abstract), uniform Plummer softening eps >= 0.
 * Allocates the structure-of-arrays state in device memory.  Defaults:
 * NB_MIXED, eta = 0.2, eta_s = 0.01, dt_max = 1/16, dt_min = 2^-40.       */
int nb_create(nb_ctx** out, int64_t n, int order, double eps);

/* Free every device and host resource of ctx.  NULL is ignored.            */
void nb_destroy(nb_ctx* ctx);

/* Message for the last failed call on ctx; with ctx NULL, the last failed
 * context-free call (nb_create, nb_force_static, ...) of the calling host
 * thread.                                                                  */
const char* nb_last_error(const nb_ctx* ctx);

/* Order later device work on this CUDA stream (a cudaStream_t); NULL = the
 * legacy default stream.                                                   */
int nb_set_stream(nb_ctx* ctx, void* cuda_stream);

/* ------------------------------------------------------------ parameters */

/* NB_FP64 or NB_MIXED (mixed fp32 + fp64 force, captions of the paper's speed
 * figures).  Takes effect at the next nb_predict.                          */
int nb_set_precision(nb_ctx* ctx, int mode);

/* Per-particle softening eps_i (host [n], each >= 0) or NULL for the uniform
 * eps of nb_create.  Pairs use max(eps_i^2, eps_j^2).  Call before
 * nb_set_particles.                                                        */
int nb_set_softening(nb_ctx* ctx, const double* eps_i);

/* Time-step parameters: accuracy eta > 0, start-up eta_s > 0, maximum step
 * dt_max (a power of two), minimum dt_min > 0 (smaller steps fail with
 * NB_ERR_DT_UNDERFLOW).  Individual block steps are powers of two
 * (abstract: "individual hierarchically block time-steps").               */
int nb_set_params(nb_ctx* ctx, double eta, double eta_s, double dt_max, double dt_min);

/* ------------------------------------------------------------- the method */

/* Load masses m [n] (>= 0), positions x [n][3] and velocities v [n][3] (host)
 * at t = 0, then start the integration: force with every particle active
 * (acc, jerk, snap and, for order 8, crackle), start-up step
 * eta_s |a| / |jerk| quantised to a power of two <= dt_max.               */
int nb_set_particles(nb_ctx* ctx, const double* m, const double* x, const double* v);

/* Block scheduler (abstract: individual hierarchical block time-steps).
 * t_blk = min_i (t_i + dt_i); the active set is every i with
 * t_i + dt_i == t_blk, in ascending index order, kept on the device for the
 * next nb_force.  Writes *t_blk, *n_act and, if idx_out != NULL, the indices
 * to idx_out (host, capacity n).                                          */
int nb_next_block(nb_ctx* ctx, double* t_blk, int32_t* idx_out, int64_t* n_act);

/* Predictor: advance every particle's position and velocity (and, for orders
 * 6 and 8, acceleration; for 8, jerk) from its own time t_i to t by the
 * Taylor series in the derivatives it holds, and write the j-particle store
 * the force kernel reads.  t must be >= every t_i.  With a j range set
 * after nb_next_block: only the range's and the block's particles
 * (nb_set_jrange).                                                         */
int nb_predict(nb_ctx* ctx, double t);

/* Force: for each listed particle i, sum over all j != i of the Plummer-
 * softened Newtonian acceleration and its time derivatives up to the order's
 * needs, plus the potential ("Codes description": the GPUs compute the
 * gravitational forces between particles).  active_idx: n_act distinct
 * indices in [0, n), host or device memory (detected), or NULL to use the
 * list of the last nb_next_block.  Must follow nb_predict.                 */
int nb_force(nb_ctx* ctx, const int32_t* active_idx, int64_t n_act);

/* Corrector and time step for the particles of the last nb_force: Hermite
 * correction of order p, Hermite interpolation of the higher derivatives,
 * new step by the generalised Aarseth criterion quantised to a power of two
 * commensurate with the block time (abstract: 4th/6th/8th-order Hermite with
 * hierarchical block steps).  Sets t_i to the predicted time.              */
int nb_correct(nb_ctx* ctx);

/* One block step: nb_next_block, nb_predict(t_blk), nb_force(NULL),
 * nb_correct.  Optional outputs (NULL to skip).                           */
int nb_block_step(nb_ctx* ctx, double* t_blk, int64_t* n_act);

/* Block steps until the next block time would exceed t_end.  Optional
 * outputs: blocks taken and pairwise interactions evaluated (n_act * n per
 * block).                                                                  */
int nb_step_until(nb_ctx* ctx, double t_end, int64_t* n_blocks, int64_t* n_interactions);

/* Kinetic and potential energy, E = sum m v^2 / 2 - sum_{i<j} m_i m_j / R_ij,
 * evaluated on the device in the context's precision.  Every particle must
 * be at the same time (a synchronised block), else NB_ERR_NOT_SYNC.        */
int nb_energy(nb_ctx* ctx, double* ekin, double* epot);

/* -------------------------------------------------------- state exchange */

/* Copy the state to host arrays (any may be NULL): x, v [n][3];
 * d [n][6][3] = acc, jerk, snap, crackle, a^(4), a^(5) (unused ones zero);
 * t, dt [n].  The reordering runs on the device (a staging buffer of 26 n
 * doubles is allocated on first use); page-locked host arrays copy fastest.
 * Synchronises.                                                            */
int nb_get_state(nb_ctx* ctx, double* x, double* v, double* d, double* t, double* dt);

/* Replace the state from host arrays with the nb_get_state layout (all
 * required; masses and softening are kept).  For checkpoint/restart.  The
 * values are checked on the device first: NB_ERR_NAN for a non-finite one,
 * NB_ERR_ARG for a dt <= 0, and then the old state is left unchanged.
 * Synchronises.                                                            */
int nb_set_state(nb_ctx* ctx, const double* x, const double* v, const double* d, const double* t,
                 const double* dt);

/* Result of the last nb_force for its n_act particles, in list order (any
 * output may be NULL): acc, jerk, snap, crackle [n_act][3], pot [n_act].
 * Unused derivatives are zero.  Synchronises.                              */
int nb_get_force(nb_ctx* ctx, double* acc, double* jerk, double* snap, double* crackle, double* pot);

/* The predicted j-particle store of the last nb_predict, converted to double
 * exactly as the force kernel sees it (mixed: hi + lo positions, FP32
 * velocity/acc/jerk): xp, vp, ap, jp [n][3] (NULL to skip).  After a
 * prediction restricted by a j range (nb_set_jrange) the records outside the
 * range and the block hold earlier predictions.  Synchronises.             */
int nb_get_predicted(nb_ctx* ctx, double* xp, double* vp, double* ap, double* jp);

/* Kernel launch shape of the last nb_force: CTAs along i, j-splits and
 * i-particles per CTA -- the launch variant: 256 (128 threads holding two
 * particles each), 128 (one each), 32 or 4 (j-parallel: 4 or 32 threads per
 * particle, for active sets of up to 256 or 24); any output may be NULL.   */
int nb_get_launch(nb_ctx* ctx, int* i_tiles, int* j_splits, int* i_per_cta);

/* Test hook with no counterpart in the paper: warps of the mixed force
 * kernels that took the per-pair softening form since nb_create or the
 * previous call, which resets the count; n_warps must not be NULL.  With
 * per-particle softening the pair value is max(eps_i^2, eps_j^2) (this
 * library's reading; the paper gives only the star and hole values).  A warp
 * whose i-particles all carry the system's largest eps^2 has that maximum in
 * eps_i^2 and takes it without a per-pair max; only the other warps take the
 * per-pair form.  Synchronises; NB_ERR_ARG on a NULL argument, NB_ERR_CUDA
 * on a CUDA failure.                                                       */
int nb_get_pair_warps(nb_ctx* ctx, int64_t* n_warps);

/* cycles > 0: nb_step_until replays a CUDA graph of that many device-driven
 * block cycles (scheduler, predictor, force, corrector with the active-set
 * size, block time and force launch shape decided on the device), checking
 * on the host only once per replay; 0 (default): one host-driven cycle per
 * block.  Both take the same blocks with the same kernels' arithmetic.  The
 * graph is captured on first use and again after a parameter change.       */
int nb_set_graph(nb_ctx* ctx, int cycles);

/* Autotuner of the force launch shape.  For active-set sizes 1, 2, 4, ...
 * up to N it times candidate launch variants (i-particles per CTA) and
 * j-split counts on the context's own store (CUDA events on its stream, best
 * of `reps` runs each) and keeps per size class the fastest, if it beat the
 * analytic rule's own shape by 3 % at that size (else the class keeps the
 * rule: variant 0 in nb_get_tuning, with the rule's time).  It times the
 * kernels of the context's current mode: after nb_set_graph(cycles > 0) the
 * persistent kernels of device-driven cycles, otherwise the per-launch
 * kernels of host-driven ones (call nb_set_graph first to tune graph
 * replays).  Later forces of
 * the context in the current precision (host- and device-driven alike) take
 * their shape from that table: class floor(log2(n_act)), the tuned variant,
 * the split count scaled to keep the tuned number of CTAs.  reps <= 0 drops
 * the current precision's table (back to the analytic makespan rule).  The
 * particle state is untouched (predicted store and force result are
 * scratch); needs nb_set_particles and the whole j range (NB_ERR_ARG while
 * nb_set_jrange holds one).  Synchronises.                                 */
#define NB_TUNE_MAX 32
int nb_autotune(nb_ctx* ctx, int reps);

/* The current precision's table: *n_classes (0: none), and for class k
 * (active sets of 2^k .. 2^(k+1) - 1) the variant ni[k], split count js[k]
 * and measured force time ms[k] at n_act = 2^k (arrays of NB_TUNE_MAX; any
 * may be NULL).                                                            */
int nb_get_tuning(nb_ctx* ctx, int* n_classes, int32_t* ni, int32_t* js, double* ms);

/* Install a table for the current precision -- one nb_get_tuning returned,
 * e.g. from an earlier run on the same N: n_classes <= NB_TUNE_MAX classes,
 * ni[k] the variant of class k (0: untuned, the analytic rule; else 4, 32,
 * 128 or 256 mixed, 128 FP64), js[k] >= 1 its split count at n_act = 2^k.
 * n_classes = 0 drops the table.                                           */
int nb_set_tuning(nb_ctx* ctx, int n_classes, const int32_t* ni, const int32_t* js);

/* Self-test of the bounded waits (failure detection without a fault): one
 * CTA waits on an mbarrier that nothing completes, with a limit of `seconds`
 * (0 < seconds <= 5) instead of the kernels' 2 s.  Returns NB_ERR_TIMEOUT --
 * the wait ran out, the kernel reported it and returned, and the context
 * stays usable -- or another error code if the probe misbehaved.
 * Synchronises.                                                            */
int nb_selftest_wait(nb_ctx* ctx, double seconds);

/* Self-check of the format conversions of the mixed path (the reading of
 * the mixed precision: FP32 values truncated toward zero from FP64, with
 * results below the normal float range flushed to zero and those from
 * |x| >= 2^128 taken to inf; FP32 widened exactly, subnormals flushed): the
 * predictor and the corrector convert in integer arithmetic; this compares
 * that form bit for bit with the hardware's cvt instruction on n seeded
 * inputs (any bit pattern, and exponents across and at the edges of the
 * float range; NaN skipped); *mismatches = the count (0 when they agree).
 * Synchronises.                                                            */
int nb_selftest_convert(nb_ctx* ctx, int64_t n, uint64_t seed, int64_t* mismatches);

/* Force the j-split count of later nb_force calls (0 = automatic).         */
int nb_set_jsplit(nb_ctx* ctx, int j_splits);

/* ------------------------------------------- j decomposition across ranks */

/* The paper's multi-GPU scheme ("Codes description": MPI between the GPUs,
 * each GPU computing forces; the log(N_GPU) communication term of the
 * performance model): every rank holds all particles and the same active
 * set, sums the force over its own contiguous share of the j particles, the
 * partial results are exchanged once per block, and every rank adds them in
 * the same order and runs the same corrector, so the states stay identical.
 *
 * nb_set_jrange: later nb_force calls sum over the j particles
 * [j_begin, j_end) only; j_begin and j_end multiples of NB_JTILE (j_end may
 * also be n).  (0, 0) or (0, n) restores the whole range.  The start-up
 * passes and nb_energy always use every particle.  While a range is set,
 * nb_block_step, nb_step_until, graph cycles and nb_autotune fail with
 * NB_ERR_ARG: step
 * with nb_next_block, nb_predict, nb_force(NULL), the exchange,
 * nb_reduce_force and nb_correct.  nb_predict after nb_next_block then
 * predicts only the range's particles and the block's active ones (each rank
 * predicts its own share of the j particles), and nb_force takes the
 * scheduled list only (an explicit list fails with NB_ERR_ARG); a changed
 * range asks for a new nb_predict.  With the ranges [r T / G, (r + 1) T / G)
 * tiles (T = tiles of the store, G ranks) and one j-split per rank, the
 * reduced force is bit for bit the single-rank force with G j-splits.      */
#define NB_JTILE 128
int nb_set_jrange(nb_ctx* ctx, int64_t j_begin, int64_t j_end);

/* Copy the last nb_force result, ncomp x n_act doubles component-major
 * (acc xyz, jerk xyz[, snap xyz[, crackle xyz]], potential, sum_j m_j/R_ij^2),
 * to dst (device or host memory), ordered on the context's stream (the
 * caller synchronises, or orders its exchange on that stream).  Optional
 * outputs: ncomp and n_act.                                                 */
int nb_copy_force(nb_ctx* ctx, double* dst, int64_t* ncomp, int64_t* n_act);

/* Replace the last nb_force result by the sum of n_parts results in device
 * memory, parts[n_parts][ncomp][n_act] (each laid out as nb_copy_force
 * writes it), added in part order; nb_correct then uses it.               */
int nb_reduce_force(nb_ctx* ctx, const double* parts, int n_parts);

/* Give every particle the step dt, so that the next block is the whole
 * system -- the synchronised block that occurs at every multiple of dt_max of
 * a hierarchical block-step run (abstract).  All particles must be at one
 * common time t divisible by dt, and dt must be a power of two <= dt_max;
 * violations raise NB_ERR_NOT_SYNC / NB_ERR_ARG at the next synchronising
 * call.  Device-side, no synchronisation.                                  */
int nb_set_block_step(nb_ctx* ctx, double dt);

/* Relative precision eps[4] of the force components (acc, jerk, snap,
 * crackle) for the given precision mode, per unit of the particle's
 * conditioning kappa = sum_j m_j/R_ij^2 / |a| (>= 1).  The time-step criterion
 * uses each interpolated derivative net of the rounding its closed form can
 * carry from inputs of that precision (its noise floor): an unresolved
 * derivative counts as zero.  Defaults: NB_FP64 all 0 (the plain criterion);
 * NB_MIXED 5e-7, 1e-6, 2e-6, 2e-5, the measured error of the FP32 chain.   */
int nb_set_noise_floor(nb_ctx* ctx, int precision, const double* eps);
int nb_get_noise_floor(nb_ctx* ctx, int precision, double* eps);

/* ------------------------------------------------------------- profiling */

/* Phases of the per-phase timers: scheduler, predictor, force kernel, j-split
 * reduction, corrector, everything else (start-up, energy, step reset).
 * Inside nb_block_step and nb_step_until the predictor runs fused into the
 * scheduler's second pass, so its time counts as scheduler time there.     */
#define NB_NPHASES 6
#define NB_PHASE_SCHED 0
#define NB_PHASE_PREDICT 1
#define NB_PHASE_FORCE 2
#define NB_PHASE_REDUCE 3
#define NB_PHASE_CORRECT 4
#define NB_PHASE_OTHER 5

/* enable != 0: reset the totals and time every later kernel launch with CUDA
 * events recorded on the context's stream around it; 0: stop timing.       */
int nb_set_profiling(nb_ctx* ctx, int enable);

/* Device milliseconds and kernel launches per phase since profiling was
 * enabled (arrays of NB_NPHASES; either may be NULL), and the number of
 * kernel launches since nb_create (NULL to skip).  Synchronises.           */
int nb_get_profile(nb_ctx* ctx, double* ms, int64_t* launches, int64_t* total_launches);

/* Histogram of block sizes: counts[k] = corrector passes (block steps; for
 * an ensemble, cycles) whose active set had 2^k .. 2^(k+1) - 1 particles,
 * k < NB_NACT_CLASSES, counted on the device since nb_create or the last
 * reset (host- and device-driven cycles alike).  counts may be NULL; reset
 * != 0 zeroes the counts after reading them.  Synchronises.  The profiling
 * phases also open NVTX ranges ("nb:force", ...) around their launches, and
 * nb_block_step, nb_step_until and the graph replays around their calls,
 * for profilers that filter by range.                                      */
#define NB_NACT_CLASSES 48
int nb_get_nact_histogram(nb_ctx* ctx, int64_t* counts, int reset);

/* FMA-throughput microbenchmark on the context's GPU (a measurement aid for
 * roofline fractions, not part of the method): every SM runs independent
 * multiply-add chains in FP32 (fp64 = 0) or FP64 (fp64 != 0); *tflops = the
 * best of three timed launches, 2 flops per multiply-add.  Synchronises.   */
int nb_fma_peak(nb_ctx* ctx, int fp64, double* tflops);

/* Library version string.                                                  */
const char* nb_version(void);

/* ------------------------------------------------------------- ensembles */

/* Many independent clusters integrated side by side, each with its own
 * hierarchical block times (abstract: individual block time-steps): every
 * cycle advances each unfinished cluster by one of its blocks, with one launch
 * per kernel for all clusters (the force runs over a table of (cluster,
 * i-tile, j-split) items, each restricted to its cluster's particles).       */
typedef struct nb_batch nb_batch;

/* n_clusters >= 1 clusters of n_per_cluster[k] >= 1 particles, Hermite order
 * 4/6/8, uniform softening eps; defaults as nb_create.                      */
int nb_batch_create(nb_batch** out, int n_clusters, const int64_t* n_per_cluster, int order, double eps);
void nb_batch_destroy(nb_batch* b);
const char* nb_batch_last_error(const nb_batch* b);
int nb_batch_set_stream(nb_batch* b, void* cuda_stream);
int nb_batch_set_precision(nb_batch* b, int mode);
int nb_batch_set_params(nb_batch* b, double eta, double eta_s, double dt_max, double dt_min);

/* Host arrays of all clusters concatenated in cluster order (no padding):
 * m [N], x, v [N][3] with N = sum n_per_cluster.  Starts every cluster at
 * t = 0 as nb_set_particles does for one system.                            */
int nb_batch_set_particles(nb_batch* b, const double* m, const double* x, const double* v);

/* One cycle: each cluster whose next block time is <= t_end takes that block.
 * The whole cycle is planned on the device: active list, per-cluster
 * segments, the force's (cluster, i-tile, j-split) items, predictor, one
 * persistent force kernel over the items, reduction, corrector.  Outputs
 * (NULL to skip): clusters stepped (0 once all are past t_end) and
 * interactions evaluated (sum of n_act_k * n_k).  Synchronises.            */
int nb_batch_cycle(nb_batch* b, double t_end, int* n_stepped, int64_t* n_interactions);

/* Cycles until no cluster has a block at or before t_end: one nb_batch_cycle
 * after another, or with nb_batch_set_graph(b, c > 0) replays of a CUDA graph
 * of c such cycles, checked on the host once per replay (same cycles, same
 * arithmetic).                                                             */
int nb_batch_step_until(nb_batch* b, double t_end, int64_t* n_cycles, int64_t* n_interactions);

/* cycles > 0: nb_batch_step_until replays a CUDA graph of that many cycles;
 * 0 (default): one host-checked cycle at a time.  Captured on first use and
 * again after a parameter change.                                          */
int nb_batch_set_graph(nb_batch* b, int cycles);

/* The force plan of a cycle (nb_batch_cycle) cuts each cluster's work into
 * (i-tile, j-split) items of about equal size, about `waves` times as many
 * as the persistent force kernel has resident CTAs (default 4; 1 .. 8).
 * nb_batch_set_waves sets it; nb_batch_get_waves reads it.                  */
int nb_batch_set_waves(nb_batch* b, int waves);
int nb_batch_get_waves(nb_batch* b, int* waves);

/* Autotuner of the ensemble's force plan (how its work is cut into items):
 * for each of the next `cycles` cycles, the force and split
 * reduction are timed (CUDA events, best of reps) with the plans of 1, 2, 4
 * and 8 waves, then the cycle is completed with the wave count in use; the
 * count with the least total time is kept if it beats 4 by 3 %.  The tuning
 * cycles are real cycles of the run (the state advances by them), so tune
 * on a copy of the ensemble and pass the result to nb_batch_set_waves when
 * the run itself must start from the initial state.  ms_per_wave (nullable,
 * [4]): total milliseconds of 1, 2, 4, 8 waves.                            */
int nb_batch_autotune(nb_batch* b, int cycles, int reps, double* ms_per_wave);

/* Per-cluster kinetic and potential energy (arrays [n_clusters]); every
 * cluster must be synchronised within itself, else NB_ERR_NOT_SYNC.         */
int nb_batch_energy(nb_batch* b, double* ekin, double* epot);

/* State of all clusters concatenated as in nb_batch_set_particles (any
 * output may be NULL): x, v [N][3], t, dt [N].  Synchronises.               */
int nb_batch_get_state(nb_batch* b, double* x, double* v, double* t, double* dt);

/* ----------------------------------------------------- allocation-free call */

/* The paper has no counterpart to this call: it serves callers that cannot
 * allocate device memory when they need a force -- code running inside
 * another framework's memory pool or arena that forbids allocations outside
 * its own allocator, or a loop that must not allocate once it has started.
 *
 * Force of the n_act particles idx[] (device int32, in [0, n)) from all n
 * particles given at one instant, with the pair arithmetic of nb_force (its
 * one-particle-per-thread kernels, not the autotuned or two-per-thread
 * launch shapes), so results agree with nb_force's within the parity
 * tolerances, not bit for bit.  Every
 * pointer is device memory owned by the caller: m, eps2 [n]; x, v [n][3];
 * a [n][3] (order >= 6, else may be NULL); jerk [n][3] (order 8, else NULL);
 * out [ncomp][n_act], component-major: acc xyz, jerk xyz, snap xyz (order
 * >= 6), crackle xyz (order 8), potential, sum_j m_j/R_ij^2.  ncomp = 8, 11,
 * 14 for orders 4, 6, 8.  Pair softening max(eps2_i, eps2_j).
 *
 * It allocates nothing: the packed records, the j-split partial sums and the
 * status word live in one fixed array of NB_STATIC_SCRATCH_BYTES that every
 * GPU loading this part of the library holds until the process exits; n is
 * limited to NB_STATIC_MAX_N (larger n fails with NB_ERR_ARG).  The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current.  All calls share the array and it keeps the last
 * call's contents: calls that overlap on the GPU race, so order them (one
 * stream, or synchronise).  Work runs on `stream` (a cudaStream_t, NULL =
 * legacy default) and the call synchronises with it before returning, to
 * report device-side errors (an index out of range gives NB_ERR_ARG); so it
 * must not be called while that stream is being captured into a graph.
 * Messages: nb_last_error(NULL), kept per host thread.                       */
#define NB_STATIC_MAX_N 16384
#define NB_STATIC_SCRATCH_BYTES (16384 * 128 + (1 << 20) * 8 + 256)
int nb_force_static(int order, int precision, int64_t n, const double* m, const double* eps2, const double* x,
                    const double* v, const double* a, const double* jerk, const int32_t* idx, int64_t n_act,
                    double* out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* NB_H */
