/*
 * muca.h - C ABI of the GB300 (sm_103a) parallel multicanonical simulation of the 2D
 * Ising model, after Gross, Zierenberg, Weigel and Janke, "Massively parallel
 * multicanonical simulations" (arXiv:1707.00919).
 *
 * Many independent walkers, each a periodic L x L Ising lattice (Eq. 5, J = 1), run
 * sequential single-spin-flip Metropolis updates accepted with the multicanonical
 * weight ratio W(E')/W(E) (Sec. 2.1, Sec. 2.3).  All walkers share one weight function
 * and add their energies to one histogram H(E) (Sec. 2.2); the host turns H into the
 * next weights, ln W <- ln W - ln H (Eq. 4), until H is flat, and a production run with
 * fixed weights estimates ln g(E) (Sec. 3.3).
 *
 * Conventions shared by every call
 *   - N = L*L sites, site i = y*L + x (x fastest).  Energies live on the grid
 *     E = -2N + 4e, e = 0 .. N ("energy index", Sec. 3); arrays over energies have
 *     n_bins = N + 1 entries.  e = 1 and e = N - 1 are never visited (Sec. 3).
 *   - Update order is typewriter: attempt t of a walker flips site t mod N, where t is
 *     the instance's attempt counter, shared by all walkers and advanced by every
 *     update call (thermalization included).  This is the shared site sequence of
 *     Sec. 2.3 in its deterministic form.
 *   - Random numbers: Philox4x32-10 (Salmon et al., cited in Sec. 2.3), key = the
 *     64-bit seed, counter = (t >> 2 as 64 bits, walker index, tag), word t & 3; tag 0
 *     drives the updates, tag 1 the initial spins (+1 iff the top bit of the word for
 *     t = site is clear).
 *   - Acceptance (Sec. 2.3, integer form): for a flip at a site with k antiparallel
 *     neighbours the energy index moves to e' = e + 2 - k; with dw = lnW[e'] - lnW[e]
 *     the threshold is 0xFFFFFFFF if dw >= 0, else min(floor(exp(dw) * 2^32), 2^32 - 1)
 *     in FP64, and 0 if e' is off the grid.  A draw r is accepted iff r < T or
 *     T == 0xFFFFFFFF.
 *   - exp (thresholds) and ln (the Eq. (4) recursion, the Eq. (6) measure) are a fixed
 *     sequence of IEEE double operations: Cody-Waite reduction with the Taylor series of
 *     exp, and the atanh series of ln (within 1 and 3 units in the last place of the C
 *     library's exp and log), so the host and the device compute the same bits.
 *   - Recording: each recorded attempt adds its post-decision energy index to H.
 *
 * Memory and threads
 *   - The library owns all device memory of an instance (allocated at create, freed at
 *     destroy) through the allocator set with muca_set_allocator (cudaMalloc by
 *     default).  Host buffers passed in are copied and never retained.
 *   - Calls on one instance run in order on the instance's CUDA stream (a stream of its
 *     own unless muca_set_stream gives another).  Update calls are asynchronous; calls
 *     that return data to the host synchronize that stream first.
 *   - An instance must not be used from two host threads at the same time.
 *
 * Errors: every int-returning call returns MUCA_OK (0) or a negative MUCA_E* code and
 * then sets a thread-local message readable with muca_last_error().  MUCA_EDEVICE means
 * a kernel found an invalid state (an energy index off the grid); the instance should
 * then be destroyed.
 */
#ifndef MUCA_H
#define MUCA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MUCA_OK 0
#define MUCA_EINVAL (-1)         /* bad argument: L, sizes, NULL pointers, non-finite weights */
#define MUCA_ENOMEM (-2)         /* device or host allocation failed                        */
#define MUCA_ECUDA (-3)          /* a CUDA runtime call failed                              */
#define MUCA_ETIMEOUT (-4)       /* the deadline of muca_iterate_until_flat passed          */
#define MUCA_ENOTCONVERGED (-5)  /* the iteration budget ran out before H was flat          */
#define MUCA_EDEVICE (-6)        /* a kernel reported an invalid state                      */
#define MUCA_EIO (-7)            /* a checkpoint file could not be written or read, or is not one */

/* Lattice storage layouts in device memory (both walker-minor, Sec. 2.3: all walkers'
 * copies of one site are adjacent, so a warp's accesses coalesce). */
#define MUCA_LAYOUT_INT8 0       /* int8 spin[site][walker], values +1 / -1                  */
#define MUCA_LAYOUT_PACKED 1     /* row[y][walker] bit words (bit x set = spin -1);
                                    uint32 words for L <= 32, uint64 for L <= 64          */
#define MUCA_LAYOUT_AUTO 2       /* muca_create_ex only: time both layouts, keep the faster */

/* walkers_per_block value of muca_create_ex that times every block size from 32 to 256
 * (two recorded sweeps each on a temporary instance) and keeps the fastest.  0 picks
 * one from the kernel's occupancy without timing. */
#define MUCA_WPB_TUNE (-1)

/* n_walkers value of muca_create / muca_create_ex that asks for the walker count of
 * muca_optimal_walkers (the paper's default when W is not given, Sec. 3.1). */
#define MUCA_WALKERS_OPTIMAL (-1)

/* Stop rules of the weight iteration. */
#define MUCA_STOP_MIN_MEAN 0     /* min H / mean H over accessible energies >= threshold    */
#define MUCA_STOP_KL 1           /* Kullback-Leibler d_k < threshold (Eq. 6)                */
#define MUCA_STOP_CHEBYSHEV 2    /* Chebyshev distance d_c < threshold (Eq. A.1)            */

/* Update schedules of the weight iteration. */
#define MUCA_SCHEDULE_SWEEPS 0   /* fixed sweeps per iteration                              */
#define MUCA_SCHEDULE_PAPER 1    /* N_therm = f_therm w, N_updates of Eq. (7) (Sec. 3)      */

typedef struct muca_s *muca_t;

/* Options for muca_create_ex.  Zero-initialise, then set what differs from the
 * defaults (layout MUCA_LAYOUT_INT8, walkers_per_block chosen from the occupancy). */
typedef struct {
    int32_t L;                   /* lattice side: multiple of 4, 4 <= L <= 64               */
    int64_t n_walkers;           /* 1 <= n_walkers <= 2^31 - 1, or MUCA_WALKERS_OPTIMAL     */
    uint64_t seed;               /* Philox key                                              */
    int32_t layout;              /* MUCA_LAYOUT_* (AUTO: measured choice)                   */
    int32_t walkers_per_block;   /* 0 = from occupancy, MUCA_WPB_TUNE = measured, else a
                                    multiple of 32 in [32, 256]                            */
    int64_t first_walker;        /* global index of this instance's walker 0 (default 0):
                                    instances holding disjoint walker ranges of one
                                    simulation draw the random numbers of one instance
                                    holding them all; first_walker + n_walkers <= 2^31    */
} muca_options;

/* Parameters of muca_iterate_until_flat.  muca_default_params fills the paper's values
 * (Sec. 3: f_therm = 30, z = 2.25, factor 6, growth 1.1, d_k < 1e-4) with the fixed-sweep
 * schedule and the min/mean >= 0.8 stop rule. */
typedef struct {
    int32_t schedule;            /* MUCA_SCHEDULE_*                                         */
    int32_t stop_rule;           /* MUCA_STOP_*                                             */
    double flat_threshold;       /* 0.8 (min/mean), 1e-4 (KL) or 0.05 (Chebyshev)           */
    uint64_t therm_sweeps;       /* SWEEPS: unrecorded sweeps before each iteration        */
    uint64_t sweeps_per_iter;    /* SWEEPS: recorded sweeps per iteration                  */
    double f_therm;              /* PAPER: N_therm = f_therm * w attempts                  */
    double z;                    /* PAPER: N_updates = floor(factor * w^z / W) + 1         */
    double factor;
    double growth;               /* PAPER: after full coverage N <- floor(growth N) + 1    */
    int32_t max_iterations;      /* stop with MUCA_ENOTCONVERGED after this many           */
    double deadline_s;           /* > 0: stop with MUCA_ETIMEOUT after this wall time      */
    int32_t resume;              /* 1: continue the iteration state the instance keeps (see
                                    below), 0: start afresh (w' = 0, no range visited)    */
} muca_params;

/* Iteration state kept by an instance between calls of muca_iterate_until_flat, updated
 * after every weight update and stored by muca_save: the width w' and the range
 * [lo, hi] of the energies visited in the previous iteration (the w of Sec. 3 and the
 * Kullback-Leibler reference width of Eq. (6)), whether the whole range had been covered
 * (Eq. (7) then gives way to the growth rule) and the previous N_updates.  With
 * params.resume = 1 a run stopped by max_iterations or the deadline, or restored from a
 * checkpoint, continues the schedule as one uninterrupted call would have.
 * muca_iterate_device (fixed-sweep schedule) and muca_batch_iterate (both schedules) keep
 * and continue the same state; served requests start afresh (muca_server_submit rejects
 * resume = 1). */

/* Statistics of a weight iteration. */
typedef struct {
    int32_t iterations;          /* iterations run                                         */
    int32_t converged;           /* 1 if the last histogram met the stop rule              */
    double last_metric;          /* stop metric of the last iteration                      */
    uint64_t attempts_per_walker;/* attempts per walker spent (thermalization included)    */
    double seconds;              /* wall time of the call                                  */
} muca_stats;

/* Fills p with the defaults described at muca_params.  Returns MUCA_EINVAL for NULL. */
int muca_default_params(muca_params *p);

/* Creates an instance (Sec. 2.2: p walkers with identical weights): allocates the
 * lattices, energies, threshold table and histogram on the current device, draws the
 * initial spins (tag 1 stream), computes their energies, sets ln W = 0 (every flip
 * accepted) and the attempt counter t = 0.  *out receives the handle.
 * Errors: MUCA_EINVAL (L not a multiple of 4 in [4, 64], n_walkers out of range,
 * out == NULL), MUCA_ENOMEM, MUCA_ECUDA. */
int muca_create(int32_t L, int64_t n_walkers, uint64_t seed, muca_t *out);
int muca_create_ex(const muca_options *opt, muca_t *out);

/* Walker count of full occupancy (Sec. 3.1: the first minimum of the time per attempted
 * flip lies where every multiprocessor holds its maximal number of resident blocks, and
 * the program uses that count when W is not given).  For lattice side L and layout
 * (MUCA_LAYOUT_INT8 or MUCA_LAYOUT_PACKED) on the current device: the block size whose
 * resident blocks per SM (whole-sweep kernel, shared memory and registers) hold the
 * most walkers, ties to the larger block; *n_walkers = SMs x resident blocks x block
 * size, *walkers_per_block (may be NULL) = that block size.  Nothing is allocated.
 * Errors: MUCA_EINVAL (L as in muca_create, other layout, n_walkers NULL, no block size
 * fits), MUCA_ECUDA. */
int muca_optimal_walkers(int32_t L, int32_t layout, int64_t *n_walkers, int32_t *walkers_per_block);

/* Frees all device and host memory of the instance (NULL is accepted). */
int muca_destroy(muca_t h);

/* State and checkpoints.  The state of an instance is its lattices, energies, ln W, the
 * histogram, the attempt counter and the site order (the random numbers are a function of
 * seed, walker and attempt counter, Sec. 2.3), so a restored instance continues bit for
 * bit as the saved one would have.
 * muca_set_lattice: replaces the lattices by spins[walker][site] (int8 +1 / -1,
 * n = n_walkers * N) and recomputes the energies on the device.
 * muca_set_attempt_counter: sets t, the counter of the next attempt.
 * muca_save: writes the state and the creation options to a binary file (little-endian:
 * 8-byte magic "MUCACKP2", L, layout, n_walkers, seed, walkers_per_block, site order, t,
 * first_walker, the iteration state (int32 w', lo, hi, covered; uint64 previous N_updates),
 * ln W[N+1] FP64, H[N+1] uint64, energies int32[n_walkers], then per walker N bits,
 * rounded up to whole bytes, bit i of byte i/8 set for a down spin at site i).
 * muca_load: creates an instance from such a file (same options) and restores the state;
 * the stored energies must equal those recomputed from the stored lattices.  Files of the
 * earlier format "MUCACKP1" (no iteration state) load with a fresh iteration state.
 * Errors: MUCA_EINVAL (NULL, wrong n, a spin other than +1 / -1), MUCA_EIO (file
 * cannot be opened, written or read; not a checkpoint; inconsistent content),
 * MUCA_ENOMEM, MUCA_ECUDA. */
int muca_set_lattice(muca_t h, const int8_t *spins, size_t n);
int muca_set_attempt_counter(muca_t h, uint64_t t);
int muca_save(muca_t h, const char *path);
int muca_load(const char *path, muca_t *out);

/* Measurement helper (no counterpart in the paper): the rate at which the current
 * device issues one integer instruction class when every SM sub-partition has 16 warps
 * of independent work, for the integer roofline of the sweep kernels.  kind:
 * MUCA_PROBE_XOR (three-input XOR: the integer ALU pipe), MUCA_PROBE_MAD (32-bit
 * multiply-add), MUCA_PROBE_MIXED (the two alternating), MUCA_PROBE_PHILOX
 * (Philox4x32-10 words, Sec. 2.3's generator), MUCA_PROBE_MIXED_ONE_WARP (the
 * alternating mix with one warp per sub-partition, sixteen independent chains per thread:
 * what a single warp can issue, the situation of the sweep kernels at 16384 walkers).
 * *per_second receives thread instructions per second (words per second for
 * MUCA_PROBE_PHILOX).  Runs for about 0.1 s; allocates 4 KiB of device memory.
 * Errors: MUCA_EINVAL (unknown kind, NULL), MUCA_ECUDA. */
#define MUCA_PROBE_XOR 0
#define MUCA_PROBE_MAD 1
#define MUCA_PROBE_MIXED 2
#define MUCA_PROBE_PHILOX 3
#define MUCA_PROBE_MIXED_ONE_WARP 4
int muca_measure_issue_rate(int32_t kind, double *per_second);

/* Site order of later updates (sweeps, attempts, iterations, production):
 * MUCA_ORDER_TYPEWRITER (default): attempt t flips site t mod N;
 * MUCA_ORDER_RANDOM: the paper's scheme (Sec. 2.3), one random site sequence shared by
 * all walkers, the site of attempt t being floor(u N / 2^32) with u the Philox word t & 3
 * of counter (t >> 2, 0xFFFFFFFF, tag 2); acceptance words as in typewriter order.
 * Random order runs on its own kernel (any L and attempt range); the batched entry
 * points run typewriter order only and reject instances in random order.
 * Errors: MUCA_EINVAL (NULL, unknown order). */
#define MUCA_ORDER_TYPEWRITER 0
#define MUCA_ORDER_RANDOM 1
int muca_set_site_order(muca_t h, int32_t order);
int muca_get_site_order(muca_t h, int32_t *order);

/* Runs the instance's work on the given cudaStream_t (passed as void*; NULL = the
 * instance's own stream).  Work already queued on the old stream is synchronized first. */
int muca_set_stream(muca_t h, void *cuda_stream);

/* Replaces the device allocator used by later muca_create calls (alloc == NULL restores
 * cudaMalloc/cudaFree).  alloc(size, ctx) returns device memory or NULL. */
int muca_set_allocator(void *(*alloc)(size_t size, void *ctx), void (*release)(void *ptr, void *ctx),
                       void *ctx);

/* Copies ln W(e), e = 0 .. N (FP64, n_bins = N + 1), into the instance and rebuilds the
 * acceptance-threshold table (Sec. 2.3) on the device, on the instance's stream (the
 * thresholds equal muca_build_table's bit for bit).  Errors: MUCA_EINVAL (wrong n_bins,
 * NULL, non-finite value). */
int muca_set_weights(muca_t h, const double *lnW, size_t n_bins);

/* Histogram reduction for a simulation spread over several instances (Sec. 2.2: the
 * walkers' histograms are summed before the weights are updated), e.g. one instance per
 * GPU with disjoint walker ranges (muca_options.first_walker).  fn(H, n_bins, ctx) is
 * called on the host with the instance's histogram after every recorded phase of
 * muca_iterate_until_flat, muca_production and muca_production_jackknife, before it is
 * used, and must replace it by the sum over all instances of the simulation (an
 * all-reduce); every instance then takes the same stop decision and computes the same
 * weights.  total_walkers (>= n_walkers) is the simulation's walker count, used by the
 * Eq. (7) schedule.  fn == NULL removes it.  muca_get_histogram still returns the
 * instance's own counts.  muca_iterate_device and muca_batch_create refuse instances
 * with a reducer (MUCA_EINVAL). */
typedef void (*muca_histogram_reducer)(uint64_t *H, size_t n_bins, void *ctx);

/* Observer of the weight iteration (for convergence traces such as the paper's Fig. A.1):
 * fn(iteration, H, n_bins, metric, n_therm, n_updates, ctx) is called by
 * muca_iterate_until_flat after the stop metric of every iteration (iteration counts
 * from 1; H is the histogram the metric was computed from, valid during the call;
 * n_therm and n_updates are the attempts per walker of that iteration).  fn == NULL
 * removes it. */
typedef void (*muca_iteration_observer)(int32_t iteration, const uint64_t *H, size_t n_bins, double metric,
                                        uint64_t n_therm, uint64_t n_updates, void *ctx);
int muca_set_iteration_observer(muca_t h, muca_iteration_observer fn, void *ctx);
int muca_set_histogram_reducer(muca_t h, muca_histogram_reducer fn, void *ctx, int64_t total_walkers);

/* Copies the current ln W into lnW_out[n_bins]. */
int muca_get_weights(muca_t h, double *lnW_out, size_t n_bins);

/* Copies the threshold table T[e*5 + k] (uint32, n = 5 * (N + 1)) into T_out. */
int muca_get_table(muca_t h, uint32_t *T_out, size_t n);

/* Every walker performs n_sweeps * N further attempts (Sec. 2.3); record = 0 is
 * thermalization, record != 0 adds each post-decision energy to H.  Asynchronous. */
int muca_sweep(muca_t h, uint64_t n_sweeps, int record);

/* Same as muca_sweep for any number of attempts per walker (partial sweeps, as the
 * schedule of Eq. (7) asks for). */
int muca_attempts(muca_t h, uint64_t n_attempts, int record);

/* Copies H (uint64, n_bins = N + 1, summed over walkers, Sec. 2.2) into out.  Syncs. */
int muca_get_histogram(muca_t h, uint64_t *out, size_t n_bins);

/* Sets H to zero (asynchronous). */
int muca_reset_histogram(muca_t h);

/* The sampling of one weight iteration (Sec. 3: N_therm thermalization attempts, then
 * N_updates recorded ones): zeroes H, then every walker performs n_therm attempts
 * without recording and n_record recorded attempts.  The results (lattices, energies,
 * attempt counter, H) equal those of muca_reset_histogram, muca_attempts(h, n_therm, 0)
 * and muca_attempts(h, n_record, 1).  In typewriter order, when both counts are whole
 * sweeps starting at a sweep boundary, the two phases run in one kernel launch (the
 * lattices are read and written once); otherwise as two launches.  Asynchronous. */
int muca_thermalize_and_record(muca_t h, uint64_t n_therm, uint64_t n_record);

/* The weight iteration of Sec. 2.2 and Sec. 3: repeat { thermalize; zero H; record;
 * stop if H meets the stop rule; else ln W(e) -= ln H(e) where H(e) > 0 (Eq. 4) }.
 * On success the instance holds the weights that produced the flat histogram.
 * Returns MUCA_OK, MUCA_ENOTCONVERGED or MUCA_ETIMEOUT (stats filled in every case),
 * or another error.  p == NULL uses muca_default_params; stats may be NULL. */
int muca_iterate_until_flat(muca_t h, const muca_params *p, muca_stats *stats);

/* The same weight iteration with its host-side steps on the device: after each recorded
 * phase kernels test the stop rule, apply Eq. (4) and build the next threshold table,
 * so no histogram or table crosses to the host between iterations.  The host enqueues
 * iterations_per_sync (>= 1) iterations at a time and then reads a small state record;
 * iterations enqueued after the stop do nothing.  Fixed-sweep schedule only
 * (MUCA_SCHEDULE_SWEEPS; the Eq. (7) schedule sizes each iteration from the previous
 * histogram on the host).  Weights, table, histogram, lattices, energies, attempt
 * counter and stats equal those of muca_iterate_until_flat bit for bit, except that a
 * deadline is checked only every iterations_per_sync iterations.  Returns as
 * muca_iterate_until_flat; MUCA_EINVAL also for another schedule or
 * iterations_per_sync < 1.  Allocates (N + 1) doubles and a state record on the device
 * at the first call. */
int muca_iterate_device(muca_t h, const muca_params *p, int32_t iterations_per_sync, muca_stats *stats);

/* Host computations of the library without an instance (no device needed).
 * muca_build_table: thresholds T_out[e*5 + k] (n_bins = L*L + 1 weights in, 5 n_bins
 * thresholds out) by the rule above.  muca_update_weights: Eq. (4) in logarithms,
 * lnW[e] -= ln H[e] where H[e] > 0, in place.  Errors: MUCA_EINVAL (L as in muca_create,
 * wrong n_bins, NULL, non-finite weight). */
int muca_build_table(int32_t L, const double *lnW, size_t n_bins, uint32_t *T_out);
int muca_update_weights(int32_t L, double *lnW, const uint64_t *H, size_t n_bins);

/* The three flatness measures of a histogram H[n_bins] (n_bins = L*L + 1), host FP64 as
 * the iteration computes them: *min_over_mean = min H / mean H over the accessible
 * energies; *kl = d_k of Eq. (6) with the reference width taken from the union of
 * [prev_lo, prev_hi] (the previous iteration's visited range, prev_lo = -1 for none) and
 * the visited range of H; *chebyshev = d_c of Eq. (A.1); *lo, *hi = the visited range of H
 * (-1, -1 when empty).  Every output may be NULL.  For per-iteration logs (the
 * convergence traces of App. A).  Errors: MUCA_EINVAL (L as in muca_create, wrong
 * n_bins, NULL H, prev_hi < prev_lo or outside the grid when prev_lo >= 0). */
int muca_flatness(int32_t L, const uint64_t *H, size_t n_bins, int32_t prev_lo, int32_t prev_hi,
                  double *min_over_mean, double *kl, double *chebyshev, int32_t *lo, int32_t *hi);

/* Production run (Sec. 3.3) with the current weights: therm_sweeps unrecorded sweeps,
 * zero H, n_sweeps recorded sweeps, then ln g(e) = ln H(e) - ln W(e) on visited energies
 * shifted so that sum_e exp(ln g(e)) = 2^N; unvisited energies get -inf.  H_out (may
 * be NULL) receives the histogram, ln_g_out[n_bins] the estimate. */
int muca_production(muca_t h, uint64_t therm_sweeps, uint64_t n_sweeps, uint64_t *H_out,
                    double *ln_g_out, size_t n_bins);

/* Production with error bars (Sec. 3.3): thermalize, then n_chunks >= 2 recorded
 * chunks of sweeps_per_chunk sweeps, each with its own histogram (H_chunks_out, may be
 * NULL, receives them as [chunk][bin]).  ln_g_out is the estimate from all chunks
 * (as muca_production); ln_g_err_out the jackknife error over leave-one-chunk-out
 * estimates, sqrt((n-1)/n sum_c (x_c - mean)^2), +inf where an energy is missing from
 * some leave-one-out histogram and NaN where it was never visited. */
int muca_production_jackknife(muca_t h, uint64_t therm_sweeps, int32_t n_chunks, uint64_t sweeps_per_chunk,
                              uint64_t *H_chunks_out, double *ln_g_out, double *ln_g_err_out, size_t n_bins);

/* Reweighting ln g (n_bins = L*L + 1, -inf entries skipped) to the canonical ensemble,
 * P(E) ~ g(E) exp(-beta E) (Eq. 1): energy per spin <E>/N and specific heat per spin
 * beta^2 (<E^2> - <E>^2)/N (may be NULL) at each of n_betas inverse temperatures.
 * Host-only arithmetic in FP64 (log-sum-exp); no instance or GPU needed. */
int muca_reweight(int32_t L, const double *ln_g, size_t n_bins, const double *betas, size_t n_betas,
                  double *energy_per_spin, double *specific_heat_per_spin);

/* Copies the walkers' energy indices (int32, n = n_walkers).  Syncs. */
int muca_get_energies(muca_t h, int32_t *e_out, size_t n);

/* Copies the lattices as int8 spins out[walker][site] (+1 / -1, n = n_walkers * N). */
int muca_get_lattice(muca_t h, int8_t *out, size_t n);

/* Instance facts: lattice side, walkers, attempt counter, layout, walkers per block. */
int muca_get_info(muca_t h, int32_t *L, int64_t *n_walkers, uint64_t *attempt_counter,
                  int32_t *layout, int32_t *walkers_per_block);

/* Waits for the instance's queued work; reports MUCA_EDEVICE if a kernel flagged an
 * invalid state. */
int muca_synchronize(muca_t h);

/* Waits at most `seconds` for the work queued so far on the instance's stream (polling,
 * no blocking wait), then checks the device error word as muca_synchronize does.
 * Returns MUCA_ETIMEOUT if the work is still running (it keeps running; a later call
 * can wait again), MUCA_EINVAL for NULL or a negative limit. */
int muca_synchronize_timeout(muca_t h, double seconds);

/* Evaluates the library's device Philox4x32-10 on n counters (ctr[4*i .. 4*i+3]) with
 * one key (key[0] low, key[1] high 32 bits of the seed) into out[4*n].  Host buffers;
 * used to check the generator against independent implementations. */
int muca_philox(const uint32_t *ctr, const uint32_t key[2], size_t n, uint32_t *out);

/* ----------------------------------------------------------------------------------
 * Batches (Sec. 2.2 applied to many independent simulations at once): one launch of a
 * persistent kernel advances every member instance; each block takes work items
 * (instance, 256 or fewer walkers) from a global counter, so instances of uneven L and
 * walker count share the GPU.  Member instances must have L in {8, 16, 24, 32, 48, 64}.
 * Results are the same as running each instance alone (walkers and histograms of
 * different instances never interact).
 * -------------------------------------------------------------------------------- */
typedef struct muca_batch_s *muca_batch_t;

/* Groups n existing instances.  The batch does not own them; while it exists their
 * work runs on the batch's stream (ordered with batch launches); muca_batch_destroy
 * gives each instance its stream back.  Allocates the launch descriptors, the work list
 * and the work counters on the device.  Errors: MUCA_EINVAL (NULL, duplicates, L
 * without a whole-sweep kernel), MUCA_ENOMEM, MUCA_ECUDA. */
int muca_batch_create(const muca_t *instances, int32_t n, muca_batch_t *out);
int muca_batch_destroy(muca_batch_t b);

/* Every member performs n_sweeps further sweeps (record as in muca_sweep) in one
 * batched launch (more if the 32-bit per-block counts require it).  Asynchronous. */
int muca_batch_sweep(muca_batch_t b, uint64_t n_sweeps, int record);

/* The weight iteration of muca_iterate_until_flat for every member at once (either
 * schedule; with MUCA_SCHEDULE_PAPER each member follows Eq. (7) from its own visited
 * ranges, and launches may start and end inside sweeps).  Each iteration is one replay of
 * a CUDA graph (table uploads, zeroed histograms, one launch in which every member's
 * walkers thermalize and then record, histogram reads), or, when a member records more
 * than 0xFFFFFFFF / 256 attempts per walker, the same steps issued directly with a
 * thermalization launch and several recording launches;
 * a member leaves the work list when its histogram is flat or it reached max_iterations.
 * stats[i] (may be NULL) receives member i's result, seconds being the wall time until
 * its last iteration finished.  Returns MUCA_OK if every member became flat, else
 * MUCA_ENOTCONVERGED or MUCA_ETIMEOUT. */
int muca_batch_iterate(muca_batch_t b, const muca_params *p, muca_stats *stats);

/* Members, persistent grid size and dynamic shared memory per block of the batch. */
int muca_batch_info(muca_batch_t b, int32_t *n_instances, int32_t *grid, size_t *smem_bytes);

/* ----------------------------------------------------------------------------------
 * Serving: weight iterations requested over time.  A request is admitted (its instance
 * created and kept resident on the device) as soon as its device memory fits the
 * server's budget; every muca_server_step advances all admitted requests by one
 * batched weight iteration (one graph replay of the batched kernel, so requests that
 * arrive while others run share the GPU), and a request leaves when its histogram is
 * flat or it reached its max_iterations, freeing its memory for queued requests.  Each
 * request's result equals that of muca_iterate_until_flat on the same instance alone.
 * -------------------------------------------------------------------------------- */
typedef struct muca_server_s *muca_server_t;

#define MUCA_REQ_QUEUED 0
#define MUCA_REQ_ACTIVE 1
#define MUCA_REQ_DONE 2

typedef struct {
    int32_t L;                   /* one of 8, 16, 24, 32, 48, 64                           */
    int64_t n_walkers;
    uint64_t seed;
    int32_t layout;              /* MUCA_LAYOUT_INT8 or MUCA_LAYOUT_PACKED                 */
    int32_t walkers_per_block;   /* 0 = from occupancy                                     */
    muca_params params;          /* either schedule, no resume                             */
} muca_request;

typedef struct {
    int32_t state;               /* MUCA_REQ_*                                             */
    int32_t code;                /* when done: MUCA_OK (flat), MUCA_ENOTCONVERGED, error   */
    muca_stats stats;            /* iterations, flatness, attempts; seconds while admitted */
    double seconds_queued;       /* arrival -> admission (so far)                          */
    double seconds_total;        /* arrival -> done: the time to converged weights         */
} muca_request_status;

/* Creates a server that keeps at most hbm_budget_bytes of instance device memory. */
int muca_server_create(size_t hbm_budget_bytes, muca_server_t *out);
int muca_server_destroy(muca_server_t s);

/* Enqueues a request (arrival time = now) and returns its id.  Errors: MUCA_EINVAL
 * (L not in the list, bad parameters), MUCA_ENOMEM (larger than the whole budget). */
int muca_server_submit(muca_server_t s, const muca_request *r, int64_t *id);

/* Admits what fits, runs one batched iteration of all admitted requests, retires the
 * finished ones.  Reports the admitted and queued counts afterwards. */
int muca_server_step(muca_server_t s, int32_t *n_active, int32_t *n_queued);

/* State and timing of a request; its final ln W (n_bins = L*L + 1) once done. */
int muca_server_status(muca_server_t s, int64_t id, muca_request_status *out);
int muca_server_weights(muca_server_t s, int64_t id, double *lnW_out, size_t n_bins);

/* Walker-attempts run so far, seconds since creation, steps, device bytes in use. */
int muca_server_totals(muca_server_t s, uint64_t *walker_attempts, double *seconds, int32_t *steps,
                       size_t *bytes_in_use);

/* ----------------------------------------------------------------------------------
 * Allocation-free batched sweep.  The paper has no counterpart: this entry point exists
 * for callers that must not allocate device memory while they run, for instance an
 * application that owns the GPU's memory and lends out fixed buffers reserved at start-up,
 * a plugin whose host forbids allocation after initialisation, or a loop that cannot
 * afford the device-wide synchronisation a cudaMalloc/cudaFree may cause.  Such a caller
 * passes its own device buffers; the call allocates nothing (no cudaMalloc, cudaFree or
 * allocating library routine).  The kernel's one piece of scratch, its work counter, sits
 * in a fixed array of MUCA_NOALLOC_SCRATCH_BYTES in device memory that every GPU loading
 * this library keeps until the process exits; the instance descriptors travel in the
 * kernel's launch parameters.
 * -------------------------------------------------------------------------------- */
#define MUCA_NOALLOC_MAX_INSTANCES 64
#define MUCA_NOALLOC_SCRATCH_BYTES 256

/* One instance's state in caller-owned device memory, in the layouts of this header:
 * lattice in `layout`, energy indices int32[n_walkers], thresholds uint32[(L*L+1)*5]
 * (as muca_get_table returns them), histogram uint64[L*L+1] (added to), error word
 * uint32 (bits OR-ed in, 0 = fine).  t0 is the attempt counter of the first attempt and
 * must lie on a sweep boundary (a multiple of L*L).  A walker whose energy index lies
 * outside 0..L*L sets bit 0 of the error word and is left unchanged; an index inside
 * that range that does not match the walker's lattice is used as given (flips whose
 * target energy leaves the grid are rejected: their thresholds are 0). */
typedef struct {
    int32_t L;                   /* one of 8, 16, 24, 32, 48, 64                           */
    int32_t layout;              /* MUCA_LAYOUT_INT8 or MUCA_LAYOUT_PACKED                 */
    int64_t n_walkers;
    uint64_t seed;
    uint64_t t0;
    void *lattice;
    int32_t *energy;
    const uint32_t *table;
    unsigned long long *hist;
    uint32_t *err;
} muca_raw_instance;

/* Every one of the n instances (at most MUCA_NOALLOC_MAX_INSTANCES) performs n_sweeps
 * whole sweeps (record as in muca_sweep) in one launch of the batched kernel on
 * cuda_stream (NULL = the default stream); results are those of muca_batch_sweep on the
 * same state.  The caller advances its t0 by n_sweeps * L * L afterwards.
 *  - The first call on a device looks up the scratch array's device address (once per
 *    device, with that device current); make that first call before any stream capture.
 *  - The instance array is read during the call (its descriptors become the kernel's
 *    launch parameters), so it may be reused as soon as the call returns.
 *  - All calls share the one scratch array, which keeps the last call's contents (each
 *    call zeroes the work counter on cuda_stream before its launch): calls that overlap
 *    on the GPU (other streams, other host threads) race and must not be issued.
 * Errors: MUCA_EINVAL (NULL, more than MUCA_NOALLOC_MAX_INSTANCES instances, L outside
 * the list, t0 off a sweep boundary, a recorded launch longer than 0xFFFFFFFF / 256
 * attempts per walker, more than 2^31 - 1 work items of up to 256 walkers, two instances
 * whose lattice or energy buffers overlap, the same instance given twice included),
 * MUCA_ECUDA. */
int muca_batch_sweep_noalloc(const muca_raw_instance *instances, int32_t n, uint64_t n_sweeps, int record,
                             void *cuda_stream);

/* Message of the last failed call on this host thread ("" if none). */
const char *muca_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MUCA_H */
