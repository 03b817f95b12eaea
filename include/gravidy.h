/*
 * gravidy.h -- C ABI of the GB300 Hermite-4 block-time-step N-body library
 * (libgravidy_gb300.so).
 *
 * The library integrates the Newtonian N-body problem with Plummer softening
 * (GraviDy, arXiv 1702.00440, Sec. 2.1 Eq. 1 and its softened form in
 * Sec. 2.4) by the 4th-order Hermite predictor-corrector (Sec. 2.1) with
 * power-of-two block time steps (Sec. 2.4) and Aarseth's time-step criterion
 * with parameter eta (Sec. 3.2).  One block step follows Sec. 2.4 steps 5-7:
 * find the active particles, predict all N particles, compute the force and
 * jerk of the active ones against all N predicted ones (the O(N_act N) part,
 * Sec. 2.5), correct the active particles and give them new steps.  Every
 * step runs on the GPU; the host only launches work and reads results.
 *
 * Conventions
 *   - G = 1.  Units are whatever the caller uses (N-body units in the tests).
 *   - Host arrays at this boundary are AoS: x, v, a, jerk are n*3 doubles
 *     (x0 y0 z0 x1 y1 z1 ...); m is n doubles.  Inside, the library keeps
 *     structure-of-arrays copies on the device.
 *   - Time is kept as integer ticks of dt_min (a power of two): a particle's
 *     time is tau * dt_min and its step dtau * dt_min, dtau a power of two.
 *   - Ownership: the caller owns every host array; the library copies in and
 *     out and never keeps a caller pointer.  gd_ctx owns all device memory.
 *   - Errors: every int-returning call returns GD_OK (0) or a negative
 *     gd_status; gd_last_error() gives a message.  Faults found on the device
 *     (a non-finite value, a bounded wait that ran out) are recorded in a
 *     device flag and returned by the next call that synchronises.
 *   - Threading: a gd_ctx is not thread-safe; distinct contexts are
 *     independent.
 */
#ifndef GRAVIDY_H
#define GRAVIDY_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gd_status {
    GD_OK = 0,
    GD_EINVAL = -1,      /* bad argument */
    GD_ENOMEM = -2,      /* device or host allocation failed */
    GD_ECUDA = -3,       /* a CUDA runtime call failed */
    GD_ENONFINITE = -4,  /* a corrected state or step was NaN/Inf */
    GD_ETIMEOUT = -5,    /* a bounded device-side wait gave up */
    GD_ESTATE = -6       /* call not valid in the current state */
} gd_status;

typedef enum gd_precision {
    /* all pair arithmetic in FP64 */
    GD_FP64 = 0,
    /* pair arithmetic in FP32 on double-single (hi+lo float) positions with
     * compensated sums; positions and velocities kept double-single (about 48
     * significant bits, every value an FP64 number, so gd_get_state /
     * gd_set_state round trips are exact), accelerations and jerks FP32;
     * prediction and correction in FP32/double-single arithmetic, energy sums in
     * FP64 (the mixed-precision alternative of Sec. 2.3).  Needs dt_min >= 2^-24
     * and dt_max/dt_min <= 2^24. */
    GD_MIXED = 1
} gd_precision;

typedef struct gd_opts {
    double dt_min;      /* smallest block step, a power of two (default 2^-22) */
    double dt_max;      /* largest block step, a power of two >= dt_min (default 1/8) */
    int32_t precision;  /* gd_precision (default GD_MIXED) */
    int32_t device;     /* CUDA device ordinal (default 0) */
    void *stream;       /* cudaStream_t to run on; NULL = a stream owned by the context */
    int32_t use_graph;  /* 1 = run gd_evolve through a captured CUDA graph (default 1) */
    int32_t graph_steps;/* block steps per graph launch, a multiple of 1..64 (default 16) */
    int32_t jsplit;     /* > 0 forces the j-split factor of the force kernel; 0 = tuned */
    int32_t mode_cut;   /* active count at/above which the i-parallel force mode is used
                           (0 = default: 1024 mixed, 256 FP64); per-bucket autotuned choices
                           override it */
    int32_t time_force; /* 1 = record CUDA events around every force launch (gd_kernel_time) */
    int32_t autotune;   /* 1 = run gd_autotune(c, 3) at the end of gd_init */
    int32_t fused;      /* GD_MIXED: 1 = gd_evolve runs many block steps per cooperative launch of
                           one fused kernel with grid barriers; 0 = three kernels per block step
                           (graph or eager, see use_graph; the default, faster on GB300 at the
                           sizes measured).  Both compute the same results bit for bit. */
    int32_t pdl;        /* three-kernel path: 1 = launch the step kernels with programmatic
                           dependent launch (each may start while the previous finishes) */
    int32_t tail_correct; /* three-kernel path: 1 = the force kernel corrects warp-mode tiles in
                           their reduction tails and finalizes the step (k_correct then only
                           handles i-parallel plans); 0 = k_correct always corrects */
    int32_t cluster;    /* GD_MIXED, gd_evolve: 1 (default) = block steps with few active
                           particles run inside one thread-block cluster that holds the whole
                           system in its shared memory (no kernel launch per step), larger
                           steps on the full GPU; used when n fits (about 20000 particles with
                           16-CTA clusters) and the GPU can launch the cluster, else ignored.
                           0 = every step on the full GPU.  The two differ in the order of
                           the force sums (last bits); each is deterministic. */
    int32_t corrector;  /* GD_CORR_HERMITE (default): the 4th-order Hermite corrector of Sec. 2.4
                           step 7d; GD_CORR_TIMESYM: its time-symmetric form (Hut, Makino &
                           McMillan 1995), with h = dt/2, v1 = v0 + h (a1 + a0) - h^2/3 (j1 - j0),
                           x1 = x0 + h (v1 + v0) - h^2/3 (a1 - a0); the same force, Aarseth step
                           and block quantisation, in every path (three kernels, small-step
                           cluster, fused kernel, ensembles) and both precisions */
    int32_t pn_terms;   /* post-Newtonian terms of one pair (Sec. 5: corrections for a binary):
                           0 (default) none; a combination of GD_PN_1, GD_PN_2 and GD_PN_25: the
                           1PN, 2PN and 2.5PN (radiation reaction) relative accelerations of the
                           two-body problem in harmonic coordinates (Kidder 1995; Blanchet 2014),
                           added with their time derivative to the force and jerk of particles
                           pn_p (share m_q/M) and pn_q (share -m_p/M) whenever they are active,
                           in every path (three kernels, small-step cluster, fused kernel).
                           gd_init only (not ensembles) */
    int32_t pn_p, pn_q; /* the pair, distinct indices in [0, n) */
    double pn_c;        /* speed of light in the caller's units (G = 1), > 0 */
    int32_t n_iter;     /* evaluation-correction passes per block step, 1 (default) to 16: with
                           n_iter > 1 (P(EC)^n, Kokubo, Yoshinaga & Makino 1998; needs the
                           time-symmetric corrector) every pass but the last evaluates the
                           active particles' force and jerk and writes their corrected position
                           and velocity over their predicted ones, which the next pass evaluates
                           against; the last pass corrects as usual.  Each pass counts its
                           N_act * N interactions.  The three-kernel step and the small-step
                           cluster take the passes (not the fused kernel or ensembles; no
                           post-Newtonian pair) */
} gd_opts;

enum { GD_CORR_HERMITE = 0, GD_CORR_TIMESYM = 1 };
enum { GD_PN_1 = 1, GD_PN_2 = 2, GD_PN_25 = 4 };

typedef struct gd_stats {
    int64_t tick;          /* time of the last block step, in ticks */
    int64_t block_steps;   /* block steps taken (Sec. 2.4 "Iter") */
    int64_t particle_steps;/* sum of N_act over block steps ("Nsteps") */
    double interactions;   /* sum of N_act * N over all force evaluations */
    int64_t last_nact;     /* N_act of the last block step */
    int64_t kernel_launches; /* CUDA kernels this context has launched (host count) */
    double phase_ms[3];    /* time spent in the select/predict, force (+ small-set correction)
                              and correction phases of the fused gd_evolve kernel and of the
                              small-step cluster kernel, each up to and including its grid or
                              cluster barrier (one CTA's device clock); 0 on the three-kernel
                              path */
} gd_stats;

typedef struct gd_ctx gd_ctx;

/* Fill *o with the defaults listed in gd_opts. */
void gd_opts_default(gd_opts *o);

/* Sec. 2.4 steps 1-4: allocate the device store, copy m, x, v in, compute the
 * initial force and jerk of all n particles (O(n^2)) and the first block step
 * of each, dt = eta |a| / |jerk| rounded down to a power of two in
 * [dt_min, dt_max].  eps is the Plummer softening length (>= 0; eps = 0 gives
 * the unsoftened Eq. 1 with the self term excluded), eta > 0.  An eps whose
 * square is below the smallest normal number of the pair arithmetic (FP32 for
 * GD_MIXED, FP64 for GD_FP64) changes no resolvable r^2 and runs as eps = 0;
 * an eps with max(m) / eps^3 beyond that precision's range (the self term of
 * the softened sum would overflow) is GD_EINVAL.  opt may be NULL for the
 * defaults.  On success *out is a new context (time 0). */
int gd_init(gd_ctx **out, int64_t n, const double *m, const double *x, const double *v,
            double eps, double eta, const gd_opts *opt);

/* Advance by block steps (Sec. 2.4 steps 5-7) until no particle's next time
 * is <= t_end.  With t_end a multiple of dt_max every particle ends exactly
 * at t_end (synchronised).  t_end must not be below the current time. */
int gd_evolve(gd_ctx *c, double t_end);

/* One block step; *t_out (nullable) receives its time and *nact_out
 * (nullable) its number of active particles. */
int gd_step_block(gd_ctx *c, double *t_out, int64_t *nact_out);

/* Kinetic and potential energy (Sec. 2.1 Eq. 2, with the potential softened
 * like the force: -sum_{i<j} m_i m_j / sqrt(r_ij^2 + eps^2)) at the time of
 * the last block step; particles behind it are predicted to it first.  GD_FP64
 * computes every pair term in FP64; GD_MIXED computes the pair terms in FP32 on
 * double-single positions (one Newton step on rsqrt, about 8 units of 2^-24 per
 * term) and sums them with compensation; both return FP64 totals. */
int gd_energy(gd_ctx *c, double *K, double *U);

/* Copy the state out: x, v, a, jerk as n*3 AoS doubles (each particle at its
 * own time), tau and dtau as n int64 ticks.  Any pointer may be NULL. */
int gd_get_state(gd_ctx *c, double *x, double *v, double *a, double *jerk, int64_t *tau,
                 int64_t *dtau);

/* Replace the state (checkpoint restart); same layouts as gd_get_state.  All
 * pointers are required.  Every dtau must be a power of two in
 * [1, dt_max/dt_min] and every tau a non-negative multiple of its dtau. */
int gd_set_state(gd_ctx *c, const double *x, const double *v, const double *a,
                 const double *jerk, const int64_t *tau, const int64_t *dtau);

/* Force-kernel autotuner: for every active-count bucket floor(log2 N_act) up to
 * 2^34 interactions, times the force kernel (CUDA events, median of reps
 * launches, 1 <= reps <= 100) on the current particles for both work
 * decompositions (i-parallel tiles; warp j-parallel tiles, their j-split sums
 * taken in the force kernel or in the corrector) and a ladder of
 * j-split factors (the j-range split of Sec. 2.5), and keeps the fastest choice
 * for later steps.  The integration state is not changed. */
int gd_autotune(gd_ctx *c, int32_t reps);

/* The tuning table: *mode_cut, and for buckets b < nbuckets (<= 32) the j-split
 * factor split[b] (0 = rule), the mode mode[b] (0 i-parallel, 1 warp, 2 warp with
 * the j-split partials summed in the corrector, -1 rule)
 * and the autotuner's best force-kernel time ms[b] for N_act = 2^b (0 = not
 * measured).  Any pointer may be NULL. */
int gd_get_tuning(gd_ctx *c, int32_t *mode_cut, int16_t *split, int8_t *mode, float *ms,
                  int32_t nbuckets);

/* Replace the tuning table (the inverse of gd_get_tuning): mode_cut >= 1, and
 * for buckets b < nbuckets (<= 32) split[b] >= 0 and mode[b] in {-1, 0, 1, 2}
 * (meanings as in gd_get_tuning; NULL leaves that column unchanged).  Two
 * contexts with the same table and state take the same block steps with the
 * same arithmetic.  The integration state is not changed. */
int gd_set_tuning(gd_ctx *c, int32_t mode_cut, const int16_t *split, const int8_t *mode, int32_t nbuckets);

/* Counters since gd_init. */
int gd_get_stats(gd_ctx *c, gd_stats *s);

/* Device time of the full-GPU force-kernel launches recorded (CUDA events on
 * the context's stream) since the last call, for launches with a non-empty
 * active set (needs opts.time_force = 1; the small-step cluster's steps are
 * timed by gd_cluster_time): *ms_total summed milliseconds, *launches
 * their count, *interactions the sum of N_act * N they computed.  With the fused
 * gd_evolve path the timed kernel is the fused block-step kernel (prediction,
 * force and correction together).  Any pointer may be NULL.  Resets the
 * counters. */
int gd_kernel_time(gd_ctx *c, double *ms_total, int64_t *launches, double *interactions);

/* The small-step cluster gd_evolve uses (opts.cluster): *csize CTAs per
 * cluster (0 = not used: FP64 context, option off, n too large for its shared
 * memory, or no such cluster can be launched), *per_cta particles each CTA
 * holds, *max_nact the largest active count a cluster step takes (larger steps
 * run on the full GPU).  Any pointer may be NULL. */
int gd_cluster_info(gd_ctx *c, int32_t *csize, int32_t *per_cta, int32_t *max_nact);

/* Where the small-step cluster's time goes: SM cycles of CTA 0 (accumulated
 * since gd_init) in the phases of every small block step it finished --
 * [0] predict and list the CTA's active particles, [1] publish the count,
 * cluster barrier, offsets, [2] gather the active records, [3] force tasks,
 * [4] segment sums and partial push, [5] cluster barrier, [6] correction,
 * [7] publish the next-time minimum, cluster barrier, [8] next block time --
 * then [9] the launches' prologues (state into shared memory), [10] their
 * epilogues (write-back, hand-over) and [11] the number of small steps.  The
 * first count (<= 12) values go to cycles; *clock_khz (nullable) receives the
 * device's maximum SM clock. */
int gd_cluster_phases(gd_ctx *c, double *cycles, int32_t count, int32_t *clock_khz);

/* Device time of the small-step cluster launches of gd_evolve's graph or eager
 * path recorded since the last call (needs opts.time_force = 1): *ms_total
 * summed milliseconds, *launches their count (a launch takes zero or more block
 * steps).  The block steps and interactions of the cluster are the context's
 * totals (gd_get_stats) minus those gd_kernel_time reports.  Any pointer may be
 * NULL.  Resets the counters. */
int gd_cluster_time(gd_ctx *c, double *ms_total, int64_t *launches);

void gd_free(gd_ctx *c);

/* Message of the last error on c (or, for c NULL, of the calling thread's last
 * failed gd_init or gd_force_noalloc). */
const char *gd_last_error(const gd_ctx *c);

/* ---- hooks for tests and measurement (no integration state changes) ---- */

/* Force and jerk (Sec. 2.4, softened Eq. 1 and its time derivative) of the
 * nact particles idx[] (host int32, each in [0, n), duplicates allowed)
 * against all n particles predicted to tick; acc and jerk are nact*3 host
 * doubles in the order of idx.  State is unchanged. */
int gd_force(gd_ctx *c, int64_t tick, const int32_t *idx, int64_t nact, double *acc,
             double *jerk);

/* Positions and velocities of all n particles predicted to tick (Sec. 2.4
 * step 7a), n*3 AoS doubles each; either pointer may be NULL. */
int gd_predict(gd_ctx *c, int64_t tick, double *xp, double *vp);

/* The next block step taken inside the small-step cluster that gd_evolve uses
 * for steps with few active particles (gd_cluster_info), the same kernel and
 * arithmetic, stopped after that one step.  A step with more active particles
 * than the cluster takes is left untaken: *nact_out = 0 and *t_out = 0 (the
 * state is unchanged; gd_step_block takes it).  Otherwise *t_out (nullable) is
 * the step's time and *nact_out (nullable) its active count.  GD_ESTATE if the
 * context does not use the cluster. */
int gd_step_block_small(gd_ctx *c, double *t_out, int64_t *nact_out);

/* Positions and velocities of all n particles predicted to tick exactly as the
 * block step's predictor (Sec. 2.4 step 7a) stores them for the force kernel,
 * n*3 AoS doubles each; either pointer may be NULL.  GD_MIXED: the double-single
 * position of the j-record (hi + lo, an FP64 sum) and its FP32 velocity, from
 * the double-single / FP32 Taylor series of the mixed path; GD_FP64: the same as
 * gd_predict. */
int gd_predict_records(gd_ctx *c, int64_t tick, double *xp, double *vp);

/* The active set of the next block step (Sec. 2.4 step 5) without taking it:
 * idx (host, n int32) receives the list exactly as the block step's compaction
 * writes it on the device (ascending particle order), *nact its length,
 * *tick_next the block time. */
int gd_active(gd_ctx *c, int32_t *idx, int64_t *nact, int64_t *tick_next);

/* One block step with a given block time and active list (host int32,
 * ascending, distinct, each particle's next time must not be before
 * tick_next): used to replay another integrator's schedule.  The new steps
 * are computed and stored as usual but the block times come from the caller. */
int gd_replay_step(gd_ctx *c, int64_t tick_next, const int32_t *idx, int64_t nact);

/* Failure-detection probe: one GPU thread waits, with the bounded wait the
 * fused kernel's grid barrier uses, for a device counter that nothing
 * advances; after `limit` polls (limit in [1, 2^24]) it gives up, records
 * GD_ETIMEOUT in the device flag and ends.  Returns GD_ETIMEOUT, read back by
 * the same synchronisation as every other call; the context then refuses
 * further work, as after any device fault, while the CUDA context and the GPU
 * stay usable.  GD_EINVAL for a null context or a limit out of range. */
int gd_test_wait_timeout(gd_ctx *c, int32_t limit);

/* FP32 FMA throughput of the GPU (the roofline denominator of the FP32-bound
 * force kernels): a kernel whose threads run 8 independent FMA chains of
 * `iters` rounds each on every SM at full occupancy, timed with CUDA events
 * (best of three launches after a warm one).  *tflops (nullable) receives
 * 2 flop per FMA per lane over that time, *ms (nullable) the time.  iters in
 * [1, 2^24]; the calling thread's current device becomes `device`. */
int gd_probe_fma(int32_t device, int32_t iters, double *tflops, double *ms);

/* Allocation-failure injection for tests: the nth allocation of `kind` (0 = host,
 * pageable or pinned; 1 = device) that the calling thread's next context set-ups
 * (gd_init, gd_ens_init, gd_h6_init, gd_h6_init_scheme) make fails, once, as if
 * the allocator had run out; the set-up then frees what it holds and returns
 * GD_ENOMEM.  nth = 0 cancels a pending injection.  GD_EINVAL for kind not 0 or 1
 * or nth outside [0, 2^20].  Needs no GPU. */
int gd_test_fail_alloc(int32_t kind, int32_t nth);

/* ---- ensembles of independent clusters -------------------------------------
 *
 * nclusters independent N-body systems advanced together: every cluster follows
 * the same scheme as gd_init/gd_evolve (Sec. 2.4, Hermite-4 with block steps and
 * Aarseth's criterion, Plummer softening eps, parameter eta) and feels only its
 * own particles.  A global block step is the smallest next time over all clusters;
 * the active particles of every cluster whose next time equals it are advanced in
 * the same kernels (one captured graph replays many such steps).  GD_MIXED only.
 * Cluster q has n_per[q] particles, 1 <= n_per[q] <= 2^24, 1 <= nclusters <= 2048;
 * m, x, v are the clusters' arrays concatenated in cluster order (m: sum n_per
 * doubles, x and v: sum n_per * 3 doubles AoS).  Same ownership and error rules
 * as the single-system calls; gd_ens_last_error(NULL) reports a failed init. */
typedef struct gd_ens gd_ens;

int gd_ens_init(gd_ens **out, int32_t nclusters, const int64_t *n_per, const double *m, const double *x,
                const double *v, double eps, double eta, const gd_opts *opt);

/* Advance every cluster until no particle's next time is <= t_end.  With
 * opts.cluster = 1 (the default), opts.fused = 0 and every cluster small enough
 * (at most 16 x 1280 particles), each cluster is integrated on its own, without a
 * global block time: one launch per size class of thread-block clusters (the
 * fewest CTAs of up to 1280 particles that hold a cluster: 1, 2, 4, 8 or 16), whose
 * thread-block clusters take whole clusters from the class's work queue, largest
 * first, and run all of a cluster's block steps in shared memory; the same schedule and arithmetic per particle as the global steps, force
 * sums split over those CTAs.  Otherwise global block steps, as above. */
int gd_ens_evolve(gd_ens *s, double t_end);

/* One global block step; *t_out its time, *nact_out its active particles (all clusters). */
int gd_ens_step_block(gd_ens *s, double *t_out, int64_t *nact_out);

/* Per-cluster kinetic and potential energy (nclusters doubles each) at the time of
 * the last global block step (Eq. 2 with the softened potential, FP32 pair terms
 * on double-single positions summed with compensation, FP64 totals). */
int gd_ens_energy(gd_ens *s, double *K, double *U);

/* Concatenated state (cluster order, as given to gd_ens_init); any pointer may be NULL. */
int gd_ens_get_state(gd_ens *s, double *x, double *v, int64_t *tau, int64_t *dtau);

/* Counters over all clusters (interactions count only pairs within a cluster).
 * block_steps counts global block steps, except that gd_ens_evolve on the
 * independent-cluster path adds every cluster's own block steps. */
int gd_ens_get_stats(gd_ens *s, gd_stats *st);

void gd_ens_free(gd_ens *s);
const char *gd_ens_last_error(const gd_ens *s);

/* ---- allocation-free variant ---------------------------------------------
 *
 * The paper has no counterpart of this entry point; it exists for callers that
 * cannot call cudaMalloc -- code running where another component owns the
 * device memory budget (a framework's caching allocator, a hard memory cap),
 * or on a latency-critical path where an allocation and the device-wide
 * synchronisation it may imply are not acceptable.
 *
 * gd_force_noalloc computes what gd_force computes with GD_MIXED precision --
 * the softened acceleration and jerk of the particles idx[0..nact) against all
 * n particles, in FP32 pair arithmetic on double-single positions -- but from
 * caller-owned DEVICE arrays and without allocating anything.  Its scratch
 * (3,949,056 bytes, 3.77 MiB: j-records, j-split partial sums, summed forces,
 * a control block) is a fixed array compiled into the library, which every GPU
 * that loads the library holds until the process exits.
 *
 *   n      number of particles, 1 <= n <= 32768 (larger n returns GD_EINVAL)
 *   m      device, n doubles;  x, v  device, n*3 doubles (AoS xyz)
 *   eps    Plummer softening >= 0; eps^2 below FLT_MIN runs as eps = 0.  With
 *          eps > 0 the row of particle i is finite only while m_i / eps^3 is
 *          finite in FP32 (its self term); the masses are not inspected
 *   idx    device, nact int32 particle indices (duplicates allowed); an entry
 *          outside [0, n) yields NaN in its output rows
 *   nact   1 <= nact <= n
 *   acc, jerk  device, nact*3 doubles (AoS), written in the order of idx
 *   stream cudaStream_t to run on (NULL = the legacy default stream)
 *
 * All pointers refer to memory on the current device.  The call only queues
 * kernels: results are ready once the stream has reached them.  The first call
 * on a device does a one-time set-up for that device (it looks up the scratch
 * array's device address and the kernel's occupancy), so make that first call
 * before any stream capture.  All calls on a device share the one scratch
 * array, and each call re-initialises everything it reads from it; calls whose
 * work overlaps on the GPU (different streams, or different host threads)
 * race on that array and give wrong results, so serialise them.  Errors are
 * reported by the return value, with a message from gd_last_error(NULL). */
int gd_force_noalloc(int64_t n, const double *m, const double *x, const double *v, double eps,
                     const int32_t *idx, int64_t nact, double *acc, double *jerk, void *stream);

/* ---- sixth-order Hermite integrator (FP64) ---------------------------------
 *
 * The same block-step scheme (Sec. 2.4: active set, prediction of all N, force
 * of the active set from predicted values, correction, power-of-two steps)
 * raised to sixth order as in the sixth-order Hermite scheme the paper cites
 * among the higher-order Hermite integrators (Nitadori & Makino 2008): the force
 * evaluation returns acceleration, jerk and snap (the first two time derivatives
 * of the softened Eq. 1, which need the predicted accelerations of all
 * particles); positions, velocities and accelerations are predicted with the
 * crackle; the corrector is the time-symmetric sixth-order formula; the step is
 *     dt = eta ( (|a||snap| + |jerk|^2) / (|crackle||a^(5)| + |pop|^2) )^(1/6)
 * with crackle, pop and a^(5) from the quintic interpolant of (a, jerk, snap) at
 * both ends of the step, quantised as in the fourth-order path.  The first steps
 * are eta_init |a| / |jerk| (quantised); the initial crackle is zero.  All
 * arithmetic is FP64.  Arrays and ownership as for gd_init; opt may be NULL
 * (dt_min, dt_max, device and stream are used, the rest ignored); errors as for
 * the other calls, gd_h6_last_error(NULL) after a failed init. */
typedef struct gd_h6 gd_h6;

int gd_h6_init(gd_h6 **out, int64_t n, const double *m, const double *x, const double *v,
               double eps, double eta, double eta_init, const gd_opts *opt);

/* The same engine with a choice of scheme.  order 6 is the scheme above;
 * order 4 is GraviDy's fourth-order scheme (Sec. 2.1: cubic predictor, force
 * and jerk, Aarseth's step from the cubic interpolant) with the time-symmetric
 * corrector of Hut, Makino & McMillan (1995), the fourth-order member of the
 * nm08 family: with h = dt / 2,
 *     v1 = v0 + h (a1 + a0) - (h^2 / 3) (j1 - j0),
 *     x1 = x0 + h (v1 + v0) - (h^2 / 3) (a1 - a0);
 * snap and crackle stay zero (gd_h6_force returns a zero snap).  n_iter in
 * [1, 16] is the number of evaluation-correction passes per block step
 * (P(EC)^n, Kokubo, Yoshinaga & Makino 1998): every pass but the last puts the
 * corrected position and velocity and the new acceleration of each active
 * particle in place of its prediction before the next evaluation.  With shared
 * constant steps and n_iter >= 2 the map is time-reversible to round-off.
 * gd_h6_init(...) is gd_h6_init_scheme(..., 6, 1, opt).  An order other than 4
 * or 6, or n_iter outside [1, 16], is GD_EINVAL. */
int gd_h6_init_scheme(gd_h6 **out, int64_t n, const double *m, const double *x, const double *v,
                      double eps, double eta, double eta_init, int32_t order, int32_t n_iter,
                      const gd_opts *opt);

/* Advance until no particle's next time is <= t_end (as gd_evolve). */
int gd_h6_evolve(gd_h6 *s, double t_end);

/* One block step; *t_out its time, *nact_out its number of active particles. */
int gd_h6_step_block(gd_h6 *s, double *t_out, int64_t *nact_out);

/* One block step with a given block time and active list (host int32,
 * ascending, distinct), as gd_replay_step. */
int gd_h6_replay_step(gd_h6 *s, int64_t tick_next, const int32_t *idx, int64_t nact);

/* Acceleration, jerk and snap (nact*3 host doubles each, order of idx) of the
 * particles idx against all n predicted to tick; state unchanged. */
int gd_h6_force(gd_h6 *s, int64_t tick, const int32_t *idx, int64_t nact, double *acc,
                double *jerk, double *snap);

/* Kinetic and softened potential energy with every particle predicted to the
 * time of the last block step. */
int gd_h6_energy(gd_h6 *s, double *K, double *U);

/* State at each particle's own time (n*3 AoS doubles; tau, dtau n int64);
 * any pointer may be NULL. */
int gd_h6_get_state(gd_h6 *s, double *x, double *v, double *a, double *jerk, double *snap,
                    double *crackle, int64_t *tau, int64_t *dtau);

/* Counters (as gd_get_stats; phase_ms zero). */
int gd_h6_get_stats(gd_h6 *s, gd_stats *st);

void gd_h6_free(gd_h6 *s);
const char *gd_h6_last_error(const gd_h6 *s);

#ifdef __cplusplus
}
#endif

#endif /* GRAVIDY_H */
