/*
 * frost.h -- C-ABI of the GB300 (sm_103a) HHS-FSI hot path.
 *
 * The library integrates a self-gravitating N-body system with the hierarchical fourth-
 * order forward symplectic integrator HHS-FSI of Rantala, Naab & Springel (2021, "FROST"):
 * direct-summation Newtonian accelerations (Eq. acc-newton), the force-gradient term of the
 * FSI (Eqs. acc-gradient-g, acc-gradient, force-gradient-inter-1/2), symmetrised free-fall /
 * fly-by time-steps (Eqs. dt-freefall, dt-flyby, their derivatives, Eq. time-step-factor),
 * the slow/fast partition (Sec. 3.1), kick/drift and the recursion of Algorithm hhs-fsi.
 *
 * Conventions shared by every entry point
 *  - Positions and velocities cross the boundary as [n][3] row-major doubles, masses as [n]
 *    doubles.  Inside, the library keeps its own FP64 structure-of-arrays copy on the GPU.
 *  - Index lists are int32 particle indices in [0, n).  A NULL list with a count k means the
 *    first k particles in order (0, 1, ..., k-1).
 *  - Pointers marked "device" must be readable/writable by the GPU (cudaMalloc, torch CUDA
 *    tensors, managed or mapped pinned memory).  Pointers marked "host or device" may be
 *    either; the library copies with cudaMemcpyDefault.  The caller owns every pointer it
 *    passes; the library never frees caller memory and keeps no caller pointer after a
 *    call returns.
 *  - Work is issued on the stream given in frost_opts (the caller's stream); entry points
 *    that return results to the host synchronise that stream before returning.
 *  - Every call returns a frost_status; no C++ exception crosses the boundary.  The message
 *    of the last failure in the calling thread is available from frost_last_error().
 *    Kernels report problems through a device error word that the library reads at its
 *    synchronisation points; the first error is sticky until frost_clear_error().
 *  - A frost_ctx is not thread-safe; use one context per host thread or serialise calls.
 */
#ifndef FROST_H
#define FROST_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct frost_ctx frost_ctx;

typedef enum {
    FROST_OK = 0,
    FROST_EINVAL = 1,      /* bad argument: size, index out of range, overlapping lists */
    FROST_ENOMEM = 2,      /* device or pinned host allocation failed */
    FROST_ECUDA = 3,       /* a CUDA runtime call failed (message has the CUDA error) */
    FROST_ENONFINITE = 4,  /* a non-finite input, or a pass produced a non-finite value */
    FROST_ECOINCIDENT = 5, /* two distinct particles at zero separation (unsoftened) */
    FROST_EDEPTH = 6,      /* hhs_fsi recursion deeper than frost_opts.max_depth */
    FROST_ETIMEOUT = 7     /* reserved for a bounded device-side wait that gives up; no entry
                              point of this version returns it: no kernel waits on a flag or
                              on another block (teams synchronise through hardware block and
                              cluster barriers only) */
} frost_status;

typedef enum {
    FROST_PREC_FP64 = 0,   /* every pair body in FP64 */
    FROST_PREC_MIXED = 1   /* FP32 pair bodies on float-float separations, FP64 state and sums */
} frost_precision;

typedef enum {
    FROST_SYM_HARMONIC = 0,   /* harmonic symmetrisation, Eq. time-step-factor (second line) */
    FROST_SYM_ARITHMETIC = 1, /* arithmetic symmetrisation, Eq. time-step-factor (first line) */
    FROST_SYM_NONE = 2,       /* no symmetrisation (factor 1) */
    /* flag or-ed into one of the above: the exact fly-by derivative, Eq. dt-flyby-derivative
     * (first line) with the relative acceleration of the pair, instead of its two-body
     * approximation (second line, the default).  The accelerations are those of the level's
     * set due to itself (a Newtonian pass before each time-step pass, softened like the
     * dynamics). */
    FROST_FLYBY_EXACT = 4
} frost_sym;

typedef struct {
    int32_t precision;  /* frost_precision */
    int32_t sym;        /* frost_sym value, optionally | FROST_FLYBY_EXACT */
    double eps_soft;    /* Plummer softening length eps_P (Sec. 2.3); 0 = unsoftened */
    int32_t max_depth;  /* deepest hhs_fsi level allowed (top level = 0); <= 0 means 40 */
    void *cuda_stream;  /* cudaStream_t for all work; NULL = the legacy default stream */
    int32_t subtree_max;/* hhs_fsi calls on sets of at most this many particles run their whole
                           subtree in one thread block (one launch, no host synchronisation);
                           0 = default (384), negative = never */
    int32_t integrator; /* frost_integrator: what frost_step advances with */
    int32_t subtree_blocks; /* thread blocks that share one subtree-solver set (a thread-block
                               cluster, 1..8); 0 = default */
    int32_t branch_streams; /* 0 (default) or 1: in every hhs_fsi call above the subtree
                               threshold, the two fsi(S) steps run on a stream of their own,
                               concurrently with the recursion hhs_fsi(F) on the context stream
                               (they act on disjoint particles, so the results are those of the
                               serial order, bit for bit); likewise, inside the single-block
                               subtree solver, a set's two fsi(S) steps run on warps 1..7 while
                               warp 0 advances its fast set of at most 32 particles;
                               -1: everything on the context stream, in the serial order.
                               With per-kernel timing on, the branches run serially.  The
                               branch streams take the device's lowest priority: give the
                               context a stream of higher priority (cudaStreamCreateWithPriority)
                               so that the recursion, the step's critical path, is scheduled
                               first (64k Plummer: 64.5 against 65.1 ms per step). */
    int32_t sym_cross;      /* 0 (default): the kick_sf passes of a hierarchy level evaluate
                               each S x F pair once for both sides where that grid fills the
                               GPU, else two one-sided passes on two streams: the Newtonian
                               kicks (see frost_accel_pairwise) and, in the mixed mode, the
                               force-gradient kick (see frost_accel_gradient_pairwise); and, in
                               the mixed mode, the time-step pass of a set of at least 8192
                               particles evaluates each pair once for both particles (the same
                               result bits: the pair criteria are symmetric and a minimum does
                               not depend on the order).  1: all always; -1: never */
} frost_opts;

typedef enum {
    FROST_HHS_FSI = 0,  /* the fourth-order hierarchical FSI, Algorithm hhs-fsi (default) */
    FROST_HOLD2 = 1     /* the second-order HOLD integrator of Eq. hhs2, the paper's point of
                           comparison: e^{eps/2 H_F} e^{eps/2 H_S} e^{eps U_FS} e^{eps/2 H_S}
                           e^{eps/2 H_F} with leapfrog for H_S and the fast set recursively;
                           host recursion only (no subtree solver, not for batch contexts) */
} frost_integrator;

/* Default options: mixed precision, harmonic symmetrisation, no softening, depth 40,
 * legacy default stream, subtree threshold 384, the HHS-FSI integrator, concurrent branches. */
void frost_default_opts(frost_opts *opt);

/*
 * Create a context holding n particles with masses m[n], positions x[n][3] and velocities
 * v[n][3] (host or device; copied), Newton's constant G and accuracy parameter eta
 * (eta = eta_ff = eta_fb, Sec. 4.3).  opt may be NULL for the defaults.  n >= 1 and
 * n < 2^31.  Non-finite inputs or non-positive masses give FROST_ENONFINITE / FROST_EINVAL.
 * The context allocates about (330 + 32 * levels_used) bytes per particle of device memory,
 * plus about 350 bytes per particle for each hierarchy level above the subtree threshold
 * whose FSI steps run on a stream of their own (frost_opts.branch_streams, allocated on
 * first use).
 * On failure *ctx is NULL.
 */
frost_status frost_init(frost_ctx **ctx, int64_t n, const double *m, const double *x,
                        const double *v, double G, double eta, const frost_opts *opt);

/*
 * Create a context holding n_clusters independent clusters (no force between clusters):
 * cluster k is the particles [offsets[k], offsets[k+1]) of m, x, v (host or device; copied;
 * offsets is a host array of n_clusters + 1 entries with offsets[0] = 0, increasing).  On
 * such a context frost_step advances every cluster by n_steps top-level HHS-FSI steps in
 * one launch (one thread block per cluster, Algorithm hhs-fsi inside the block), and
 * frost_energy_clusters reports per-cluster E, P, L; frost_energy_momentum reports the sum of
 * the per-cluster values.  The remaining calls see the particles as one set.
 */
frost_status frost_init_batch(frost_ctx **ctx, int32_t n_clusters, const int64_t *offsets,
                              const double *m, const double *x, const double *v, double G,
                              double eta, const frost_opts *opt);

/* Per-cluster kinetic and potential energy, momentum and angular momentum of a batch
 * context (host outputs: E_kin[n_clusters], E_pot[n_clusters], P[n_clusters][3],
 * L[n_clusters][3]; any may be NULL), FP64.  FROST_EINVAL on a single-set context. */
frost_status frost_energy_clusters(frost_ctx *ctx, double *E_kin, double *E_pot, double *P,
                                   double *L);

/* Replace positions x[n][3] and velocities v[n][3] (host or device; either may be NULL to
 * keep the current values) and set the simulation time to t. */
frost_status frost_set_state(frost_ctx *ctx, const double *x, const double *v, double t);

/* Copy positions and velocities out (host or device [n][3]; either may be NULL) and the
 * simulation time (host pointer, may be NULL).  Synchronises. */
frost_status frost_get_state(frost_ctx *ctx, double *x, double *v, double *t);

/*
 * Newtonian and gradient accelerations of the active particles against the source
 * particles (Eq. acc-newton; Eqs. acc-gradient-g, acc-gradient; Eqs. force-newton-inter,
 * force-gradient-inter-1/2):
 *   acc[k]       = a_i       = G sum_{j in source, j != i} m_j x_ji / r_ji^3
 *   grad[k]      = g_i       = 2 G sum_j m_j r_ji^-5 (r_ji^2 a_ji - 3 (x_ji . a_ji) x_ji)
 *   acc_tilde[k] = a~_i      = a_i + eps_grad^2 g_i / 48
 * for i = active[k].  Two cases are accepted:
 *   - active and source are the same set (any order): the intra-set pass of fsi; the a_j in
 *     a_ji = a_j - a_i are the same set's accelerations;
 *   - active and source are disjoint: the inter-level pass of hhs_fsi; the a_j are the
 *     sources' accelerations due to the active set (Eq. force-newton-inter, second line).
 * Partial overlap or a repeated index returns FROST_EINVAL.  active/source are device
 * int32 lists (or NULL = identity); acc, acc_tilde, grad are device [n_active][3] doubles,
 * each may be NULL (if acc_tilde and grad are both NULL only the Newtonian pass runs).
 * With softening eps_P, r^2 -> r^2 + eps_P^2 everywhere in both sums.  Pairs at zero
 * separation give FROST_ECOINCIDENT when unsoftened.  Synchronises.
 * Accuracy: FP64 mode, 1e-12 relative.  Mixed mode: the Newtonian pass runs a prepass for
 * max_j m_j / r^3 and sums the terms above 1/16 of it (up to 8 per particle) in
 * double-float, and so does the gradient pass; the rest are FP32 terms in compensated sums.
 * That gives a_i to about 1e-7 and g_i to below 1e-6 at the 99.9th percentile of a set of a
 * few thousand particles or more.  The relative error of one g_i grows as
 * sum_j |term_ij| / |g_i| where the gradient nearly vanishes.
 */
frost_status frost_accel_gradient(frost_ctx *ctx, const int32_t *active, int64_t n_active,
                                  const int32_t *source, int64_t n_source, double eps_grad,
                                  double *acc, double *acc_tilde, double *grad);

/*
 * Newtonian accelerations of two disjoint sets due to each other, both lines of Eq.
 * force-newton-inter, with every pair evaluated once (Sec. 3.3: the inter-level kick is
 * pairwise):
 *   acc_a[k] = G sum_{j in b} m_j x_ji / r_ji^3   for i = a[k]
 *   acc_b[k] = G sum_{i in a} m_i x_ij / r_ij^3   for j = b[k]
 * Each pair's separation, r^2 and r^-3 are formed once and weighted by m_j for the a-side and
 * by -m_i for the b-side; the a-side (the longer list) is summed per thread, the b-side by a
 * fixed-order reduction over the threads, so results are deterministic.  a, b: device int32
 * lists (or NULL = identity) of n_a and n_b indices with no index in both (else
 * FROST_EINVAL); acc_a, acc_b: device [n][3] doubles (either may be NULL).  Softened like
 * frost_accel_gradient.  Accuracy: as the Newtonian pass of frost_accel_gradient (FP64:
 * 1e-12 relative; mixed: ~1e-7 at the 99.9th percentile).  Synchronises.
 */
frost_status frost_accel_pairwise(frost_ctx *ctx, const int32_t *a, int64_t n_a, const int32_t *b,
                                  int64_t n_b, double *acc_a, double *acc_b);

/*
 * The force-gradient kick between two disjoint sets, both lines of Eqs.
 * force-gradient-inter-1/2 (the 2 tau/3 kick_sf of Algorithm hhs-fsi): the Newtonian
 * accelerations of each set due to the other (Eq. force-newton-inter), then the gradient of
 * each set against the other with those accelerations,
 *   g_i = 2G sum_{j in b} m_j r^-5 (r^2 a_ji - 3 (x_ji . a_ji) x_ji),  a_ji = a_j - a_i,
 * and a~ = a + eps_grad^2 / 48 g, for i in a (a_i due to b, a_j due to a) and likewise for b.
 * Mixed mode: every pair is evaluated once for both sets, in both passes (a pair's term for
 * b is the term for a with the other mass and the opposite sign, Sec. 3.3); each side keeps
 * its dominant terms (above 1/16 of its max m / r^3) out of the FP32 sums and evaluates them
 * in double-float, as frost_accel_gradient does, with no limit on their number for the set
 * summed by the reduction; sums are in a fixed order, so results are deterministic.  With
 * frost_opts.sym_cross = -1, and in FP64 mode, two one-sided passes per kind.  a, b: device
 * int32 lists (or NULL = identity) of n_a and n_b indices with no index in both (else
 * FROST_EINVAL); outputs: device [n][3] doubles, each may be NULL.  Softened like
 * frost_accel_gradient.  Accuracy: as frost_accel_gradient.  Synchronises.
 */
frost_status frost_accel_gradient_pairwise(frost_ctx *ctx, const int32_t *a, int64_t n_a, const int32_t *b,
                                           int64_t n_b, double eps_grad, double *acc_a, double *acc_b,
                                           double *acc_tilde_a, double *acc_tilde_b, double *grad_a,
                                           double *grad_b);

/*
 * Symmetrised time-steps of the members of `set` (device list or NULL), Sec. 4:
 *   tau[k] = min_{j in set, j != i} min( s(eta dt_ff/dt) eta t_ff, s(eta dt_fb/dt) eta t_fb )
 * with t_ff = (r^3 / (G (m_i + m_j)))^(1/2), t_fb = r / |v_ij|, their time derivatives
 * (fly-by in the two-body approximation of Eq. dt-flyby-derivative) and the symmetrisation
 * factor s of Eq. time-step-factor chosen by frost_opts.sym.  tau is device [n_set] doubles;
 * a set of one particle gets +inf; v_ij = 0 drops the fly-by criterion of that pair.
 * Two distinct members at the same position give FROST_ECOINCIDENT.  Synchronises.
 */
frost_status frost_timesteps(frost_ctx *ctx, const int32_t *set, int64_t n_set, double *tau);

/*
 * Slow/fast partition by the pivot step (Sec. 3.1): S = {set[k] : tau[k] >= tau_pivot},
 * F = the rest, both in the order of `set`.  set, tau (device) have n_set entries; S and F
 * are device int32 buffers of capacity n_set; *n_slow and *n_fast (host) receive the
 * sizes.  Synchronises.
 */
frost_status frost_partition(frost_ctx *ctx, const int32_t *set, int64_t n_set,
                             const double *tau, double tau_pivot, int32_t *S, int32_t *F,
                             int64_t *n_slow, int64_t *n_fast);

/* Kick v_i += dt a[k] for i = set[k] (a device [n_set][3]) and drift x_i += dt v_i for the
 * members of set (Sec. 5.3).  Asynchronous on the context stream. */
frost_status frost_kick(frost_ctx *ctx, const int32_t *set, int64_t n_set, const double *a,
                        double dt);
frost_status frost_drift(frost_ctx *ctx, const int32_t *set, int64_t n_set, double dt);

/*
 * One FSI step (Algorithm fsi, Eq. fsi) of the particles in `set` (device list or NULL)
 * with step dt, ignoring every particle outside the set.  Asynchronous; errors are reported
 * by the next synchronising call.
 */
frost_status frost_fsi(frost_ctx *ctx, const int32_t *set, int64_t n_set, double dt);

/*
 * n_steps top-level HHS-FSI steps (Algorithm hhs-fsi called with all particles and
 * tau_pivot = dt_pivot, as in the main loop of Algorithm frost); the simulation time
 * advances by n_steps * dt_pivot.  Returns FROST_EDEPTH if the hierarchy would go deeper
 * than max_depth (the state is then partially advanced).  Synchronises.
 */
frost_status frost_step(frost_ctx *ctx, double dt_pivot, int64_t n_steps);

/*
 * Kinetic energy T = 1/2 sum m v^2, potential U = -G sum_{i<j} m_i m_j / r_ij (softened as
 * configured), momentum P = sum m v and angular momentum L = sum m x cross v (host
 * outputs; any may be NULL).  Computed in FP64 in every precision mode.  Synchronises.
 */
frost_status frost_energy_momentum(frost_ctx *ctx, double *E_kin, double *E_pot, double P[3],
                                   double L[3]);

/* Counters since frost_init or frost_reset_stats. */
#define FROST_STATS_LEVELS 48
typedef struct {
    int64_t acc_pairs;      /* Newtonian pair interactions evaluated */
    int64_t grad_pairs;     /* gradient pair interactions evaluated */
    int64_t tstep_pairs;    /* time-step pair interactions evaluated */
    int64_t kernel_launches;/* kernels launched by the library */
    int64_t hhs_calls;      /* hhs_fsi invocations with a non-empty set */
    int64_t fsi_calls;      /* fsi invocations with a non-empty set */
    int32_t max_depth_seen; /* deepest hhs_fsi level reached */
    int32_t timing_enabled; /* 1 if per-kernel CUDA-event timing is on */
    /* per-kernel-kind CUDA-event totals (only when timing is enabled):
     * index 0 = Newtonian pass, 1 = gradient pass, 2 = time-step pass, 3 = single-block
     * subtree launches (all passes of a small set; their pairs are in the totals above) */
    int64_t timed_launches[4];
    double timed_ms[4];
    int64_t timed_pairs[4];
    int64_t subtree_launches;  /* hhs_fsi calls handed to the single-block subtree solver */
    /* per hierarchy depth d (top level 0; the last entry collects d >= FROST_STATS_LEVELS-1):
     * hhs_fsi calls with a non-empty set, and the summed sizes of those sets */
    int64_t level_calls[FROST_STATS_LEVELS];
    int64_t level_particles[FROST_STATS_LEVELS];
    /* Newtonian pair interactions of the second fsi(S) of each hhs_fsi call that were not
     * recomputed: S has not moved since the end of the first fsi(S), whose final a^SS is
     * reused bit for bit (acc_pairs counts evaluated pairs only) */
    int64_t acc_pairs_reused;
    /* the pair interactions evaluated inside single-block subtree-solver launches (Newtonian,
     * gradient, time-step; also part of acc_pairs, grad_pairs and tstep_pairs) */
    int64_t subtree_pairs[3];
    /* Newtonian pairs evaluated once for both sides (symmetric S x F passes; counted once in
     * acc_pairs, and each served two interactions) */
    int64_t acc_pairs_symmetric;
    /* gradient pairs evaluated once for both sides (symmetric gradient kick_sf; counted once
     * in grad_pairs, and each served two interactions) */
    int64_t grad_pairs_symmetric;
    /* fsi(S) steps of the single-block subtree solver that ran on warps 1..7 while warp 0
     * advanced the fast set F (at most 32 particles) of the same hhs_fsi call: the two
     * operators act on disjoint particles and commute (Algorithm hhs-fsi); off with
     * frost_opts.branch_streams = -1 (the serial order, the same result bits) */
    int64_t subtree_fsi_beside;
} frost_stats;

frost_status frost_get_stats(frost_ctx *ctx, frost_stats *out);
frost_status frost_reset_stats(frost_ctx *ctx);

/* Enable (1) or disable (0) CUDA-event timing of every pair-pass kernel launch on the
 * context stream (a pair of events per launch; totals in frost_stats). */
frost_status frost_set_timing(frost_ctx *ctx, int32_t enable);

/* Autotuner of the pair kernels' launch shapes (the paper has no counterpart; its kernels use
 * one fixed layout).  For every power-of-two set size 2^k, 512 <= 2^k <= N, and each pass
 * kind (0 = Newtonian, 1 = gradient, 2 = time-step), it times an intra-set pass and its
 * finalisation over the context's particles 0 .. 2^k-1 with the j-split chosen for at most
 * 1, 2, 4, 8 or 16 full waves of blocks, and keeps the fastest.  In the mixed mode each bound
 * is timed with two kernel layouts: 128 threads and 128-source tiles, and one warp and
 * 32-source tiles (the small-tile layout, which spreads a pass of a few hundred particles
 * over all SMs).  Later passes with an active list of [2^k, 2^(k+1)) particles use that
 * choice; untuned sizes take 8 waves, and the small-tile layout where the other cannot fill
 * one wave.  Synchronous.  Results are unchanged to rounding: only the split of the sources
 * (the summation order of the partials) differs.
 * In the mixed mode, the Newtonian pass that feeds a gradient (its wmax prepass and
 * deferred double-float terms) is tuned as a fourth kind (3).
 * waves_out: NULL, or int32[4][32] receiving the chosen bound per kind and k (0 = untuned;
 * negative = the small-tile layout with that many waves).
 * On a batch context (frost_init_batch) it tunes the team split instead: every cluster of at
 * least min_n particles runs on a thread-block cluster of `blocks` blocks, the others on one
 * block each.  It times one batch step (the pivot of the last frost_step call, else 2^-7)
 * for min_n in {256, 384, 512, 768, 1024, 1536, 2048} x blocks in {2, 4, 8} and for one block
 * per cluster, from the same saved state, keeps the fastest (by 2%) and restores the state
 * and time; waves_out[0] = min_n (INT32_MAX: no teams) and waves_out[1] = blocks, the rest 0.
 * The default split (before tuning) is min_n = 768, 8 blocks. */
frost_status frost_autotune(frost_ctx *ctx, int32_t *waves_out);

/* Wait for all work of the context and report the sticky device error, if any. */
frost_status frost_synchronize(frost_ctx *ctx);
frost_status frost_clear_error(frost_ctx *ctx);

/* Release the context and all its device memory (NULL is ignored). */
void frost_destroy(frost_ctx *ctx);

/* Message of the last failure in the calling thread ("" if none). */
const char *frost_last_error(void);

/* Library version string.  0.2: frost_autotune writes int32[4][32] (was [3][32]).
 * 0.3: frost_peak_probe. */
const char *frost_version(void);

/*
 * Throughput probe of the arithmetic pipes that bound the pair passes (the paper has no
 * counterpart; it is the denominator of their roofline).  On the current device it times,
 * with CUDA events on cuda_stream (NULL = legacy default stream), kernels that fill every SM
 * at full occupancy with independent chains of one operation, and writes to out (host, 6
 * doubles): [0] scalar FP32 FMA TFLOP/s, [1] packed FP32x2 FMA TFLOP/s (two lanes per
 * instruction), [2] FP64 FMA TFLOP/s, [3] MUFU reciprocal square roots per second, [4] the
 * SM count, [5] the resident threads per SM of the probe.  An FMA counts as 2 flops.  It
 * allocates and frees a 2 KB device buffer and synchronises cuda_stream; about 50 ms.
 */
frost_status frost_peak_probe(double *out, void *cuda_stream);

/*
 * Entry point that allocates nothing (the paper has no counterpart; it serves callers that
 * may not allocate device memory, e.g. inside an application or allocator that owns all
 * device memory, or in time-critical code where an allocation is not allowed).
 *
 * Computes the mixed-precision Newtonian accelerations of all n particles against all n
 * particles, a_i = G sum_{j != i} m_j x_ji / (r_ji^2 + eps_soft^2)^(3/2), with the same
 * kernels as frost_accel_gradient in FROST_PREC_MIXED mode (same tolerance), but without a
 * context: m[n], x[n][3] (inputs) and acc[n][3] (output) are caller-owned device pointers,
 * and all scratch lives in one static device array of FROST_NOALLOC_MAX_N particles
 * (8 MiB), which every GPU that loads the library holds until the process exits.
 *  - n outside [1, FROST_NOALLOC_MAX_N] returns FROST_EINVAL; nothing is launched.
 *  - No cudaMalloc, cudaFree or other allocating call is made.
 *  - The first call on each device looks up the scratch array's device address on that
 *    device (the device current at the call) and keeps it for the life of the process; make
 *    that first call before any stream capture.  A cudaDeviceReset of the device invalidates
 *    the kept address: do not call this entry point on that device afterwards.
 *  - Every call shares the scratch array, which keeps the previous call's contents (the only
 *    part that must start at zero, the status word, is cleared by every call); calls whose
 *    GPU work may overlap (other streams or host threads without ordering) race and must be
 *    serialised by the caller.
 *  - Work runs on cuda_stream (NULL = legacy default stream); the call synchronises that
 *    stream before returning, to read the status word of its kernels.  Non-finite inputs or
 *    non-positive masses give FROST_ENONFINITE, two particles at zero separation
 *    (eps_soft = 0) FROST_ECOINCIDENT.  Every failure sets the message of
 *    frost_last_error() (without allocating).
 */
#define FROST_NOALLOC_MAX_N 65536
frost_status frost_accel_noalloc(int64_t n, const double *m, const double *x, double G,
                                 double eps_soft, double *acc, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* FROST_H */
