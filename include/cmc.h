/*
 * cmc.h - C ABI of the GB300 library for the per-timestep hot path of the
 * Henon Monte Carlo method for collisional star clusters (Pattabiraman et
 * al., "A Parallel Monte Carlo Code for Simulating Collisional N-body
 * Systems", section 2.1 and section 3.3).
 *
 * One timestep (cmc_step) advances every bound star of every cluster:
 *   1. relaxation timestep: Eq. 7 averaged on bins of bin_size consecutive
 *      stars (section 3.3), dt = minimum over bins;
 *   2. two-body relaxation of radial neighbours (2j, 2j+1) (section 2.1
 *      step 3(i));
 *   3. new orbits: turning points by bisection on Q of Eq. 12 and a new
 *      radius by the rejection of Eqs. 13-15 (section 2.1 step 5);
 *      stars with E >= 0 escape;
 *   4. sort by radius (section 2.1 step 6), ties by id, escaped stars last;
 *   5. shell potential of Eqs. 1-5 and the energy correction for the orbit
 *      having been drawn in the old potential (section 2.1 step 6).
 * Random numbers come from a counter-based generator (Philox4x32-10) keyed
 * by the cluster seed and indexed by (star id, step, stream tag, trial), so
 * results do not depend on thread layout, batching or resumption.
 *
 * Units: G = 1 (Henon N-body units).  State arrays are structure-of-arrays:
 * r (radius), vr (radial velocity), vt (transverse speed, >= 0), m (mass)
 * as double, id as uint32.  An ensemble of clusters is stored back to back;
 * cluster c owns n_per_cluster[c] consecutive entries.  After every call
 * the stars of each cluster are sorted by (r, id) with escaped stars
 * (r = +inf) at the end ordered by id.
 *
 * Conventions for every function:
 *   - Status codes only; nothing aborts or throws across the ABI.
 *   - ptr_kind 0: the array arguments are host pointers; 1: device
 *     pointers (for example from torch tensors) on the library's device.
 *   - Work is ordered on the context's CUDA stream (the caller's stream,
 *     or the legacy default stream when NULL).  Calls that return host
 *     data or a status that depends on device results synchronise it.
 *   - The library owns all memory it allocates; caller arrays are copied
 *     and never retained.  A context is used by one host thread at a time.
 *   - A device-side error (bounded wait expired, invalid state) poisons the
 *     context: later calls return CMC_EPOISONED.  cmc_last_error() gives
 *     text for the last failure.
 */
#ifndef CMC_H
#define CMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cmc_ctx cmc_ctx;

typedef enum {
    CMC_OK = 0,
    CMC_EINVAL = 1,     /* bad argument or invalid input state */
    CMC_ENOMEM = 2,     /* device or host allocation failed */
    CMC_ECUDA = 3,      /* a CUDA runtime call failed */
    CMC_ENOCONV = 4,    /* reserved: a bounded iteration did not converge */
    CMC_ETIMEOUT = 5,   /* a bounded device wait gave up (context poisoned) */
    CMC_EPOISONED = 6   /* an earlier device error poisoned the context */
} cmc_status;

/* Per-cluster counters returned by cmc_get_stats (cumulative). */
enum {
    CMC_STAT_ESCAPED = 0,     /* stars that reached E >= 0 and left */
    CMC_STAT_DEGENERATE = 1,  /* orbits with rmax <= rmin or F = 0, kept in place */
    CMC_STAT_CAP_HITS = 2,    /* rejection ran out of trials, star kept in place */
    CMC_STAT_TRIALS = 3,      /* rejection trials drawn */
    CMC_STAT_VIOLATIONS = 4,  /* trials with g(s) > F (bound exceeded) */
    CMC_STAT_CLAMPS = 5,      /* energy corrections with T' < 0 set to 0 */
    CMC_STAT_ANGLE_FAILS = 6, /* 64 failed unit-disk draws (never expected) */
    CMC_STAT_TIES = 7,        /* runs of equal radii ordered by id */
    CMC_STAT_FP64_TRIALS = 8, /* mixed mode: trials whose FP32 accept test could
                                 not be decided within its error bound, taken
                                 in FP64 (0 in FP64 mode) */
    CMC_STAT_CLAMP_ENERGY = 9,  /* energy the clamps of T' < 0 to 0 added to the
                                   cluster (section 2.1 step 6's correction):
                                   the sum of m_k |T'_k| over clamped stars, as
                                   an integer in units of 2^-62 */
    CMC_STAT_COLLISIONS = 10,   /* sticky-sphere mergers (cfg.collisions); the
                                   merged-away partners left the cluster but
                                   are not counted as escapers */
    CMC_STAT_COLLISION_ENERGY = 11, /* what the mergers changed of K + W (the
                                   relative kinetic energy dissipated and the
                                   shell-model W of the moved mass), as a signed
                                   integer in units of 2^-62: K + W + E_esc
                                   minus this is what the method conserves */
    CMC_STAT_ENVELOPE_FP64 = 12,    /* FP64 mode (precision 0): envelope samples
                                   evaluated in FP64 because their FP32 bounds
                                   could not rule them out of the maximum */
    CMC_NSTATS = 13
};

typedef struct {
    int32_t precision;          /* 0: FP64: every result the FP64 method's
                                   (searches, bounds and accept tests
                                   screened in FP32 with error bounds, each
                                   decision they cannot certify taken in
                                   FP64); 1: mixed (as 0, but the envelope F
                                   from FP32 samples: an equally valid
                                   bound, a different accept sequence);
                                   2: FP64 by bisection on the FP64 table
                                   (Appendix A's kernels; the same results
                                   as 0, slower) */
    int32_t bin_size;           /* stars per timestep bin, even, >= 2 (20) */
    double theta_max;           /* maximum deflection angle of Eq. 7 (pi/2) */
    double gamma;               /* Coulomb logarithm ln(gamma N) (0.1, Eq. 20) */
    int32_t max_trials;         /* rejection trials per star per step (1000) */
    int32_t energy_correction;  /* 1: apply the section 2.1 step 6 correction */
    int32_t orbit_block;        /* threads per block of the orbit kernel: 0 (auto) or a multiple of 32 up to 256 */
    int32_t autotune;           /* 1: at cmc_init, time the sort shapes (and the
                                   orbit block size when orbit_block is 0) on
                                   the real state and keep the fastest; results
                                   do not depend on the choice (default 1) */
    int32_t orbit_variant;      /* FP32 sampler kernel variant, precision 0 and 1 (listed at
                                   cmc_get_tuning): -1 = the autotuner's choice
                                   (0 without autotune), or 0..6 (default -1) */
    int32_t rng;                /* 0: counter-based Philox4x32-10 draws keyed by
                                   (star id, step, purpose, trial) (default);
                                   1: the paper's combined Tausworthe generator
                                   (section 3.6; L'Ecuyer 1999), one stream per
                                   star id, the streams 2^80 apart in one
                                   sequence seeded from the cluster seed, each
                                   star's draws taken in a fixed order
                                   (relaxation, orbit trials, v_r sign); ids must
                                   then be below 4 N_c + 64 in every cluster
                                   (stream slots are indexed by id); the mixed
                                   sampler runs one launch shape */
    int32_t relax_variant;      /* relaxation kernel variant (listed at
                                   cmc_get_tuning): -1 = the autotuner's choice
                                   (0 without autotune), or 0..2 (default -1) */
    int32_t collisions;         /* 1: stars carry radii (cmc_set_radii): the
                                   collision timestep of Eq. 8 joins Eq. 7's, and
                                   relaxation pairs may merge as sticky spheres
                                   (section 2.1 step 3(iii)); default 0 */
    int32_t diag_ring;          /* records per cluster of the per-step
                                   diagnostics ring (cmc_get_diagnostics), 0 =
                                   off (default); on, every step also computes
                                   K and W (four more kernels per step) */
    int32_t binaries;           /* 1: stars carry semi-major axes
                                   (cmc_set_binaries; 0 for a single star, a
                                   binary's mass its total): the binary-binary
                                   and binary-single timesteps of Eqs. 9 and 10
                                   join Eq. 7's; default 0 */
    double x_bb;                /* strong-interaction parameter X_bb of Eq. 9 (1) */
    double x_bs;                /* strong-interaction parameter X_bs of Eq. 10 (1) */
    int32_t sort_packed;        /* 1: when every cluster has at most 2^24 stars, the
                                   timestep's sort moves 8-byte keys that carry
                                   each star's index in their low 24 bits (bits
                                   the radix passes leave to the tie fix) instead
                                   of keys and 4-byte values (default 1); 0: keys
                                   and values.  Results do not depend on it. */
} cmc_config;

/* Fill cfg with the defaults shown above. */
void cmc_config_default(cmc_config *cfg);

/*
 * Create a context holding n_clusters clusters.
 *   n_per_cluster (host, n_clusters): stars per cluster, each >= 1.
 *   seeds (host, n_clusters): generator key of each cluster.
 *   r, vr, vt, m (ptr_kind, sum n doubles), id (ptr_kind, sum n uint32):
 *     the stars, concatenated cluster by cluster, in any order.  Requires
 *     r > 0 finite, vt >= 0, m >= 0, all finite, ids unique per cluster.
 *   stream: cudaStream_t to order work on (NULL: legacy default stream).
 * The stars are sorted by (r, id) and their potential computed.  The
 * Coulomb logarithm of cluster c is ln(gamma * n_per_cluster[c]).
 * Errors: CMC_EINVAL (arguments or state), CMC_ENOMEM, CMC_ECUDA.
 * On error *out is NULL.
 */
cmc_status cmc_init(cmc_ctx **out, const cmc_config *cfg, int32_t n_clusters,
                    const int64_t *n_per_cluster, const uint64_t *seeds,
                    const double *r, const double *vr, const double *vt,
                    const double *m, const uint32_t *id, int32_t ptr_kind,
                    void *stream);

/* Advance every cluster by n_steps timesteps (n_steps >= 0).  The step
 * sequence is captured once in a CUDA graph and replayed.  Synchronises
 * the stream at the end to check device error flags. */
cmc_status cmc_step(cmc_ctx *ctx, int32_t n_steps);

/* Total energies per cluster of the bound stars (section 2.1 step 6):
 * out (host, n_clusters x 3) = {K, W, E} with K = 1/2 sum m v^2,
 * W = -G sum_{i<j} m_i m_j / max(r_i, r_j), E = K + W. */
cmc_status cmc_energy(cmc_ctx *ctx, double *out);

/* Lagrangian radii: for each cluster and each fraction f in fracs (host,
 * nf values in [0, 1]) the radius r_k of the first bound star whose
 * enclosed mass M_k = sum_{i<=k} m_i reaches f times the bound mass.
 * out: host, n_clusters x nf. */
cmc_status cmc_lagrange_radii(cmc_ctx *ctx, const double *fracs, int32_t nf, double *out);

/* The stream states of the Tausworthe mode (rng = 1): slots of four
 * 32-bit words, cluster by cluster, slot = the cluster's first slot + id.
 * cmc_get_rng_state writes them to out (host, may be NULL) and their
 * number of words to *n_words; cmc_set_rng_state reads n_words words (the
 * same count) from in (host).  With cmc_get_state / cmc_set_state they make
 * a checkpoint from which the run continues bit for bit.  CMC_EINVAL in
 * the counter mode or for a wrong count. */
cmc_status cmc_get_rng_state(cmc_ctx *ctx, uint32_t *out, int64_t *n_words);
cmc_status cmc_set_rng_state(cmc_ctx *ctx, const uint32_t *in, int64_t n_words);

/* Core diagnostics (section 4.2, Eq. 19) per cluster of the bound stars:
 * out (host, n_clusters x 3) = {rho_c, r_c, n_est}.  The density around
 * sorted bound star k (3 <= k < N_bound - 3) is the 6th-order estimator of
 * Casertano & Hut taken in the radial order, rho_k = (m_{k-2} + ... +
 * m_{k+2}) / (4 pi / 3 (r_{k+3}^3 - r_{k-3}^3)) (shells of no volume are
 * skipped); rho_c = sum rho_k^2 / sum rho_k (Eq. 19), r_c = sum rho_k r_k /
 * sum rho_k (the density-weighted core radius), n_est = the number of
 * estimates (0 when N_bound < 7, rho_c = r_c = 0 then).  Units G = M = 1
 * (rho_c in M r_vir^-3 for Henon units, r_vir = 1).  Synchronous. */
cmc_status cmc_core(cmc_ctx *ctx, double *out);

/* Copy the state out (sorted as described above).  Any array may be NULL.
 * phi receives the potential at each star (0 for escaped stars); step the
 * number of steps taken so far (host pointer, may be NULL). */
cmc_status cmc_get_state(cmc_ctx *ctx, double *r, double *vr, double *vt, double *m,
                         uint32_t *id, double *phi, int64_t *step, int32_t ptr_kind);

/* Replace the state of every cluster (same sizes as at cmc_init) and set
 * the step counter; the stars are re-sorted and the potential recomputed.
 * Escaped stars may be passed with r = +inf.  A state obtained from
 * cmc_get_state resumes bit for bit. */
cmc_status cmc_set_state(cmc_ctx *ctx, const double *r, const double *vr, const double *vt,
                         const double *m, const uint32_t *id, int64_t step,
                         int32_t ptr_kind);

/* Bound stars per cluster: out (host, n_clusters). */
cmc_status cmc_get_nbound(cmc_ctx *ctx, int64_t *out);

/* Last timestep per cluster: out (host, n_clusters). */
cmc_status cmc_get_dt(cmc_ctx *ctx, double *out);

/* Cumulative counters: out (host, n_clusters x CMC_NSTATS). */
cmc_status cmc_get_stats(cmc_ctx *ctx, int64_t *out);

/* What the escapers have carried off since cmc_init (the energy budget of
 * section 4.2: K + W of the bound stars plus E_esc is what the method
 * conserves).  out (host, n_clusters x 2): M_esc, E_esc.  A star k leaving
 * in a step adds m_k and m_k e_k, e_k = Phi_k + m_k / r_k + v_k^2 / 2 (its
 * energy in the field of the others, from the state before its orbit
 * step), summed in a fixed order, so the figures are reproducible.
 * cmc_set_state leaves them as they are; cmc_set_escaped (in: host,
 * n_clusters x 2, finite) restores them when a run is resumed. */
cmc_status cmc_get_escaped(cmc_ctx *ctx, double *out);
cmc_status cmc_set_escaped(cmc_ctx *ctx, const double *in);

/* Per-step diagnostics ring (cmc_config.diag_ring = capacity R > 0): at the
 * end of every step each cluster appends one record of CMC_DIAG_FIELDS
 * doubles, written on the device inside the step (no host round trip):
 * the step count after the step, its timestep, N_bound, K and W of the
 * bound stars (as cmc_energy), K + W + E_esc, M_esc, E_esc, the cumulative
 * rejection trials and the context's device error bits.  out (host,
 * n_clusters x R x CMC_DIAG_FIELDS, may be NULL) receives the last
 * min(R, steps) records of each cluster, oldest first, and *n_records
 * their count.  CMC_EINVAL when the ring is off. */
enum {
    CMC_DIAG_STEP = 0, CMC_DIAG_DT = 1, CMC_DIAG_NBOUND = 2, CMC_DIAG_K = 3, CMC_DIAG_W = 4,
    CMC_DIAG_ETOTAL = 5, CMC_DIAG_MESC = 6, CMC_DIAG_EESC = 7, CMC_DIAG_TRIALS = 8,
    CMC_DIAG_ERR = 9, CMC_DIAG_FIELDS = 10
};
cmc_status cmc_get_diagnostics(cmc_ctx *ctx, double *out, int32_t *n_records);

/* Debug builds (libcmc_debug.so, compiled with -DCMC_DEBUG): every table
 * probe and scatter index that a wrong bracket, bucket or segment offset
 * could send out of range is checked on the device; a failed check skips
 * the access and records its site.  cmc_debug_check writes to *site (host)
 * the first failed site since the last call (translation unit x 100000 +
 * source line; 0: none) and clears the records; in a release build it
 * always writes 0.  cmc_is_debug_build returns 1 in a debug build. */
cmc_status cmc_debug_check(uint32_t *site);
int32_t cmc_is_debug_build(void);

/* Stages of one timestep, as timed by cmc_step_profiled. */
enum {
    CMC_STAGE_TIMESTEP = 0,    /* Eq. 7 bins and the minimum over bins */
    CMC_STAGE_RELAX = 1,       /* two-body relaxation of neighbour pairs */
    CMC_STAGE_TURNING = 2,     /* turning points (mixed mode; FP64 mode: in ORBIT) */
    CMC_STAGE_ORBIT = 3,       /* rejection sampling (FP64 mode: and turning points) */
    CMC_STAGE_SORT = 4,        /* radix passes and the id order of ties */
    CMC_STAGE_GATHER = 5,      /* payload into the sorted arrays */
    CMC_STAGE_POTENTIAL = 6,   /* shell potential (Eqs. 1-5) and mixed-mode tables */
    CMC_STAGE_CORRECTION = 7,  /* energy correction */
    CMC_STAGE_END = 8,         /* bookkeeping of the step */
    CMC_NSTAGES = 9
};

/* Advance by n_steps timesteps like cmc_step, but launch the kernels one
 * by one (no graph) with a CUDA event after each stage; stage_ms (host,
 * CMC_NSTAGES) receives the summed device time of each stage.  Results are
 * identical to cmc_step. */
cmc_status cmc_step_profiled(cmc_ctx *ctx, int32_t n_steps, double *stage_ms);

/* Kernel shapes in use (chosen by autotune or the configuration): out
 * (host, 5) = {orbit threads per block, sort keys per thread, sort
 * multisplit (0: match, 1: ballot), mixed-mode orbit variant (registers per
 * thread capped for 1 (no cap), 2, 3, 4, 5, 6 or 8 resident 256-thread
 * blocks per SM: variants 0..6), relaxation variant (registers per thread
 * capped for 1 (no cap), 6 or 8 resident 128-thread blocks per SM:
 * variants 0..2)}.  All shapes give bit-identical results. */
cmc_status cmc_get_tuning(const cmc_ctx *ctx, int32_t *out);

/* Number of kernels one cmc_step timestep launches. */
int32_t cmc_kernels_per_step(const cmc_ctx *ctx);

/* Order later work on another stream (cudaStream_t, NULL: default). */
cmc_status cmc_set_stream(cmc_ctx *ctx, void *stream);

/* Text of the last failure of this context ("" if none); ctx may be NULL
 * for failures of cmc_init or of the stage functions below. */
const char *cmc_last_error(const cmc_ctx *ctx);

/* Release the context and its device memory (NULL is allowed). */
void cmc_destroy(cmc_ctx *ctx);

/* ---------------------------------------------------------------------
 * Stage functions: one step of the hot path on caller-owned DEVICE
 * arrays of a single cluster of n stars, ordered on `stream`.  They
 * allocate their scratch with cudaMallocAsync on that stream and return
 * once the work is enqueued (except where stated).  Arrays are device
 * pointers; sorted inputs are sorted by (r, id).
 * ------------------------------------------------------------------- */

/* Counter-based RNG (section 3.6's per-star streams): out[4i..4i+3] =
 * Philox4x32-10 of counter ctr[4i..4i+3] under key seed. */
cmc_status cmc_rng_philox(int64_t n, const uint32_t *ctr, uint64_t seed, uint32_t *out,
                          void *stream);

/* Sort by radius (section 2.1 step 6): perm[j] = input index of the star
 * that goes to slot j, order (r, id) with r = +inf last by id.  This is the
 * timestep's sort: a stable radix sort by r followed by ordering equal
 * radii by id. */
cmc_status cmc_sort_radius(int64_t n, const double *r, const uint32_t *id, uint32_t *perm,
                           void *stream);

/* Shell potential, Eqs. 1-5 (scan form), of n sorted stars (all bound).
 * phi: n doubles out.  M (may be NULL): enclosed mass M_k out. */
cmc_status cmc_potential(int64_t n, const double *r, const double *m, double *phi, double *M,
                         void *stream);

/* Relaxation timestep, Eq. 7 on bins (section 3.3), of n sorted stars:
 * nbin (ceil(n/bin_size) doubles out) bin densities, dt (1 double out,
 * device) the minimum over bins.  pref = (theta_max/(pi/2)) (pi/32). */
cmc_status cmc_timestep(int64_t n, const double *r, const double *vr, const double *vt,
                        const double *m, int32_t bin_size, double theta_max, double lnL,
                        double *nbin, double *dt, void *stream);

/* Two-body relaxation (section 2.1 step 3) of pairs (2j, 2j+1) of n
 * sorted stars, in place on vr, vt; nbin from cmc_timestep; dt, lnL on
 * the host. */
cmc_status cmc_relax(int64_t n, double *vr, double *vt, const double *m, const uint32_t *id,
                     const double *nbin, int32_t bin_size, double dt, double lnL,
                     uint64_t seed, uint32_t step, void *stream);

/* New orbits (section 2.1 step 5) of n sorted stars with potential phi:
 * per star r_new, vr_new, vt_new, phi_new (= Phi_old(r_new)), rmin, rmax,
 * F and code (0 moved, 1 escaped, 2 degenerate, 3 trial cap); escaped
 * stars get r_new = +inf.  Any output except r_new may be NULL.
 * precision: 0 FP64, 1 mixed, 2 FP64 by bisection (as cmc_config). */
cmc_status cmc_orbit(int64_t n, const double *r, const double *phi, const double *vr,
                     const double *vt, const uint32_t *id, uint64_t seed, uint32_t step,
                     int32_t max_trials, int32_t precision, double *r_new, double *vr_new,
                     double *vt_new, double *phi_new, double *rmin, double *rmax, double *F,
                     int32_t *code, void *stream);

/* Energy correction (section 2.1 step 6) of n sorted stars in the new
 * potential phi, in place on vr, vt; r_old and c = Phi_old(r_old) -
 * Phi_old(r_new) per star (sorted with the stars). */
cmc_status cmc_energy_correction(int64_t n, const double *r, const double *phi, double *vr,
                                 double *vt, const double *r_old, const double *c,
                                 void *stream);

/* Stellar radii (configuration collisions = 1; in Henon length units) of
 * the stars in the order cmc_get_state returns them: R (n, host or device
 * per ptr_kind) in, finite and >= 0; 0 means no radius.  With radii the
 * collision timestep of Eq. 8 (section 2.1 step 2), over the innermost 300
 * bound stars, joins the minimum with Eq. 7's, and a relaxation pair
 * (section 2.1 step 3(iii)) merges with probability
 * n pi (R1 + R2)^2 (1 + 2 G (m1 + m2) / ((R1 + R2) |w|^2)) |w| dt (the bin
 * density n, the pair's 3-D relative speed |w|; one draw per pair): the
 * first star keeps the pair's mass and momentum and takes the radius
 * (R1^3 + R2^3)^(1/3), the second leaves the cluster (radius -1 afterwards).
 * Radii travel with the stars through every sort; cmc_set_state sets them
 * to 0.  CMC_EINVAL without collisions or for bad radii. */
cmc_status cmc_set_radii(cmc_ctx *ctx, const double *R, int32_t ptr_kind);
/* The stellar radii in state order (n doubles out, host or device). */
cmc_status cmc_get_radii(cmc_ctx *ctx, double *R, int32_t ptr_kind);

/* Semi-major axes of binaries (configuration binaries = 1; Henon length
 * units) of the stars in the order cmc_get_state returns them: a (n, host
 * or device per ptr_kind) in, finite and >= 0; 0 marks a single star, and a
 * binary's entry of m is the pair's total mass.  With them the binary
 * timesteps of section 2.1 step 2 join the minimum with Eq. 7's, over the
 * innermost P = min(300, N_bound) stars of each cluster (Eqs. 9 and 10):
 *   1/T_bb = 16 sqrt(pi) n_b X_bb^2 <a^2> sigma
 *            (1 + G <M a> / (2 sigma^2 X_bb <a^2>)),
 *   1/T_bs = 4 sqrt(pi) n_s X_bs^2 <a^2> sigma
 *            (1 + G <M> <a> / (sigma^2 X_bs <a^2>)),
 * with n = 3 (P - 1) / (4 pi (r_{P-1}^3 - r_0^3)), n_b and n_s that density
 * times the binaries' and the single stars' shares of the P stars, <a^2>,
 * <M a>, <a> means over the binaries among them, <M> the mean mass of all
 * P, sigma^2 = <v_r^2 + v_t^2> / 3 over all P.  No binary: no T_bb or T_bs;
 * no single star: no T_bs.  The axes travel with the stars through every
 * sort (the interactions that would change them are outside this
 * library); cmc_set_state sets them to 0.  CMC_EINVAL without binaries or
 * for bad values (checked for host input). */
cmc_status cmc_set_binaries(cmc_ctx *ctx, const double *a, int32_t ptr_kind);
/* The semi-major axes in state order (n doubles out, host or device). */
cmc_status cmc_get_binaries(cmc_ctx *ctx, double *a, int32_t ptr_kind);

/* An outside bound on the next steps of each cluster (host, n_clusters
 * doubles, each finite and >= 0; 0 = none, the initial value): every later
 * step of cluster c takes min(its timestep, cap[c]).  It carries the
 * timesteps that other processes put on the step (section 2.1 step 2: Eq.
 * 11's stellar-evolution step, say, from cmc_tse).  Stays until set again.
 * CMC_EINVAL for bad values. */
cmc_status cmc_set_dt_cap(cmc_ctx *ctx, const double *cap);

/* The stellar-evolution timestep of Eq. 11: the step in which stellar
 * evolution, having taken dm_se of mass in the previous step of length
 * T_prev, takes 0.1% of the cluster mass M:
 * T_se = ((0.001 M) T_prev) / dm_se, in that order of operations;
 * +inf when dm_se <= 0 (no loss).  Host arithmetic only. */
double cmc_tse(double M, double T_prev, double dm_se);

/* Limits of the sort's bounded device waits on the current device, for all
 * contexts and stage calls there (read by the kernels at launch, so graphs
 * captured earlier follow them): lookback_polls = polls of an earlier
 * tile's look-back word before a tile gives up on it (the step then
 * returns CMC_ETIMEOUT and the context is poisoned; cmc_sort_radius
 * returns CMC_ETIMEOUT); tie_moves = moves of the insertion sort that puts a
 * run of equal sort keys in id order before it gives up on the run (a step
 * then fails, cmc_sort_radius falls back to sorting by id, then by radius).
 * Values <= 0 restore the defaults (2^22 each).  Returns CMC_ECUDA if the
 * device cannot be reached. */
cmc_status cmc_set_wait_limits(int32_t lookback_polls, int64_t tie_moves);

/* ---------------------------------------------------------------------
 * Allocation-free shell potential.  The paper has no counterpart: this is
 * cmc_potential (the same scan over the same tiles, with summation orders
 * of its own inside a tile: results agree with cmc_potential's to rounding
 * and repeat bit for bit from call to call) for callers that may not
 * allocate device memory: real-time loops that forbid allocation after
 * start-up (an allocation can block, synchronise or fail at any time),
 * programs that give all device memory to their own pool, and plug-ins
 * whose host application owns the allocator.  cmc_potential takes scratch
 * from cudaMallocAsync; this function allocates nothing.  Its only scratch,
 * the per-tile sums of the scan, is one fixed array of the library's own
 * device memory (2 * CMC_STATIC_MAX_STARS / 4096 doubles, 64 KiB) that
 * every GPU that loads the library holds until the process exits.
 *   n <= CMC_STATIC_MAX_STARS sorted stars; r, m (device, n doubles) in;
 *   phi (device, n doubles) out; M (device, may be NULL) enclosed mass out.
 * The first call on each device looks up the array's device address with
 * that device current (and may load the library's kernels); make that first
 * call before any stream capture.  The address is kept for the life of the
 * process: after cudaDeviceReset on a device, do not call this function
 * on that device again.
 * Every call shares the one array and overwrites it (nothing in it needs
 * to start at zero), so calls whose work overlaps on the GPU (different
 * streams) race: order them on one stream.  Returns CMC_EINVAL for
 * n > CMC_STATIC_MAX_STARS or bad pointers, CMC_ECUDA if the launch fails
 * (or an earlier error is pending on the device; it is reported, not
 * cleared); returns once the work is enqueued on `stream`.
 * ------------------------------------------------------------------- */
#define CMC_STATIC_MAX_STARS 16777216
cmc_status cmc_potential_static(int64_t n, const double *r, const double *m, double *phi,
                                double *M, void *stream);

/* -------------------------------------------------------------------
 * Self-check of the integer-pipe FP64 arithmetic.  GB300 issues FP64
 * arithmetic on two lanes per SM and clock, so the kernels compute their
 * correctly rounded quotients, square roots and some products from 64-bit
 * integer operations on the significands (normal operands with a normal
 * result; anything else takes the FP64 instruction).  These must
 * equal IEEE-754 round-to-nearest-even exactly, which is what keeps the
 * FP64 path bit for bit equal to an FP64 statement of the method (§2.1).
 * This call compares one of them with the FP64 hardware operation:
 *   op: 0 = a * b, 1 = a / b, 2 = sqrt(a);
 *   n operand pairs, hashed from `seed` (splitmix64) in three families in
 *   turn: any 64-bit pattern (NaN, infinities, zeros, subnormals, and the
 *   fallbacks), random values with exponents in [2^-40, 2^40], and the same
 *   with 0..52 trailing significand bits cleared (exact results and ties);
 *   *mismatches (host) receives the number of results whose bit patterns
 *   differ (NaN against NaN counts as equal).
 * Runs on the current device and the legacy default stream; synchronous.
 * Returns CMC_EINVAL for an op outside 0..2 or a NULL pointer, CMC_ECUDA
 * on a CUDA error.
 * ------------------------------------------------------------------- */
cmc_status cmc_check_arith(int32_t op, uint64_t n, uint64_t seed, uint64_t *mismatches);

#ifdef __cplusplus
}
#endif

#endif /* CMC_H */
