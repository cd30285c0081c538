/*
 * bz.h -- C ABI of the GB300 electron-swarm Monte Carlo library (libbz.so).
 *
 * The library runs the per-electron step loop of "Betaboltz: a Monte-Carlo
 * simulation tool for gas scattering processes" (Renda, Ciubotaru, Banu,
 * arXiv:1901.08140) on one NVIDIA GB300 GPU (sm_103a): electrons drift
 * through a user-defined gas mixture under static uniform E and B fields
 * (Sec. 2; "Nature of problem" in the program summary), by null-collision
 * free flights (Eqs. 3-4), analytic classical motion (Sec. 3.6), a collision
 * channel drawn from the mixture's cross-section tables (Eq. 2), scattering
 * (Eqs. 5, 8, 9) and FP64 swarm tallies (Sec. 2.3, Eqs. 15-27).
 *
 * Conventions used by every call:
 *   - SI units, except energies in eV and reduced fields in Td
 *     (1 Td = 1e-21 V m^2).
 *   - Axes: the electric force on the electron points along +z, so the
 *     reported drift velocity W is positive (the paper aligns z with the
 *     field and prints W > 0).  B lies in the xz plane at angle
 *     b_angle_rad from +z: B = |B| (sin a, 0, cos a) (Sec. 2.3).
 *   - Pointers named *_dev are device pointers on the context's device;
 *     all other pointers are host pointers.
 *   - Every call returns a bz_status.  On failure the thread-local message
 *     of bz_last_error() says why; outputs are left untouched.
 *   - No call falls back to the CPU.  If the CUDA device or kernels are not
 *     usable, calls return BZ_ECUDA.
 */
#ifndef BZ_H
#define BZ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BZ_ABI_VERSION 8

typedef enum {
    BZ_OK = 0,
    BZ_EINVAL = 1,    /* invalid argument or table */
    BZ_ENOMEM = 2,    /* device or host allocation failed */
    BZ_EBUDGET = 3,   /* request exceeds an admission or size limit */
    BZ_ETRIAL = 4,    /* fixed trial frequency was exceeded (Sec. 6.1) */
    BZ_ETIMEOUT = 5,  /* a bounded device wait gave up */
    BZ_ECUDA = 6,     /* CUDA runtime or kernel error */
    BZ_ECANCEL = 7,   /* request cancelled */
    BZ_ENOTREADY = 8  /* result not available yet (non-blocking query) */
} bz_status;

typedef enum { BZ_ELASTIC = 0, BZ_EXCITATION = 1, BZ_ATTACHMENT = 2, BZ_IONIZATION = 3 } bz_kind;
/* Scattering angle (Sec. 2): isotropic; screened Coulomb (Eq. 5, atoms);
 * XI, the xi form of non-polar molecules (Eq. 6), whose xi solves Eq. 7
 * for the ratio of the gas's momentum-transfer cross section (its one
 * elastic channel) to its total elastic cross section (bz_gas.sigma_el_m2). */
typedef enum { BZ_ANG_ISOTROPIC = 0, BZ_ANG_SCREENED_COULOMB = 1, BZ_ANG_XI = 2 } bz_angular;
/* Trial frequency nu' of the null-collision flights (Sec. 6):
 *  LAZY   -- one constant nu' = exact max of nu over [0, eps_cap] (Sec. 6.2);
 *  FIXED  -- the caller's constant nu_trial; exceeding it is an error (Sec. 6.1);
 *  WINDOW -- a local nu' per time window: the max of nu over the energies the
 *            electron can reach within the window (rigorous speed bound under
 *            E and B, per-bin maxima of nu); a flight that outlasts the window
 *            restarts at its end (exact by memorylessness).  Same statistics as
 *            LAZY with far fewer null collisions. */
/* Trial frequency nu' (Sec. 6).  LAZY: the exact maximum of nu over the
 * tables (a fail -- nu > nu' past the tables -- goes back to the last real
 * collision and raises the particle's nu' to 1.25 nu).  FIXED: nu_trial, a
 * fail is an error.  WINDOW: a local majorant over the energies reachable
 * before the end of a short time window, renewed at window ends and real
 * collisions (exact, never fails).  VARIABLE (Sec. 6.4): nu' = (1 + zeta)
 * nu(eps), queried at the start, after every `grace` collisions (null or
 * real) and on a fail.  BINNED (Sec. 6.3): nu' = the maximum of nu over the
 * energy bin of eps (bins_per_decade bins per decade), queried likewise; a
 * fail retries with the larger maximum of the two bins, and a fail under
 * that retry value is an error (BZ_ERR_TRIAL).  VARIABLE and BINNED follow
 * the paper and are not exact: a fail goes back to the last real collision. */
typedef enum {
    BZ_TRIAL_LAZY = 0,
    BZ_TRIAL_FIXED = 1,
    BZ_TRIAL_WINDOW = 2,
    BZ_TRIAL_VARIABLE = 3,
    BZ_TRIAL_BINNED = 4
} bz_trial_mode;

typedef struct bz_ctx bz_ctx;
typedef struct bz_mixture bz_mixture;
typedef struct bz_swarm bz_swarm;

/* Device-memory provider.  alloc returns a device pointer of at least
 * `bytes` usable on `stream` (NULL on failure); free releases it.  Passing
 * NULL to bz_create uses cudaMallocAsync / cudaFreeAsync. */
typedef struct {
    void *(*alloc)(size_t bytes, void *stream, void *user);
    void (*free)(void *ptr, size_t bytes, void *stream, void *user);
    void *user;
} bz_allocator;

/* Creates a context on CUDA device `device`.  The allocator is copied.
 * Errors: BZ_EINVAL (bad device), BZ_ECUDA. */
bz_status bz_create(int device, const bz_allocator *alloc, bz_ctx **out);
/* Releases the caller's hold on the context.  Mixtures and swarms created
 * from it keep it alive; it is freed when the last of them is destroyed. */
void bz_destroy(bz_ctx *ctx);
/* Message of the last failure on the calling thread ("" if none). */
const char *bz_last_error(void);
int bz_abi_version(void);

/* ------------------------------------------------------------------------
 * Gas mixtures (Eq. 2; Sec. 3.5 GasMixture by number density).
 *
 * A gas is a set of channels with its molecule mass M and number density
 * n_k.  A channel is a cross-section table sigma(eps) on strictly increasing
 * energies, interpolated linearly (Sec. 5) and extended per Sec. 2.2:
 * elastic tables continue to the left with their first value, inelastic
 * ones are zero below threshold (and rise linearly from (threshold, 0) when
 * the table starts above it); to the right a power law sigma = A eps^K goes
 * through the last two points (Eqs. 12-14), or the last value continues when
 * one of them is zero.  threshold_eV is the energy loss eps_k of Eq. (9)
 * (the ionization potential for ionization; ignored for elastic).
 * ------------------------------------------------------------------------ */
typedef struct {
    int32_t kind;             /* bz_kind */
    int32_t n_points;         /* >= 1 */
    double threshold_eV;      /* >= 0 */
    const double *energy_eV;  /* host, n_points, strictly increasing, >= 0 */
    const double *sigma_m2;   /* host, n_points, >= 0; 0 below threshold */
} bz_channel;

typedef struct {
    double mass_kg;           /* > 0 */
    double number_density_m3; /* > 0 */
    int32_t angular;          /* bz_angular of every channel of this gas */
    int32_t n_channels;       /* >= 1; BZ_ANG_XI: exactly one BZ_ELASTIC channel */
    const bz_channel *channels;
    /* BZ_ANG_XI only (ignored otherwise): the total elastic cross section,
     * host, el_n_points >= 1, energies strictly increasing, extended like
     * an elastic table (Sec. 2.2) */
    int32_t el_n_points;
    int32_t reserved;
    const double *el_energy_eV;
    const double *sigma_el_m2;
} bz_gas;

typedef struct {
    double eps_cap_eV;        /* majorant range [0, eps_cap]; <= 0: largest table energy */
    double majorant_guard;    /* nu' = (1 + guard) max nu; < 0: default 1e-6 */
    int32_t channels_in_smem; /* -1 auto, 0 channel tables stay in L2, 1 stage them in shared memory */
    int32_t smem_budget;      /* bytes of shared memory per block for tables; <= 0: auto */
} bz_mixture_opts;

/* Validates and compiles a mixture: union energy grid over all channels and
 * thresholds, per-interval density sums and slopes, per-channel interval
 * coefficients, power-law tails, a log-energy bucket index and the exact
 * trial frequency nu' = max over [0, eps_cap] of nu(eps) (Sec. 6.2,
 * LazyTrialFrequency made exact).  Tables are deep-copied to the device;
 * the caller's arrays may be freed on return.  opts may be NULL (defaults).
 * Errors: BZ_EINVAL (non-monotone grid, negative or non-finite sigma, sigma
 * > 0 below threshold, mass or density <= 0, > 65535 union points),
 * BZ_ENOMEM, BZ_ECUDA. */
bz_status bz_create_gas_mixture(bz_ctx *ctx, const bz_gas *gases, int32_t n_gases,
                                const bz_mixture_opts *opts, bz_mixture **out);
void bz_destroy_mixture(bz_mixture *mix);

typedef struct {
    double nu_max;            /* majorant before the guard [1/s] */
    double nu_trial;          /* nu' used by lazy mode [1/s] */
    double eps_at_max;        /* energy of the maximum [eV] */
    double eps_cap;           /* [eV] */
    double n_total;           /* sum of number densities [1/m^3] */
    int32_t n_gases, n_channels, n_records, n_buckets;
    int32_t smem_bytes;       /* shared memory the step kernel stages */
    int32_t channels_in_smem;
    int32_t first_tail_record;
    int32_t table_bytes;      /* device bytes of the compiled tables (FP32 + FP64 copies) */
    int32_t n_xi_gases;       /* gases with the xi form of the angle */
    int32_t reserved;
} bz_mixture_info;

bz_status bz_mixture_get_info(const bz_mixture *mix, bz_mixture_info *out);

/* Host only: validates and compiles a mixture exactly as
 * bz_create_gas_mixture does and reports its info, without touching a
 * device (smem_bytes and channels_in_smem are left 0).  Same errors. */
bz_status bz_mixture_compile_info(const bz_gas *gases, int32_t n_gases, const bz_mixture_opts *opts,
                                  bz_mixture_info *out);

/* ------------------------------------------------------------------------
 * Swarm runs (Sec. 2.3: N primaries at the origin, I real collisions each;
 * Sec. 3.2 limiters: interactions, time).
 * ------------------------------------------------------------------------ */
typedef struct {
    double e_over_n_Td;       /* set by bz_set_fields */
    double b_T;
    double b_angle_rad;
    uint64_t n_electrons;     /* N >= 1 */
    uint32_t real_collisions; /* I: InteractionBulletLimiter; >= 1 */
    int32_t precision;        /* 32: FP32 flights and scattering, FP64 tallies; 64: FP64 throughout */
    int32_t trial_mode;       /* bz_trial_mode */
    int32_t attach_keep_state;/* 1: a dummy attachment leaves the electron unchanged */
    double nu_trial;          /* fixed mode: nu' [1/s]; lazy mode: > 0 overrides the start value */
    double eps0_mean_eV;      /* isotropic Maxwellian start with this mean energy (0: at rest) */
    double t_end_s;           /* > 0: TimeBulletLimiter, the last flight is cut at t_end */
    uint64_t max_trials;      /* per particle, 0: 2^31 - 1 */
    uint64_t seed;            /* Philox key of the swarm */
    uint64_t id_offset;       /* first particle id: ids id_offset .. id_offset + N - 1 */
    int32_t block_threads;    /* threads per block: 0 or 256; 128, 384 or 768 for FP32 swarms without spawn
                                 mode whose mixture and trial mode run the lean step kernel (same results) */
    int32_t blocks_per_sm;    /* 0: auto (occupancy) */
    double window_c;          /* WINDOW mode: window = window_c / nu of the current energy bin; 0: 2 */
    int32_t spawn;            /* 1: ionizations create electrons, attachments remove them (Sec. 2) */
    int32_t reserved0;
    uint64_t pop_cap;         /* spawn mode: at most this many electrons in all; 0: 64 x n_electrons */
    double zeta;              /* VARIABLE: overhead, nu' = (1 + zeta) nu(eps); >= 0 */
    uint32_t grace;           /* VARIABLE, BINNED: collisions between queries of nu'; >= 1 */
    int32_t bins_per_decade;  /* BINNED: 1, 2, 4, 8, 16 or 32 */
    double gas_temperature_K; /* > 0: the targets move, Maxwell-Boltzmann at this temperature, and every
                                 collision but attachment is worked in the centre-of-momentum frame
                                 (Sec. 2.1); 0: targets at rest (Eqs. 8-9) */
    double spawn_wait_s;      /* spawn mode: a warp with no electron to run gives up after waiting this long for a
                                 created one (sets BZ_ERR_SPAWN_WAIT, bz_read_tallies returns BZ_ETIMEOUT);
                                 <= 0: 60 s */
    uint32_t hold_pending;    /* spawn mode, for tests of that bounded wait: this many electrons are counted as
                                 pending and never arrive, so lanes that run out of work wait until spawn_wait_s;
                                 0 in normal use */
    uint32_t hold_stage;      /* tests of the table staging wait: 1 = once a block's tables are in, it waits on
                                 a further copy that is never issued, so the wait runs out after stage_wait_s
                                 (BZ_ERR_STAGE_TIMEOUT; the read returns BZ_ETIMEOUT) with no copy in flight;
                                 0 in normal use */
    double stage_wait_s;      /* a block gives up waiting for its tables (TMA bulk copy into shared memory) after
                                 this long, sets BZ_ERR_STAGE_TIMEOUT and exits once no copy is in flight (at most
                                 1 s more); <= 0: 10 s; at most 3600 */
} bz_swarm_config;

/* Fills *cfg with defaults: N = 1e4, I = 1000, FP32, lazy mode, Maxwellian
 * start with mean 0.1 eV, no time limit, seed 1901081400, fields zero;
 * zeta = 0.25, grace = 5000, bins_per_decade = 8. */
void bz_config_defaults(bz_swarm_config *cfg);

/* Sets the fields of a configuration: reduced field E/N [Td] (E = (E/N) N
 * with N the mixture's total density), |B| [T] and the angle of B from +z
 * in the xz plane [rad].  Errors: BZ_EINVAL (negative or non-finite). */
bz_status bz_set_fields(bz_swarm_config *cfg, double e_over_n_Td, double b_T, double b_angle_rad);

/* Launches one swarm on `stream` (cudaStream_t; NULL: the legacy default
 * stream) and returns at once.  The swarm owns its device buffers until
 * bz_destroy_swarm.  Each electron starts at the origin with an isotropic
 * Maxwellian velocity and runs until its I-th real collision (or t_end).
 * With spawn = 0, ionizations and attachments are dummy (counted, Sec.
 * 2.3).  With spawn = 1 (ChildrenBulletLimiter, Sec. 3.2) an ionization
 * creates an electron at the collision point with the fraction u of the
 * energy left after Eq. (9), leaving isotropically (u and the direction from
 * the second draw of that step), with id derived from (parent id, step); an
 * attachment removes the electron; past pop_cap electrons, ionizations are
 * only counted.  Every electron has its own limiters (I real collisions,
 * absolute t_end) and reports position and time relative to its birth.  In
 * spawn mode one persistent launch runs every electron: lanes that finish
 * an electron take the next created one as soon as its birth record is
 * published, until none is left; the call returns at once here too.
 * Errors: BZ_EINVAL, BZ_ENOMEM, BZ_ECUDA. */
bz_status bz_run_swarm(bz_ctx *ctx, const bz_mixture *mix, const bz_swarm_config *cfg,
                       void *stream, bz_swarm **out);

/* Swarm results (Sec. 2.3 and the Drifter fields of the worked example in
 * Sec. 7).  Per-particle ratio means as the paper writes them; "_flux"
 * fields are ratios of sums; "_se" fields are standard errors from 32 batch
 * groups (particle id mod 32).  d_n = x_n - t_n W_vec (full drift vector). */
typedef struct {
    double W, W_se;           /* <z/t> [m/s] (Eq. 15) */
    double Wx, Wy;            /* <x/t>, <y/t> (E x B drift) */
    double W_flux;            /* sum z / sum t */
    double lorentz_angle;     /* atan2(|W_perp|, W) [rad] */
    double mu, mu_N, mu_0;    /* W/E; mu N; mu N / N_Loschmidt */
    double eps, eps_se;       /* mean energy just before real collisions [eV] (Eq. 18) */
    double eps_after, eps_after_se; /* just after (Eq. 19) */
    double alpha, alpha_se, eta, eta_se; /* <G/z>, <D/z> [1/m] (Eqs. 16-17) */
    double alpha_flux, eta_flux;
    double D, D_se, D_L, D_L_se, D_T, D_T_se; /* [m^2/s] (Eqs. 22-24) */
    double D_L_flux, D_T_flux;
    double sig, sig_se, sig_L, sig_L_se, sig_T, sig_T_se; /* [m] (Eqs. 25-27) */
    double efficiency;        /* real / (real + null + fail) (Eq. 28) */
    double E_V_m, n_total, nu_trial, t_mean;
    uint64_t n_particles, n_real, n_null, n_fail, n_ion, n_att, n_incomplete;
    uint64_t n_window;        /* WINDOW mode: flights restarted at a window end */
    uint64_t n_spawned;       /* spawn mode: electrons created by ionization */
    uint64_t n_alive;         /* electrons stopped by the time limit (alive at t_end) */
    uint64_t n_removed;       /* spawn mode: electrons removed by attachment */
    uint64_t n_capped;        /* spawn mode: ionizations that found the population at its cap */
    int32_t error_flags;      /* device error bits (see BZ_ERR_*) */
    int32_t reserved;
} bz_tallies;

#define BZ_ERR_STAGE_TIMEOUT 1u /* table staging wait gave up */
#define BZ_ERR_TRIAL 2u         /* fixed nu' exceeded, or a BINNED retry failed again */
#define BZ_ERR_NONFINITE 4u     /* non-finite energy met; particle stopped */
#define BZ_ERR_MAX_TRIALS 8u    /* a particle reached max_trials */
#define BZ_ERR_SPAWN_WAIT 16u   /* spawn mode: a warp waited longer than spawn_wait_s for work */

/* Waits for the swarm and copies its tallies into *out.
 * Errors: BZ_ETRIAL (fixed mode exceeded), BZ_ETIMEOUT (a bounded device
 * wait gave up: table staging, or spawn mode's wait for created electrons;
 * the tallies are still copied), BZ_ECUDA. */
bz_status bz_read_tallies(bz_swarm *sw, bz_tallies *out);
/* Non-blocking: BZ_ENOTREADY while the swarm runs, else as bz_read_tallies. */
bz_status bz_query_tallies(bz_swarm *sw, bz_tallies *out);

/* Per-particle final state (slot i = particle id_offset + i), copied into
 * caller-owned host arrays of length >= N; any pointer may be NULL.  Waits
 * for the swarm. */
typedef struct {
    double *x, *y, *z, *t;         /* position [m] and time [s] at the end, relative to birth */
    double *sum_e, *sum_e2;        /* energy sums before / after real collisions [eV] */
    float *vx, *vy, *vz;           /* final velocity [m/s] */
    float *nu_p;                   /* final trial frequency of the particle [1/s] */
    uint32_t *n_real, *n_null, *n_fail, *n_ion, *n_att, *steps, *status;
    uint64_t *id;                  /* particle id (secondaries: derived from parent id and step) */
    double *t_birth;               /* birth time [s] (0 for the initial electrons) */
} bz_particles;

/* Status codes of bz_particles.status. */
#define BZ_ST_DONE 0     /* reached I real collisions */
#define BZ_ST_TIME 1     /* stopped at t_end */
#define BZ_ST_STEPS 2    /* reached max_trials */
#define BZ_ST_TRIAL 3    /* fixed nu' exceeded */
#define BZ_ST_ERROR 4    /* non-finite state */
#define BZ_ST_ATTACHED 5 /* removed by attachment (spawn mode) */

/* Number of electrons of the swarm (initial + created); waits for it. */
bz_status bz_swarm_size(bz_swarm *sw, uint64_t *n);

bz_status bz_read_particles(bz_swarm *sw, const bz_particles *out);

/* Device time of the swarm's step kernel and of its tally kernels [ms],
 * from CUDA events recorded around them on the swarm's stream.  Waits for
 * the swarm. */
bz_status bz_swarm_timing(bz_swarm *sw, double *step_ms, double *tally_ms);
void bz_destroy_swarm(bz_swarm *sw);

/* ------------------------------------------------------------------------
 * Batched swarms: many swarms of uneven size and different mixtures in one
 * persistent launch (the GPU counterpart of the paper's many independent
 * particles of Sec. 4).  Work is split into tiles (swarm, particle range)
 * ordered by mixture; a block re-stages tables only when the mixture
 * changes.  The launch, the FP64 tallies of every swarm and the copy of
 * the tallies to the host are captured once in a CUDA graph and replayed
 * by bz_launch_batch.  Every swarm's results equal those of bz_run_swarm
 * with the same configuration when the batch's swarms all have a magnetic
 * field or all lack one, and their mixtures all stage their channel tables
 * in shared memory or all leave them in global memory
 * (bz_mixture_info.channels_in_smem).  Otherwise the batch runs the field's
 * build, or searches every mixture's cumulative channel table in global
 * memory, and a swarm that runs differently alone matches its run alone to
 * FP32 rounding (a channel choice differs only where a draw falls within
 * rounding of a channel boundary).
 * ------------------------------------------------------------------------ */
typedef struct bz_batch bz_batch;

typedef struct {
    int32_t tile_particles;   /* electrons per tile at most (the last tiles shrink as the work left runs out,
                                 to 256 electrons or the block's threads rounded up to a multiple of 256);
                                 <= 0: about 16 tiles per resident block */
    int32_t blocks_per_sm;    /* <= 0: as many as fit */
    int32_t use_graph;        /* 1: CUDA graph (default when opts is NULL), 0: plain launches */
    int32_t channels_in_l2;   /* table-staging policy: 1 = every mixture's channels are chosen from its cumulative
                                 table in global memory, even where its channel coefficients would fit shared
                                 memory (smaller staged prefix; results then match runs alone to FP32 rounding
                                 of channel boundaries); 0 = stage them where every mixture's fit */
    int32_t block_threads;    /* threads per block: 0 or 256; 128, 384 or 768 for FP32 batches of the lean step
                                 kernel (no VARIABLE / BINNED trial frequency, no xi-form gas), at the register cap
                                 of the 256-thread build (6 x 128, 2 x 384 or 1 x 768 threads per SM).  Results do
                                 not depend on it; other values: BZ_EINVAL */
} bz_batch_opts;

/* Prepares a batch of n swarms (1 <= n <= 65535): mixtures[i] and cfgs[i]
 * as for bz_run_swarm (all the same precision, no spawn mode; either every
 * swarm or none needs the feature instance).  Allocates the device state of
 * all swarms once.  Errors: BZ_EINVAL, BZ_EBUDGET (tables too large for
 * shared memory), BZ_ENOMEM, BZ_ECUDA. */
bz_status bz_create_batch(bz_ctx *ctx, int32_t n, const bz_mixture *const *mixtures, const bz_swarm_config *cfgs,
                          const bz_batch_opts *opts, bz_batch **out);
/* Runs the batch on `stream` (asynchronous); may be called again after the
 * previous run finished (same results: counters are keyed by the seeds). */
bz_status bz_launch_batch(bz_batch *b, void *stream);
/* Non-blocking: BZ_ENOTREADY while the last launch runs, BZ_OK when done. */
bz_status bz_batch_query(bz_batch *b);
/* Waits for the last launch and copies the n swarms' tallies into out[n]. */
bz_status bz_batch_read_tallies(bz_batch *b, bz_tallies *out);
/* Waits, then copies swarm i's per-particle results (as bz_read_particles). */
bz_status bz_batch_read_particles(bz_batch *b, int32_t i, const bz_particles *out);
/* Device time of the last launch: the batch kernel and the tally kernels [ms]. */
bz_status bz_batch_timing(bz_batch *b, double *step_ms, double *tally_ms);
void bz_destroy_batch(bz_batch *b);

/* ------------------------------------------------------------------------
 * Merging one swarm run in parts.  Electrons never interact (the paper
 * neglects Coulomb forces between them, Sec. 9) and every random number is
 * keyed by the swarm seed and the particle id, so a swarm can run as id
 * ranges (id_offset) on several GPUs or in several launches and be merged
 * into the tallies of one run.  The estimators of Sec. 2.3 are sums over
 * electrons, grouped by batch group (id mod 32) for the standard errors:
 *   pass 1: BZ_GROUP_Q1 sums per group -- count, x/t, y/t, z/t, G/z, D/z,
 *           x, y, z, t, the energy sums, the counts of real, null and failed
 *           trials, ionizations, attachments, incomplete electrons, steps,
 *           electrons stopped at t_end and removed;
 *   pass 2: BZ_GROUP_Q2 sums per group about the swarm's drift vectors --
 *           |d|^2/t, d_z^2/(2t), |d_perp|^2/(4t), 2|d|, 2|d_z|, 2|d_perp| with
 *           d = x - t W_vec (Eqs. 21-27), and the two flux forms' squares.
 * Because pass 2 needs the drift of the whole swarm, a merge takes two
 * exchanges: add every part's pass-1 sums (FP64) and derive the drift
 * (bz_drift_from_group_sums); have every part sum pass 2 about it and add
 * those; then bz_finalize_group_sums.  Sums are [32][Q] row-major host
 * arrays.  The drift vector is {<x/t>, <y/t>, <z/t>, sum x/sum t,
 * sum y/sum t, sum z/sum t}.
 * ------------------------------------------------------------------------ */
#define BZ_GROUPS 32
#define BZ_GROUP_Q1 21
#define BZ_GROUP_Q2 8

typedef struct {
    double e_over_n_Td;       /* for E in the mobility fields */
    double n_total_m3;        /* the mixture's total number density */
    double nu_trial;          /* copied into the result */
    uint64_t n_spawned;       /* spawn mode: created electrons, summed over the parts */
    uint64_t n_capped;        /* spawn mode: capped ionizations, summed over the parts */
    int32_t error_flags;      /* the parts' error bits, or-ed */
    int32_t reserved;
} bz_merge_info;

/* Pass-1 group sums of a finished swarm (waits for it): out[32][21]. */
bz_status bz_swarm_group_sums1(bz_swarm *sw, double *out);
/* Pass-2 group sums of a finished swarm about drift[6] (runs the second
 * pass again on the swarm's stream and waits): out[32][8]. */
bz_status bz_swarm_group_sums2(bz_swarm *sw, const double *drift, double *out);
/* The same for swarm i of a launched batch (waits for the launch). */
bz_status bz_batch_group_sums1(bz_batch *b, int32_t i, double *out);
bz_status bz_batch_group_sums2(bz_batch *b, int32_t i, const double *drift, double *out);
/* Host only: the drift vector from (summed) pass-1 group sums. */
bz_status bz_drift_from_group_sums(const double *g1, double *drift);
/* Host only: the tallies of (summed) pass-1 and pass-2 group sums; the
 * same arithmetic the device reduction ends with.  Errors: BZ_EINVAL. */
bz_status bz_finalize_group_sums(const double *g1, const double *g2, const bz_merge_info *info, bz_tallies *out);

/* ------------------------------------------------------------------------
 * Serving: a request loop with continuous batching.  The paper has no
 * counterpart (its drifter runs one swarm per process, Sec. 7); this is the
 * form in which many independent swarm requests share one GPU.
 *
 * Requests (a compiled mixture and a configuration, as for bz_run_swarm)
 * are queued in submission order.  A worker thread of the server owns
 * n_slots launch slots, one non-blocking CUDA stream each.  Whenever a slot
 * is free it takes queued requests in order -- as many as fit the
 * device-memory budget, at most max_group, all of one step-kernel class
 * (precision; the feature instance or the lean one; the lean one with or
 * without the magnetic field's paths) -- and runs them as one batched
 * persistent launch (bz_create_batch); a spawn-mode request runs alone
 * (bz_run_swarm).  Launches are polled without blocking, so requests that
 * arrive while others run are admitted as soon as a slot and memory free up.
 * A request's tallies equal those of bz_run_swarm with its configuration.
 *
 * Device bytes of a request, counted against the budget while it runs:
 * 92 per electron slot (its results), 40 per created electron's birth
 * record in spawn mode (pop_cap - n_electrons), plus 2 MiB.
 * ------------------------------------------------------------------------ */
typedef struct bz_server bz_server;

typedef struct {
    double memory_budget_bytes; /* device bytes running requests may hold at once; <= 0: 60e9 */
    int32_t n_slots;            /* concurrent launches, at most 64; <= 0: 3 */
    int32_t max_group;          /* requests per batched launch, at most 65535; <= 0: 512 */
    int32_t simulate;           /* 0: run on the context's GPU.  n > 0: host-only scheduling test -- no
                                   device is touched, ctx and mixtures may be NULL, a launch ends after
                                   n polls of the worker and reports n_particles and n_real only */
    int32_t reserved;
} bz_server_opts;

typedef struct {
    double t_submit, t_admit, t_done; /* seconds since the server was created (monotonic clock) */
    uint64_t launch;                  /* index of the launch that ran the request (0, 1, ...) */
    int32_t group_size;               /* requests in that launch */
    int32_t status;                   /* bz_status of the request's run */
} bz_request_info;

typedef struct {
    uint64_t submitted, completed, cancelled, launches;
    int32_t queued, running, max_running, reserved; /* requests waiting / on the GPU / most at once */
    double bytes_in_use, peak_bytes_in_use;         /* device bytes held by running requests */
} bz_server_stats;

/* Creates a server on ctx's device and starts its worker thread.  The
 * context (and the mixtures of submitted requests) must outlive the
 * server.  Errors: BZ_EINVAL, BZ_ENOMEM, BZ_ECUDA (stream creation). */
bz_status bz_server_create(bz_ctx *ctx, const bz_server_opts *opts, bz_server **out);
/* Queues a request and returns its id (> 0) at once.  The configuration is
 * copied.  Errors: BZ_EINVAL (as bz_run_swarm's checks), BZ_EBUDGET (the
 * request alone needs more device memory than the budget: it could never
 * run). */
bz_status bz_submit(bz_server *s, const bz_mixture *mix, const bz_swarm_config *cfg, uint64_t *request_id);
/* Non-blocking: BZ_ENOTREADY while the request is queued or running.  When
 * it has run, copies its tallies into *out and its times into *info (either
 * may be NULL), forgets the request and returns the run's status (BZ_OK, or
 * the error its launch reported).  BZ_ECANCEL if it was cancelled (the id is
 * then forgotten); BZ_EINVAL for an unknown or already delivered id. */
bz_status bz_poll(bz_server *s, uint64_t request_id, bz_tallies *out, bz_request_info *info);
/* Cancels a request: a queued one never starts; a running one's launch goes
 * on with the rest of its group and its result is dropped (its memory is
 * released when the launch ends); a finished one's result is dropped.
 * bz_poll then reports BZ_ECANCEL.  Errors: BZ_EINVAL (unknown id). */
bz_status bz_cancel(bz_server *s, uint64_t request_id);
/* Holds (paused != 0) or resumes admission: while held, queued requests
 * wait and launches already running go on (draining, maintenance, or a set
 * of submissions that should be grouped together).  Errors: BZ_EINVAL. */
bz_status bz_server_pause(bz_server *s, int32_t paused);
bz_status bz_server_get_stats(bz_server *s, bz_server_stats *out);
/* Stops the server: queued requests are cancelled, running launches are
 * waited for, and every undelivered result is dropped. */
void bz_server_destroy(bz_server *s);

/* ------------------------------------------------------------------------
 * Allocation-free tally reduction.  The paper has no counterpart: this entry
 * exists for callers that cannot allocate device memory at the point where
 * they need swarm statistics -- code whose device memory is entirely held by
 * another allocator (a framework's caching pool or a serving process with a
 * fixed HBM plan, where cudaMalloc fails or fragments the pool), and
 * latency-sensitive loops in which cudaMalloc / cudaFree would synchronize
 * the device.  It computes the same bz_tallies as bz_read_tallies from
 * caller-owned per-particle device arrays (the layout bz_read_particles
 * returns), using scratch that lives in a fixed static device array of
 * libbz.so (BZ_NOALLOC_SCRATCH_BYTES, held by every GPU that loads the
 * library until the process exits) instead of allocating.
 * ------------------------------------------------------------------------ */
#define BZ_NOALLOC_SPAN 32768u              /* particles per reduction block */
#define BZ_NOALLOC_MAX_BLOCKS 512u
#define BZ_NOALLOC_MAX_PARTICLES (BZ_NOALLOC_SPAN * BZ_NOALLOC_MAX_BLOCKS) /* 16777216 */
#define BZ_NOALLOC_SCRATCH_BYTES (8u * (BZ_NOALLOC_MAX_BLOCKS * 32u * 29u + 32u * 29u + 8u) + 256u)

typedef struct {
    const double *x, *y, *z, *t;      /* device, n each: final position [m], time [s] */
    const double *sum_e, *sum_e2;     /* device, n each: energy sums [eV] */
    const uint32_t *n_real, *n_null, *n_fail, *n_ion, *n_att, *status;  /* device, n each */
    const uint32_t *steps;            /* device, n, or NULL (then n_window is 0) */
} bz_particle_arrays;

/* Reduces n particles (ids id_offset .. id_offset + n - 1) into *out_dev (a
 * device bz_tallies) on `stream`, asynchronously, without allocating:
 * it calls no cudaMalloc, cudaFree or allocating library routine.
 * e_over_n_Td and n_total_m3 give E for the mobility fields; nu_trial is
 * copied into the result.  The first call on a device looks up the scratch
 * array's device address (cudaGetSymbolAddress with that device current) and
 * caches it; make that first call before any stream capture.  All calls on
 * a device share the one scratch array and overwrite it, so calls whose
 * kernels overlap on the GPU (concurrent streams, or threads) race: order
 * them on one stream.  The reduction sees only the per-particle arrays,
 * not the step kernel's error word, so the result's error_flags reads 0:
 * the run's outcome is in the per-particle status array (BZ_ST_*).
 * Errors: BZ_EINVAL (null pointer, n = 0), BZ_EBUDGET
 * (n > BZ_NOALLOC_MAX_PARTICLES), BZ_ECUDA. */
bz_status bz_reduce_tallies_noalloc(const bz_particle_arrays *in, uint64_t n, uint64_t id_offset,
                                    double e_over_n_Td, double n_total_m3, double nu_trial,
                                    bz_tallies *out_dev, void *stream);

/* ------------------------------------------------------------------------
 * Verification entry points.
 * ------------------------------------------------------------------------ */

/* One trial step per particle from a state at a real collision (single-step
 * replay, Sec. 2): state_in_dev[8 n] holds, per particle i, at 8i..8i+7:
 * x, y, z, vx, vy, vz, t, nu'.  The step draws Philox counter
 * (id, steps[i], 0), flies, and takes the fail / null / real decision.
 * Outputs: state_out_dev[8 n] the state after the step; decision_dev[n] the
 * global channel index, -1 null, -2 fail; eps_dev[2 n] the energy before and
 * after the collision.  Uses cfg's fields, precision, seed and trial mode
 * (cfg is validated as for bz_run_swarm).  Asynchronous on `stream`.
 * Errors: BZ_EINVAL (null pointer, n < 0, an invalid configuration, the
 * VARIABLE or BINNED trial frequency), BZ_EBUDGET, BZ_ENOMEM, BZ_ECUDA. */
bz_status bz_step_replay(bz_ctx *ctx, const bz_mixture *mix, const bz_swarm_config *cfg, int64_t n,
                         const double *state_in_dev, const uint64_t *ids_dev, const uint32_t *steps_dev,
                         double *state_out_dev, int32_t *decision_dev, double *eps_dev, void *stream);

/* Philox4x32-10 (Salmon et al., SC'11) on the device: out_dev[4 i..] =
 * Philox(ctr_dev[4 i..], key) for i < n.  Asynchronous on `stream`. */
bz_status bz_philox(bz_ctx *ctx, int64_t n, const uint32_t *ctr_dev, uint64_t key, uint32_t *out_dev,
                    void *stream);

#ifdef __cplusplus
}
#endif

#endif /* BZ_H */
