// kernels.h -- host-side launch interface of the CUDA kernels (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "bz_impl.h"

namespace bz {

enum { ST_DONE = 0, ST_TIME = 1, ST_STEPS = 2, ST_TRIAL = 3, ST_ERROR = 4, ST_ATTACHED = 5 };
enum { DEC_WINDOW = -3, DEC_FAIL = -2, DEC_NULL = -1 };
enum { TF_NONE = 0, TF_VARIABLE = 1, TF_BINNED = 2 };

// Uniform static fields in the force frame (force on the electron along +z).
// The field constants rounded to FP32 by the host, for the FP32 step: it
// reads them as they are and never converts from FP64 in the loop (GB300
// runs FP64, conversions included, at a small fraction of the FP32 rate).
struct Fields32 {
    float a, b0, b1, b2, w, inv_w, vD0, vD1, vD2, vDn, a_par, Ke;
    float inv_a, inv_apar;  // 1/a and 1/|a_par| (0 where those vanish)
};

struct Fields {
    double a;        // eE/m [m/s^2]
    int32_t has_b;
    double b[3];     // unit vector of B
    double w;        // e|B|/m [rad/s]
    double vD[3];    // E x B drift (b x a z)/w
    double a_par;    // a (z . b)
    Fields32 f32;
};

struct ParticlesDev {
    double *x, *y, *z, *t, *se, *se2;
    float *vx, *vy, *vz, *nup;
    uint32_t *n_real, *n_null, *n_fail, *n_ion, *n_att, *steps, *status;
};

struct RunArgs {
    const uint8_t *blob;     // compiled mixture (device)
    Layout lay;
    uint32_t stage_bytes;    // prefix of the blob staged into shared memory
    uint32_t key0, key1;     // Philox key (swarm seed)
    uint32_t rk[20];         // its round keys: key + r (0x9E3779B9, 0xBB67AE85), r = 0..9
    uint64_t id_offset, n;
    uint32_t I;              // real collisions per particle
    int32_t fixed;           // fixed trial frequency: a fail stops the particle
    int32_t attach_keep;
    double nu0;              // starting trial frequency
    double eps0_mean;        // Maxwellian start, mean energy [eV]
    double v0_scale;         // sqrt(2 eps0_mean / (3 m)) [m/s]: the Maxwellian's per-component spread
    float v0_scale32, nu0_32;  // it and nu0 rounded to FP32 by the host, for the FP32 step
    double t_end;            // > 0: time limit [s]
    uint64_t max_trials;
    int32_t window;          // windowed local trial frequency
    float win_c;             // window length in units of 1/nu of the current energy bin
    double nu_floor;         // lower bound of any trial frequency [1/s]
    float nu_floor32;        // nu_floor rounded to FP32, and
    int32_t timed;           // t_end > 0: the FP32 step reads these and does no FP64 work per trial
    // the paper's adaptive trial frequencies (Sec. 6): tf = TF_VARIABLE or
    // TF_BINNED (0 otherwise), run by the ADAPT instance of the step kernel
    int32_t tf;
    double tf_zeta1;         // VARIABLE: 1 + zeta
    uint32_t tf_grace;       // collisions between queries of nu'
    int32_t tf_B;            // BINNED: bins per decade (divides lay.bins_per_decade)
    double kT_m;             // > 0: moving targets (Sec. 2.1), k T / m_e [(m/s)^2]; 0: targets at rest
    float kT_m32;            // kT_m rounded to FP32, and
    int32_t thermal;         // kT_m > 0, for the FP32 step
    // spawn mode: slots [0, n_primary) are the initial electrons; secondaries
    // take slots from *n_total (up to cap) and their birth state from
    // b*[slot - n_primary]; bid[] != 0 marks a published birth record
    int32_t spawn;
    uint64_t n_primary, cap;
    unsigned long long *n_total;
    unsigned long long *pending;  // electrons created and not finished
    unsigned int *n_capped;
    double *bt;
    double *bvx, *bvy, *bvz;
    uint64_t *bid;
    Fields f;
    unsigned long long *counter;  // spawn mode: next slot ticket
    uint64_t spawn_wait_ns;       // spawn mode: a warp without work gives up after this long
    uint64_t stage_wait_ns;       // a block gives up waiting for its tables after this long
    uint32_t stage_hold;          // tests of that wait: a second phase that no copy completes
    uint32_t pad0;
    uint32_t *err;
    ParticlesDev out;
};

struct ReplayArgs {
    RunArgs run;
    int64_t n;
    const double *state_in;
    const uint64_t *ids;
    const uint32_t *steps;
    double *state_out;
    int32_t *decision;
    double *eps_io;
};

struct TallyArgs {
    const double *x, *y, *z, *t, *se, *se2;
    const uint32_t *n_real, *n_null, *n_fail, *n_ion, *n_att, *status;
    const uint32_t *steps;   // may be null (no window-restart count)
    const uint64_t *ids;     // spawn mode: ids of slots >= n_primary (null otherwise)
    const unsigned int *capped;  // spawn mode: capped-ionization counter (may be null)
    uint64_t n, id_offset, n_primary;
    const unsigned long long *n_dev;  // spawn mode: particles = min(*n_dev, n) (may be null)
    double *part1, *part2;   // [blocks][kGroups][kQ1 | kQ2] scratch
    double *gsum;            // [kGroups][kQ1 + kQ2] + 8 summary values, scratch
    int32_t blocks;
    double E_V_m, n_total, nu_trial;
    const uint32_t *err;
    bz_tallies *out;         // device
};

// Batched launch: tiles (x = swarm, y = first particle, z = count) over the
// per-swarm parameters desc[] (RunArgs without the counter).
struct BatchArgs {
    const RunArgs *desc;     // null: one swarm, described by `single`
    const uint4 *tiles;      // null: tiles of tile_size electrons over `single`
    int32_t n_tiles;
    uint32_t tile_size;
    unsigned int *tile_counter;
    uint64_t slot_lo;        // implicit tiles start at this slot
    RunArgs single;
};

// Scalars of a run that its group sums do not hold.
struct GroupScalars {
    double E_V_m, n_total, nu_trial;
    uint64_t n_spawned, n_capped;
    int32_t error_flags;
};

// Group-sum layout: gsum[g * kGS + q], q < kQ1 pass 1, kQ1 <= q < kGS pass
// 2; the drift vectors S[0..5] follow at gsum + kGroups * kGS.
constexpr int kGS = kQ1 + kQ2;
// The swarm's drift vectors from pass-1 group sums, and the tallies from
// both passes' group sums (kernels.cu; host and device).
__host__ __device__ void drift_of_groups(const double *gsum, double *S);
__host__ __device__ void tallies_of_groups(const double *gsum, const double *S, const GroupScalars &X, bz_tallies *out);

// Launch helpers (kernels.cu).  precision is 32 or 64.
cudaError_t launch_replay(int precision, bool ch_smem, const ReplayArgs &a, int grid, int block, cudaStream_t s);
cudaError_t launch_philox(int64_t n, const uint32_t *ctr, uint64_t key, uint32_t *out, cudaStream_t s);
cudaError_t launch_tallies(const TallyArgs &a, cudaStream_t s);
// Pass 2 of a finished run's tallies about the given drift vectors
// (drift_host[6], as S above), summed into the group sums' pass-2 columns.
cudaError_t launch_group_sums2(const TallyArgs &a, const double *drift_host, cudaStream_t s);
// ext: the instance with the paper's adaptive trial frequencies and the xi
// form of the angle; the lean instance (the hot path of Lazy, Fixed and
// windowed swarms in mixtures without xi-form gases) compiles without them.
// wide: the 4-block build of the lean FP32 kernel may be taken (where its
// blocks fit); callers allow it without B, and with B for single-gas
// mixtures.  bfield: some swarm of the launch has a magnetic field (else the
// lean build without the field's paths runs).  block: 256 threads, or 128,
// 384 or 768 for the lean FP32 build (precision 32, not ext; never the
// 4-block build); any other value returns cudaErrorInvalidValue.
cudaError_t launch_batch(int precision, bool ch_smem, bool ext, bool wide, bool bfield, const BatchArgs &a,
                         size_t smem, int grid, int block, cudaStream_t s);
// Spawn mode: one persistent launch runs the primaries and every electron
// created from them (slots handed out as tickets from a.counter).
cudaError_t launch_spawn(int precision, bool ch_smem, bool ext, bool wide, bool bfield, const RunArgs &a, size_t smem,
                         int grid, int block, cudaStream_t s);
int spawn_occupancy(int precision, bool ch_smem, bool ext, bool wide, bool bfield, int block, size_t smem);
// Blocks of `block` threads that fit on one SM with `smem` bytes of tables.
// (a negative value is minus the CUDA error of the query)
int batch_occupancy(int precision, bool ch_smem, bool ext, bool wide, bool bfield, int block, size_t smem);
// Tallies of n_swarms swarms; args_dev is a device array of TallyArgs.
cudaError_t launch_tallies_multi(const TallyArgs *args_dev, int n_swarms, int max_blocks, cudaStream_t s);
int tally_blocks(uint64_t n, int sm_count);

}  // namespace bz
