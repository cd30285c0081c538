// bz_impl.h -- internal layout shared by the mixture compiler (host C++) and
// the CUDA kernels.  Not part of the public ABI.
#pragma once

#include <stdint.h>

#include <string>
#include <vector>

#include "bz.h"

namespace bz {

// Physical constants (CODATA 2018).
constexpr double kQe = 1.602176634e-19;       // C
constexpr double kMe = 9.1093837015e-31;      // kg
constexpr double kHartreeEv = 27.211386245988;
constexpr double kTownsend = 1e-21;           // V m^2
constexpr double kLoschmidt = 2.686780111e25; // m^-3 (273.15 K, 101.325 kPa)

constexpr int kMaxGases = 16;  // gases per mixture
constexpr int kGroups = 32;   // batch groups for standard errors (id mod 32)
constexpr int kQ1 = 21;       // first-pass tally quantities
constexpr int kQ2 = 8;        // second-pass tally quantities
// Shared-memory budgets of a mixture's staged tables: three FP32 step blocks
// of 256 threads per SM (each also holds ~2 KB of static and reserved shared
// memory out of a GB300 SM's 228 KB), and one FP64 block.
constexpr size_t kStageBudget32 = 72 * 1024;
constexpr size_t kStageBudget64 = 200 * 1024;
constexpr int kGuide = 256;  // buckets of the channel-search guide

// One interval [e_lo, e_hi) of the union energy grid: the density sum
// S(eps) = sum n_k sigma_kj(eps) of all channels not in their power-law
// tail is S_lo + slope (eps - e_lo) there.
template <typename R>
struct alignas(4 * sizeof(R)) Rec {
    R e_lo, e_hi, S_lo, slope;
};

// Per-channel constants.  bits: kind | angular << 4 | tail_zero << 8, and
// for xi-form gases gas << 12 | (the gas's elastic channel) << 16.
// Tail: n sigma(eps) = exp(tail_logc + tail_K ln eps) for eps >= e_last.
template <typename R>
struct alignas(16) ChParam {
    R kappa2;     // 2 m M / (m + M)^2            (Eq. 8)
    R mfrac;      // M / (m + M)                  (Eq. 9)
    R minv;       // (m + M) / M                  (Eq. 9)
    R eps_k;      // energy loss [eV]             (Eq. 9)
    R e_last;     // last table energy [eV]
    R tail_logc;
    R tail_K;
    int32_t bits;
};

// Per-interval, per-channel density n sigma_j = val + slope (eps - e_lo).
template <typename R>
struct alignas(2 * sizeof(R)) ChVal {
    R val, slope;
};

// Where each section of a compiled mixture sits in its device blob.  The
// blob is [records | buckets | channel params | bin maxima | channel values
// | per-gas sums | xi tables | cumulative channel values]; the prefix up to
// stage_tables (or stage_all) is copied into shared memory.  Bin maxima: the
// maximum of nu(eps) over each of n_bins log-uniform energy bins from
// 2^bin_lo to the last union point (windowed trial frequency); nu_low is the
// maximum below the first bin.  The compiler sizes the bucket index (1 to 4
// entries per record) and decides whether the bin maxima are staged so that
// stage_tables fits a shared-memory budget (the step kernels then keep
// three blocks per SM); bin maxima outside the staged prefix are read from
// global memory through L1.
struct Layout {
    int32_t n_rec, n_buckets, n_ch, first_tail_rec;
    float log2_lo, inv_bw;
    uint32_t off_bucket, off_chp, off_chval;
    uint32_t stage_tables;   // bytes of records + buckets + channel params (+ bin maxima when they fit)
    uint32_t stage_all;      // everything but the cumulative channel values
    uint32_t total;
    uint32_t off_bin;
    uint32_t bin_end;        // off_bin + bytes of the bin maxima: staged iff the staged prefix reaches it
    // cumulative channel values per record ({val, slope}, n_rec x n_ch, in
    // the order of Eq. 2): entry j is the sum of channels 0..j, searched by
    // bisection on real collisions when the channel values are not staged
    uint32_t off_cum;
    // guide of the search (mixtures of at most 255 channels, else 0): per
    // record r a row of kGuide bytes at off_guide + r kGuide; entry b of row r
    // is the first channel whose cumulative value reaches b/kGuide of the
    // density sum at the lower edge of record r (row r + 1: at its upper edge)
    uint32_t off_guide;
    int32_t buckets_per_record;
    double s_min;            // speed at the first bin edge [m/s]
    int32_t n_bins, bin_levels;  // sparse table: level l at [l * n_bins + b] = max over bins [b, b + 2^l)
    float bin_lo, inv_binw;  // log2 energy of the first bin edge, bins per unit log2
    double nu_low;           // max nu over [0, 2^bin_lo]
    double g_top;            // last union point [eV]
    // bin edges lie on the lattice 10^(j / bins_per_decade), the first at
    // j = bin_j0; low_sqrt: below it nu = nu_low sqrt(eps / 2^bin_lo)
    int32_t bin_j0, bins_per_decade, low_sqrt;
    double nu_first;         // nu at the first positive union point (floor of the adaptive nu')
    // per-gas density sums per record ({val, slope}, n_rec x n_gases, global
    // memory) and each gas's channel range, for a two-level channel search
    uint32_t off_gval;
    int32_t n_gases;
    // xi-form gases (Eqs. 6-7): the total elastic cross section per record
    // and gas ({val, slope}, n_rec x n_gases) and per gas its tail constants
    // (ChParam: e_last, tail_logc, tail_K, bits & 0x100 = no tail), global memory
    uint32_t off_elval, off_elp;
    int16_t gas_first[kMaxGases], gas_count[kMaxGases];
};

struct CompiledMixture {
    std::vector<uint8_t> blob32, blob64;
    Layout lay32, lay64;
    bz_mixture_info info;
    double n_total;
    double nu_max, nu_trial;
};

// Sets the calling thread's message returned by bz_last_error (api.cpp).
void set_last_error(const std::string &msg);

// Context and configuration queries shared by the C ABI's translation units
// (api.cpp): the context's CUDA device; the checks bz_run_swarm applies to a
// configuration (BZ_OK or BZ_EINVAL with the message set); whether a swarm
// runs in the step kernel's feature instance (the paper's adaptive trial
// frequencies, xi-form gases or moving targets).
int ctx_device(const bz_ctx *ctx);
bz_status check_config(const bz_swarm_config *cfg);
bool needs_feature_instance(const bz_mixture *mix, const bz_swarm_config *cfg);
// Whether a launch of this mixture alone stages its channel tables in shared
// memory (the CH_SMEM instance of the step kernel) at this precision.
bool stages_channels(const bz_mixture *mix, int precision);

// Host mixture compiler (mixture.cpp).  Returns BZ_OK or an error with *err.
bz_status compile_mixture(const bz_gas *gases, int32_t n_gases, const bz_mixture_opts *opts,
                          CompiledMixture *out, std::string *err);

}  // namespace bz
