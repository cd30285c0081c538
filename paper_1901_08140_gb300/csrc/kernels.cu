// kernels.cu -- the electron-swarm step loop on sm_103a.
//
// One thread owns one electron at a time and runs it from the origin to its
// I-th real collision (Sec. 2.3), then takes the next electron from a
// per-swarm counter (warp-aggregated atomic).  A trial step (Sec. 2):
//   1. Philox4x32-10 at counter (id, step, 0) gives four uniforms;
//   2. free flight t_c = -ln(1-R)/nu' (Eq. 3);
//   3. analytic motion in uniform static E and B (Sec. 3.6), evaluated from
//      the state at the last real collision and the time since then, so null
//      collisions touch no position state;
//   4. nu(eps) = |v| S(eps) from the union-grid record that a log-energy
//      bucket index points at (Eq. 2, Sec. 5, Sec. 2.2 tails);
//   5. fail if nu > nu' (Sec. 6): back to the last real collision and raise
//      nu' to 1.25 nu; else null if R nu' > nu (Eq. 4);
//   6. on a real collision: the channel whose cumulative frequency reaches
//      R nu', angle (Eq. 5 or isotropic), energy exchange (Eqs. 8, 9;
//      attachment plastic; ionization split with a second draw), rotation,
//      and the per-collision energy tallies (Eqs. 18-19).
// The mixture's tables (records, bucket index, channel constants and, when
// they fit, the per-channel coefficients) are staged into shared memory by
// one TMA bulk copy per block (cp.async.bulk + mbarrier, bounded wait).
// FP32 kernels keep position and time at real collisions, and the energy
// sums, as compensated float pairs; all tallies are reduced in FP64.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.h"

namespace bz {
namespace {

constexpr int kBlock = 256;
#ifndef BZ_SWARM_MIN_BLOCKS
#define BZ_SWARM_MIN_BLOCKS 3  // FP32: resident blocks per SM the register allocation must allow
#endif
// The lean FP32 step kernel is also built for 4 resident blocks per SM (64
// registers, more spills).  A launch takes it when the caller allows it and
// the tables leave room for 4 blocks.  Measured on GB300: +6 % on a
// single-gas sweep, +6 % on a two-gas mixture without B and +27 % on
// avalanches, but -10 % on two-gas mixtures with B, whose field paths keep
// more registers live -- so callers allow it without B, and with B for
// single-gas mixtures only.
constexpr int kMinBlocksWide = 4;
// The lean FP32 batch kernel is also built for blocks of 128, 384 and 768
// threads at the register cap of the default build (3 x 256 threads per SM:
// 6 x 128, 2 x 384, 1 x 768): fewer, larger blocks hold fewer copies of the
// staged tables (more of the SM's shared memory is left to L1, which caches
// the channel tables read from global memory) but wait on more warps at the
// end of each tile.
template <int BS>
constexpr int blocks_at_default_cap() { return BZ_SWARM_MIN_BLOCKS * kBlock / BS; }
constexpr uint32_t kStageChunk = 32768;
constexpr uint32_t kWaitLimit = 1u << 24;
constexpr uint64_t kDrainNs = 1000000000ull;  // 1 s for a staging copy in flight after a timeout

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of the
// multiply-xor S-P network; the key is bumped by the Weyl constants after
// each round.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                        uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return make_uint4(c0, c1, c2, c3);
}

// The same generator with the round keys read from the swarm's parameters
// (precomputed by the host) instead of stepped in registers on every call:
// the step draws once per trial, and the 20 key additions were a few per
// cent of its instructions.
__device__ __forceinline__ uint4 philox_rk(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, const uint32_t *rk)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ rk[2 * r], n2 = hi0 ^ c3 ^ rk[2 * r + 1];
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return make_uint4(c0, c1, c2, c3);
}

// ((w >> 9) + 1/2) 2^-23: an odd multiple of 2^-24 in (0,1), exact in FP32.
// FP32 builds it from the bits, with no integer conversion: 1 + k 2^-23
// (k = w >> 9 as the mantissa of an exponent-0 float) minus 1 - 2^-24 is
// (2k + 1) 2^-24 exactly, since that difference is representable -- the
// same value for every k.
template <typename R>
__device__ __forceinline__ R uni(uint32_t w)
{
    if constexpr (sizeof(R) == 4) return __int_as_float(0x3f800000u | (w >> 9)) - 0.99999994f;
    return ((R)(w >> 9) + (R)0.5) * (R)(1.0 / 8388608.0);
}

// Math wrappers resolved per precision.
__device__ __forceinline__ float log_(float x) { return logf(x); }
__device__ __forceinline__ double log_(double x) { return log(x); }
__device__ __forceinline__ float exp_(float x) { return expf(x); }
__device__ __forceinline__ double exp_(double x) { return exp(x); }
__device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
__device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
__device__ __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }
// Division where the quotient may be a few ulp off (a window's length, which
// any positive value makes exact; 1/nu'; 1 - cos under B, the inelastic
// energy ratio and the screened-Coulomb angle, whose denominators lie in
// [1, 2^126)): the FP32 form takes the hardware reciprocal (2 ulp), FP64
// divides exactly.
__device__ __forceinline__ float fdiv_(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double fdiv_(double a, double b) { return a / b; }
__device__ __forceinline__ double rsqrt_(double x) { return rsqrt(x); }
__device__ __forceinline__ float log10_(float x) { return log10f(x); }
__device__ __forceinline__ double log10_(double x) { return log10(x); }
__device__ __forceinline__ float exp10_(float x) { return exp10f(x); }
__device__ __forceinline__ double exp10_(double x) { return exp10(x); }
__device__ __forceinline__ float floor_(float x) { return floorf(x); }
__device__ __forceinline__ double floor_(double x) { return floor(x); }
__device__ __forceinline__ void sincos_(float x, float *s, float *c) { sincosf(x, s, c); }
__device__ __forceinline__ void sincos_(double x, double *s, double *c) { sincos(x, s, c); }
__device__ __forceinline__ void sincospi_(float x, float *s, float *c) { sincospif(x, s, c); }
__device__ __forceinline__ void sincospi_(double x, double *s, double *c) { sincospi(x, s, c); }
__device__ __forceinline__ float max_(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double max_(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float min_(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double min_(double a, double b) { return fmin(a, b); }

// (sin, cos) of the azimuth 2 pi u.  FP32: the fast hardware sine and
// cosine of 2 pi u - pi, which lies in (-pi, pi) where their absolute error
// is below 4e-7, with both signs flipped; FP64: sincospi.
__device__ __forceinline__ void azimuth(float u, float &sn, float &cs)
{
    float s, c;
    __sincosf(6.28318530717958647692f * u - 3.14159265358979323846f, &s, &c);
    sn = -s;
    cs = -c;
}
__device__ __forceinline__ void azimuth(double u, double &sn, double &cs) { sincospi(2.0 * u, &sn, &cs); }

// Compensated accumulator: a float pair (TwoSum) for FP32, a double for FP64.
template <typename R>
struct Acc;
// FP32: increments go into a short float sum `s` (one add each) that fold()
// moves into the compensated pair (hi, lo) with TwoSum every 64 additions.
// Each add to the short sum rounds by at most 2^-24 |s| <= 2^-18 of the
// largest increment, so over a run the sum carries at most 2^-18 relative
// error (much less on average, the roundings being of both signs), and the
// pair adds nothing more.  A fold costs the whole warp while one or two of
// its lanes need it, so it is kept rare.
template <>
struct Acc<float> {
    float hi, lo, s;
    __device__ __forceinline__ void set(double v)
    {
        hi = (float)v;
        lo = (float)(v - (double)hi);
        s = 0.0f;
    }
    __device__ __forceinline__ void add(float b) { s += b; }
    __device__ __forceinline__ void fold()
    {
        const float t = hi + s;
        const float bb = t - hi;
        const float e = (hi - (t - bb)) + (s - bb);
        hi = t;
        lo += e;
        s = 0.0f;
    }
    __device__ __forceinline__ double value() const { return ((double)hi + (double)s) + (double)lo; }
};
template <>
struct Acc<double> {
    double v;
    __device__ __forceinline__ void set(double x) { v = x; }
    __device__ __forceinline__ void add(double b) { v += b; }
    __device__ __forceinline__ void fold() {}
    __device__ __forceinline__ double value() const { return v; }
};

// ---------------------------------------------------------------------------
// Tables
// ---------------------------------------------------------------------------
template <typename R>
struct Tab {
    const Rec<R> *rec;
    const uint16_t *bucket;
    const ChParam<R> *chp;
    const ChVal<R> *chval;
    const ChVal<R> *cum;   // cumulative channel values (global memory)
    const uint8_t *guide;  // guide rows of the search (null: bisection only)
    const R *binmax;  // sparse table of per-bin maxima (level-major)
    const ChVal<R> *gval;  // per-record, per-gas density sums (global memory)
    const Layout *lay;     // gas channel ranges
    int n_rec, n_buckets, n_ch, first_tail, n_bins, n_gases;
    int ch_steps;          // bisection steps over n_ch channels: ceil(log2 n_ch)
    float log2_lo, inv_bw, bin_lo, inv_binw;
    R nu_low, g_top, s_min;  // s_min: speed at the first bin edge [m/s]
};

// Table views of a mixture: the staged prefix (`staged` bytes) in shared
// memory, the rest in global memory.  Every constant comes from the host's
// layout, so setting up a tile does no FP64 arithmetic.
template <typename R>
__device__ __forceinline__ Tab<R> make_tab(const uint8_t *smem, const uint8_t *blob, const Layout &L, bool ch_smem,
                                           uint32_t staged)
{
    Tab<R> T;
    T.rec = (const Rec<R> *)smem;
    T.bucket = (const uint16_t *)(smem + L.off_bucket);
    T.chp = (const ChParam<R> *)(smem + L.off_chp);
    T.chval = (const ChVal<R> *)((ch_smem ? smem : blob) + L.off_chval);
    T.cum = (const ChVal<R> *)(blob + L.off_cum);
    T.guide = L.off_guide ? blob + L.off_guide : nullptr;
    T.n_rec = L.n_rec;
    T.n_buckets = L.n_buckets;
    T.n_ch = L.n_ch;
    T.ch_steps = L.n_ch > 1 ? 32 - __clz(L.n_ch - 1) : 0;
    T.first_tail = L.first_tail_rec;
    T.log2_lo = L.log2_lo;
    T.inv_bw = L.inv_bw;
    T.binmax = (const R *)((staged >= L.bin_end ? smem : blob) + L.off_bin);
    T.n_bins = L.n_bins;
    T.bin_lo = L.bin_lo;
    T.inv_binw = L.inv_binw;
    T.nu_low = (R)L.nu_low;
    T.g_top = (R)L.g_top;
    T.s_min = (R)L.s_min;
    T.gval = (const ChVal<R> *)(blob + L.off_gval);
    T.lay = &L;
    T.n_gases = L.n_gases;
    return T;
}

// Sum of the power-law tails of the channels whose table ends at or below
// the record's lower edge (Sec. 2.2, Eqs. 12-14).
template <typename R>
__device__ __noinline__ R tail_sum(const Tab<R> &T, R eps, R e_lo)
{
    const R le = log_(eps);
    R S = 0;
    for (int j = 0; j < T.n_ch; ++j) {
        const ChParam<R> p = T.chp[j];
        if (e_lo >= p.e_last && !(p.bits & 0x100)) S += exp_(p.tail_logc + p.tail_K * le);
    }
    return S;
}

// Density sum S(eps) = sum n_k sigma_kj(eps) [1/m] and the record holding eps.
template <typename R>
__device__ __forceinline__ R density(const Tab<R> &T, R eps, int &ri, R &e_lo)
{
    float fb = (__log2f((float)eps) - T.log2_lo) * T.inv_bw;
    fb = fminf(fmaxf(fb, 0.0f), (float)(T.n_buckets - 1));
    int i = T.bucket[(int)fb];
    Rec<R> r = T.rec[i];
    while (i > 0 && eps < r.e_lo) r = T.rec[--i];
    while (i < T.n_rec - 1 && eps >= r.e_hi) r = T.rec[++i];
    R S = r.S_lo + r.slope * (eps - r.e_lo);
    if (i >= T.first_tail) S += tail_sum(T, eps, r.e_lo);
    ri = i;
    e_lo = r.e_lo;
    return S;
}

// One {val, slope} pair: from shared memory, or from global memory in one
// 8-byte (FP32) or 16-byte (FP64) read-only load.
__device__ __forceinline__ ChVal<float> ldg_chval(const ChVal<float> *p)
{
    const float2 v = __ldg(reinterpret_cast<const float2 *>(p));
    ChVal<float> c;
    c.val = v.x;
    c.slope = v.y;
    return c;
}
__device__ __forceinline__ ChVal<double> ldg_chval(const ChVal<double> *p)
{
    const double2 v = __ldg(reinterpret_cast<const double2 *>(p));
    ChVal<double> c;
    c.val = v.x;
    c.slope = v.y;
    return c;
}

template <typename R>
__device__ __forceinline__ ChVal<R> load_chval(const ChVal<R> *p, bool ch_smem)
{
    if (ch_smem) return *p;
    return ldg_chval(p);
}

// First channel whose cumulative density reaches `target` (= R nu'/|v|),
// in the order of Eq. (2): gas by gas, channel by channel.  Outside the
// power-law tails the search is two-level: per-gas sums find the gas, then
// that gas's channels are scanned (the same cumulative partition).
//
// Where the channel values are not staged (many channels, read through L1
// from global memory), the search runs on the record's cumulative values
// instead: the first j whose cumulative value reaches the target.  A guide
// proposes where to look: the target's fraction u of the density sum S
// names one of kGuide buckets, and each record end's guide row names the
// first channel that reaches the bucket's lower fraction there; every
// channel's share of the cumulative sum varies monotonically between the
// record's ends, so the answer cannot lie below the smaller of the two ends'
// entries (L) nor above the larger of the next bucket's (U).  One round trip
// reads the guide bytes and the record's total, a second the cumulative
// values at L - 1, L and L + 1; 97 % of the searches end there (256
// buckets, the 256-swarm workload's mixtures).  The cumulative values
// decide, not the guide: if rounding left the answer below L or above U,
// or in a wide bucket, a bisection finishes the search, so the result is
// always the first index reaching the target.  (Bisecting the whole row took
// ceil(log2 n_ch) dependent trips to L2 per real collision; a 16-ary search
// tree took two, but read four times the bytes and needed more registers:
// 12 % slower.)  The target is first clamped to the record's total: where
// rounding leaves it a hair above, the search lands on the last channel that
// adds to the total (the first entry equal to it).  Every entry is evaluated
// with the same fused multiply-add, so the clamp and the search agree.
__device__ __forceinline__ float fma_(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_(double a, double b, double c) { return fma(a, b, c); }

template <typename R>
__device__ __forceinline__ R cum_at(const ChVal<R> &c, R de)
{
    return fma_(c.slope, de, c.val);
}

// First j in [lo, hi] whose cumulative value reaches the target, or hi
// (whose value the caller knows to reach it).
template <typename R>
__device__ __noinline__ int cum_lower_bound(const ChVal<R> *row, int lo, int hi, R de, R target)
{
    int base = lo, len = hi - lo + 1;
    while (len > 1) {
        const int half = len >> 1;
        if (cum_at(ldg_chval(row + base + half - 1), de) < target) base += half;
        len -= half;
    }
    return base;
}

template <typename R, bool CH_SMEM>
__device__ __forceinline__ int select_channel(const Tab<R> &T, int ri, R e_lo, R eps, R target, R S)
{
    const R de = eps - e_lo;
    if (!CH_SMEM && ri < T.first_tail) {
        const int n = T.n_ch;
        const ChVal<R> *row = T.cum + (size_t)ri * n;
        const ChVal<R> top = ldg_chval(row + n - 1);
        if (T.guide) {
            const uint8_t *gl = T.guide + (size_t)ri * kGuide, *gh = gl + kGuide;
            const float u = (S > (R)0) ? (float)(target / S) : 0.0f;
            const int b = min(max((int)(u * (float)kGuide), 0), kGuide - 1);
            const int L = min((int)__ldg(gl + b), (int)__ldg(gh + b));
            const int U = (b + 1 < kGuide) ? max((int)__ldg(gl + b + 1), (int)__ldg(gh + b + 1)) : n - 1;
            target = min_(target, cum_at(top, de));
            const R v0 = cum_at(ldg_chval(row + L), de);
            const R v1 = cum_at(ldg_chval(row + min(L + 1, n - 1)), de);
            const R vm = cum_at(ldg_chval(row + max(L - 1, 0)), de);
            if (L > 0 && !(vm < target)) return cum_lower_bound(row, 0, L - 1, de, target);  // below L (rounding)
            if (!(v0 < target)) return L;
            if (!(v1 < target)) return min(L + 1, n - 1);
            // a bucket with several channels, or the answer above U by rounding
            const int hi = min(max(U, L + 2), n - 1);
            if (cum_at(ldg_chval(row + hi), de) < target) return cum_lower_bound(row, hi + 1, n - 1, de, target);
            return cum_lower_bound(row, L + 2, hi, de, target);
        }
        target = min_(target, cum_at(top, de));
        int base = 0, len = n;
        // the answer lies in [base, base + len): each step halves len
        for (int k = 0; k < T.ch_steps; ++k) {
            const int half = len >> 1;
            if (cum_at(ldg_chval(row + base + half - 1), de) < target) base += half;
            len -= half;
        }
        return base;
    }
    if (ri < T.first_tail && T.n_gases > 1) {
        const ChVal<R> *grow = T.gval + (size_t)ri * T.n_gases;
        R cum = 0;
        int g = 0;
        for (; g < T.n_gases - 1; ++g) {
            const ChVal<R> gv = load_chval(grow + g, false);
            const R d = gv.val + gv.slope * de;
            if (cum + d >= target) break;
            cum += d;
        }
        const int j0 = T.lay->gas_first[g], j1 = j0 + T.lay->gas_count[g];
        const ChVal<R> *row = T.chval + (size_t)ri * T.n_ch;
        int last = j0;
        for (int j = j0; j < j1; ++j) {
            const ChVal<R> cv = load_chval(row + j, CH_SMEM);
            const R d = cv.val + cv.slope * de;
            if (d > (R)0) last = j;
            cum += d;
            if (cum >= target) return j;
        }
        return last;  // rounding left the sum a hair short: last open channel of that gas
    }
    const ChVal<R> *row = T.chval + (size_t)ri * T.n_ch;
    const bool tails = ri >= T.first_tail;
    const R le = tails ? log_(eps) : (R)0;
    R cum = 0;
    int last = 0;
    for (int j = 0; j < T.n_ch; ++j) {
        const ChVal<R> cv = load_chval(row + j, CH_SMEM);
        R d = cv.val + cv.slope * de;
        if (tails) {
            const ChParam<R> p = T.chp[j];
            if (e_lo >= p.e_last && !(p.bits & 0x100)) d += exp_(p.tail_logc + p.tail_K * le);
        }
        if (d > (R)0) last = j;
        cum += d;
        if (cum >= target) return j;
    }
    return last;  // rounding left the sum a hair short of S: last channel that is open
}

// Right side of Eq. 7, r(xi) = (1 - xi)/(2 xi^2) ((1 + xi) ln((1 + xi)/(1 - xi)) - 2 xi),
// and its derivative; for |xi| < 0.2, where the bracket cancels, from the
// series 1 - 2 sum_k xi^(2k+1) / ((2k+1)(2k+3)) (the logarithm expanded).
template <typename R>
__device__ __forceinline__ void xi_ratio(R xi, R &f, R &df)
{
    if (fabs(xi) < (R)0.2) {
        const R x2 = xi * xi;
        R p = 1, s = 0, ds = 0;
#pragma unroll
        for (int k = 0; k < 14; ++k) {
            ds += p / (R)(2 * k + 3);
            s += p * xi / (R)((2 * k + 1) * (2 * k + 3));
            p *= x2;
        }
        f = (R)1 - (R)2 * s;
        df = (R)-2 * ds;
    } else {
        const R L = log_(((R)1 + xi) / ((R)1 - xi));
        const R A = ((R)1 + xi) * L - (R)2 * xi;
        f = ((R)1 - xi) * A / ((R)2 * xi * xi);
        df = ((R)2 - L) / xi - ((R)1 - xi) * A / (xi * xi * xi);
    }
}

// xi with r(xi) = r: Newton steps kept inside a bisection bracket of
// (-1, 1), on which r falls from 2 to 0.
template <typename R>
__device__ __forceinline__ R xi_solve(R r)
{
    const R lim = (sizeof(R) == 4) ? (R)0.9999 : (R)0.99999999;
    R lo = -lim, hi = lim;
    R x = min_(max_((R)1.5 * ((R)1 - r), (R)-0.9), (R)0.9);
    const R tol = (sizeof(R) == 4) ? (R)1e-6 : (R)1e-14;
    for (int it = 0; it < 80; ++it) {
        R f, df;
        xi_ratio(x, f, df);
        const R d = f - r;
        if (d > (R)0) lo = x;  // r falls with xi: the root lies above
        else hi = x;
        R xn = x - d / df;
        if (!(xn > lo && xn < hi)) xn = (R)0.5 * (lo + hi);
        const bool done = fabs(xn - x) <= tol;
        x = xn;
        if (done || hi - lo <= tol) break;
    }
    return x;
}

// Eq. 6 for a channel of an xi-form gas: xi from the ratio of the gas's
// momentum-transfer cross section (its elastic channel) to its total
// elastic one at eps, both read on record ri (or from their tails).
template <typename R, bool CH_SMEM>
__device__ __noinline__ R xi_cos_theta(const Tab<R> &T, const RunArgs &P, int bits, int ri, R e_lo, R eps, R u)
{
    const int g = (bits >> 12) & 15, cel = (bits >> 16) & 0xFFFF;
    const R de = eps - e_lo;
    const ChVal<R> cv = load_chval(T.chval + (size_t)ri * T.n_ch + cel, CH_SMEM);
    R smt = cv.val + cv.slope * de;
    const ChParam<R> pm = T.chp[cel];
    if (e_lo >= pm.e_last && !(pm.bits & 0x100)) smt += exp_(pm.tail_logc + pm.tail_K * log_(eps));
    const ChVal<R> *elv = (const ChVal<R> *)(P.blob + P.lay.off_elval);
    const ChParam<R> *elp = (const ChParam<R> *)(P.blob + P.lay.off_elp);
    const ChVal<R> ev = load_chval(elv + (size_t)ri * T.n_gases + g, false);
    R sel = ev.val + ev.slope * de;
    const R e_last = __ldg(&elp[g].e_last);
    if (e_lo >= e_last && !(__ldg(&elp[g].bits) & 0x100))
        sel += exp_(__ldg(&elp[g].tail_logc) + __ldg(&elp[g].tail_K) * log_(eps));
    const R xi = (sel > (R)0) ? xi_solve(smt / sel) : (R)0;
    return (R)1 - (R)2 * u * ((R)1 - xi) / ((R)1 + xi * ((R)1 - (R)2 * u));
}

template <typename R>
struct Fld {
    R a, b0, b1, b2, w, inv_w, vD0, vD1, vD2, vDn, a_par, Ke;
    R inv_a, inv_apar;  // 1/a and 1/|a_par| (0 where those vanish)
    int has_b;
};

template <typename R>
__device__ __forceinline__ Fld<R> make_fld(const Fields &f)
{
    Fld<R> F;
    F.has_b = f.has_b;
    if constexpr (sizeof(R) == 4) {  // the host's FP32 copies
        const Fields32 &g = f.f32;
        F.a = g.a;
        F.b0 = g.b0;
        F.b1 = g.b1;
        F.b2 = g.b2;
        F.w = g.w;
        F.inv_w = g.inv_w;
        F.vD0 = g.vD0;
        F.vD1 = g.vD1;
        F.vD2 = g.vD2;
        F.vDn = g.vDn;
        F.a_par = g.a_par;
        F.Ke = g.Ke;
        F.inv_a = g.inv_a;
        F.inv_apar = g.inv_apar;
        return F;
    }
    F.a = (R)f.a;
    F.b0 = (R)f.b[0];
    F.b1 = (R)f.b[1];
    F.b2 = (R)f.b[2];
    F.w = (R)f.w;
    F.inv_w = f.has_b ? (R)(1.0 / f.w) : (R)0;
    F.vD0 = (R)f.vD[0];
    F.vD1 = (R)f.vD[1];
    F.vD2 = (R)f.vD[2];
    F.vDn = (R)sqrt(f.vD[0] * f.vD[0] + f.vD[1] * f.vD[1] + f.vD[2] * f.vD[2]);
    F.a_par = (R)f.a_par;
    F.Ke = (R)(0.5 * kMe / kQe);  // eV per (m/s)^2
    F.inv_a = f.a > 0.0 ? (R)(1.0 / f.a) : (R)0;
    F.inv_apar = f.a_par != 0.0 ? (R)(1.0 / fabs(f.a_par)) : (R)0;
    return F;
}

// ---------------------------------------------------------------------------
// Particle state
// ---------------------------------------------------------------------------
template <typename R>
struct PState {
    R vr0, vr1, vr2;         // velocity right after the last real collision
    R T;                     // time since then
    R nu_p, inv_nu;          // trial frequency of this particle
    R T_wend;                // windowed trial frequency: end of the current window (time since last real)
    R u0x, u0y, u0z, bux, buy, buz;  // B != 0: u0 = v_perp - vD and b x u0 at the last real collision
    Acc<R> x, y, z, t;       // position and time at the last real collision, relative to birth
    Acc<R> se, se2;          // energy sums before / after real collisions
    double t0;               // birth time (absolute)
    R t_left;                // FP32 runs with t_end: time from the last real collision to t_end
    uint32_t id_lo, id_hi, k, n_real, n_null, n_fail, n_ion, n_att, status;
    bool done;
    uint32_t grace;          // adaptive trial frequencies: collisions left before the next query
    bool retried;            // BINNED: nu' comes from a retry after a fail
};

// Time left until t_end, from the last real collision.  The FP32 step keeps it
// in FP32 and takes the flight time of each real collision off it; it is set
// exactly (in FP64) at birth and again at every fold of the time sum, so it
// carries at most 64 FP32 roundings of the remaining time.
template <typename R>
__device__ __forceinline__ void set_t_left(const RunArgs &P, PState<R> &s)
{
    if (P.timed) s.t_left = (R)(P.t_end - s.t0 - s.t.value());
}

template <typename R, bool BF = true>
__device__ __forceinline__ void set_b_cache(const Fld<R> &F, PState<R> &s)
{
    if (!BF || !F.has_b) return;
    const R vpar = s.vr0 * F.b0 + s.vr1 * F.b1 + s.vr2 * F.b2;
    s.u0x = s.vr0 - vpar * F.b0 - F.vD0;
    s.u0y = s.vr1 - vpar * F.b1 - F.vD1;
    s.u0z = s.vr2 - vpar * F.b2 - F.vD2;
    s.bux = F.b1 * s.u0z - F.b2 * s.u0y;
    s.buy = F.b2 * s.u0x - F.b0 * s.u0z;
    s.buz = F.b0 * s.u0y - F.b1 * s.u0x;
}

// Velocity after time T since the last real collision.  With B != 0 the
// velocity splits into the part along b (accelerated by a_par), the E x B
// drift vD and u = v_perp - vD rotating about b at w; written as a change of
// the velocity at the last collision,
//   v(T) = v_r + a_par T b - u0 (1 - cos wT) + (b x u0) sin wT,
// so that rounding stays relative to the change even when |vD| >> |v|.
// Returns sn = sin wT and omc = 1 - cos wT (without cancellation).
template <typename R, bool BF = true>
__device__ __forceinline__ void velocity_at(const Fld<R> &F, const PState<R> &s, R T, R &v0, R &v1, R &v2, R &sn,
                                            R &omc)
{
    if (BF && F.has_b) {
        R cs;
        sincos_(F.w * T, &sn, &cs);
        omc = (cs > (R)0) ? fdiv_(sn * sn, (R)1 + cs) : (R)1 - cs;  // 1 - cos, no cancellation
        const R ap = F.a_par * T;
        v0 = s.vr0 + ap * F.b0 - s.u0x * omc + s.bux * sn;
        v1 = s.vr1 + ap * F.b1 - s.u0y * omc + s.buy * sn;
        v2 = s.vr2 + ap * F.b2 - s.u0z * omc + s.buz * sn;
    } else {
        sn = 0;
        omc = 0;
        v0 = s.vr0;
        v1 = s.vr1;
        v2 = s.vr2 + F.a * T;
    }
}

// sin(x) - x, accurate also for small x (Taylor series below |x| = 3/4).
template <typename R>
__device__ __forceinline__ R sin_minus_x(R x, R sn)
{
    if (fabs(x) >= (R)0.75) return sn - x;
    const R y = x * x;
    R p = (R)(1.0 / 1307674368000.0);
    p = (R)(1.0 / 6227020800.0) - y * p;
    p = (R)(1.0 / 39916800.0) - y * p;
    p = (R)(1.0 / 362880.0) - y * p;
    p = (R)(1.0 / 5040.0) - y * p;
    p = (R)(1.0 / 120.0) - y * p;
    p = (R)(1.0 / 6.0) - y * p;
    return -x * y * p;
}

// Displacement after time T since the last real collision:
//   dx = v_r T + a_par T^2/2 b + [u0 (sin wT - wT) + (b x u0)(1 - cos wT)] / w.
template <typename R, bool BF = true>
__device__ __forceinline__ void displacement(const Fld<R> &F, const PState<R> &s, R T, R sn, R omc, R &dx, R &dy,
                                             R &dz)
{
    if (BF && F.has_b) {
        const R smx = sin_minus_x(F.w * T, sn);
        const R hp = (R)0.5 * F.a_par * T * T;
        dx = s.vr0 * T + hp * F.b0 + (s.u0x * smx + s.bux * omc) * F.inv_w;
        dy = s.vr1 * T + hp * F.b1 + (s.u0y * smx + s.buy * omc) * F.inv_w;
        dz = s.vr2 * T + hp * F.b2 + (s.u0z * smx + s.buz * omc) * F.inv_w;
    } else {
        dx = s.vr0 * T;
        dy = s.vr1 * T;
        dz = s.vr2 * T + (R)0.5 * F.a * T * T;
    }
}

// ---------------------------------------------------------------------------
// Windowed local trial frequency.  Over a window of length dt that starts
// with speed |v|, the speed stays within |v| +- g with g = a dt (B = 0) or
// g = |a_par| dt + |u0| min(2, w dt) (B != 0: |u(t) - u(t0)| = 2|u0||sin(w(t-t0)/2)|),
// so the maximum of nu over the energies [eps(|v|-g), eps(|v|+g)] -- read
// from per-bin maxima of nu, 1/32 of a bin of margin on each side, plus a bound
// of the power-law tails above the last union point -- is a trial frequency
// that holds for the whole window.  A flight longer than the window stops
// at its end and a new window starts there: by the memorylessness of the
// exponential flight this samples the same process as a constant nu'
// (Eqs. 3-4), with fewer null collisions.
// ---------------------------------------------------------------------------
// The lower bound of any trial frequency in the step's precision.  GB300 runs
// FP64 at a small fraction of the FP32 rate, so the FP32 step takes the FP32
// copy the host made rather than converting the double on every trial.
template <typename R>
__device__ __forceinline__ R nu_floor_of(const RunArgs &P);
template <>
__device__ __forceinline__ float nu_floor_of<float>(const RunArgs &P) { return P.nu_floor32; }
template <>
__device__ __forceinline__ double nu_floor_of<double>(const RunArgs &P) { return P.nu_floor; }
// The Maxwellian start's per-component spread and the starting nu', in the
// step's precision (the FP32 step reads the host's FP32 copies).
template <typename R>
__device__ __forceinline__ R v0_scale_of(const RunArgs &P);
template <>
__device__ __forceinline__ float v0_scale_of<float>(const RunArgs &P) { return P.v0_scale32; }
template <>
__device__ __forceinline__ double v0_scale_of<double>(const RunArgs &P) { return P.v0_scale; }
template <typename R>
__device__ __forceinline__ R nu0_of(const RunArgs &P);
template <>
__device__ __forceinline__ float nu0_of<float>(const RunArgs &P) { return P.nu0_32; }
template <>
__device__ __forceinline__ double nu0_of<double>(const RunArgs &P) { return P.nu0; }
template <typename R>
__device__ __forceinline__ R kT_m_of(const RunArgs &P);
template <>
__device__ __forceinline__ float kT_m_of<float>(const RunArgs &P) { return P.kT_m32; }
template <>
__device__ __forceinline__ double kT_m_of<double>(const RunArgs &P) { return P.kT_m; }

template <typename R>
__device__ __forceinline__ float bin_pos(const Tab<R> &T, R eps)
{
    return (__log2f((float)eps) - T.bin_lo) * T.inv_binw;
}

template <typename R>
__device__ __forceinline__ int bin_of(const Tab<R> &T, R eps)
{
    const float fb = fminf(fmaxf(bin_pos(T, eps), -1.0f), (float)T.n_bins);
    return (int)floorf(fb);  // -1 below the first bin, n_bins above the last
}

// Upper bound of nu over [a, b] with a >= g_top: every channel is on its
// power-law tail there, each term is monotone, so it peaks at an end.
template <typename R>
__device__ __noinline__ R tail_bound(const Tab<R> &T, R a, R b)
{
    const R la = log_(a), lb = log_(b);
    R S = 0;
    for (int j = 0; j < T.n_ch; ++j) {
        const ChParam<R> p = T.chp[j];
        if (p.bits & 0x100) continue;
        S += max_(exp_(p.tail_logc + p.tail_K * la), exp_(p.tail_logc + p.tail_K * lb));
    }
    return sqrt_(b * (R)(2.0 * kQe / kMe)) * S;
}

template <typename R>
__device__ __forceinline__ R window_majorant(const Tab<R> &T, R e_lo, R e_hi)
{
    // Bins met by [e_lo, e_hi], the positions widened by 1/32 of a bin (0.2 %
    // in energy): many times the FP32 rounding of the positions, of the
    // energy bounds and of the energies the flight then reaches.
    const float pl = fmaxf(bin_pos(T, e_lo) - 0.03125f, -1.0f), ph = fminf(bin_pos(T, e_hi) + 0.03125f, (float)T.n_bins);
    int bl = (int)floorf(pl), bh = (int)floorf(ph);
    R m = 0;
    if (bl < 0) {
        m = T.nu_low;
        bl = 0;
    }
    if (bh > T.n_bins - 1) bh = T.n_bins - 1;
    if (bh >= bl) {  // range maximum from two entries of the sparse table
        const int len = bh - bl + 1, l = 31 - __clz(len);
        const R *lev = T.binmax + (size_t)l * T.n_bins;
        m = max_(m, max_(lev[bl], lev[bh - (1 << l) + 1]));
    }
    if (e_hi >= T.g_top) m = max_(m, tail_bound(T, max_(e_lo, T.g_top), e_hi));
    return m;
}

// The window lasts win_c / nu of the current energy bin, and at most as long
// as the speed bound needs to grow by a quarter of the speed (plus the speed
// of the lowest table energy), so that a strong field cannot stretch the
// energy range -- and the tails of the tables -- far beyond the electron's.
// With B != 0 a second bound holds for any window length: the velocity is
// v_par(t) b + vD + u(t) with vD, u perpendicular to b and |u| = |u0|, so
// |v|^2 lies between v_par^2 + (|vD| - |u0|)^2 and v_par^2 + (|vD| + |u0|)^2;
// the window then only has to bound the change of v_par, and the tighter of
// the two bounds is used.
template <typename R, bool BF = true>
__device__ __forceinline__ void window_of(const Tab<R> &T, const Fld<R> &F, const RunArgs &P, const PState<R> &s, R v0,
                                          R v1, R v2, R t0, R &nu_p, R &inv_nu, R &t_wend)
{
    const R speed = sqrt_(v0 * v0 + v1 * v1 + v2 * v2);
    const R eps = F.Ke * speed * speed;
    const int b = bin_of(T, eps);
    const R nub = max_((b < 0) ? T.nu_low : T.binmax[b < T.n_bins ? b : T.n_bins - 1], nu_floor_of<R>(P));
    R dt = fdiv_((R)P.win_c, nub);  // any positive length is exact
    const R grow_max = (R)0.25 * speed + T.s_min;
    R s_hi, s_lo;
    if (BF && F.has_b) {
        const R u0n = sqrt_(s.u0x * s.u0x + s.u0y * s.u0y + s.u0z * s.u0z);
        const R apar = fabs(F.a_par);
        if (apar * dt > grow_max) dt = grow_max * F.inv_apar;
        R wdt = F.w * dt;
        if (wdt > (R)2) wdt = (R)2;
        const R grow = apar * dt + u0n * wdt;  // |v(t) - v(t0)| <= |a_par| dt + |u0| min(2, w dt)
        const R vp = fabs(v0 * F.b0 + v1 * F.b1 + v2 * F.b2);
        const R vp_hi = vp + apar * dt, vp_lo = max_((R)0, vp - apar * dt);
        const R g_hi = F.vDn + u0n, g_lo = F.vDn - u0n;
        s_hi = min_(speed + grow, sqrt_(vp_hi * vp_hi + g_hi * g_hi));
        s_lo = max_(max_((R)0, speed - grow), sqrt_(vp_lo * vp_lo + g_lo * g_lo));
    } else {
        if (F.a * dt > grow_max) dt = grow_max * F.inv_a;
        const R grow = F.a * dt;
        s_hi = speed + grow;
        s_lo = max_((R)0, speed - grow);
    }
    const R m = max_(window_majorant(T, F.Ke * s_lo * s_lo, F.Ke * s_hi * s_hi) * (R)(1.0 + 1e-5), nu_floor_of<R>(P));
    nu_p = m;
    inv_nu = fdiv_((R)1, m);  // 2 ulp in FP32: the flights' rate is nu' to ~1e-7
    t_wend = t0 + dt;
}

template <typename R, bool BF = true>
__device__ __forceinline__ void new_window(const Tab<R> &T, const Fld<R> &F, const RunArgs &P, PState<R> &s, R v0,
                                           R v1, R v2, R t0)
{
    window_of<R, BF>(T, F, P, s, v0, v1, v2, t0, s.nu_p, s.inv_nu, s.T_wend);
}

// BinnedTrialFrequency (Sec. 6.3): the maximum of nu over the energy bin of
// eps, bin j = [10^(j/B), 10^((j+1)/B)) with j = floor(B log10 eps).  The
// compiled bins lie on the lattice 10^(i/fpd) and B divides fpd, so bin j is
// the run of compiled bins [j fpd/B, (j+1) fpd/B): its maximum comes from
// two entries of the sparse table.  Below the compiled bins nu grows as
// sqrt(eps) (a constant density sum) when the layout says so, else nu_low
// bounds it; above them the power-law tails are bounded per channel.
template <typename R>
__device__ R binned_max(const Tab<R> &T, const RunArgs &P, R eps)
{
    if (!(eps > (R)0)) return (R)0;
    const int fpd = P.lay.bins_per_decade, B = P.tf_B, m = fpd / B, j0 = P.lay.bin_j0;
    const int j = (int)floor_((R)B * log10_(eps));
    int lo = j * m - j0;
    const int hi = lo + m - 1;
    if (hi < 0) {
        if (!P.lay.low_sqrt) return T.nu_low;
        // nu_low is nu at the first compiled edge 10^(j0/fpd)
        return T.nu_low * exp10_((R)0.5 * ((R)(j + 1) / (R)B - (R)j0 / (R)fpd));
    }
    if (lo < 0) lo = 0;  // the part below is dominated by the first compiled bin
    R mx = (R)0;
    if (lo < T.n_bins) {
        const int h = hi < T.n_bins ? hi : T.n_bins - 1;
        const int l = 31 - __clz(h - lo + 1);
        const R *lev = T.binmax + (size_t)l * T.n_bins;
        mx = max_(lev[lo], lev[h - (1 << l) + 1]);
    }
    if (hi >= T.n_bins) {
        const R a = max_(exp10_((R)(j0 + T.n_bins) / (R)fpd), exp10_((R)j / (R)B));
        mx = max_(mx, tail_bound(T, a, exp10_((R)(j + 1) / (R)B)));
    }
    return mx;
}

// nu' of the adaptive strategies at energy eps where nu = nu(eps) is known
// (Sec. 6): VARIABLE (1 + zeta) nu, BINNED the maximum over eps's bin; not
// below nu_floor, nu at the lowest table energy (nu vanishes at rest).
template <typename R>
__device__ __forceinline__ R adaptive_nu(const Tab<R> &T, const RunArgs &P, R eps, R nu)
{
    if (P.tf == TF_VARIABLE) return (R)P.tf_zeta1 * max_(nu, nu_floor_of<R>(P));
    return max_(binned_max(T, P, eps), nu_floor_of<R>(P));
}

// nu(eps) from the tables (Eq. 2), for queries at an energy the step has
// not evaluated.
template <typename R>
__device__ __forceinline__ R nu_at(const Tab<R> &T, const Fld<R> &F, R eps)
{
    int ri;
    R elo;
    return sqrt_(eps / F.Ke) * density(T, eps, ri, elo);
}

template <typename R>
__device__ __forceinline__ R density_at(const Tab<R> &T, R eps)
{
    int ri;
    R elo;
    return density(T, eps, ri, elo);
}

// First query of an electron's nu' (VARIABLE, BINNED) at its start.
template <typename R>
__device__ __forceinline__ void adaptive_start(const Tab<R> &T, const Fld<R> &F, const RunArgs &P, PState<R> &s)
{
    const R eps = F.Ke * (s.vr0 * s.vr0 + s.vr1 * s.vr1 + s.vr2 * s.vr2);
    s.nu_p = adaptive_nu(T, P, eps, P.tf == TF_VARIABLE ? nu_at(T, F, eps) : (R)0);
    s.inv_nu = (R)1 / s.nu_p;
    s.grace = P.tf_grace;
    s.retried = false;
}

template <typename R, bool BF = true>
__device__ __forceinline__ void init_particle(const Tab<R> &T, const RunArgs &P, const Fld<R> &F, PState<R> &s,
                                              uint64_t id)
{
    s.id_lo = (uint32_t)id;
    s.id_hi = (uint32_t)(id >> 32);
    const uint4 w = philox(s.id_lo, s.id_hi, 0u, 2u, P.key0, P.key1);
    // isotropic Maxwellian with mean energy eps0 = 3/2 kT (Box-Muller)
    const R sv = v0_scale_of<R>(P);
    const R r0 = sqrt_((R)-2 * log_(uni<R>(w.x))), r1 = sqrt_((R)-2 * log_(uni<R>(w.z)));
    R s1, c1, s3, c3;
    sincospi_((R)2 * uni<R>(w.y), &s1, &c1);
    sincospi_((R)2 * uni<R>(w.w), &s3, &c3);
    s.vr0 = sv * r0 * c1;
    s.vr1 = sv * r0 * s1;
    s.vr2 = sv * r1 * c3;
    s.T = 0;
    s.nu_p = nu0_of<R>(P);
    s.inv_nu = (R)1 / s.nu_p;
    s.x.set(0.0);
    s.y.set(0.0);
    s.z.set(0.0);
    s.t.set(0.0);
    s.se.set(0.0);
    s.se2.set(0.0);
    s.k = 0;
    s.n_real = s.n_null = s.n_fail = s.n_ion = s.n_att = 0;
    s.status = ST_DONE;
    s.done = false;
    s.t0 = 0.0;
    set_t_left(P, s);
    set_b_cache<R, BF>(F, s);
    s.T_wend = (R)0;
    if (P.window) new_window<R, BF>(T, F, P, s, s.vr0, s.vr1, s.vr2, (R)0);
}

// Spawn mode: the electron in secondary slot j starts from its birth record.
template <typename R, bool BF = true>
__device__ __forceinline__ void init_secondary(const Tab<R> &T, const RunArgs &P, const Fld<R> &F, PState<R> &s,
                                               uint64_t j)
{
    // the record was published by another SM: read it from L2
    const uint64_t id = __ldcg(P.bid + j);
    s.id_lo = (uint32_t)id;
    s.id_hi = (uint32_t)(id >> 32);
    s.vr0 = (R)__ldcg(P.bvx + j);
    s.vr1 = (R)__ldcg(P.bvy + j);
    s.vr2 = (R)__ldcg(P.bvz + j);
    s.T = 0;
    s.nu_p = nu0_of<R>(P);
    s.inv_nu = (R)1 / s.nu_p;
    s.x.set(0.0);
    s.y.set(0.0);
    s.z.set(0.0);
    s.t.set(0.0);
    s.se.set(0.0);
    s.se2.set(0.0);
    s.k = 0;
    s.n_real = s.n_null = s.n_fail = s.n_ion = s.n_att = 0;
    s.status = ST_DONE;
    s.done = false;
    s.t0 = __ldcg(P.bt + j);
    set_t_left(P, s);
    set_b_cache<R, BF>(F, s);
    s.T_wend = (R)0;
    if (P.window) new_window<R, BF>(T, F, P, s, s.vr0, s.vr1, s.vr2, (R)0);
}

// Id of the electron created by the ionization at `step` of electron
// `parent`: the SplitMix64 finaliser (Steele, Lea, Flood 2014) of
// parent * 0x9E3779B97F4A7C15 + step + 1, top bit set (never a primary id).
__device__ __forceinline__ uint64_t secondary_id(uint64_t parent, uint32_t step)
{
    uint64_t z = parent * 0x9E3779B97F4A7C15ull + (uint64_t)step + 1ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return z | 0x8000000000000000ull;
}

__device__ __forceinline__ void st_release(uint64_t *p, uint64_t v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint64_t ld_acquire(const uint64_t *p)
{
    uint64_t v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Appends the secondary of an ionization: one atomic per group of lanes
// that ionize in the same step (warp-aggregated) takes their slots and
// counts them as pending before any of them can finish; the birth record
// is written at the slot and published by storing the id last (release).
template <typename R>
__device__ __noinline__ void spawn_secondary(const RunArgs &P, R Ke, double t_birth, uint64_t parent, uint32_t step,
                                             R es, R u_cos, R u_phi)
{
    namespace cg = cooperative_groups;
    cg::coalesced_group g = cg::coalesced_threads();
    unsigned long long base = 0;
    if (g.thread_rank() == 0) {
        base = atomicAdd(P.n_total, (unsigned long long)g.size());
        const unsigned long long made = base >= P.cap ? 0ull : min((unsigned long long)g.size(), P.cap - base);
        if (made) atomicAdd(P.pending, made);
    }
    g.sync();
    base = g.shfl(base, 0);
    const unsigned long long k = base + g.thread_rank();
    if (k >= P.cap) {
        atomicAdd(P.n_capped, 1u);
        return;
    }
    const uint64_t j = k - P.n_primary;
    const R ss = sqrt_(es / Ke), ct = (R)1 - (R)2 * u_cos, st = sqrt_(max_((R)0, (R)1 - ct * ct));
    R sp, cp;
    azimuth(u_phi, sp, cp);
    P.bt[j] = t_birth;
    P.bvx[j] = (double)(ss * st * cp);
    P.bvy[j] = (double)(ss * st * sp);
    P.bvz[j] = (double)(ss * ct);
    st_release(P.bid + j, secondary_id(parent, step));
}

// Sec. 2.1: a collision with a moving target, in the centre-of-momentum
// frame.  The target's velocity is Maxwell-Boltzmann at the gas temperature
// (each component normal with variance kT/M; Box-Muller on the step's
// fourth draw, sub-counter 3); the bullet's velocity relative to the centre
// of momentum keeps its length less what the energy loss eps_k takes,
// |g'|^2 = |g|^2 - 2 eps_k M / ((m + M) m), and turns by (ct, azimuth u)
// about its own direction, with the azimuth origin of the lab rotation.
// m/(m+M) comes from kappa2 / (2 M/(m+M)), which does not cancel in FP32.
template <typename R>
__device__ __noinline__ void thermal_collide(const RunArgs &P, uint32_t id_lo, uint32_t id_hi, uint32_t step,
                                             const ChParam<R> &p, bool elastic, R v0, R v1, R v2, R ct, R u, R Ke,
                                             R &o0, R &o1, R &o2)
{
    const uint4 w = philox(id_lo, id_hi, step, 3u, P.key0, P.key1);
    const R a = p.mfrac, b = p.kappa2 / ((R)2 * p.mfrac);  // M/(m+M), m/(m+M)
    const R st = sqrt_(kT_m_of<R>(P) * (b / a));              // sqrt(kT/M) = sqrt(kT/m * m/M)
    const R r0 = sqrt_((R)-2 * log_(uni<R>(w.x))), r1 = sqrt_((R)-2 * log_(uni<R>(w.z)));
    R s1, c1, s3, c3;
    sincospi_((R)2 * uni<R>(w.y), &s1, &c1);
    sincospi_((R)2 * uni<R>(w.w), &s3, &c3);
    const R V0 = st * r0 * c1, V1 = st * r0 * s1, V2 = st * r1 * c3;
    const R c0 = b * v0 + a * V0, cc1 = b * v1 + a * V1, c2 = b * v2 + a * V2;  // centre of momentum
    const R g0 = v0 - c0, g1 = v1 - cc1, g2 = v2 - c2;
    const R gsq = g0 * g0 + g1 * g1 + g2 * g2;
    R d0 = 0, d1 = 0, d2 = 1;
    if (gsq > (R)0) {
        const R ig = rsqrt_(gsq);
        d0 = g0 * ig;
        d1 = g1 * ig;
        d2 = g2 * ig;
    }
    const R ek = elastic ? (R)0 : p.eps_k;
    const R gp = sqrt_(max_((R)0, gsq - ek * a / Ke));  // 2 eps_k QE M/((m+M) m) = eps_k a / Ke
    // azimuth origin e1 = (x x d)/|x x d|, x the axis of the smallest |d_i|
    const R ax = fabs(d0), ay = fabs(d1), az = fabs(d2);
    R e0, e1, e2;
    if (ax <= ay && ax <= az) {
        e0 = 0;
        e1 = -d2;
        e2 = d1;
    } else if (ay <= az) {
        e0 = d2;
        e1 = 0;
        e2 = -d0;
    } else {
        e0 = -d1;
        e1 = d0;
        e2 = 0;
    }
    const R ie = rsqrt_(e0 * e0 + e1 * e1 + e2 * e2);
    e0 *= ie;
    e1 *= ie;
    e2 *= ie;
    const R f0 = d1 * e2 - d2 * e1, f1 = d2 * e0 - d0 * e2, f2 = d0 * e1 - d1 * e0;
    const R sn = sqrt_(max_((R)0, (R)1 - ct * ct));
    R sp3, cp3;
    azimuth(u, sp3, cp3);
    o0 = c0 + gp * (ct * d0 + sn * (cp3 * e0 + sp3 * f0));
    o1 = cc1 + gp * (ct * d1 + sn * (cp3 * e1 + sp3 * f1));
    o2 = c2 + gp * (ct * d2 + sn * (cp3 * e2 + sp3 * f2));
}

// One trial step.  Returns the decision (channel, DEC_NULL, DEC_FAIL or
// DEC_WINDOW); eps_i / eps_f receive the energy before and after a real
// collision.  The velocity at the end of the flight is computed once for
// every lane, and every lane that needs a new trial-frequency window (window
// end, real collision, fail) computes it at one common point after the
// branches, so divergent lanes do not repeat that code.
template <typename R, bool CH_SMEM, bool EXT = false, bool BF = true>
__device__ __forceinline__ int trial(const Tab<R> &T, const Fld<R> &F, const RunArgs &P, PState<R> &s, R &eps_i,
                                     R &eps_f)
{
    const uint32_t step = s.k++;
    const uint4 w = philox_rk(s.id_lo, s.id_hi, step, 0u, P.rk);
    // Eq. (3): the draw stands for 1 - R
    R Tn = s.T - log_(uni<R>(w.x)) * s.inv_nu;
    // a flight that outlasts the window stops at its end (its nu' holds only there) ...
    bool restart = P.window && Tn >= s.T_wend;
    if (restart) Tn = s.T_wend;
    // ... unless t_end comes first: TimeBulletLimiter, the flight stops at t_end
    bool cut = false;
    if (P.timed) {
        bool over;
        if constexpr (sizeof(R) == 4)
            over = Tn >= s.t_left;  // no FP64 work per trial in the FP32 step
        else
            over = s.t0 + s.t.value() + (double)Tn >= P.t_end;
        if (over) {
            Tn = (R)(P.t_end - s.t0 - s.t.value());
            cut = true;
            restart = false;
        }
    }
    R v0, v1, v2, sn, omc;
    velocity_at<R, BF>(F, s, Tn, v0, v1, v2, sn, omc);
    const R vsq = v0 * v0 + v1 * v1 + v2 * v2;
    const R eps = F.Ke * vsq;
    eps_i = eps;
    eps_f = 0;
    if (cut) {
        R dx, dy, dz;
        displacement<R, BF>(F, s, Tn, sn, omc, dx, dy, dz);
        s.x.add(dx);
        s.y.add(dy);
        s.z.add(dz);
        s.t.set(P.t_end - s.t0);
        s.vr0 = v0;
        s.vr1 = v1;
        s.vr2 = v2;
        s.T = 0;
        s.status = ST_TIME;
        s.done = true;
        return DEC_NULL;
    }
    // No branch below returns early: every lane of the warp meets again
    // before the window, which they then compute together.
    int dec;
    bool need_window = false, stop = false;
    R wt0 = 0, nu_fail = 0;
    R w0 = v0, w1 = v1, w2 = v2;  // velocity at the start of a new window
    if (restart) {
        s.T = Tn;  // a new window starts where the old one ended
        need_window = true;
        wt0 = Tn;
        dec = DEC_WINDOW;
    } else {
        int ri;
        R elo;
        const R S = density(T, eps, ri, elo);
        const R inv_sp = vsq > (R)0 ? rsqrt_(vsq) : (R)0;
        const R sp = vsq * inv_sp;
        const R nu = sp * S;
        const R r = uni<R>(w.y) * s.nu_p;
        if (!(nu <= s.nu_p)) {
            dec = DEC_FAIL;
            if (!(nu == nu)) {  // non-finite state: stop this particle, flag it
                atomicOr(P.err, BZ_ERR_NONFINITE);
                s.status = ST_ERROR;
                stop = true;
            } else {
                ++s.n_fail;
                bool error = P.fixed;  // FixedTrialFrequency (Sec. 6.1): an error
                if constexpr (EXT) {
                    // BinnedTrialFrequency (Sec. 6.3): one retry, then an error
                    if (P.tf == TF_BINNED) {
                        error = s.retried;
                        s.retried = true;
                    }
                }
                if (error) {
                    atomicOr(P.err, BZ_ERR_TRIAL);
                    s.status = ST_TRIAL;
                    stop = true;
                } else {
                    s.T = 0;  // fail (Sec. 6): back to the last real collision
                    nu_fail = nu;
                    need_window = P.window;
                    w0 = s.vr0;
                    w1 = s.vr1;
                    w2 = s.vr2;
                }
            }
        } else if (r > nu) {  // Eq. (4): null collision
            ++s.n_null;
            s.T = Tn;
            dec = DEC_NULL;
            if constexpr (EXT) {
                if (P.tf != TF_NONE && --s.grace == 0) {  // end of the grace period: query nu' here
                    s.nu_p = adaptive_nu(T, P, eps, nu);
                    s.inv_nu = (R)1 / s.nu_p;
                    s.grace = P.tf_grace;
                    s.retried = false;
                }
            }
        } else {
            // ---- real collision ----
            const int c = select_channel<R, CH_SMEM>(T, ri, elo, eps, r * inv_sp, S);
            {
                R dx, dy, dz;
                displacement<R, BF>(F, s, Tn, sn, omc, dx, dy, dz);
                s.x.add(dx);
                s.y.add(dy);
                s.z.add(dz);
                s.t.add(Tn);
                if (sizeof(R) == 4 && P.timed) s.t_left -= Tn;
                s.T = 0;
            }
            const R u2 = uni<R>(w.z);
            const ChParam<R> p = T.chp[c];
            const int kind = p.bits & 15;
            R ct;
            const int ang = (p.bits >> 4) & 15;
            if (ang == BZ_ANG_SCREENED_COULOMB) {  // Eq. (5), eps in Hartree
                ct = (R)1 - fdiv_((R)2 * u2, (R)1 + (R)8 * (eps * (R)(1.0 / kHartreeEv)) * ((R)1 - u2));
            } else if (EXT && ang == BZ_ANG_XI) {  // Eqs. (6)-(7)
                ct = xi_cos_theta<R, CH_SMEM>(T, P, p.bits, ri, elo, eps, u2);
            } else {
                ct = (R)1 - (R)2 * u2;
            }
            // Isotropic scattering sends the electron in a direction uniform on
            // the sphere whatever its incident one: the direction is drawn in
            // the lab frame (polar cosine ct, the azimuth from w.w), which
            // needs no frame about the incident direction, and Eqs. (8)-(9)
            // take its cosine to the incident direction.
            const bool lab = ang == BZ_ANG_ISOTROPIC && !(EXT && P.thermal && kind != BZ_ATTACHMENT);
            R n0 = 0, n1 = 0, n2 = 0;
            if (lab) {
                const R st = sqrt_(max_((R)0, (R)1 - ct * ct));
                R sp3, cp3;
                azimuth(uni<R>(w.w), sp3, cp3);
                n0 = st * cp3;
                n1 = st * sp3;
                n2 = ct;
                ct = vsq > (R)0 ? (v0 * n0 + v1 * n1 + v2 * n2) * inv_sp : n2;
            }
            R ratio;
            bool rotate = true;
            bool moved = false;  // moving targets: the new velocity is set directly
            R e_after = 0;
            if (EXT && P.thermal && kind != BZ_ATTACHMENT) {
                R t0, t1, t2;
                thermal_collide<R>(P, s.id_lo, s.id_hi, step, p, kind == BZ_ELASTIC, v0, v1, v2, ct, uni<R>(w.w),
                                   F.Ke, t0, t1, t2);
                const R efl = F.Ke * (t0 * t0 + t1 * t1 + t2 * t2);
                R keep = 1;
                if (kind == BZ_IONIZATION) {  // the secondary takes u4 of the lab energy
                    const uint4 w2 = philox_rk(s.id_lo, s.id_hi, step, 1u, P.rk);
                    const R u4 = uni<R>(w2.x);
                    if (P.spawn)
                        spawn_secondary(P, F.Ke, s.t0 + s.t.value(), ((uint64_t)s.id_hi << 32) | s.id_lo, step,
                                        u4 * efl, uni<R>(w2.y), uni<R>(w2.z));
                    keep = (R)1 - u4;
                    ++s.n_ion;
                }
                const R sk = sqrt_(keep);
                s.vr0 = t0 * sk;
                s.vr1 = t1 * sk;
                s.vr2 = t2 * sk;
                e_after = keep * efl;
                ratio = 0;
                moved = true;
            } else if (kind == BZ_ELASTIC) {
                ratio = (R)1 - p.kappa2 * ((R)1 - ct);  // Eq. (8)
            } else if (kind == BZ_ATTACHMENT) {
                ++s.n_att;
                if (P.attach_keep) {
                    ratio = 1;
                    rotate = false;
                } else {
                    ratio = 0;  // plastic collision: the electron stops
                    if (P.spawn) {  // ... and is removed
                        s.status = ST_ATTACHED;
                        s.done = true;
                    }
                }
            } else {
                const R x = fdiv_(p.eps_k, eps);  // Eq. (9), radicand clamped at 0
                const R rad = max_((R)0, (R)1 - p.minv * x);
                ratio = max_((R)0, (R)1 - p.mfrac * x + p.kappa2 * (sqrt_(rad) * ct - (R)1));
                if (kind == BZ_IONIZATION) {
                    const uint4 w2 = philox_rk(s.id_lo, s.id_hi, step, 1u, P.rk);
                    const R u4 = uni<R>(w2.x);
                    if (P.spawn)
                        spawn_secondary(P, F.Ke, s.t0 + s.t.value(), ((uint64_t)s.id_hi << 32) | s.id_lo, step,
                                        u4 * ratio * eps, uni<R>(w2.y), uni<R>(w2.z));
                    ratio *= (R)1 - u4;  // the secondary takes the rest
                    ++s.n_ion;
                }
            }
            const R nsp = sp * sqrt_(ratio);
            if (moved) {
            } else if (rotate && lab) {
                s.vr0 = nsp * n0;
                s.vr1 = nsp * n1;
                s.vr2 = nsp * n2;
            } else if (rotate) {
                R d0 = v0 * inv_sp, d1 = v1 * inv_sp, d2 = v2 * inv_sp;
                if (!(vsq > (R)0)) {
                    d0 = 0;
                    d1 = 0;
                    d2 = 1;
                }
                // azimuth origin e1 = (a x d)/|a x d|, a the axis of the smallest |d_i|
                const R ax = fabs(d0), ay = fabs(d1), az = fabs(d2);
                R e0, e1, e2;
                if (ax <= ay && ax <= az) {
                    e0 = 0;
                    e1 = -d2;
                    e2 = d1;
                } else if (ay <= az) {
                    e0 = d2;
                    e1 = 0;
                    e2 = -d0;
                } else {
                    e0 = -d1;
                    e1 = d0;
                    e2 = 0;
                }
                const R ie = rsqrt_(e0 * e0 + e1 * e1 + e2 * e2);
                e0 *= ie;
                e1 *= ie;
                e2 *= ie;
                const R f0 = d1 * e2 - d2 * e1, f1 = d2 * e0 - d0 * e2, f2 = d0 * e1 - d1 * e0;  // d x e1
                const R st = sqrt_(max_((R)0, (R)1 - ct * ct));
                R sp3, cp3;
                azimuth(uni<R>(w.w), sp3, cp3);
                s.vr0 = nsp * (ct * d0 + st * (cp3 * e0 + sp3 * f0));
                s.vr1 = nsp * (ct * d1 + st * (cp3 * e1 + sp3 * f1));
                s.vr2 = nsp * (ct * d2 + st * (cp3 * e2 + sp3 * f2));
            } else {
                s.vr0 = v0;
                s.vr1 = v1;
                s.vr2 = v2;
            }
            set_b_cache<R, BF>(F, s);
            eps_f = moved ? e_after : ratio * eps;
            s.se.add(eps);
            s.se2.add(eps_f);
            if (++s.n_real >= P.I) s.done = true;
            if ((s.n_real & 63u) == 0u) {
                s.x.fold();
                s.y.fold();
                s.z.fold();
                s.t.fold();
                s.se.fold();
                s.se2.fold();
                set_t_left(P, s);
            }
            need_window = P.window;
            w0 = s.vr0;
            w1 = s.vr1;
            w2 = s.vr2;
            dec = c;
            if constexpr (EXT) {
                s.retried = false;
                if (P.tf != TF_NONE && --s.grace == 0) {  // query at the energy the electron leaves with
                    s.nu_p = adaptive_nu(T, P, eps_f, P.tf == TF_VARIABLE ? nsp * density_at(T, eps_f) : (R)0);
                    s.inv_nu = (R)1 / s.nu_p;
                    s.grace = P.tf_grace;
                }
            }
        }
    }
    if (P.window) {
        // taken by every lane (the warp is whole again here), kept by those
        // that start a window: after a restart, a real collision or a fail
        R m, im, we;
        window_of<R, BF>(T, F, P, s, w0, w1, w2, wt0, m, im, we);
        if (need_window) {
            s.nu_p = m;
            s.inv_nu = im;
            s.T_wend = we;
        }
    }
    if (stop) {
        s.done = true;
        return DEC_FAIL;
    }
    if (dec == DEC_FAIL) {
        if (EXT && P.tf != TF_NONE) {
            // VARIABLE: (1 + zeta) nu at the fail; BINNED: the larger of the two bins' maxima
            const R q = adaptive_nu(T, P, eps, nu_fail);
            s.nu_p = (P.tf == TF_VARIABLE) ? q : max_(s.nu_p, q);
            s.grace = P.tf_grace;
        } else {
            s.nu_p = max_(s.nu_p, (R)1.25 * nu_fail);
        }
        s.inv_nu = (R)1 / s.nu_p;
    }
    return dec;
}

template <typename R>
__device__ __forceinline__ void write_particle(const RunArgs &P, const PState<R> &s, uint64_t slot)
{
    const ParticlesDev &o = P.out;
    o.x[slot] = s.x.value();
    o.y[slot] = s.y.value();
    o.z[slot] = s.z.value();
    o.t[slot] = s.t.value();
    o.se[slot] = s.se.value();
    o.se2[slot] = s.se2.value();
    o.vx[slot] = (float)s.vr0;
    o.vy[slot] = (float)s.vr1;
    o.vz[slot] = (float)s.vr2;
    o.nup[slot] = (float)s.nu_p;
    o.n_real[slot] = s.n_real;
    o.n_null[slot] = s.n_null;
    o.n_fail[slot] = s.n_fail;
    o.n_ion[slot] = s.n_ion;
    o.n_att[slot] = s.n_att;
    o.steps[slot] = s.k;
    o.status[slot] = s.status;
}

// ---------------------------------------------------------------------------
// Table staging: one TMA bulk copy (global -> shared) per block, completion
// tracked by an mbarrier; every wait is bounded and a timeout is reported.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t mb, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(mb), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for phase `parity` of the block's mbarrier, at most wait_ns of the
// global timer (and at most kWaitLimit polls).  On a timeout in any thread
// the block sets BZ_ERR_STAGE_TIMEOUT, waits (bounded by kDrainNs) for a
// copy still in flight, so that none lands after the block has exited, and
// returns false.
__device__ bool stage_wait(uint32_t mb, uint32_t parity, uint64_t wait_ns, uint32_t *err)
{
    bool ok = mbar_try_wait(mb, parity);
    if (!ok) {
        const uint64_t t0 = global_ns();
        for (uint32_t it = 0; it < kWaitLimit && !ok && global_ns() - t0 < wait_ns; ++it)
            ok = mbar_try_wait(mb, parity);
    }
    if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) atomicOr(err, BZ_ERR_STAGE_TIMEOUT);
        bool done = ok;
        const uint64_t t1 = global_ns();
        for (uint32_t it = 0; it < kWaitLimit && !done && global_ns() - t1 < kDrainNs; ++it)
            done = mbar_try_wait(mb, parity);
        __syncthreads();
        return false;
    }
    return true;
}

// Tests of the bounded staging wait (stage_hold): once the tables are in,
// thread 0 opens the next phase expecting 16 bytes that no copy sends, and
// the block waits on it.  No copy is in flight, so the wait can only run out.
__device__ bool stage_hold_wait(uint32_t mb, uint32_t parity, uint64_t wait_ns, uint32_t *err)
{
    if (threadIdx.x == 0)
        asm volatile(
            "{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(mb),
            "r"(16u)
            : "memory");
    return stage_wait(mb, parity, wait_ns, err);
}

__device__ void issue_stage_copy(const uint8_t *src, uint8_t *dst, uint32_t bytes, uint32_t mb)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(mb),
                 "r"(bytes)
                 : "memory");
    const uint32_t d = smem_u32(dst);
    for (uint32_t off = 0; off < bytes; off += kStageChunk) {
        const uint32_t sz = (bytes - off < kStageChunk) ? bytes - off : kStageChunk;
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(d + off),
            "l"(src + off), "r"(sz), "r"(mb)
            : "memory");
    }
}

__device__ bool stage_tables(const uint8_t *src, uint8_t *dst, uint32_t bytes, uint64_t *mbar, uint64_t wait_ns,
                             uint32_t hold, uint32_t *err)
{
    const uint32_t mb = smem_u32(mbar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (bytes == 0) return true;
    if (threadIdx.x == 0) issue_stage_copy(src, dst, bytes, mb);
    if (!stage_wait(mb, 0, wait_ns, err)) return false;
    if (hold) return stage_hold_wait(mb, 1, wait_ns, err);
    return true;
}

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------
// Re-stages the tables of a new mixture into shared memory through the
// block's mbarrier (already initialised), waiting on phase `parity`.
__device__ bool restage_tables(const uint8_t *src, uint8_t *dst, uint32_t bytes, uint32_t mb, uint32_t parity,
                               uint64_t wait_ns, uint32_t hold, uint32_t *err)
{
    if (threadIdx.x == 0) {
        // the generic-proxy reads of the previous tables are ordered before
        // the asynchronous copy that overwrites them
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue_stage_copy(src, dst, bytes, mb);
    }
    if (!stage_wait(mb, parity, wait_ns, err)) return false;
    if (hold) return stage_hold_wait(mb, parity ^ 1u, wait_ns, err);
    return true;
}

// The step kernel: one persistent launch over tiles (swarm, first particle,
// count), ordered by mixture -- of many swarms (batched form) or of one
// (bz_run_swarm), so that a swarm's results do not depend on how it was
// launched.  A block takes a tile, copies that swarm's parameters into
// shared memory, re-stages the tables only if the mixture differs from the
// one it holds, runs the tile's electrons with per-lane refill (a lane that
// finishes an electron takes the next one of the tile), and synchronises
// before the next tile.
template <typename R, bool CH_SMEM, bool EXT, int MINB, bool BF, int BS = kBlock>
__global__ void __launch_bounds__(BS, MINB) batch_kernel(const __grid_constant__ BatchArgs B)
{
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ __align__(16) RunArgs P;
    __shared__ int s_tile;
    __shared__ unsigned int s_next;
    const uint32_t mb = smem_u32(&mbar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    uint32_t phase = 0;
    const uint8_t *staged = nullptr;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    for (;;) {
        if (threadIdx.x == 0) {
            s_tile = (int)atomicAdd(B.tile_counter, 1u);
            s_next = 0;
        }
        __syncthreads();
        const int ti = s_tile;
        if (ti >= B.n_tiles) break;
        uint4 tile;
        if (B.tiles) {
            tile = B.tiles[ti];
        } else {
            const uint64_t first = B.slot_lo + (uint64_t)ti * B.tile_size;
            const uint64_t left = B.single.n - first;
            tile = make_uint4(0u, (uint32_t)first, (uint32_t)(left < B.tile_size ? left : B.tile_size), 0u);
        }
        {
            const uint32_t *src = (const uint32_t *)(B.desc ? B.desc + tile.x : &B.single);
            uint32_t *dst = (uint32_t *)&P;
            for (int i = threadIdx.x; i < (int)(sizeof(RunArgs) / 4); i += blockDim.x) dst[i] = src[i];
        }
        __syncthreads();
        if (P.blob != staged) {
            if (!restage_tables(P.blob, smem, P.stage_bytes, mb, phase, P.stage_wait_ns, P.stage_hold, P.err))
                return;
            phase ^= 1u;
            staged = P.blob;
        }
        const Tab<R> T = make_tab<R>(smem, P.blob, P.lay, CH_SMEM, P.stage_bytes);
        const Fld<R> F = make_fld<R>(P.f);
        PState<R> s;
        bool have = false, exhausted = false;
        uint64_t slot = 0;
        for (;;) {
            const unsigned need = __ballot_sync(FULL, !have);
            if (need && !exhausted) {
                const int leader = __ffs(need) - 1;
                unsigned int base = 0;
                if (lane == leader) base = atomicAdd(&s_next, (unsigned int)__popc(need));
                base = __shfl_sync(FULL, base, leader);
                if (base >= tile.z) exhausted = true;
                if (!have) {
                    const unsigned int idx = base + __popc(need & ((1u << lane) - 1u));
                    if (idx < tile.z) {
                        slot = (uint64_t)tile.y + idx;
                        init_particle<R, BF>(T, P, F, s, P.id_offset + slot);
                        if constexpr (EXT) {
                            if (P.tf != TF_NONE) adaptive_start(T, F, P, s);
                        }
                        have = true;
                    }
                }
            }
            if (!__any_sync(FULL, have)) break;
#pragma unroll 1
            for (int it = 0; it < 8 && have; ++it) {
                if (s.k >= P.max_trials) {
                    s.status = ST_STEPS;
                    s.done = true;
                    atomicOr(P.err, BZ_ERR_MAX_TRIALS);
                } else {
                    R ei, ef;
                    trial<R, CH_SMEM, EXT, BF>(T, F, P, s, ei, ef);
                }
                if (s.done) {
                    write_particle<R>(P, s, slot);
                    have = false;
                }
            }
        }
        __syncthreads();
    }
}

__device__ __forceinline__ uint64_t ld_acquire_ull(const unsigned long long *p)
{
    uint64_t v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}



// Spawn mode (ChildrenBulletLimiter, Sec. 3.2): one persistent launch runs
// the primaries and every electron created from them.  A lane without an
// electron holds a ticket k, a slot handed out in increasing order by one
// warp-aggregated atomic.  Slot k < n_primary is a primary; a created slot
// starts once its birth record is published (id != 0, acquire).  Every
// created electron is counted as pending before its parent can finish and
// uncounted when it finishes, so once pending reads 0 nothing more can be
// created: a ticket whose record is still missing is void, and so is every
// later one.  Tickets are taken only by lanes that are running, and every
// slot below the largest ticket has a holder, so a waiting lane waits only
// on electrons that are being run.
template <typename R, bool CH_SMEM, bool EXT, int MINB, bool BF>
__global__ void __launch_bounds__(kBlock, MINB) spawn_kernel(const __grid_constant__ RunArgs P)
{
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ __align__(8) uint64_t mbar;
    if (!stage_tables(P.blob, smem, P.stage_bytes, &mbar, P.stage_wait_ns, P.stage_hold, P.err)) return;
    const Tab<R> T = make_tab<R>(smem, P.blob, P.lay, CH_SMEM, P.stage_bytes);
    const Fld<R> F = make_fld<R>(P.f);
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    PState<R> s;
    bool have = false, ticket = false, over = false;
    uint64_t k = 0, wait_since = 0;
    uint32_t nap = 64;
    for (;;) {
        const bool idle = !have && !ticket && !over;
        const unsigned want = __ballot_sync(FULL, idle);
        if (want) {
            const int leader = __ffs(want) - 1;
            unsigned long long base = 0;
            if (lane == leader) base = atomicAdd(P.counter, (unsigned long long)__popc(want));
            base = __shfl_sync(FULL, base, leader);
            if (idle) {
                k = base + __popc(want & ((1u << lane) - 1u));
                ticket = true;
            }
        }
        bool ready = false;
        if (ticket) {
            if (k >= P.cap) {
                ticket = false;
                over = true;
            } else {
                ready = k < P.n_primary || ld_acquire(P.bid + (k - P.n_primary)) != 0;
            }
        }
        const unsigned blocked = __ballot_sync(FULL, ticket && !ready);
        if (blocked) {
            const int first = __ffs(blocked) - 1;
            unsigned long long pend = 1;
            if (lane == first) pend = ld_acquire_ull(P.pending);
            pend = __shfl_sync(FULL, pend, first);
            __syncwarp(FULL);  // orders the other lanes' loads after that acquire
            if (pend == 0 && ticket && !ready) {
                // every record was published before the last electron finished
                ready = ld_acquire(P.bid + (k - P.n_primary)) != 0;
                if (!ready) {
                    ticket = false;
                    over = true;
                }
            }
        }
        if (ready) {
            if (k < P.n_primary) init_particle<R, BF>(T, P, F, s, P.id_offset + k);
            else init_secondary<R, BF>(T, P, F, s, k - P.n_primary);
            have = true;
            ticket = false;
        }
        if (!__any_sync(FULL, have)) {
            if (__all_sync(FULL, over)) break;
            const uint64_t now = global_ns();
            if (wait_since == 0) {
                wait_since = now;
            } else if (now - wait_since > P.spawn_wait_ns) {  // a warp without work gives up
                if (lane == 0) atomicOr(P.err, BZ_ERR_SPAWN_WAIT);
                break;
            }
            __nanosleep(nap);
            nap = nap < 8192 ? 2 * nap : nap;
            continue;
        }
        wait_since = 0;
        nap = 64;
#pragma unroll 1
        for (int it = 0; it < 8 && have; ++it) {
            if (s.k >= P.max_trials) {
                s.status = ST_STEPS;
                s.done = true;
                atomicOr(P.err, BZ_ERR_MAX_TRIALS);
            } else {
                R ei, ef;
                trial<R, CH_SMEM, EXT, BF>(T, F, P, s, ei, ef);
            }
            if (s.done) {
                write_particle<R>(P, s, k);
                __threadfence();
                atomicAdd(P.pending, ~0ull);  // this electron is finished
                have = false;
            }
        }
    }
}

template <typename R, bool CH_SMEM>
__global__ void __launch_bounds__(kBlock) replay_kernel(const ReplayArgs A)
{
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ __align__(8) uint64_t mbar;
    const RunArgs &P = A.run;
    if (!stage_tables(P.blob, smem, P.stage_bytes, &mbar, P.stage_wait_ns, P.stage_hold, P.err)) return;
    const Tab<R> T = make_tab<R>(smem, P.blob, P.lay, CH_SMEM, P.stage_bytes);
    const Fld<R> F = make_fld<R>(P.f);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < A.n; i += (int64_t)gridDim.x * blockDim.x) {
        const double *in = A.state_in + 8 * i;
        PState<R> s;
        const uint64_t id = A.ids[i];
        s.id_lo = (uint32_t)id;
        s.id_hi = (uint32_t)(id >> 32);
        s.x.set(in[0]);
        s.y.set(in[1]);
        s.z.set(in[2]);
        s.vr0 = (R)in[3];
        s.vr1 = (R)in[4];
        s.vr2 = (R)in[5];
        s.t.set(in[6]);
        s.nu_p = (R)in[7];
        s.inv_nu = (R)1 / s.nu_p;
        s.T = 0;
        s.se.set(0.0);
        s.se2.set(0.0);
        s.k = A.steps[i];
        s.n_real = s.n_null = s.n_fail = s.n_ion = s.n_att = 0;
        s.status = ST_DONE;
        s.done = false;
        s.t0 = 0.0;
        set_t_left(P, s);
        set_b_cache(F, s);
        s.T_wend = (R)0;
        if (P.window) new_window(T, F, P, s, s.vr0, s.vr1, s.vr2, (R)0);
        R ei, ef;
        const int dec = trial<R, CH_SMEM, true>(T, F, P, s, ei, ef);
        // state at the trial point: last real collision advanced by s.T
        R v0, v1, v2, sn, omc, dx, dy, dz;
        velocity_at(F, s, s.T, v0, v1, v2, sn, omc);
        displacement(F, s, s.T, sn, omc, dx, dy, dz);
        double *o = A.state_out + 8 * i;
        o[0] = s.x.value() + (double)dx;
        o[1] = s.y.value() + (double)dy;
        o[2] = s.z.value() + (double)dz;
        o[3] = (double)v0;
        o[4] = (double)v1;
        o[5] = (double)v2;
        o[6] = s.t.value() + (double)s.T;
        o[7] = (double)s.nu_p;
        A.decision[i] = dec;
        A.eps_io[2 * i] = (double)ei;
        A.eps_io[2 * i + 1] = (double)ef;
    }
}

__global__ void philox_kernel(int64_t n, const uint32_t *ctr, uint32_t k0, uint32_t k1, uint32_t *out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint4 c = reinterpret_cast<const uint4 *>(ctr)[i];
        reinterpret_cast<uint4 *>(out)[i] = philox(c.x, c.y, c.z, c.w, k0, k1);
    }
}

// ---------------------------------------------------------------------------
// FP64 tallies (Sec. 2.3).  Pass 1 sums, per batch group (id mod 32), the
// per-particle quantities whose means give W_vec, alpha, eta, <eps>, the flux
// forms and the collision counts.  The middle step fixes W_vec; pass 2 sums
// the displacement terms d = x - t W_vec of Eqs. (22)-(27).  Per-block
// partial sums are reduced in a fixed order, so results are reproducible.
// Threads keep one group each: blocks and the grid stride are multiples of 32.
// ---------------------------------------------------------------------------
constexpr int kTallyBlock = 256;

template <int Q>
__device__ void block_group_reduce(double (&acc)[Q], double *out_block, uint64_t id_offset)
{
    __shared__ double red[kTallyBlock / 32][32][Q > kQ1 ? Q : kQ1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < Q; ++q) red[warp][lane][q] = acc[q];
    __syncthreads();
    if (warp == 0) {
        const int g = (int)((id_offset + (uint64_t)lane) & 31u);
        for (int q = 0; q < Q; ++q) {
            double v = 0.0;
            for (int w = 0; w < kTallyBlock / 32; ++w) v += red[w][lane][q];
            out_block[g * Q + q] = v;
        }
    }
}

// Pass-1 quantities of particle i (see the layout comment below).
__device__ __forceinline__ void pass1_contrib(const TallyArgs &A, uint64_t i, double (&c)[kQ1])
{
#pragma unroll
    for (int q = 0; q < kQ1; ++q) c[q] = 0.0;
    const double t = A.t[i];
    const uint32_t st = A.status[i];
    c[17] = (st != ST_DONE && st != ST_TIME && st != ST_ATTACHED) ? 1.0 : 0.0;
    c[19] = (st == ST_TIME) ? 1.0 : 0.0;
    c[20] = (st == ST_ATTACHED) ? 1.0 : 0.0;
    if (!(t > 0.0)) return;
    const double x = A.x[i], y = A.y[i], z = A.z[i];
    const double G = (double)A.n_ion[i], D = (double)A.n_att[i];
    c[0] = 1.0;
    c[1] = x / t;
    c[2] = y / t;
    c[3] = z / t;
    c[4] = G / z;
    c[5] = D / z;
    c[6] = x;
    c[7] = y;
    c[8] = z;
    c[9] = t;
    c[10] = A.se[i];
    c[11] = A.se2[i];
    c[12] = (double)A.n_real[i];
    c[13] = (double)A.n_null[i];
    c[14] = (double)A.n_fail[i];
    c[15] = G;
    c[16] = D;
    c[18] = A.steps ? (double)A.steps[i] : 0.0;
}

// Particles to reduce: in spawn mode the population the step kernel left.
__device__ __forceinline__ uint64_t tally_n(const TallyArgs &A)
{
    if (!A.n_dev) return A.n;
    const uint64_t v = *A.n_dev;
    return v < A.n ? v : A.n;
}

// Batch group (id mod 32) of particle i; secondaries carry their own ids.
__device__ __forceinline__ int group_of(const TallyArgs &A, uint64_t i)
{
    const uint64_t id = (A.ids && i >= A.n_primary) ? A.ids[i - A.n_primary] : A.id_offset + i;
    return (int)(id & 31u);
}

// Groups by particle id through shared-memory atomics (spawn mode, where a
// thread's particles do not share one group).
template <int Q, typename Fn>
__device__ void id_group_reduce(const TallyArgs &A, int bx, int nbx, double *out_block, Fn contrib)
{
    __shared__ double gs[kGroups * (kQ1 > kQ2 ? kQ1 : kQ2)];
    for (int k = threadIdx.x; k < kGroups * Q; k += blockDim.x) gs[k] = 0.0;
    __syncthreads();
    const uint64_t stride = (uint64_t)nbx * blockDim.x, n = tally_n(A);
    for (uint64_t i = (uint64_t)bx * blockDim.x + threadIdx.x; i < n; i += stride) {
        double c[Q];
        contrib(i, c);
        const int g = group_of(A, i);
        for (int q = 0; q < Q; ++q)
            if (c[q] != 0.0) atomicAdd(&gs[g * Q + q], c[q]);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kGroups * Q; k += blockDim.x) out_block[k] = gs[k];
}

__device__ void tally_pass1_body(const TallyArgs &A, int bx, int nbx)
{
    double *out = A.part1 + (size_t)bx * kGroups * kQ1;
    if (A.ids) {
        id_group_reduce<kQ1>(A, bx, nbx, out, [&](uint64_t i, double(&c)[kQ1]) { pass1_contrib(A, i, c); });
        return;
    }
    double acc[kQ1];
#pragma unroll
    for (int q = 0; q < kQ1; ++q) acc[q] = 0.0;
    const uint64_t stride = (uint64_t)nbx * blockDim.x, n = tally_n(A);
    for (uint64_t i = (uint64_t)bx * blockDim.x + threadIdx.x; i < n; i += stride) {
        double c[kQ1];
        pass1_contrib(A, i, c);
#pragma unroll
        for (int q = 0; q < kQ1; ++q) acc[q] += c[q];
    }
    block_group_reduce<kQ1>(acc, out, A.id_offset);
}

// gsum layout: [g][0..kQ1) pass 1, [g][kQ1..kQ1+kQ2) pass 2, then summary
// values at kGroups*(kQ1+kQ2): Wx, Wy, Wz, Wfx, Wfy, Wfz.

}  // namespace

// The swarm's drift vectors from the pass-1 group sums (gsum[g][q], row
// stride kGS): S[0..2] = W_vec = <x/t, y/t, z/t> (Eq. 15 per component),
// S[3..5] = the flux form (sum x, sum y, sum z) / sum t.  Host and device.
__host__ __device__ void drift_of_groups(const double *gsum, double *S)
{
    double c = 0, sx = 0, sy = 0, sz = 0, X = 0, Y = 0, Z = 0, Tt = 0;
    for (int k = 0; k < kGroups; ++k) {
        const double *r = gsum + k * kGS;
        c += r[0];
        sx += r[1];
        sy += r[2];
        sz += r[3];
        X += r[6];
        Y += r[7];
        Z += r[8];
        Tt += r[9];
    }
    S[0] = c > 0 ? sx / c : 0.0;
    S[1] = c > 0 ? sy / c : 0.0;
    S[2] = c > 0 ? sz / c : 0.0;
    S[3] = Tt > 0 ? X / Tt : 0.0;
    S[4] = Tt > 0 ? Y / Tt : 0.0;
    S[5] = Tt > 0 ? Z / Tt : 0.0;
}

namespace {

__device__ void tally_mid_body(const TallyArgs &A)
{
    const int g = threadIdx.x / kQ1, q = threadIdx.x % kQ1;
    if (threadIdx.x < kGroups * kQ1) {
        double v = 0.0;
        for (int b = 0; b < A.blocks; ++b) v += A.part1[((size_t)b * kGroups + g) * kQ1 + q];
        A.gsum[g * kGS + q] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) drift_of_groups(A.gsum, A.gsum + kGroups * kGS);
}

__device__ __forceinline__ void pass2_contrib(const TallyArgs &A, uint64_t i, const double *S, double (&c)[kQ2])
{
#pragma unroll
    for (int q = 0; q < kQ2; ++q) c[q] = 0.0;
    const double t = A.t[i];
    if (!(t > 0.0)) return;
    const double Wx = S[0], Wy = S[1], Wz = S[2], Fx = S[3], Fy = S[4], Fz = S[5];
    const double x = A.x[i], y = A.y[i], z = A.z[i];
    const double dx = x - t * Wx, dy = y - t * Wy, dz = z - t * Wz;
    const double dp2 = dx * dx + dy * dy, d2 = dp2 + dz * dz;
    c[0] = d2 / t;
    c[1] = dz * dz / (2.0 * t);
    c[2] = dp2 / (4.0 * t);
    c[3] = 2.0 * sqrt(d2);
    c[4] = 2.0 * fabs(dz);
    c[5] = 2.0 * sqrt(dp2);
    const double fz = z - Fz * t, fx = x - Fx * t, fy = y - Fy * t;
    c[6] = fz * fz;
    c[7] = fx * fx + fy * fy;
}

__device__ void tally_pass2_body(const TallyArgs &A, int bx, int nbx)
{
    const double *S = A.gsum + kGroups * kGS;
    double *out = A.part2 + (size_t)bx * kGroups * kQ2;
    if (A.ids) {
        id_group_reduce<kQ2>(A, bx, nbx, out, [&](uint64_t i, double(&c)[kQ2]) { pass2_contrib(A, i, S, c); });
        return;
    }
    double acc[kQ2];
#pragma unroll
    for (int q = 0; q < kQ2; ++q) acc[q] = 0.0;
    const uint64_t stride = (uint64_t)nbx * blockDim.x, n = tally_n(A);
    for (uint64_t i = (uint64_t)bx * blockDim.x + threadIdx.x; i < n; i += stride) {
        double c[kQ2];
        pass2_contrib(A, i, S, c);
#pragma unroll
        for (int q = 0; q < kQ2; ++q) acc[q] += c[q];
    }
    block_group_reduce<kQ2>(acc, out, A.id_offset);
}

}  // namespace

__host__ __device__ static double group_se(const double *v, const bool *has, int G)
{
    int n = 0;
    double m = 0.0;
    for (int g = 0; g < G; ++g)
        if (has[g]) {
            m += v[g];
            ++n;
        }
    if (n < 2) {
        const unsigned long long nan_bits = 0x7ff8000000000000ull;
        double x;
        memcpy(&x, &nan_bits, sizeof x);
        return x;
    }
    m /= n;
    double s = 0.0;
    for (int g = 0; g < G; ++g)
        if (has[g]) s += (v[g] - m) * (v[g] - m);
    return sqrt(s / (n - 1)) / sqrt((double)n);
}

// Swarm tallies (Eqs. 15-28, the Drifter fields of Sec. 7) from the group
// sums of both passes (gsum[g][0..kQ1) pass 1, gsum[g][kQ1..kGS) pass 2 about
// the drift vectors S[0..5]) and the run's scalars.  Host and device.
__host__ __device__ void tallies_of_groups(const double *gsum, const double *S, const GroupScalars &X, bz_tallies *out)
{
    double tot[kGS];
    for (int k = 0; k < kGS; ++k) {
        tot[k] = 0.0;
        for (int gg = 0; gg < kGroups; ++gg) tot[k] += gsum[gg * kGS + k];
    }
    bz_tallies o;
    memset(&o, 0, sizeof o);
    const double N = tot[0];
    const double inv = N > 0 ? 1.0 / N : 0.0;
    o.W = tot[3] * inv;
    o.Wx = tot[1] * inv;
    o.Wy = tot[2] * inv;
    o.W_flux = S[5];
    o.lorentz_angle = atan2(sqrt(o.Wx * o.Wx + o.Wy * o.Wy), o.W);
    o.alpha = tot[4] * inv;
    o.eta = tot[5] * inv;
    o.alpha_flux = tot[15] / tot[8];
    o.eta_flux = tot[16] / tot[8];
    o.eps = tot[12] > 0 ? tot[10] / tot[12] : 0.0;
    o.eps_after = tot[12] > 0 ? tot[11] / tot[12] : 0.0;
    o.D = tot[kQ1 + 0] * inv;
    o.D_L = tot[kQ1 + 1] * inv;
    o.D_T = tot[kQ1 + 2] * inv;
    o.sig = tot[kQ1 + 3] * inv;
    o.sig_L = tot[kQ1 + 4] * inv;
    o.sig_T = tot[kQ1 + 5] * inv;
    o.D_L_flux = tot[9] > 0 ? tot[kQ1 + 6] / (2.0 * tot[9]) : 0.0;
    o.D_T_flux = tot[9] > 0 ? tot[kQ1 + 7] / (4.0 * tot[9]) : 0.0;
    const double trials = tot[12] + tot[13] + tot[14];
    o.efficiency = trials > 0 ? tot[12] / trials : 0.0;
    o.E_V_m = X.E_V_m;
    o.n_total = X.n_total;
    o.nu_trial = X.nu_trial;
    o.t_mean = tot[9] * inv;
    o.mu = X.E_V_m > 0 ? o.W / X.E_V_m : 0.0;
    o.mu_N = o.mu * X.n_total;
    o.mu_0 = o.mu_N / kLoschmidt;
    o.n_particles = (uint64_t)(N + 0.5);
    o.n_real = (uint64_t)(tot[12] + 0.5);
    o.n_null = (uint64_t)(tot[13] + 0.5);
    o.n_fail = (uint64_t)(tot[14] + 0.5);
    o.n_ion = (uint64_t)(tot[15] + 0.5);
    o.n_att = (uint64_t)(tot[16] + 0.5);
    o.n_incomplete = (uint64_t)(tot[17] + 0.5);
    o.n_alive = (uint64_t)(tot[19] + 0.5);
    o.n_removed = (uint64_t)(tot[20] + 0.5);
    o.n_spawned = X.n_spawned;
    o.n_capped = X.n_capped;
    const double other = tot[18] - trials;  // steps that were neither real, null nor fail: window restarts
    o.n_window = other > 0.5 ? (uint64_t)(other + 0.5) : 0;
    o.error_flags = X.error_flags;
    // batch-mean standard errors
    bool has[kGroups];
    double v[kGroups];
    for (int k = 0; k < kGroups; ++k) has[k] = gsum[k * kGS] > 0.0;
    auto se_of = [&](int num, int den, double scale) {
        for (int k = 0; k < kGroups; ++k) {
            const double *r = gsum + k * kGS;
            v[k] = has[k] && r[den] > 0 ? scale * r[num] / r[den] : 0.0;
        }
        return group_se(v, has, kGroups);
    };
    o.W_se = se_of(3, 0, 1.0);
    o.alpha_se = se_of(4, 0, 1.0);
    o.eta_se = se_of(5, 0, 1.0);
    o.eps_se = se_of(10, 12, 1.0);
    o.eps_after_se = se_of(11, 12, 1.0);
    o.D_se = se_of(kQ1 + 0, 0, 1.0);
    o.D_L_se = se_of(kQ1 + 1, 0, 1.0);
    o.D_T_se = se_of(kQ1 + 2, 0, 1.0);
    o.sig_se = se_of(kQ1 + 3, 0, 1.0);
    o.sig_L_se = se_of(kQ1 + 4, 0, 1.0);
    o.sig_T_se = se_of(kQ1 + 5, 0, 1.0);
    *out = o;
}

namespace {

// Pass 2's per-block sums added over the blocks into the group sums.
__device__ void tally_sum2_body(const TallyArgs &A)
{
    const int g = threadIdx.x / kQ2, q = threadIdx.x % kQ2;
    if (threadIdx.x < kGroups * kQ2) {
        double v = 0.0;
        for (int b = 0; b < A.blocks; ++b) v += A.part2[((size_t)b * kGroups + g) * kQ2 + q];
        A.gsum[g * kGS + kQ1 + q] = v;
    }
}

__device__ void tally_final_body(const TallyArgs &A)
{
    tally_sum2_body(A);
    __syncthreads();
    if (threadIdx.x != 0) return;
    const uint64_t n = tally_n(A);
    GroupScalars X;
    X.E_V_m = A.E_V_m;
    X.n_total = A.n_total;
    X.nu_trial = A.nu_trial;
    X.n_spawned = n > A.n_primary && A.ids ? n - A.n_primary : 0;
    X.n_capped = A.capped ? (uint64_t)*A.capped : 0;
    X.error_flags = (int32_t)*A.err;
    tallies_of_groups(A.gsum, A.gsum + kGroups * kGS, X, A.out);
}


__global__ void __launch_bounds__(kTallyBlock) tally_pass1(const TallyArgs A) { tally_pass1_body(A, blockIdx.x, gridDim.x); }
__global__ void tally_mid(const TallyArgs A) { tally_mid_body(A); }
__global__ void __launch_bounds__(kTallyBlock) tally_pass2(const TallyArgs A) { tally_pass2_body(A, blockIdx.x, gridDim.x); }
__global__ void tally_final(const TallyArgs A) { tally_final_body(A); }
__global__ void tally_sum2(const TallyArgs A) { tally_sum2_body(A); }

// Many swarms at once: blockIdx.y (passes) or blockIdx.x (the one-block
// steps) selects the swarm's arguments.
__global__ void __launch_bounds__(kTallyBlock) tally_pass1_multi(const TallyArgs *As)
{
    const TallyArgs &A = As[blockIdx.y];
    if ((int)blockIdx.x < A.blocks) tally_pass1_body(A, blockIdx.x, A.blocks);
}
__global__ void tally_mid_multi(const TallyArgs *As) { tally_mid_body(As[blockIdx.x]); }
__global__ void __launch_bounds__(kTallyBlock) tally_pass2_multi(const TallyArgs *As)
{
    const TallyArgs &A = As[blockIdx.y];
    if ((int)blockIdx.x < A.blocks) tally_pass2_body(A, blockIdx.x, A.blocks);
}
__global__ void tally_final_multi(const TallyArgs *As) { tally_final_body(As[blockIdx.x]); }

}  // namespace

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
// Lets `kernel` take up to the device's opt-in shared memory per block minus
// its static shared memory (dynamic plus static above 48 KB needs the
// opt-in); the limit only ever rises to that one value, so concurrent
// launches of the same kernel with different table sizes cannot race on it.
template <typename K>
static cudaError_t prep_smem(K kernel, size_t smem)
{
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    const int limit = optin - (int)fa.sharedSizeBytes;
    if ((long long)smem > (long long)limit) return cudaErrorInvalidValue;
    if (fa.maxDynamicSharedSizeBytes < limit)
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, limit);
    return e;
}

// Launching and occupancy of one build of a step kernel.
template <typename K, typename A>
static cudaError_t go(K kernel, const A &a, size_t smem, int grid, int block, cudaStream_t s)
{
    cudaError_t e = prep_smem(kernel, smem);
    if (e != cudaSuccess) return e;
    kernel<<<grid, block, smem, s>>>(a);
    return cudaGetLastError();
}

// Blocks of `kernel` resident per SM (negative: minus the CUDA error of the query).
template <typename K>
static int occ(K kernel, int block, size_t smem)
{
    int n = 0;
    cudaError_t e = prep_smem(kernel, smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, block, smem);
    return e == cudaSuccess ? n : -(int)e;
}

template <typename R, bool C, bool E, int M, bool B, bool SPAWN>
static auto kernel_of()
{
    if constexpr (SPAWN) return &spawn_kernel<R, C, E, M, B>;
    else return &batch_kernel<R, C, E, M, B>;
}

// Block sizes a launch may take: 256 for every build; 128, 384 and 768 for
// the lean FP32 batch kernel.
static bool block_supported(int precision, bool ext, bool spawn, int block)
{
    if (block == kBlock) return true;
    return (block == 128 || block == 384 || block == 768) && precision == 32 && !ext && !spawn;
}

template <int BS, typename Fn>
static auto lean_block_build(bool ch, bool bf, Fn fn)
{
    constexpr int M = blocks_at_default_cap<BS>();
    if (ch) return bf ? fn(&batch_kernel<float, true, false, M, true, BS>)
                      : fn(&batch_kernel<float, true, false, M, false, BS>);
    return bf ? fn(&batch_kernel<float, false, false, M, true, BS>)
              : fn(&batch_kernel<float, false, false, M, false, BS>);
}

// Calls fn with the build of the step kernel (batch or spawn) that a launch
// uses: FP64 and the feature build (ext) are general; the lean FP32 build
// comes without the magnetic-field paths where the launch has no field
// (bf false), and in its 4-block form where the caller allows it and 4
// blocks fit.
template <bool SPAWN, typename Fn>
static auto dispatch(int precision, bool ch, bool ext, bool bf, bool wide, int block, size_t smem, Fn fn)
{
    // (callers check block_supported first)
    if constexpr (!SPAWN) {
        if (block == 128) return lean_block_build<128>(ch, bf, fn);
        if (block == 384) return lean_block_build<384>(ch, bf, fn);
        if (block == 768) return lean_block_build<768>(ch, bf, fn);
    }
    if (precision == 64) {
        if (ch) return ext ? fn(kernel_of<double, true, true, 1, true, SPAWN>())
                           : fn(kernel_of<double, true, false, 1, true, SPAWN>());
        return ext ? fn(kernel_of<double, false, true, 1, true, SPAWN>())
                   : fn(kernel_of<double, false, false, 1, true, SPAWN>());
    }
    if (ext) return ch ? fn(kernel_of<float, true, true, BZ_SWARM_MIN_BLOCKS, true, SPAWN>())
                       : fn(kernel_of<float, false, true, BZ_SWARM_MIN_BLOCKS, true, SPAWN>());
#define BZ_LEAN(C, B)                                                                 \
    do {                                                                              \
        auto k4 = kernel_of<float, C, false, kMinBlocksWide, B, SPAWN>();            \
        if (wide && occ(k4, block, smem) >= kMinBlocksWide) return fn(k4);          \
        return fn(kernel_of<float, C, false, BZ_SWARM_MIN_BLOCKS, B, SPAWN>());      \
    } while (0)
    if (ch) {
        if (bf) BZ_LEAN(true, true);
        BZ_LEAN(true, false);
    }
    if (bf) BZ_LEAN(false, true);
    BZ_LEAN(false, false);
#undef BZ_LEAN
}

cudaError_t launch_batch(int precision, bool ch_smem, bool ext, bool wide, bool bfield, const BatchArgs &a,
                         size_t smem, int grid, int block, cudaStream_t s)
{
    if (!block_supported(precision, ext, false, block)) return cudaErrorInvalidValue;
    return dispatch<false>(precision, ch_smem, ext, bfield, wide, block, smem,
                           [&](auto k) { return go(k, a, smem, grid, block, s); });
}

int batch_occupancy(int precision, bool ch_smem, bool ext, bool wide, bool bfield, int block, size_t smem)
{
    if (!block_supported(precision, ext, false, block)) return -(int)cudaErrorInvalidValue;
    return dispatch<false>(precision, ch_smem, ext, bfield, wide, block, smem,
                           [&](auto k) { return occ(k, block, smem); });
}

cudaError_t launch_spawn(int precision, bool ch_smem, bool ext, bool wide, bool bfield, const RunArgs &a, size_t smem,
                         int grid, int block, cudaStream_t s)
{
    if (block != kBlock) return cudaErrorInvalidValue;
    return dispatch<true>(precision, ch_smem, ext, bfield, wide, block, smem,
                          [&](auto k) { return go(k, a, smem, grid, block, s); });
}

int spawn_occupancy(int precision, bool ch_smem, bool ext, bool wide, bool bfield, int block, size_t smem)
{
    if (block != kBlock) return -(int)cudaErrorInvalidValue;
    return dispatch<true>(precision, ch_smem, ext, bfield, wide, block, smem,
                          [&](auto k) { return occ(k, block, smem); });
}

cudaError_t launch_tallies_multi(const TallyArgs *args_dev, int n_swarms, int max_blocks, cudaStream_t s)
{
    if (n_swarms <= 0) return cudaSuccess;
    tally_pass1_multi<<<dim3(max_blocks, n_swarms), kTallyBlock, 0, s>>>(args_dev);
    tally_mid_multi<<<n_swarms, kGroups * kQ1, 0, s>>>(args_dev);
    tally_pass2_multi<<<dim3(max_blocks, n_swarms), kTallyBlock, 0, s>>>(args_dev);
    tally_final_multi<<<n_swarms, kGroups * kQ2, 0, s>>>(args_dev);
    return cudaGetLastError();
}

cudaError_t launch_replay(int precision, bool ch_smem, const ReplayArgs &a, int grid, int block, cudaStream_t s)
{
    if (block != kBlock) return cudaErrorInvalidValue;
    const size_t smem = a.run.stage_bytes;
    cudaError_t e;
#define BZ_LAUNCH(R, C)                                                        \
    do {                                                                       \
        e = prep_smem(replay_kernel<R, C>, smem);                              \
        if (e != cudaSuccess) return e;                                        \
        replay_kernel<R, C><<<grid, block, smem, s>>>(a);                      \
    } while (0)
    if (precision == 64) {
        if (ch_smem) BZ_LAUNCH(double, true); else BZ_LAUNCH(double, false);
    } else {
        if (ch_smem) BZ_LAUNCH(float, true); else BZ_LAUNCH(float, false);
    }
#undef BZ_LAUNCH
    return cudaGetLastError();
}

cudaError_t launch_philox(int64_t n, const uint32_t *ctr, uint64_t key, uint32_t *out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int block = 256;
    const int grid = (int)((n + block - 1) / block < 4096 ? (n + block - 1) / block : 4096);
    philox_kernel<<<grid, block, 0, s>>>(n, ctr, (uint32_t)key, (uint32_t)(key >> 32), out);
    return cudaGetLastError();
}

int tally_blocks(uint64_t n, int sm_count)
{
    uint64_t b = (n + kTallyBlock - 1) / kTallyBlock;
    uint64_t cap = (uint64_t)sm_count * 2;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

cudaError_t launch_group_sums2(const TallyArgs &a, const double *drift_host, cudaStream_t s)
{
    // the drift vectors go where pass 2 reads them; pass-1 group sums stay
    cudaError_t e = cudaMemcpyAsync(a.gsum + kGroups * kGS, drift_host, 6 * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    tally_pass2<<<a.blocks, kTallyBlock, 0, s>>>(a);
    tally_sum2<<<1, kGroups * kQ2, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_tallies(const TallyArgs &a, cudaStream_t s)
{
    tally_pass1<<<a.blocks, kTallyBlock, 0, s>>>(a);
    tally_mid<<<1, kGroups * kQ1, 0, s>>>(a);
    tally_pass2<<<a.blocks, kTallyBlock, 0, s>>>(a);
    tally_final<<<1, kGroups * kQ2, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace bz
