// mixture.cpp -- host compiler of a gas mixture into the tables the step
// kernels read.
//
// What the kernels need is nu(eps) = sqrt(2 eps/m) sum_k n_k sum_j sigma_kj(eps)
// (Eq. 2) and, on a real collision, the channel whose cumulative frequency
// reaches the drawn value.  Every table is linear between its points
// (Sec. 5) and is extended per Sec. 2.2 (Eqs. 12-14), so between two
// consecutive points of the union of all tables and thresholds each channel
// is a single linear function (or, above its last point, its power-law
// tail).  The compiler therefore emits one record per union interval holding
// the density sum and its slope, exact up to rounding; per-channel
// coefficients on the same intervals; a log-energy bucket index that lands
// within a record or two of the right one; and the exact maximum of nu over
// [0, eps_cap], which is the constant trial frequency (Sec. 6.2).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <limits>

#include "bz_impl.h"

namespace bz {
namespace {

struct Chan {
    int kind, gas;
    double th;
    std::vector<double> e, s;
    double n;            // number density of the gas
    // right extension n sigma(eps) = n s_last (eps/e_last)^K
    bool tail_zero;
    double tail_K;
};

// Linear piece a + b eps of channel c on an interval whose midpoint is m;
// returns false if the channel is in its right extension there.  *k is a
// hint of the table interval (e[k-1] <= m < e[k]); it only moves forward, so
// a caller that visits increasing m finds every interval in amortised O(1).
bool piece(const Chan &c, double m, double *a, double *b, size_t *k)
{
    const std::vector<double> &e = c.e, &s = c.s;
    size_t n = e.size();
    if (m > e[n - 1]) return false;
    if (c.kind != BZ_ELASTIC) {
        if (m < c.th) { *a = 0.0; *b = 0.0; return true; }
        if (m < e[0]) {  // linear rise from (threshold, 0) to the first point
            *b = s[0] / (e[0] - c.th);
            *a = -*b * c.th;
            return true;
        }
    } else if (m < e[0]) {
        *a = s[0]; *b = 0.0; return true;
    }
    if (*k > n || (*k > 0 && e[*k - 1] > m)) *k = 0;  // the hint ran past m: search again
    while (*k < n && e[*k] <= m) ++*k;                // e[k-1] <= m < e[k]
    size_t i = *k;
    if (i == 0) i = 1;
    if (i >= n) i = n - 1;
    double e0 = e[i - 1], e1 = e[i], s0 = s[i - 1], s1 = s[i];
    *b = (s1 - s0) / (e1 - e0);
    *a = s0 - *b * e0;
    return true;
}

bool piece(const Chan &c, double m, double *a, double *b)
{
    if (m > c.e.back()) return false;  // the right extension: no search needed
    size_t k = (size_t)(std::upper_bound(c.e.begin(), c.e.end(), m) - c.e.begin());
    return piece(c, m, a, b, &k);
}

double speed_of(double eps) { return sqrt(2.0 * eps * kQe / kMe); }

// Exact density sum at eps in record (a, b): linear part plus active tails,
// n sigma = exp(tail_logc + K ln eps) (tail_logc per channel, host FP64).
double record_density(const std::vector<Chan> &ch, const std::vector<double> &tail_logc, double a, double b,
                      double eps)
{
    double mid = 0.5 * (a + b), S = 0.0;
    const double le = log(eps);
    for (size_t j = 0; j < ch.size(); ++j) {
        const Chan &c = ch[j];
        double pa, pb;
        if (piece(c, mid, &pa, &pb)) S += c.n * (pa + pb * eps);
        else if (!c.tail_zero) S += exp(tail_logc[j] + c.tail_K * le);
    }
    return S;
}

struct Bins {
    std::vector<double> max;   // per-bin maxima, then the sparse-table levels: level l holds
    int levels;                // the max over bins [b, b + 2^l) at [l * n_bins + b]
    int n_bins;
    int j0, per_decade;        // first edge 10^(j0 / per_decade)
    float lo, inv_w;
    double nu_low;
    double nu_first;  // nu at the first positive union point
    bool low_sqrt;
};

// Total elastic cross section of an xi-form gas (Eqs. 6-7): per record and
// gas its density-weighted value and slope (zero for other gases and in the
// tail), and per gas its tail constants.
struct ElTabs {
    std::vector<std::vector<double>> val, slope;  // [n_rec][n_gases]
    std::vector<ChParam<double>> tail;            // [n_gases]
};

// Log-energy bucket index with k buckets per union point (record i holds
// [g[i-1], g[i]) for i >= 1, [0, g[0]) for i = 0).
struct BucketIndex {
    std::vector<uint16_t> bucket;
    float log2_lo, inv_bw;
};

BucketIndex bucket_index(const std::vector<double> &g, int k)
{
    const int P = (int)g.size();
    int ipos = 0;
    while (ipos < P && g[ipos] <= 0.0) ++ipos;
    double L0 = (ipos < P) ? log2(g[ipos]) : 0.0, L1 = log2(g[P - 1] > 0.0 ? g[P - 1] : 1.0);
    int nb = std::min(std::max(k * P, 64), 65535);
    double w = (L1 > L0) ? (L1 - L0) / nb : 0.0;
    if (w == 0.0) nb = 1;
    BucketIndex B;
    B.bucket.resize(nb);
    size_t i = 0;  // record of bucket b's lower edge e: g[i-1] <= e < g[i]; e grows with b
    for (int b = 0; b < nb; ++b) {
        double e = exp2(L0 + b * w);
        while (i < g.size() && g[i] <= e) ++i;
        B.bucket[b] = (uint16_t)i;
    }
    B.log2_lo = (float)L0;
    B.inv_bw = (w > 0.0) ? (float)(1.0 / w) : 0.0f;
    return B;
}

// Emits the blob of one precision.  The bucket index takes as many entries
// per record (4, 3, 2 or 1) as let records + buckets + channel params + bin
// maxima fit `budget` bytes of shared memory; if none does, the bin maxima
// stay in global memory and the densest index that fits is taken.  Four per
// record land the walk on the right record almost always (a walk step costs
// the whole warp); fewer keep large mixtures at three blocks per SM.
template <typename R>
bool emit(const std::vector<Chan> &ch, const std::vector<double> &g, const std::vector<double> &Slo,
          const std::vector<double> &Ssl, const std::vector<std::vector<double>> &cv,
          const std::vector<std::vector<double>> &cs, const std::vector<ChParam<double>> &cp, int first_tail,
          const Bins &bins, const ElTabs &el, size_t budget, std::vector<uint8_t> *blob, Layout *lay,
          std::string *err_out)
{
    const int n_rec = (int)Slo.size(), n_ch = (int)ch.size();
    const int n_bins = bins.n_bins, n_bin_vals = (int)bins.max.size();
    auto pad16 = [](size_t x) { return (x + 15) & ~(size_t)15; };
    size_t off_rec = 0;
    const size_t off_bucket = pad16(off_rec + sizeof(Rec<R>) * n_rec);
    auto prefix = [&](int k, bool with_bins) {
        const int nb = std::min(std::max(k * (int)g.size(), 64), 65535);
        const size_t ob = pad16(pad16(off_bucket + sizeof(uint16_t) * nb) + sizeof(ChParam<R>) * n_ch);
        return with_bins ? ob + sizeof(R) * n_bin_vals : ob;
    };
    int k = 0;
    for (int kk = 4; kk >= 1 && !k; --kk)
        if (prefix(kk, true) <= budget) k = kk;
    for (int kk = 4; kk >= 1 && !k; --kk)
        if (prefix(kk, false) <= budget) k = kk;
    if (!k) k = 1;
    const BucketIndex BI = bucket_index(g, k);
    const std::vector<uint16_t> &bucket = BI.bucket;
    const int nb = (int)bucket.size();
    size_t off_chp = pad16(off_bucket + sizeof(uint16_t) * nb);
    size_t off_bin = pad16(off_chp + sizeof(ChParam<R>) * n_ch);
    const size_t bin_end = off_bin + sizeof(R) * n_bin_vals;
    size_t off_chval = pad16(bin_end);
    size_t off_gval = pad16(off_chval + sizeof(ChVal<R>) * (size_t)n_rec * n_ch);
    int n_gases = 0;
    for (const Chan &c : ch) n_gases = std::max(n_gases, c.gas + 1);
    size_t off_elval = pad16(off_gval + sizeof(ChVal<R>) * (size_t)n_rec * n_gases);
    size_t off_elp = pad16(off_elval + sizeof(ChVal<R>) * (size_t)n_rec * n_gases);
    size_t off_cum = pad16(off_elp + sizeof(ChParam<R>) * (size_t)n_gases);
    const bool guided = n_ch <= 255;
    size_t off_guide = pad16(off_cum + sizeof(ChVal<R>) * (size_t)n_rec * n_ch);
    size_t total = pad16(off_guide + (guided ? (size_t)kGuide * (n_rec + 1) : 0));
    blob->assign(total, 0);
    Rec<R> *rec = (Rec<R> *)(blob->data() + off_rec);
    for (int i = 0; i < n_rec; ++i) {
        double lo = (i == 0) ? 0.0 : g[i - 1];
        double hi = (i < n_rec - 1) ? g[i] : std::numeric_limits<double>::infinity();
        rec[i].e_lo = (R)lo;
        rec[i].e_hi = (R)hi;
        rec[i].S_lo = (R)Slo[i];
        rec[i].slope = (R)Ssl[i];
    }
    memcpy(blob->data() + off_bucket, bucket.data(), sizeof(uint16_t) * nb);
    ChParam<R> *p = (ChParam<R> *)(blob->data() + off_chp);
    for (int j = 0; j < n_ch; ++j) {
        p[j].kappa2 = (R)cp[j].kappa2;
        p[j].mfrac = (R)cp[j].mfrac;
        p[j].minv = (R)cp[j].minv;
        p[j].eps_k = (R)cp[j].eps_k;
        p[j].e_last = (R)cp[j].e_last;
        p[j].tail_logc = (R)cp[j].tail_logc;
        p[j].tail_K = (R)cp[j].tail_K;
        p[j].bits = cp[j].bits;
    }
    R *bm = (R *)(blob->data() + off_bin);
    for (int b = 0; b < n_bin_vals; ++b) bm[b] = (R)bins.max[b];
    ChVal<R> *v = (ChVal<R> *)(blob->data() + off_chval);
    for (int i = 0; i < n_rec; ++i)
        for (int j = 0; j < n_ch; ++j) {
            v[(size_t)i * n_ch + j].val = (R)cv[i][j];
            v[(size_t)i * n_ch + j].slope = (R)cs[i][j];
        }
    ChVal<R> *gv = (ChVal<R> *)(blob->data() + off_gval);
    for (int i = 0; i < n_rec; ++i) {
        std::vector<double> sv(n_gases, 0.0), ss(n_gases, 0.0);
        for (int j = 0; j < n_ch; ++j) {
            sv[ch[j].gas] += cv[i][j];
            ss[ch[j].gas] += cs[i][j];
        }
        for (int gI = 0; gI < n_gases; ++gI) {
            gv[(size_t)i * n_gases + gI].val = (R)sv[gI];
            gv[(size_t)i * n_gases + gI].slope = (R)ss[gI];
        }
    }
    ChVal<R> *ev = (ChVal<R> *)(blob->data() + off_elval);
    for (int i = 0; i < n_rec; ++i)
        for (int gI = 0; gI < n_gases; ++gI) {
            ev[(size_t)i * n_gases + gI].val = (R)el.val[i][gI];
            ev[(size_t)i * n_gases + gI].slope = (R)el.slope[i][gI];
        }
    ChParam<R> *ep = (ChParam<R> *)(blob->data() + off_elp);
    for (int gI = 0; gI < n_gases; ++gI) {
        ep[gI].kappa2 = ep[gI].mfrac = ep[gI].minv = ep[gI].eps_k = (R)0;
        ep[gI].e_last = (R)el.tail[gI].e_last;
        ep[gI].tail_logc = (R)el.tail[gI].tail_logc;
        ep[gI].tail_K = (R)el.tail[gI].tail_K;
        ep[gI].bits = el.tail[gI].bits;
    }
    lay->off_elval = (uint32_t)off_elval;
    lay->off_elp = (uint32_t)off_elp;
    lay->off_gval = (uint32_t)off_gval;
    lay->n_gases = n_gases;
    for (int gI = 0; gI < kMaxGases; ++gI) {
        lay->gas_first[gI] = 0;
        lay->gas_count[gI] = 0;
    }
    for (int j = n_ch - 1; j >= 0; --j) {
        lay->gas_first[ch[j].gas] = (int16_t)j;
        lay->gas_count[ch[j].gas] += 1;
    }
    // cumulative channel values: running FP64 sums in the order of Eq. 2,
    // rounded once, so that entry j reaches the record's density sum at j =
    // n_ch - 1 and never decreases where a channel adds nothing
    ChVal<R> *cu = (ChVal<R> *)(blob->data() + off_cum);
    for (int i = 0; i < n_rec; ++i) {
        double a = 0.0, b = 0.0;
        for (int j = 0; j < n_ch; ++j) {
            a += cv[i][j];
            b += cs[i][j];
            cu[(size_t)i * n_ch + j].val = (R)a;
            cu[(size_t)i * n_ch + j].slope = (R)b;
        }
    }
    // guide rows: row 0 from the constant values of record 0 (below the first
    // grid point), row r >= 1 from record r - 1's own linear pieces at its
    // upper edge g[r - 1] -- by continuity of every channel also the lower
    // edge of record r; record i reads rows i and i + 1
    if (guided) {
        uint8_t *gd = blob->data() + off_guide;
        std::vector<double> C(n_ch);
        for (int r = 0; r <= n_rec; ++r) {
            const int src = r == 0 ? 0 : std::min(r - 1, n_rec - 1);
            const double w = (r == 0 || src >= (int)g.size()) ? 0.0 : g[src] - (src == 0 ? 0.0 : g[src - 1]);
            double a = 0.0;
            for (int j = 0; j < n_ch; ++j) C[j] = (a += cv[src][j] + cs[src][j] * w);
            const double tot = C[n_ch - 1];
            int j = 0;
            for (int b = 0; b < kGuide; ++b) {
                const double q = tot * (double)b / kGuide;
                while (j < n_ch - 1 && C[j] < q) ++j;
                gd[(size_t)r * kGuide + b] = (uint8_t)(tot > 0.0 ? j : 0);
            }
        }
    }
    lay->off_guide = guided ? (uint32_t)off_guide : 0u;
    lay->n_rec = n_rec;
    lay->n_buckets = nb;
    lay->n_ch = n_ch;
    lay->first_tail_rec = first_tail;
    lay->log2_lo = BI.log2_lo;
    lay->inv_bw = BI.inv_bw;
    lay->buckets_per_record = k;
    lay->off_bucket = (uint32_t)off_bucket;
    lay->off_chp = (uint32_t)off_chp;
    lay->off_chval = (uint32_t)off_chval;
    lay->stage_tables = (uint32_t)(bin_end <= budget ? bin_end : off_bin);
    lay->stage_all = (uint32_t)off_cum;
    lay->total = (uint32_t)total;
    lay->off_bin = (uint32_t)off_bin;
    lay->bin_end = (uint32_t)bin_end;
    lay->off_cum = (uint32_t)off_cum;
    lay->s_min = sqrt(exp2((double)bins.lo) * 2.0 * kQe / kMe);
    lay->n_bins = n_bins;
    lay->bin_levels = bins.levels;
    lay->bin_lo = bins.lo;
    lay->inv_binw = bins.inv_w;
    lay->nu_low = bins.nu_low;
    lay->bin_j0 = bins.j0;
    lay->bins_per_decade = bins.per_decade;
    lay->low_sqrt = bins.low_sqrt ? 1 : 0;
    lay->nu_first = bins.nu_first;
    lay->g_top = g.back();
    return true;
}

bool finite(double x) { return std::isfinite(x); }

}  // namespace

bz_status compile_mixture(const bz_gas *gases, int32_t n_gases, const bz_mixture_opts *opts,
                          CompiledMixture *out, std::string *err)
{
    if (!gases || n_gases < 1) { *err = "need at least one gas"; return BZ_EINVAL; }
    if (n_gases > kMaxGases) { *err = "at most 16 gases per mixture"; return BZ_EINVAL; }
    std::vector<Chan> ch;
    std::vector<ChParam<double>> cp;
    std::vector<Chan> eltab;  // per gas (xi form: the total elastic table; else empty)
    double n_total = 0.0, emax = 0.0;
    const double m = kMe;
    for (int gi = 0; gi < n_gases; ++gi) {
        const bz_gas &G = gases[gi];
        if (!(G.mass_kg > 0.0) || !finite(G.mass_kg)) { *err = "gas mass must be > 0"; return BZ_EINVAL; }
        if (!(G.number_density_m3 > 0.0) || !finite(G.number_density_m3)) {
            *err = "gas number density must be > 0"; return BZ_EINVAL;
        }
        if (G.angular != BZ_ANG_ISOTROPIC && G.angular != BZ_ANG_SCREENED_COULOMB && G.angular != BZ_ANG_XI) {
            *err = "unknown angular model"; return BZ_EINVAL;
        }
        Chan elc;  // xi form: the total elastic cross section, as an elastic table
        elc.kind = BZ_ELASTIC;
        elc.gas = gi;
        elc.th = 0.0;
        elc.n = G.number_density_m3;
        elc.tail_zero = true;
        elc.tail_K = 0.0;
        if (G.angular == BZ_ANG_XI) {
            int n_el_ch = 0;
            for (int c = 0; c < G.n_channels && G.channels; ++c) n_el_ch += G.channels[c].kind == BZ_ELASTIC;
            if (n_el_ch != 1) { *err = "an xi-form gas needs exactly one elastic channel"; return BZ_EINVAL; }
            if (G.el_n_points < 1 || !G.el_energy_eV || !G.sigma_el_m2) {
                *err = "an xi-form gas needs its total elastic cross section"; return BZ_EINVAL;
            }
            elc.e.assign(G.el_energy_eV, G.el_energy_eV + G.el_n_points);
            elc.s.assign(G.sigma_el_m2, G.sigma_el_m2 + G.el_n_points);
            for (int i = 0; i < G.el_n_points; ++i) {
                if (!finite(elc.e[i]) || elc.e[i] < 0.0 || !finite(elc.s[i]) || elc.s[i] < 0.0 ||
                    (i > 0 && !(elc.e[i] > elc.e[i - 1]))) {
                    *err = "bad total elastic cross-section table"; return BZ_EINVAL;
                }
            }
            const size_t n = elc.e.size();
            elc.tail_zero = elc.s[n - 1] == 0.0;
            if (n >= 2 && elc.s[n - 1] > 0.0 && elc.s[n - 2] > 0.0)
                elc.tail_K = log(elc.s[n - 1] / elc.s[n - 2]) / log(elc.e[n - 1] / elc.e[n - 2]);
        }
        eltab.push_back(std::move(elc));
        if (G.n_channels < 1 || !G.channels) { *err = "a gas needs at least one channel"; return BZ_EINVAL; }
        n_total += G.number_density_m3;
        const double M = G.mass_kg;
        for (int c = 0; c < G.n_channels; ++c) {
            const bz_channel &C = G.channels[c];
            if (C.kind < BZ_ELASTIC || C.kind > BZ_IONIZATION) { *err = "unknown channel kind"; return BZ_EINVAL; }
            if (C.n_points < 1 || !C.energy_eV || !C.sigma_m2) { *err = "empty cross-section table"; return BZ_EINVAL; }
            if (!(C.threshold_eV >= 0.0) || !finite(C.threshold_eV)) { *err = "threshold must be >= 0"; return BZ_EINVAL; }
            Chan k;
            k.kind = C.kind;
            k.gas = gi;
            k.th = (C.kind == BZ_ELASTIC) ? 0.0 : C.threshold_eV;
            k.n = G.number_density_m3;
            k.e.assign(C.energy_eV, C.energy_eV + C.n_points);
            k.s.assign(C.sigma_m2, C.sigma_m2 + C.n_points);
            for (int i = 0; i < C.n_points; ++i) {
                if (!finite(k.e[i]) || k.e[i] < 0.0) { *err = "energies must be finite and >= 0"; return BZ_EINVAL; }
                if (!finite(k.s[i]) || k.s[i] < 0.0) { *err = "cross sections must be finite and >= 0"; return BZ_EINVAL; }
                if (i > 0 && !(k.e[i] > k.e[i - 1])) { *err = "energies must be strictly increasing"; return BZ_EINVAL; }
                if (C.kind != BZ_ELASTIC && k.e[i] < k.th && k.s[i] > 0.0) {
                    *err = "cross section > 0 below the threshold"; return BZ_EINVAL;
                }
            }
            size_t n = k.e.size();
            double sl = k.s[n - 1];
            k.tail_zero = (sl == 0.0);
            k.tail_K = 0.0;
            if (n >= 2 && k.s[n - 1] > 0.0 && k.s[n - 2] > 0.0)
                k.tail_K = log(k.s[n - 1] / k.s[n - 2]) / log(k.e[n - 1] / k.e[n - 2]);
            emax = std::max(emax, k.e[n - 1]);
            ChParam<double> p;
            p.kappa2 = 2.0 * m * M / ((m + M) * (m + M));
            p.mfrac = M / (m + M);
            p.minv = (m + M) / M;
            p.eps_k = k.th;
            p.e_last = k.e[n - 1];
            p.tail_K = k.tail_K;
            p.tail_logc = k.tail_zero ? 0.0 : log(k.n * sl) - k.tail_K * log(k.e[n - 1]);
            p.bits = C.kind | (G.angular << 4) | ((k.tail_zero ? 1 : 0) << 8);
            ch.push_back(std::move(k));
            cp.push_back(p);
        }
    }
    const int n_ch = (int)ch.size();
    std::vector<double> tail_logc(n_ch);
    for (int j = 0; j < n_ch; ++j) tail_logc[j] = cp[j].tail_logc;
    // union grid of all table energies and inelastic thresholds
    std::vector<double> g;
    for (const Chan &c : ch) {
        g.insert(g.end(), c.e.begin(), c.e.end());
        if (c.kind != BZ_ELASTIC) g.push_back(c.th);
    }
    for (const Chan &c : eltab) g.insert(g.end(), c.e.begin(), c.e.end());
    // xi-form gases: each channel names its gas and the gas's elastic channel
    if (n_ch > 0xFFFF) { *err = "at most 65535 channels"; return BZ_EINVAL; }
    for (int j = 0; j < n_ch; ++j) {
        const int gI = ch[j].gas;
        if (gases[gI].angular != BZ_ANG_XI) continue;
        int el = 0;
        for (int k = 0; k < n_ch; ++k)
            if (ch[k].gas == gI && ch[k].kind == BZ_ELASTIC) el = k;
        cp[j].bits |= (gI << 12) | (el << 16);
    }
    std::sort(g.begin(), g.end());
    g.erase(std::unique(g.begin(), g.end()), g.end());
    const int P = (int)g.size();
    const int n_rec = P + 1;
    if (n_rec > 65535) { *err = "more than 65535 union grid points"; return BZ_EINVAL; }
    std::vector<double> Slo(n_rec), Ssl(n_rec);
    std::vector<std::vector<double>> cv(n_rec, std::vector<double>(n_ch, 0.0)), cs = cv;
    int first_tail = n_rec - 1;
    std::vector<size_t> cursor(n_ch, 0);  // per channel: its table interval, moving up with the records
    for (int i = 0; i < n_rec; ++i) {
        double lo = (i == 0) ? 0.0 : g[i - 1];
        double hi = (i < n_rec - 1) ? g[i] : lo * 2.0 + 1.0;
        // record 0 is [0, g0): every channel is on its left extension there
        double mid = (i == 0) ? 0.5 * g[0] : 0.5 * (lo + hi);
        double S = 0.0, sl = 0.0;
        bool any_tail = false;
        for (int j = 0; j < n_ch; ++j) {
            double a, b;
            if (i == n_rec - 1 || !piece(ch[j], mid, &a, &b, &cursor[j])) { any_tail = true; continue; }
            cv[i][j] = ch[j].n * (a + b * lo);
            cs[i][j] = ch[j].n * b;
            S += cv[i][j];
            sl += cs[i][j];
        }
        Slo[i] = S;
        Ssl[i] = sl;
        if (any_tail && i < first_tail) first_tail = i;
    }
    // xi-form gases: the total elastic cross section on the same records
    ElTabs elt;
    elt.val.assign(n_rec, std::vector<double>(n_gases, 0.0));
    elt.slope = elt.val;
    elt.tail.assign(n_gases, ChParam<double>());
    for (int gI = 0; gI < n_gases; ++gI) {
        ChParam<double> &t = elt.tail[gI];
        memset(&t, 0, sizeof t);
        t.bits = 0x100;  // no tail
        const Chan &c = eltab[gI];
        if (gases[gI].angular != BZ_ANG_XI) continue;
        for (int i = 0; i + 1 < n_rec; ++i) {
            double lo = (i == 0) ? 0.0 : g[i - 1];
            double mid = (i == 0) ? 0.5 * g[0] : 0.5 * (lo + g[i]);
            double a, b;
            if (!piece(c, mid, &a, &b)) continue;
            elt.val[i][gI] = c.n * (a + b * lo);
            elt.slope[i][gI] = c.n * b;
        }
        t.e_last = c.e.back();
        t.tail_K = c.tail_K;
        t.tail_logc = c.tail_zero ? 0.0 : log(c.n * c.s.back()) - c.tail_K * log(c.e.back());
        t.bits = c.tail_zero ? 0x100 : 0;
    }
    // exact maximum of nu over [0, eps_cap]
    double cap = (opts && opts->eps_cap_eV > 0.0) ? opts->eps_cap_eV : emax;
    double best = speed_of(g[0]) * Slo[0], best_eps = g[0];
    auto consider = [&](double eps, double S) {
        double v = speed_of(eps) * S;
        if (v > best) { best = v; best_eps = eps; }
    };
    for (int i = 1; i < n_rec; ++i) {
        double lo = g[i - 1];
        if (lo >= cap) break;
        double hi = (i < n_rec - 1) ? std::min(g[i], cap) : cap;
        if (i < first_tail) {
            double B = Ssl[i], A = Slo[i] - B * lo;
            consider(lo, A + B * lo);
            consider(hi, A + B * hi);
            if (B != 0.0) {
                double x = -A / (3.0 * B);
                if (x > lo && x < hi) consider(x, A + B * x);
            }
        } else {
            double rhi = (i < n_rec - 1) ? g[i] : hi;
            auto f = [&](double x) { return speed_of(x) * record_density(ch, tail_logc, lo, rhi, x); };
            const int NS = 2048;
            int arg = 0;
            double vm = -1.0;
            for (int k = 0; k <= NS; ++k) {
                double x = lo + (hi - lo) * k / NS, v = f(x);
                if (v > vm) { vm = v; arg = k; }
            }
            double a = lo + (hi - lo) * std::max(arg - 1, 0) / NS, b = lo + (hi - lo) * std::min(arg + 1, NS) / NS;
            const double gr = 0.6180339887498949;
            double x1 = b - gr * (b - a), x2 = a + gr * (b - a), f1 = f(x1), f2 = f(x2);
            for (int it = 0; it < 200 && (b - a) > 1e-14 * b; ++it) {
                if (f1 < f2) { a = x1; x1 = x2; f1 = f2; x2 = a + gr * (b - a); f2 = f(x2); }
                else { b = x2; x2 = x1; f2 = f1; x1 = b - gr * (b - a); f1 = f(x1); }
            }
            double xs[4] = {lo + (hi - lo) * arg / NS, x1, x2, hi};
            for (double x : xs) {
                double v = f(x);
                if (v > best) { best = v; best_eps = x; }
            }
        }
    }
    double guard = (opts && opts->majorant_guard >= 0.0) ? opts->majorant_guard : 1e-6;
    int ipos = 0;  // first positive union point
    while (ipos < P && g[ipos] <= 0.0) ++ipos;

    // Maximum of nu over each log-uniform energy bin (32 per decade) between
    // the first positive union point and the last one, exact per record:
    // linear records peak at an end or at eps* = -a/(3b); records with a
    // tail are sampled densely and refined.  A relative margin of 1e-9 covers
    // the refinement.
    auto record_max = [&](int i, double a, double b) {
        if (b <= a) return speed_of(b) * (i == 0 ? Slo[0] : 0.0);
        double rlo = (i == 0) ? 0.0 : g[i - 1];
        if (i < first_tail) {
            double B = Ssl[i], A = Slo[i] - B * rlo, m = std::max(speed_of(a) * (A + B * a), speed_of(b) * (A + B * b));
            if (B != 0.0) {
                double x = -A / (3.0 * B);
                if (x > a && x < b) m = std::max(m, speed_of(x) * (A + B * x));
            }
            return m;
        }
        double rhi = (i < n_rec - 1) ? g[i] : b;
        auto f = [&](double x) { return speed_of(x) * record_density(ch, tail_logc, rlo, rhi, x); };
        const int NS = 256;
        int arg = 0;
        double vm = -1.0;
        for (int k = 0; k <= NS; ++k) {
            double x = a + (b - a) * k / NS, v = f(x);
            if (v > vm) { vm = v; arg = k; }
        }
        double lo2 = a + (b - a) * std::max(arg - 1, 0) / NS, hi2 = a + (b - a) * std::min(arg + 1, NS) / NS;
        const double gr = 0.6180339887498949;
        double x1 = hi2 - gr * (hi2 - lo2), x2 = lo2 + gr * (hi2 - lo2), f1 = f(x1), f2 = f(x2);
        for (int it = 0; it < 100 && (hi2 - lo2) > 1e-13 * hi2; ++it) {
            if (f1 < f2) { lo2 = x1; x1 = x2; f1 = f2; x2 = lo2 + gr * (hi2 - lo2); f2 = f(x2); }
            else { hi2 = x2; x2 = x1; f2 = f1; x1 = hi2 - gr * (hi2 - lo2); f1 = f(x1); }
        }
        return std::max(vm, std::max(f1, f2));
    };
    // max of nu over [a, b]: every record that meets the interval
    auto range_max = [&](double a, double b) {
        int i = (int)(std::upper_bound(g.begin(), g.end(), a) - g.begin());  // record holding a
        double m = 0.0;
        for (; i < n_rec; ++i) {
            double rlo = (i == 0) ? 0.0 : g[i - 1];
            double rhi = (i < n_rec - 1) ? g[i] : std::numeric_limits<double>::infinity();
            if (rlo > b) break;
            double x0 = std::max(a, rlo), x1 = std::min(b, rhi);
            if (i == 0) m = std::max(m, speed_of(x1) * Slo[0]);
            else m = std::max(m, record_max(i, x0, x1));
        }
        return m * (1.0 + 1e-9);
    };
    // Bins are 1/fpd decade wide with edges on the lattice 10^(j/fpd)
    // (fpd = 32, halved while the tables would need more than 1024 bins), from
    // the edge at or below the first positive union point to three decades
    // above the last one, so that the maxima are exact in the tails too.
    Bins bins;
    {
        const double d0 = (ipos < P) ? log10(g[ipos]) : 0.0, d1 = log10(g[P - 1] > 0.0 ? g[P - 1] : 1.0) + 3.0;
        int fpd = 32, j0 = 0, nbins = 1;
        for (;;) {
            j0 = (int)floor(fpd * d0);
            int j1 = (int)ceil(fpd * d1);
            if (j1 <= j0) j1 = j0 + 1;
            nbins = j1 - j0;
            if (nbins <= 1024 || fpd == 1) break;
            fpd /= 2;
        }
        nbins = std::min(nbins, 1024);
        auto edge = [&](int j) { return pow(10.0, (double)j / fpd); };
        int levels = 1;
        while ((1 << levels) <= nbins) ++levels;
        bins.n_bins = nbins;
        bins.levels = levels;
        bins.j0 = j0;
        bins.per_decade = fpd;
        bins.max.assign((size_t)levels * nbins, 0.0);
        for (int b = 0; b < nbins; ++b) bins.max[b] = range_max(edge(j0 + b), edge(j0 + b + 1));
        // sparse table for O(1) range maxima
        for (int l = 1; l < levels; ++l)
            for (int b = 0; b + (1 << l) <= nbins; ++b)
                bins.max[(size_t)l * nbins + b] = std::max(bins.max[(size_t)(l - 1) * nbins + b],
                                                           bins.max[(size_t)(l - 1) * nbins + b + (1 << (l - 1))]);
        bins.lo = (float)((double)j0 / fpd * log2(10.0));
        bins.inv_w = (float)(fpd / log2(10.0));
        bins.nu_low = range_max(0.0, edge(j0));
        // below the first union point the density sum is constant, so there
        // nu grows as sqrt(eps)
        bins.low_sqrt = g[0] > 0.0 && edge(j0) <= g[0];
        // record ipos + 1 starts at the first positive union point
        if (ipos < P) {
            const double e1 = g[ipos];
            const int i1 = ipos + 1;
            const double hi1 = (i1 < n_rec - 1) ? g[i1] : 2.0 * e1 + 1.0;
            bins.nu_first = speed_of(e1) * (i1 < first_tail ? Slo[i1] : record_density(ch, tail_logc, e1, hi1, e1));
        } else {
            bins.nu_first = 0.0;
        }
    }

    // shared-memory budgets of the staged tables: three FP32 blocks per SM
    // (72 KB each on a GB300's 228 KB), one FP64 block
    const size_t budget32 = (opts && opts->smem_budget > 0) ? (size_t)opts->smem_budget : kStageBudget32;
    if (!emit<float>(ch, g, Slo, Ssl, cv, cs, cp, first_tail, bins, elt, budget32, &out->blob32, &out->lay32, err) ||
        !emit<double>(ch, g, Slo, Ssl, cv, cs, cp, first_tail, bins, elt, kStageBudget64, &out->blob64, &out->lay64,
                      err))
        return BZ_EINVAL;
    out->n_total = n_total;
    out->nu_max = best;
    out->nu_trial = best * (1.0 + guard);
    bz_mixture_info &I = out->info;
    memset(&I, 0, sizeof I);
    for (int gI = 0; gI < n_gases; ++gI) I.n_xi_gases += gases[gI].angular == BZ_ANG_XI;
    I.nu_max = best;
    I.nu_trial = out->nu_trial;
    I.eps_at_max = best_eps;
    I.eps_cap = cap;
    I.n_total = n_total;
    I.n_gases = n_gases;
    I.n_channels = n_ch;
    I.n_records = n_rec;
    I.n_buckets = out->lay32.n_buckets;
    I.first_tail_record = first_tail;
    return BZ_OK;
}

}  // namespace bz
