/*
 * oracle.c -- plain, slow, FP64 CPU reference of the electron-swarm Monte
 * Carlo step loop of "Betaboltz: a Monte-Carlo simulation tool for gas
 * scattering processes" (Renda, Ciubotaru, Banu; arXiv:1901.08140).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant with the CUDA path and never calls it.
 *
 * Everything is FP64 and follows the paper's steps in order, one particle at
 * a time, one free flight at a time:
 *   - free flight by the null-collision technique, Eq. (3) random_time,
 *     null test Eq. (4) null_fraction (Sec. 2);
 *   - real collision frequency nu(eps) channel by channel, Eq. (2) frequency,
 *     each table linearly interpolated (Sec. 5) and extended per Sec. 2.2,
 *     Eqs. (12)-(14);
 *   - classical motion in uniform static E and B (UniformFieldClassic, Sec. 3.6);
 *   - scattering angle isotropic or screened Coulomb, Eq. (5) collision_angle;
 *   - energy exchange Eq. (8) delta_energy_ela and Eq. (9) delta_energy_ine,
 *     attachment as a plastic collision and ionization with an energy split
 *     (Sec. 2);
 *   - fail detection and revert to the last real collision (Sec. 6).
 * Random numbers come from Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11),
 * implemented here from its published definition.
 *
 * Readings of points the paper leaves open, each with its reason:
 *   - the electric force on the electron points along +z, so W > 0 (the
 *     worked example of Sec. 7 prints a positive drift velocity);
 *   - the flight's uniform is used directly as 1-R (both are uniform on
 *     (0,1), and this spares a subtraction that would round);
 *   - a fail reverts the electron to its last real collision and raises its
 *     trial frequency to 1.25 nu (Sec. 6 names reverting and a 25 % margin);
 *   - the radicand of Eq. (9) is clamped at 0 (it is negative only in the
 *     kinematically closed band just above the threshold);
 *   - the ionization remainder is split uniformly between primary and
 *     secondary (the paper says only that it is shared);
 *   - a dummy attachment leaves the electron at rest (a plastic collision
 *     keeps no kinetic energy);
 *   - an inelastic table that starts above its threshold rises linearly
 *     from (threshold, 0) (Sec. 2.2 sets the cross section to zero below
 *     the threshold and interpolates linearly).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* CODATA 2018 */
#define OR_QE 1.602176634e-19      /* elementary charge [C] */
#define OR_ME 9.1093837015e-31     /* electron mass [kg] */
#define OR_HARTREE_EV 27.211386245988
#define OR_TD 1e-21                /* 1 Townsend [V m^2] */
#define OR_PI 3.14159265358979323846
#define OR_KB 1.380649e-23         /* Boltzmann constant [J/K] */

enum { OR_ELASTIC = 0, OR_EXCITATION = 1, OR_ATTACHMENT = 2, OR_IONIZATION = 3 };
enum { OR_ISOTROPIC = 0, OR_SCREENED_COULOMB = 1, OR_ANG_XI = 2 };
enum { OR_DEC_FAIL = -2, OR_DEC_NULL = -1 };
enum { OR_ST_DONE = 0, OR_ST_TIME = 1, OR_ST_STEPS = 2, OR_ST_TRIAL = 3, OR_ST_ERROR = 4, OR_ST_ATTACHED = 5 };

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11, Sec. 4): 10 rounds of the Philox      */
/* S-P network on a 4x32-bit counter with a 2x32-bit key bumped by the Weyl   */
/* constants after each round.                                                */
/* ------------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform on the open interval (0,1) from the top 23 bits of a word:
 * ((w >> 9) + 1/2) / 2^23.  Every value is an odd multiple of 2^-24 below 1,
 * exactly representable in FP32 and FP64, so an FP32 consumer of the same
 * word sees the same number. */
double or_uniform(uint32_t w) { return ((double)(w >> 9) + 0.5) * (1.0 / 8388608.0); }

static void draw4(uint64_t seed, uint64_t id, uint32_t step, uint32_t sub, double u[4])
{
    uint32_t ctr[4] = {(uint32_t)id, (uint32_t)(id >> 32), step, sub};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t w[4];
    or_philox4x32_10(ctr, key, w);
    for (int i = 0; i < 4; ++i) u[i] = or_uniform(w[i]);
}

/* ------------------------------------------------------------------------ */
/* Mixture: per-channel tables, kept exactly as given.                        */
/* ------------------------------------------------------------------------ */
typedef struct {
    int gas, kind, n;
    double threshold;
    double *e, *s;
} or_channel;

typedef struct {
    double M, n;
    int angular;
    int n_el;          /* xi form: the total elastic cross section table */
    double *e_el, *s_el;
} or_gas;

typedef struct {
    int n_gas, n_ch;
    or_gas *gas;
    or_channel *ch;
    double n_total;
    double eps_cap, nu_max, eps_at_max;
} or_mixture;

/* sigma of one channel at eps [eV] -- Sec. 5 (linear interpolation inside the
 * table) and Sec. 2.2 (extensions): elastic tables extend to the left with
 * their first value, inelastic ones are zero below threshold; to the right a
 * power law sigma = A eps^K through the last two points, Eqs. (12)-(14).
 * Where either of the two points is zero the power law is undefined and the
 * last value is continued. */
static double table_sigma(int kind, double threshold, const double *e, const double *s, int n, double eps)
{
    if (kind != OR_ELASTIC) {
        if (eps < threshold) return 0.0;
        if (eps < e[0]) return s[0] * (eps - threshold) / (e[0] - threshold);
    } else if (eps < e[0]) {
        return s[0];
    }
    if (eps >= e[n - 1]) {
        if (n < 2 || eps == e[n - 1]) return s[n - 1];
        if (s[n - 1] > 0.0 && s[n - 2] > 0.0) {
            double K = log(s[n - 1] / s[n - 2]) / log(e[n - 1] / e[n - 2]);
            double A = s[n - 1] / pow(e[n - 1], K);
            return A * pow(eps, K);
        }
        return s[n - 1];
    }
    int lo = 0, hi = n - 1; /* e[lo] <= eps < e[hi] */
    while (hi - lo > 1) {
        int mid = (lo + hi) / 2;
        if (e[mid] <= eps) lo = mid; else hi = mid;
    }
    return s[lo] + (s[hi] - s[lo]) * (eps - e[lo]) / (e[hi] - e[lo]);
}

double or_sigma(const or_mixture *m, int c, double eps)
{
    const or_channel *ch = &m->ch[c];
    return table_sigma(ch->kind, ch->threshold, ch->e, ch->s, ch->n, eps);
}

/* Total elastic cross section of gas g (xi form), extended like an elastic
 * table (Sec. 2.2). */
static double sigma_el_total(const or_mixture *m, int g, double eps)
{
    const or_gas *G = &m->gas[g];
    return table_sigma(OR_ELASTIC, 0.0, G->e_el, G->s_el, G->n_el, eps);
}

/* Eq. (2): nu(eps) = sqrt(2 eps / m) * sum_k n_k (sigma_k + sum_i sigma_ki).
 * The sum runs gas by gas, channel by channel, adding n_k sigma_kj one term at
 * a time -- the same order in which the channel is later chosen, so that the
 * last cumulative term equals nu exactly. */
static double speed_of(double eps) { return sqrt(2.0 * eps * OR_QE / OR_ME); }

double or_density_sum(const or_mixture *m, double eps)
{
    double S = 0.0;
    for (int c = 0; c < m->n_ch; ++c) S += m->gas[m->ch[c].gas].n * or_sigma(m, c, eps);
    return S;
}

double or_nu(const or_mixture *m, double eps) { return speed_of(eps) * or_density_sum(m, eps); }

/* Channel choice of a real collision: the first channel j whose cumulative
 * frequency sqrt(2 eps/m) sum_{l<=j} n sigma_l reaches r (0 < r <= nu). */
int or_select_channel(const or_mixture *m, double eps, double r)
{
    double v = speed_of(eps), cum = 0.0;
    for (int c = 0; c < m->n_ch; ++c) {
        cum += m->gas[m->ch[c].gas].n * or_sigma(m, c, eps);
        if (v * cum >= r) return c;
    }
    return m->n_ch - 1;
}

/* ------------------------------------------------------------------------ */
/* Trial frequency (Sec. 6.2, LazyTrialFrequency, made exact): the maximum of */
/* nu(eps) over [0, eps_cap].  Between consecutive breakpoints (table points  */
/* and thresholds) where no channel is in its power-law tail the density sum  */
/* is linear, S = a + b eps, so sqrt(eps) (a + b eps) peaks at an end or at   */
/* eps* = -a/(3b).  Pieces with a tail are searched by dense sampling plus a  */
/* golden-section refinement.                                                 */
/* ------------------------------------------------------------------------ */
static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

static void consider(const or_mixture *m, double eps, double *best, double *best_eps)
{
    if (!(eps >= 0.0)) return;
    double v = or_nu(m, eps);
    if (v > *best) { *best = v; *best_eps = eps; }
}

static double linear_piece_value(double a, double b, double eps) { return sqrt(eps) * (a + b * eps); }

void or_majorant(or_mixture *m, double eps_cap)
{
    int total = 0;
    for (int c = 0; c < m->n_ch; ++c) total += m->ch[c].n + 1;
    double *bp = (double *)malloc(sizeof(double) * (size_t)(total + 2));
    int nb = 0;
    for (int c = 0; c < m->n_ch; ++c) {
        for (int i = 0; i < m->ch[c].n; ++i)
            if (m->ch[c].e[i] < eps_cap) bp[nb++] = m->ch[c].e[i];
        if (m->ch[c].kind != OR_ELASTIC && m->ch[c].threshold < eps_cap) bp[nb++] = m->ch[c].threshold;
    }
    bp[nb++] = eps_cap;
    qsort(bp, (size_t)nb, sizeof(double), cmp_double);
    int u = 0;
    for (int i = 0; i < nb; ++i)
        if (u == 0 || bp[i] != bp[u - 1]) bp[u++] = bp[i];
    nb = u;

    double best = 0.0, best_eps = 0.0;
    /* below the first breakpoint the density sum is constant (its value at 0),
     * so nu grows with eps up to the breakpoint */
    {
        double v = speed_of(bp[0]) * or_density_sum(m, 0.0);
        if (v > best) { best = v; best_eps = bp[0]; }
    }
    consider(m, bp[0], &best, &best_eps);
    for (int i = 0; i + 1 < nb; ++i) {
        double lo = bp[i], hi = bp[i + 1], w = hi - lo;
        int tail = 0;
        for (int c = 0; c < m->n_ch; ++c)
            if (m->ch[c].e[m->ch[c].n - 1] < hi) tail = 1;
        if (!tail) {
            double e1 = lo + w / 3.0, e2 = lo + 2.0 * w / 3.0;
            double s1 = or_density_sum(m, e1), s2 = or_density_sum(m, e2);
            double b = (s2 - s1) / (e2 - e1), a = s1 - b * e1;
            double k = sqrt(2.0 * OR_QE / OR_ME);
            double cand[3] = {lo, hi, (b != 0.0) ? -a / (3.0 * b) : lo};
            for (int j = 0; j < 3; ++j) {
                double x = cand[j];
                if (!(x >= lo && x <= hi)) continue;
                double v = k * linear_piece_value(a, b, x);
                if (v > best) { best = v; best_eps = x; }
            }
        } else {
            const int NS = 1024;
            int arg = 0;
            double vmax = -1.0;
            for (int j = 0; j <= NS; ++j) {
                double x = lo + w * (double)j / NS;
                double v = or_nu(m, x);
                if (v > vmax) { vmax = v; arg = j; }
            }
            double a = lo + w * (double)(arg > 0 ? arg - 1 : 0) / NS;
            double b = lo + w * (double)(arg < NS ? arg + 1 : NS) / NS;
            const double g = 0.6180339887498949;
            double x1 = b - g * (b - a), x2 = a + g * (b - a);
            double f1 = or_nu(m, x1), f2 = or_nu(m, x2);
            for (int it = 0; it < 200 && (b - a) > 1e-14 * b; ++it) {
                if (f1 < f2) { a = x1; x1 = x2; f1 = f2; x2 = a + g * (b - a); f2 = or_nu(m, x2); }
                else { b = x2; x2 = x1; f2 = f1; x1 = b - g * (b - a); f1 = or_nu(m, x1); }
            }
            consider(m, lo + w * (double)arg / NS, &best, &best_eps);
            consider(m, x1, &best, &best_eps);
            consider(m, x2, &best, &best_eps);
            consider(m, hi, &best, &best_eps);
        }
    }
    free(bp);
    m->eps_cap = eps_cap;
    m->nu_max = best;
    m->eps_at_max = best_eps;
}

/* Maximum of nu over [a, b] -- the per-bin maximum of BinnedTrialFrequency
 * (Sec. 6.3) -- by the same piecewise analysis as the majorant: between two
 * consecutive breakpoints inside [a, b] with no channel in its power-law
 * tail, nu = sqrt(eps) (A + B eps) up to a constant, maximal at an end or at
 * eps* = -A/(3B); pieces with a tail are sampled densely and refined. */
double or_range_max(const or_mixture *m, double a, double b)
{
    if (!(a >= 0.0)) a = 0.0;
    if (!(b > a)) return or_nu(m, a);
    int total = 2;
    for (int c = 0; c < m->n_ch; ++c) total += m->ch[c].n + 1;
    double *bp = (double *)malloc(sizeof(double) * (size_t)total);
    int nb = 0;
    bp[nb++] = a;
    bp[nb++] = b;
    for (int c = 0; c < m->n_ch; ++c) {
        for (int i = 0; i < m->ch[c].n; ++i)
            if (m->ch[c].e[i] > a && m->ch[c].e[i] < b) bp[nb++] = m->ch[c].e[i];
        if (m->ch[c].kind != OR_ELASTIC && m->ch[c].threshold > a && m->ch[c].threshold < b)
            bp[nb++] = m->ch[c].threshold;
    }
    qsort(bp, (size_t)nb, sizeof(double), cmp_double);
    int u = 0;
    for (int i = 0; i < nb; ++i)
        if (u == 0 || bp[i] != bp[u - 1]) bp[u++] = bp[i];
    nb = u;
    double best = 0.0, dummy = 0.0;
    const double k = sqrt(2.0 * OR_QE / OR_ME);
    for (int i = 0; i + 1 < nb; ++i) {
        double lo = bp[i], hi = bp[i + 1], w = hi - lo;
        int tail = 0;
        for (int c = 0; c < m->n_ch; ++c)
            if (m->ch[c].e[m->ch[c].n - 1] < hi) tail = 1;
        if (!tail) {
            double e1 = lo + w / 3.0, e2 = lo + 2.0 * w / 3.0;
            double s1 = or_density_sum(m, e1), s2 = or_density_sum(m, e2);
            double B = (s2 - s1) / (e2 - e1), A = s1 - B * e1;
            double cand[3] = {lo, hi, (B != 0.0) ? -A / (3.0 * B) : lo};
            for (int j = 0; j < 3; ++j) {
                double x = cand[j];
                if (!(x >= lo && x <= hi)) continue;
                double v = k * linear_piece_value(A, B, x);
                if (v > best) best = v;
            }
        } else {
            const int NS = 1024;
            int arg = 0;
            double vmax = -1.0;
            for (int j = 0; j <= NS; ++j) {
                double v = or_nu(m, lo + w * (double)j / NS);
                if (v > vmax) { vmax = v; arg = j; }
            }
            double x0 = lo + w * (double)(arg > 0 ? arg - 1 : 0) / NS;
            double x3 = lo + w * (double)(arg < NS ? arg + 1 : NS) / NS;
            const double g = 0.6180339887498949;
            double x1 = x3 - g * (x3 - x0), x2 = x0 + g * (x3 - x0);
            double f1 = or_nu(m, x1), f2 = or_nu(m, x2);
            for (int it = 0; it < 200 && (x3 - x0) > 1e-14 * x3; ++it) {
                if (f1 < f2) { x0 = x1; x1 = x2; f1 = f2; x2 = x0 + g * (x3 - x0); f2 = or_nu(m, x2); }
                else { x3 = x2; x2 = x1; f2 = f1; x1 = x3 - g * (x3 - x0); f1 = or_nu(m, x1); }
            }
            consider(m, lo + w * (double)arg / NS, &best, &dummy);
            consider(m, x1, &best, &dummy);
            consider(m, x2, &best, &dummy);
            consider(m, lo, &best, &dummy);
            consider(m, hi, &best, &dummy);
        }
    }
    free(bp);
    return best;
}

/* BinnedTrialFrequency (Sec. 6.3): bins_per_decade log-uniform bins per
 * decade of energy, bin j = [10^(j/B), 10^((j+1)/B)) with j = floor(B log10 eps);
 * the trial frequency of an energy is the maximum of nu over its bin. */
static int binned_index(int B, double eps) { return (int)floor((double)B * log10(eps)); }

double or_binned_max(const or_mixture *m, int B, int j)
{
    return or_range_max(m, pow(10.0, (double)j / B), pow(10.0, (double)(j + 1) / B));
}

/* Bin maxima of the bins that hold the mixture's tables, computed once per
 * run; other bins are computed when met. */
typedef struct {
    int B, j0, n;
    double *max;
    double nu_first;  /* floor of the adaptive nu' */
} or_binned;

static void binned_setup(const or_mixture *m, int B, or_binned *bt)
{
    bt->B = B;
    bt->n = 0;
    bt->max = NULL;
    if (B <= 0) return;
    double lo = INFINITY, hi = 0.0;
    for (int c = 0; c < m->n_ch; ++c) {
        const or_channel *ch = &m->ch[c];
        for (int i = 0; i < ch->n; ++i)
            if (ch->e[i] > 0.0) { lo = fmin(lo, ch->e[i]); hi = fmax(hi, ch->e[i]); }
    }
    if (!(hi > 0.0)) return;
    bt->j0 = binned_index(B, lo) - 1;
    bt->n = binned_index(B, hi * 1e3) + 2 - bt->j0;   /* and three decades of tails */
    bt->max = (double *)malloc(sizeof(double) * (size_t)bt->n);
    for (int i = 0; i < bt->n; ++i) bt->max[i] = or_binned_max(m, B, bt->j0 + i);
}

static double binned_nu(const or_mixture *m, const or_binned *bt, double eps)
{
    if (!(eps > 0.0)) return 0.0;
    int j = binned_index(bt->B, eps);
    if (j >= bt->j0 && j < bt->j0 + bt->n) return bt->max[j - bt->j0];
    return or_binned_max(m, bt->B, j);
}

void or_mixture_destroy(or_mixture *m);

/* Mixture from flat arrays (tables are copied). Returns 0 or -1 on bad input
 * (an xi-form gas needs its total elastic cross section table). */
int or_mixture_create(int n_gas, const double *gas_mass, const double *gas_density, const int *gas_angular,
                      int n_ch, const int *ch_gas, const int *ch_kind, const double *ch_threshold,
                      const int64_t *ch_offset, const int *ch_n, const double *energy, const double *sigma,
                      const int64_t *gas_el_offset, const int *gas_el_n, const double *el_energy,
                      const double *el_sigma, double eps_cap, or_mixture **out)
{
    *out = NULL;
    if (n_gas <= 0 || n_ch <= 0) return -1;
    or_mixture *m = (or_mixture *)calloc(1, sizeof(or_mixture));
    m->n_gas = n_gas;
    m->n_ch = n_ch;
    m->gas = (or_gas *)calloc((size_t)n_gas, sizeof(or_gas));
    m->ch = (or_channel *)calloc((size_t)n_ch, sizeof(or_channel));
    double emax = 0.0;
    for (int g = 0; g < n_gas; ++g) {
        m->gas[g].M = gas_mass[g];
        m->gas[g].n = gas_density[g];
        m->gas[g].angular = gas_angular[g];
        m->n_total += gas_density[g];
        int ne = gas_el_n ? gas_el_n[g] : 0;
        if (gas_angular[g] == OR_ANG_XI && ne < 1) { or_mixture_destroy(m); return -1; }
        m->gas[g].n_el = ne;
        if (ne > 0) {
            m->gas[g].e_el = (double *)malloc(sizeof(double) * (size_t)ne);
            m->gas[g].s_el = (double *)malloc(sizeof(double) * (size_t)ne);
            memcpy(m->gas[g].e_el, el_energy + gas_el_offset[g], sizeof(double) * (size_t)ne);
            memcpy(m->gas[g].s_el, el_sigma + gas_el_offset[g], sizeof(double) * (size_t)ne);
        }
    }
    for (int c = 0; c < n_ch; ++c) {
        or_channel *ch = &m->ch[c];
        ch->gas = ch_gas[c];
        ch->kind = ch_kind[c];
        ch->threshold = ch_threshold[c];
        ch->n = ch_n[c];
        ch->e = (double *)malloc(sizeof(double) * (size_t)ch->n);
        ch->s = (double *)malloc(sizeof(double) * (size_t)ch->n);
        memcpy(ch->e, energy + ch_offset[c], sizeof(double) * (size_t)ch->n);
        memcpy(ch->s, sigma + ch_offset[c], sizeof(double) * (size_t)ch->n);
        if (ch->n > 0 && ch->e[ch->n - 1] > emax) emax = ch->e[ch->n - 1];
    }
    or_majorant(m, eps_cap > 0.0 ? eps_cap : emax);
    *out = m;
    return 0;
}

void or_mixture_destroy(or_mixture *m)
{
    if (!m) return;
    for (int c = 0; c < m->n_ch; ++c) { free(m->ch[c].e); free(m->ch[c].s); }
    for (int g = 0; g < m->n_gas; ++g) { free(m->gas[g].e_el); free(m->gas[g].s_el); }
    free(m->ch);
    free(m->gas);
    free(m);
}

double or_mixture_nu_max(const or_mixture *m) { return m->nu_max; }
double or_mixture_eps_at_max(const or_mixture *m) { return m->eps_at_max; }
double or_mixture_n_total(const or_mixture *m) { return m->n_total; }

/* ------------------------------------------------------------------------ */
/* Scattering (Sec. 2).                                                      */
/* ------------------------------------------------------------------------ */
/* Eq. (5) collision_angle (screened Coulomb, eps in Hartree) or isotropic. */
double or_cos_theta(int angular, double eps_eV, double R)
{
    if (angular == OR_SCREENED_COULOMB) {
        double e = eps_eV / OR_HARTREE_EV;
        return 1.0 - 2.0 * R / (1.0 + 8.0 * e * (1.0 - R));
    }
    return 1.0 - 2.0 * R;
}

/* Right-hand side of the xi equation (Eq. 7): the ratio sigma_mt/sigma_el
 * that the xi form (Eq. 6) yields,
 *   r(xi) = (1 - xi)/(2 xi^2) ((1 + xi) ln((1 + xi)/(1 - xi)) - 2 xi),
 * 1 at xi = 0 (isotropic), 2 at xi = -1, 0 at xi = 1.  Near 0 the bracket
 * cancels to O(xi^2); there the same function is summed from its Taylor
 * series, 1 - 2 sum_k xi^(2k+1) / ((2k+1)(2k+3)), obtained by expanding the
 * logarithm. */
double or_xi_ratio(double xi)
{
    if (fabs(xi) < 0.05) {
        double sum = 0.0, p = xi; /* xi^(2k+1) */
        for (int k = 0; k < 40; ++k) {
            sum += p / ((2.0 * k + 1.0) * (2.0 * k + 3.0));
            p *= xi * xi;
        }
        return 1.0 - 2.0 * sum;
    }
    double L = log((1.0 + xi) / (1.0 - xi));
    return (1.0 - xi) / (2.0 * xi * xi) * ((1.0 + xi) * L - 2.0 * xi);
}

/* xi with or_xi_ratio(xi) = r, by bisection on (-1, 1), where the ratio falls
 * monotonically from 2 to 0; r outside (0, 2) gives the nearer end. */
double or_xi_solve(double r)
{
    double lo = -1.0, hi = 1.0;
    for (int it = 0; it < 200 && hi - lo > 1e-16; ++it) {
        double mid = 0.5 * (lo + hi);
        if (or_xi_ratio(mid) > r) lo = mid;
        else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* Eq. (6): cos theta of the xi form for non-polar molecules. */
double or_cos_theta_xi(double xi, double R) { return 1.0 - 2.0 * R * (1.0 - xi) / (1.0 + xi * (1.0 - 2.0 * R)); }

/* xi of gas g at energy eps (Eq. 7): from the ratio of its momentum-transfer
 * cross section (the sum of its elastic channels) to its total elastic one;
 * 0 (isotropic) where the total elastic cross section vanishes. */
double or_gas_xi(const or_mixture *m, int g, double eps)
{
    if (m->gas[g].n_el < 1) return 0.0; /* no total elastic table: isotropic */
    double smt = 0.0;
    for (int k = 0; k < m->n_ch; ++k)
        if (m->ch[k].gas == g && m->ch[k].kind == OR_ELASTIC) smt += or_sigma(m, k, eps);
    double sel = sigma_el_total(m, g, eps);
    return sel > 0.0 ? or_xi_solve(smt / sel) : 0.0;
}

/* Eq. (8) delta_energy_ela: eps_f/eps_i for an elastic collision. */
double or_ratio_elastic(double m, double M, double cos_t)
{
    return 1.0 - 2.0 * m * M * (1.0 - cos_t) / ((m + M) * (m + M));
}

/* Eq. (9) delta_energy_ine: eps_f/eps_i for an inelastic collision with loss
 * eps_k.  The radicand is clamped at 0 and the result at 0 (the formula is
 * undefined in the kinematically closed band eps_k <= eps_i < eps_k (m+M)/M). */
double or_ratio_inelastic(double m, double M, double eps_i, double eps_k, double cos_t)
{
    double x = eps_k / eps_i;
    double rad = 1.0 - (m + M) / M * x;
    if (rad < 0.0) rad = 0.0;
    double r = 1.0 - M / (m + M) * x + 2.0 * m * M / ((m + M) * (m + M)) * (sqrt(rad) * cos_t - 1.0);
    return r < 0.0 ? 0.0 : r;
}

/* New direction: d rotated by polar angle theta and azimuth phi about itself.
 * The azimuth origin e1 = (a x d)/|a x d| uses the coordinate axis a along the
 * smallest |component| of d (first such axis on ties); e2 = d x e1. */
void or_rotate(const double d[3], double cos_t, double phi, double out[3])
{
    double ax = fabs(d[0]), ay = fabs(d[1]), az = fabs(d[2]);
    double e1[3];
    if (ax <= ay && ax <= az) { e1[0] = 0.0; e1[1] = -d[2]; e1[2] = d[1]; }
    else if (ay <= az) { e1[0] = d[2]; e1[1] = 0.0; e1[2] = -d[0]; }
    else { e1[0] = -d[1]; e1[1] = d[0]; e1[2] = 0.0; }
    double nrm = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
    e1[0] /= nrm; e1[1] /= nrm; e1[2] /= nrm;
    double e2[3] = {d[1] * e1[2] - d[2] * e1[1], d[2] * e1[0] - d[0] * e1[2], d[0] * e1[1] - d[1] * e1[0]};
    double st = sqrt(fmax(0.0, 1.0 - cos_t * cos_t));
    double cp = cos(phi), sp = sin(phi);
    for (int i = 0; i < 3; ++i) out[i] = cos_t * d[i] + st * (cp * e1[i] + sp * e2[i]);
}

/* ------------------------------------------------------------------------ */
/* Motion in uniform static fields (Sec. 3.6, UniformFieldClassic).          */
/* The electron (q = -e) is pushed along +z by the electric force with       */
/* acceleration a = eE/m; B = |B| (sin thB, 0, cos thB).  With B != 0 the    */
/* velocity splits into a part along b = B/|B| (uniformly accelerated), the  */
/* E x B drift v_D = (b x a z)/w and a remainder u rotating about b at       */
/* w = e|B|/m:  u(t) = u0 cos wt + (b x u0) sin wt.                           */
/* ------------------------------------------------------------------------ */
typedef struct {
    double a;              /* eE/m along +z [m/s^2] */
    double B;              /* |B| [T] */
    double b[3];           /* unit B */
    double w;              /* e|B|/m */
    double E;              /* |E| [V/m] */
} or_field;

static void field_setup(or_field *f, double e_over_n_Td, double n_total, double b_T, double angle)
{
    f->E = e_over_n_Td * OR_TD * n_total;
    f->a = OR_QE * f->E / OR_ME;
    f->B = b_T;
    f->b[0] = sin(angle); f->b[1] = 0.0; f->b[2] = cos(angle);
    f->w = OR_QE * b_T / OR_ME;
}

static void cross(const double a[3], const double b[3], double o[3])
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

void or_move(const or_field *f, double x[3], double v[3], double dt)
{
    if (f->B == 0.0) {
        x[0] += v[0] * dt;
        x[1] += v[1] * dt;
        x[2] += v[2] * dt + 0.5 * f->a * dt * dt;
        v[2] += f->a * dt;
        return;
    }
    const double *b = f->b;
    double az[3] = {0.0, 0.0, f->a};
    double bxa[3];
    cross(b, az, bxa);
    double vD[3] = {bxa[0] / f->w, bxa[1] / f->w, bxa[2] / f->w};
    double a_par = f->a * b[2];
    double v_par = v[0] * b[0] + v[1] * b[1] + v[2] * b[2];
    double u0[3], bxu[3];
    for (int i = 0; i < 3; ++i) u0[i] = v[i] - v_par * b[i] - vD[i];
    cross(b, u0, bxu);
    double wt = f->w * dt, c = cos(wt), s = sin(wt), h = sin(0.5 * wt);
    double omc = 2.0 * h * h; /* 1 - cos(wt) */
    for (int i = 0; i < 3; ++i) {
        x[i] += (v_par * dt + 0.5 * a_par * dt * dt) * b[i] + vD[i] * dt + (u0[i] * s + bxu[i] * omc) / f->w;
        v[i] = (v_par + a_par * dt) * b[i] + vD[i] + u0[i] * c + bxu[i] * s;
    }
}

/* Exported for the motion pins: one flight of duration dt. */
void or_move_flat(double e_over_n_Td, double n_total, double b_T, double angle, double *x, double *v, double dt)
{
    or_field f;
    field_setup(&f, e_over_n_Td, n_total, b_T, angle);
    or_move(&f, x, v, dt);
}

/* ------------------------------------------------------------------------ */
/* Swarm run.                                                                */
/* ------------------------------------------------------------------------ */
typedef struct {
    double e_over_n_Td, b_T, b_angle_rad;
    double nu_trial;          /* >0: start value of nu' (fixed mode: the value) */
    int fixed;                /* 1: FixedTrialFrequency -- a fail stops the particle */
    uint32_t real_collisions; /* I */
    double t_end;             /* >0: time limit [s] */
    double eps0_mean_eV;      /* Maxwellian start, mean energy */
    uint64_t seed;
    uint64_t max_trials;
    int attach_keep_state;    /* 1: a dummy attachment leaves the electron unchanged */
    int spawn;                /* 1: ionizations create electrons, attachments remove them */
    uint64_t pop_cap;         /* spawn mode: at most this many electrons in all */
    int strategy;             /* trial frequency (Sec. 6): 0 constant (Lazy / given / Fixed),
                                 1 VariableTrialFrequency, 2 BinnedTrialFrequency */
    double zeta;              /* Variable: nu' = (1 + zeta) nu(eps) */
    uint32_t grace;           /* Variable, Binned: collisions between two queries of nu' */
    int bins_per_decade;      /* Binned */
    double gas_T;             /* > 0: gas temperature [K]: targets move (Sec. 2.1); 0: targets at rest */
} or_config;

#define OR_TF_CONST 0
#define OR_TF_VARIABLE 1
#define OR_TF_BINNED 2

/* Identifier of the electron that the ionization at `step` of electron
 * `parent` creates: the SplitMix64 finaliser (Steele, Lea, Flood 2014) of
 * parent * 0x9E3779B97F4A7C15 + step + 1, with the top bit set so that it
 * never equals a primary's id. */
uint64_t or_secondary_id(uint64_t parent, uint32_t step)
{
    uint64_t z = parent * 0x9E3779B97F4A7C15ull + (uint64_t)step + 1ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return z | 0x8000000000000000ull;
}

typedef struct {
    double *x, *y, *z, *t, *vx, *vy, *vz, *sum_e, *sum_e2, *nu_p;
    uint32_t *n_real, *n_null, *n_fail, *n_ion, *n_att, *steps, *status;
} or_particles;

static void init_velocity(const or_config *cf, uint64_t id, double v[3])
{
    double u[4];
    draw4(cf->seed, id, 0u, 2u, u);
    double kT = (2.0 / 3.0) * cf->eps0_mean_eV * OR_QE; /* mean energy = 3/2 kT */
    double sv = sqrt(kT / OR_ME);
    double r0 = sqrt(-2.0 * log(u[0])), r1 = sqrt(-2.0 * log(u[2]));
    v[0] = sv * r0 * cos(2.0 * OR_PI * u[1]);
    v[1] = sv * r0 * sin(2.0 * OR_PI * u[1]);
    v[2] = sv * r1 * cos(2.0 * OR_PI * u[3]);
}

/* One real collision on channel c at energy eps (velocity v is updated).
 * For an ionization, sec_v receives the secondary's velocity (the ejected
 * electron takes the fraction w0 of the energy left after Eq. (9) and
 * leaves isotropically: cos = 1 - 2 w1, azimuth 2 pi w2). */
/* Sec. 2.1: a collision with a moving target, worked in the centre-of-
 * momentum frame.  v1, v2: bullet and target velocities (mass m, M); the
 * bullet's velocity relative to the centre of momentum keeps its length less
 * what the energy loss eps_k [eV] takes,
 *   |v1' - Vcm|^2 = |v1 - Vcm|^2 - 2 eps_k M / ((m + M) m),
 * (clamped at 0) and turns by (cos_t, phi) about its own direction; the
 * target takes the opposite momentum in that frame. */
void or_thermal_collide(const double v1[3], const double v2[3], double m, double M, double eps_k, double cos_t,
                        double phi, double v1_out[3], double v2_out[3])
{
    double vcm[3], g[3];
    for (int i = 0; i < 3; ++i) {
        vcm[i] = (m * v1[i] + M * v2[i]) / (m + M);
        g[i] = v1[i] - vcm[i];
    }
    double gn = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    double d[3] = {0.0, 0.0, 1.0};
    if (gn > 0.0) { d[0] = g[0] / gn; d[1] = g[1] / gn; d[2] = g[2] / gn; }
    double gp = sqrt(fmax(0.0, gn * gn - 2.0 * eps_k * OR_QE * M / ((m + M) * m)));
    double nd[3];
    or_rotate(d, cos_t, phi, nd);
    for (int i = 0; i < 3; ++i) {
        v1_out[i] = vcm[i] + gp * nd[i];
        if (v2_out) v2_out[i] = vcm[i] - (m / M) * gp * nd[i];
    }
}

/* Target velocity of the real collision at `step` (Sec. 2.1): Maxwell-
 * Boltzmann at temperature T, each component normal with variance kT/M
 * (Box-Muller on the fourth draw of the step, sub-counter 3). */
static void target_velocity(const or_config *cf, uint64_t id, uint32_t step, double M, double v2[3])
{
    double w[4];
    draw4(cf->seed, id, step, 3u, w);
    double st = sqrt(OR_KB * cf->gas_T / M);
    double r0 = sqrt(-2.0 * log(w[0])), r1 = sqrt(-2.0 * log(w[2]));
    v2[0] = st * r0 * cos(2.0 * OR_PI * w[1]);
    v2[1] = st * r0 * sin(2.0 * OR_PI * w[1]);
    v2[2] = st * r1 * cos(2.0 * OR_PI * w[3]);
}

static void collide(const or_mixture *m, const or_config *cf, uint64_t id, uint32_t step, int c, double eps,
                    const double u[4], double v[3], double *eps_f, int *ion, int *att, double sec_v[3])
{
    const or_channel *ch = &m->ch[c];
    const or_gas *g = &m->gas[ch->gas];
    double cos_t = (g->angular == OR_ANG_XI) ? or_cos_theta_xi(or_gas_xi(m, ch->gas, eps), u[2])
                                             : or_cos_theta(g->angular, eps, u[2]);
    double phi = 2.0 * OR_PI * u[3];
    double ratio;
    *ion = 0;
    *att = 0;
    if (cf->gas_T > 0.0 && ch->kind != OR_ATTACHMENT) {
        /* Sec. 2.1: moving targets; the lab energy after the collision, then
         * for an ionization the split with the secondary as below */
        double v2[3], v1p[3];
        target_velocity(cf, id, step, g->M, v2);
        or_thermal_collide(v, v2, OR_ME, g->M, ch->kind == OR_ELASTIC ? 0.0 : ch->threshold, cos_t, phi, v1p, NULL);
        double ef = 0.5 * OR_ME * (v1p[0] * v1p[0] + v1p[1] * v1p[1] + v1p[2] * v1p[2]) / OR_QE;
        double keep = 1.0;
        if (ch->kind == OR_IONIZATION) {
            double w[4];
            draw4(cf->seed, id, step, 1u, w);
            double es = w[0] * ef;
            double ss = sqrt(2.0 * es * OR_QE / OR_ME), cs = 1.0 - 2.0 * w[1], sn = sqrt(fmax(0.0, 1.0 - cs * cs));
            sec_v[0] = ss * sn * cos(2.0 * OR_PI * w[2]);
            sec_v[1] = ss * sn * sin(2.0 * OR_PI * w[2]);
            sec_v[2] = ss * cs;
            keep = 1.0 - w[0];
            *ion = 1;
        }
        double sk = sqrt(keep);
        for (int i = 0; i < 3; ++i) v[i] = v1p[i] * sk;
        *eps_f = keep * ef;
        return;
    }
    /* The scattered direction.  Isotropic scattering (Sec. 2) sends the
     * electron in a direction uniform on the sphere whatever its incident
     * one, so that direction is taken in the lab frame from the same two
     * draws (polar cosine cos_t, azimuth phi), and Eqs. (8)-(9) take the
     * cosine between the incident and the new direction; the other angular
     * models turn the incident direction by (cos_t, phi). */
    double speed = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    double d[3] = {0.0, 0.0, 1.0};
    if (speed > 0.0) { d[0] = v[0] / speed; d[1] = v[1] / speed; d[2] = v[2] / speed; }
    double nd[3];
    if (g->angular == OR_ISOTROPIC) {
        double st = sqrt(fmax(0.0, 1.0 - cos_t * cos_t));
        nd[0] = st * cos(phi);
        nd[1] = st * sin(phi);
        nd[2] = cos_t;
        cos_t = d[0] * nd[0] + d[1] * nd[1] + d[2] * nd[2];
    } else {
        or_rotate(d, cos_t, phi, nd);
    }
    if (ch->kind == OR_ELASTIC) {
        ratio = or_ratio_elastic(OR_ME, g->M, cos_t);
    } else if (ch->kind == OR_ATTACHMENT) {
        *att = 1;
        if (cf->attach_keep_state) { *eps_f = eps; return; }
        ratio = 0.0; /* plastic collision: all energy is given up */
    } else {
        ratio = or_ratio_inelastic(OR_ME, g->M, eps, ch->threshold, cos_t);
        if (ch->kind == OR_IONIZATION) {
            double w[4];
            draw4(cf->seed, id, step, 1u, w);
            double es = w[0] * ratio * eps;   /* the secondary's energy */
            double ss = sqrt(2.0 * es * OR_QE / OR_ME), cs = 1.0 - 2.0 * w[1], sn = sqrt(fmax(0.0, 1.0 - cs * cs));
            sec_v[0] = ss * sn * cos(2.0 * OR_PI * w[2]);
            sec_v[1] = ss * sn * sin(2.0 * OR_PI * w[2]);
            sec_v[2] = ss * cs;
            ratio *= (1.0 - w[0]); /* the secondary takes w0 of the remainder */
            *ion = 1;
        }
    }
    double sp = speed * sqrt(ratio);
    v[0] = sp * nd[0]; v[1] = sp * nd[1]; v[2] = sp * nd[2];
    *eps_f = ratio * eps;
}

static double energy_of(const double v[3]) { return 0.5 * OR_ME * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) / OR_QE; }

/* Spawn bookkeeping of one particle run (spawn mode). */
typedef struct {
    uint64_t *ids;     /* secondaries created, in order */
    double *t_birth;   /* absolute birth time */
    double *v_birth;   /* 3 per secondary */
    int64_t n, cap;    /* count, room */
} or_spawns;

/* Runs one electron from birth (time t0, velocity v0; t0 = 0 and a
 * Maxwellian start for primaries) to its limiters.  Positions and times are
 * kept relative to birth; the time limit is absolute. */
/* nu at the lowest positive energy of any table or threshold. */
static double nu_at_first_point(const or_mixture *m)
{
    double lo = INFINITY;
    for (int c = 0; c < m->n_ch; ++c) {
        const or_channel *ch = &m->ch[c];
        for (int i = 0; i < ch->n; ++i)
            if (ch->e[i] > 0.0) lo = fmin(lo, ch->e[i]);
        if (ch->kind != OR_ELASTIC && ch->threshold > 0.0) lo = fmin(lo, ch->threshold);
    }
    return isfinite(lo) ? or_nu(m, lo) : 0.0;
}

/* Trial frequency of the adaptive strategies (Sec. 6) at energy eps:
 * Variable (1 + zeta) nu(eps), Binned the maximum of nu over the bin of eps;
 * neither below nu at the lowest table energy (nu vanishes at eps = 0, and
 * the tables say nothing below their first point). */
static double adaptive_nu(const or_mixture *m, const or_config *cf, const or_binned *bt, double eps)
{
    double floor_nu = fmax(1e-9 * m->nu_max, bt->nu_first);
    if (cf->strategy == OR_TF_VARIABLE) return (1.0 + cf->zeta) * fmax(or_nu(m, eps), floor_nu);
    return fmax(binned_nu(m, bt, eps), floor_nu);
}

static void run_particle_from(const or_mixture *m, const or_config *cf, const or_field *f, const or_binned *bt,
                              uint64_t id, double t0, const double *v0, const or_particles *P, int64_t slot,
                              or_spawns *sp)
{
    double x[3] = {0.0, 0.0, 0.0}, v[3], t = 0.0;
    if (v0) { v[0] = v0[0]; v[1] = v0[1]; v[2] = v0[2]; }
    else init_velocity(cf, id, v);
    double sx[3] = {0, 0, 0}, sv[3] = {v[0], v[1], v[2]}, st = 0.0; /* last real collision */
    /* Sec. 6: the adaptive strategies query nu' at the start, keep it for
     * `grace` collisions (null or real), query again, and on a fail go back
     * to the last real collision and query with the fail's energy. */
    const int adaptive = cf->strategy == OR_TF_VARIABLE || cf->strategy == OR_TF_BINNED;
    double nu_p = adaptive ? adaptive_nu(m, cf, bt, energy_of(v)) : cf->nu_trial;
    uint32_t grace_left = cf->grace;
    int retried = 0; /* Binned: nu' comes from a retry after a fail */
    double sum_e = 0.0, sum_e2 = 0.0;
    uint32_t n_real = 0, n_null = 0, n_fail = 0, n_ion = 0, n_att = 0, k = 0, status = OR_ST_DONE;
    while (n_real < cf->real_collisions) {
        if ((uint64_t)k >= cf->max_trials) { status = OR_ST_STEPS; break; }
        double u[4];
        uint32_t step = k++;
        draw4(cf->seed, id, step, 0u, u);
        /* Eq. (3): t_c = -ln(1-R)/nu'; the draw u0 plays the role of 1-R. */
        double tau = -log(u[0]) / nu_p;
        if (cf->t_end > 0.0 && t0 + t + tau >= cf->t_end) {
            or_move(f, x, v, cf->t_end - t0 - t);
            t = cf->t_end - t0;
            status = OR_ST_TIME;
            break;
        }
        or_move(f, x, v, tau);
        t += tau;
        double eps = energy_of(v);
        double nu = or_nu(m, eps);
        if (nu > nu_p) { /* fail: Sec. 6 -- back to the last real collision */
            ++n_fail;
            int error = cf->fixed; /* FixedTrialFrequency: a fail is an error */
            if (cf->strategy == OR_TF_BINNED) {
                /* retry with the larger maximum of the two bins; a fail
                 * under that nu' (before a real collision or a new query)
                 * is an error */
                error = retried;
                retried = 1;
            }
            for (int i = 0; i < 3; ++i) { x[i] = sx[i]; v[i] = sv[i]; }
            t = st;
            if (error) { status = OR_ST_TRIAL; break; } /* stopped at its last valid state */
            if (cf->strategy == OR_TF_VARIABLE) nu_p = adaptive_nu(m, cf, bt, eps);
            else if (cf->strategy == OR_TF_BINNED) nu_p = fmax(nu_p, adaptive_nu(m, cf, bt, eps));
            else nu_p = fmax(nu_p, 1.25 * nu);
            grace_left = cf->grace;
            continue;
        }
        double r = u[1] * nu_p;
        if (r > nu) { /* Eq. (4) */
            ++n_null;
            if (adaptive && --grace_left == 0) {
                nu_p = adaptive_nu(m, cf, bt, eps);
                grace_left = cf->grace;
                retried = 0;
            }
            continue;
        }
        int c = or_select_channel(m, eps, r);
        double eps_f, sec_v[3];
        int ion, att;
        collide(m, cf, id, step, c, eps, u, v, &eps_f, &ion, &att, sec_v);
        n_ion += (uint32_t)ion;
        n_att += (uint32_t)att;
        sum_e += eps;
        sum_e2 += eps_f;
        ++n_real;
        if (cf->spawn && ion && sp && sp->n < sp->cap) {   /* a new electron at this point */
            sp->ids[sp->n] = or_secondary_id(id, step);
            sp->t_birth[sp->n] = t0 + t;
            for (int i = 0; i < 3; ++i) sp->v_birth[3 * sp->n + i] = sec_v[i];
            ++sp->n;
        }
        if (cf->spawn && att && !cf->attach_keep_state) { status = OR_ST_ATTACHED; break; }
        for (int i = 0; i < 3; ++i) { sx[i] = x[i]; sv[i] = v[i]; }
        st = t;
        if (adaptive) {
            retried = 0;
            if (--grace_left == 0) {
                nu_p = adaptive_nu(m, cf, bt, energy_of(v));
                grace_left = cf->grace;
            }
        }
    }
    P->x[slot] = x[0]; P->y[slot] = x[1]; P->z[slot] = x[2]; P->t[slot] = t;
    P->vx[slot] = v[0]; P->vy[slot] = v[1]; P->vz[slot] = v[2];
    P->sum_e[slot] = sum_e; P->sum_e2[slot] = sum_e2; P->nu_p[slot] = nu_p;
    P->n_real[slot] = n_real; P->n_null[slot] = n_null; P->n_fail[slot] = n_fail;
    P->n_ion[slot] = n_ion; P->n_att[slot] = n_att; P->steps[slot] = k; P->status[slot] = status;
}

typedef struct {
    const or_mixture *m;
    const or_config *cf;
    const or_field *f;
    const or_binned *bt;
    const or_particles *P;
    uint64_t id0;
    int64_t begin, end;
} or_job;

static void *run_range(void *arg)
{
    const or_job *j = (const or_job *)arg;
    for (int64_t i = j->begin; i < j->end; ++i)
        run_particle_from(j->m, j->cf, j->f, j->bt, j->id0 + (uint64_t)i, 0.0, NULL, j->P, i, NULL);
    return NULL;
}

/* Checks the strategy's parameters; builds the Binned tables. */
static int strategy_setup(const or_mixture *m, const or_config *c, or_binned *bt)
{
    bt->n = 0;
    bt->max = NULL;
    bt->nu_first = nu_at_first_point(m);
    if (c->strategy == OR_TF_CONST) return 0;
    if (c->strategy != OR_TF_VARIABLE && c->strategy != OR_TF_BINNED) return -1;
    if (c->grace < 1 || c->fixed) return -1;
    if (c->strategy == OR_TF_VARIABLE && !(c->zeta >= 0.0)) return -1;
    if (c->strategy == OR_TF_BINNED) {
        if (c->bins_per_decade < 1) return -1;
        binned_setup(m, c->bins_per_decade, bt);
    }
    return 0;
}

/* Spawn mode: primaries id0 .. id0+n-1 first, then every secondary in the
 * order it was created (a FIFO queue), one electron at a time, until no
 * electron is left or pop_cap electrons exist.  Output slot k holds the
 * k-th electron run; ids_out[k] its id, t_birth_out[k] its birth time.
 * Returns the number of electrons (the slots filled). */
int64_t or_run_swarm_spawn(const or_mixture *m, const or_config *cf, uint64_t id0, int64_t n, int64_t cap,
                           double *x, double *y, double *z, double *t, double *vx, double *vy, double *vz,
                           double *sum_e, double *sum_e2, double *nu_p, uint32_t *n_real, uint32_t *n_null,
                           uint32_t *n_fail, uint32_t *n_ion, uint32_t *n_att, uint32_t *steps, uint32_t *status,
                           uint64_t *ids_out, double *t_birth_out)
{
    or_particles P = {x, y, z, t, vx, vy, vz, sum_e, sum_e2, nu_p, n_real, n_null, n_fail, n_ion, n_att, steps, status};
    or_config c = *cf;
    if (c.nu_trial <= 0.0) c.nu_trial = m->nu_max * (1.0 + 1e-6);
    if (c.max_trials == 0) c.max_trials = 0x7FFFFFFFu;
    or_field f;
    field_setup(&f, c.e_over_n_Td, m->n_total, c.b_T, c.b_angle_rad);
    int64_t room = cap - n;
    if (room < 0) return -1;
    or_binned bt;
    if (strategy_setup(m, &c, &bt) != 0) return -2;
    or_spawns sp;
    sp.ids = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(room + 1));
    sp.t_birth = (double *)malloc(sizeof(double) * (size_t)(room + 1));
    sp.v_birth = (double *)malloc(sizeof(double) * 3 * (size_t)(room + 1));
    sp.n = 0;
    sp.cap = room;
    for (int64_t i = 0; i < n; ++i) {
        ids_out[i] = id0 + (uint64_t)i;
        t_birth_out[i] = 0.0;
        run_particle_from(m, &c, &f, &bt, ids_out[i], 0.0, NULL, &P, i, &sp);
    }
    for (int64_t k = 0; k < sp.n; ++k) {
        int64_t slot = n + k;
        ids_out[slot] = sp.ids[k];
        t_birth_out[slot] = sp.t_birth[k];
        run_particle_from(m, &c, &f, &bt, sp.ids[k], sp.t_birth[k], sp.v_birth + 3 * k, &P, slot, &sp);
    }
    int64_t total = n + sp.n;
    free(sp.ids);
    free(sp.t_birth);
    free(sp.v_birth);
    free(bt.max);
    return total;
}

/* Runs particles id0 .. id0+n-1; outputs go to slot i = id - id0.  Particles
 * are independent, so the result does not depend on n_threads. */
int or_run_swarm(const or_mixture *m, const or_config *cf, uint64_t id0, int64_t n, int n_threads,
                 double *x, double *y, double *z, double *t, double *vx, double *vy, double *vz,
                 double *sum_e, double *sum_e2, double *nu_p, uint32_t *n_real, uint32_t *n_null,
                 uint32_t *n_fail, uint32_t *n_ion, uint32_t *n_att, uint32_t *steps, uint32_t *status)
{
    or_particles P = {x, y, z, t, vx, vy, vz, sum_e, sum_e2, nu_p, n_real, n_null, n_fail, n_ion, n_att, steps, status};
    or_config c = *cf;
    if (c.nu_trial <= 0.0) c.nu_trial = m->nu_max * (1.0 + 1e-6);
    if (c.max_trials == 0) c.max_trials = 0x7FFFFFFFu;
    or_field f;
    field_setup(&f, c.e_over_n_Td, m->n_total, c.b_T, c.b_angle_rad);
    or_binned bt;
    if (strategy_setup(m, &c, &bt) != 0) return -1;
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    pthread_t th[256];
    or_job jobs[256];
    int64_t per = (n + n_threads - 1) / n_threads;
    int launched = 0;
    for (int i = 0; i < n_threads; ++i) {
        int64_t b = (int64_t)i * per, e = b + per < n ? b + per : n;
        if (b >= e) break;
        jobs[i] = (or_job){m, &c, &f, &bt, &P, id0, b, e};
        if (n_threads == 1) { run_range(&jobs[i]); continue; }
        pthread_create(&th[i], NULL, run_range, &jobs[i]);
        ++launched;
    }
    for (int i = 0; i < launched; ++i) pthread_join(th[i], NULL);
    free(bt.max);
    return 0;
}

/* One trial step from a state at a real collision (single-step replay).
 * state[8*i ..] = x, y, z, vx, vy, vz, t, nu'; out has the same 8 values after
 * the step; decision = channel index, -1 null, -2 fail; eps_io[2i] = energy
 * before the collision, eps_io[2i+1] = energy after (real collisions only). */
int or_step_replay(const or_mixture *m, const or_config *cf, int64_t n, const double *state,
                   const uint64_t *ids, const uint32_t *steps, double *out, int32_t *decision, double *eps_io)
{
    or_field f;
    field_setup(&f, cf->e_over_n_Td, m->n_total, cf->b_T, cf->b_angle_rad);
    for (int64_t i = 0; i < n; ++i) {
        const double *s = state + 8 * i;
        double x[3] = {s[0], s[1], s[2]}, v[3] = {s[3], s[4], s[5]}, t = s[6], nu_p = s[7];
        double u[4];
        draw4(cf->seed, ids[i], steps[i], 0u, u);
        double tau = -log(u[0]) / nu_p;
        or_move(&f, x, v, tau);
        t += tau;
        double eps = energy_of(v), nu = or_nu(m, eps);
        double eps_f = 0.0;
        int32_t dec;
        if (nu > nu_p) {
            dec = OR_DEC_FAIL;
            x[0] = s[0]; x[1] = s[1]; x[2] = s[2]; v[0] = s[3]; v[1] = s[4]; v[2] = s[5]; t = s[6];
            nu_p = fmax(nu_p, 1.25 * nu);
        } else if (u[1] * nu_p > nu) {
            dec = OR_DEC_NULL;
        } else {
            int c = or_select_channel(m, eps, u[1] * nu_p), ion, att;
            double sec_v[3];
            collide(m, cf, ids[i], steps[i], c, eps, u, v, &eps_f, &ion, &att, sec_v);
            dec = c;
        }
        double *o = out + 8 * i;
        o[0] = x[0]; o[1] = x[1]; o[2] = x[2]; o[3] = v[0]; o[4] = v[1]; o[5] = v[2]; o[6] = t; o[7] = nu_p;
        decision[i] = dec;
        eps_io[2 * i] = eps;
        eps_io[2 * i + 1] = eps_f;
    }
    return 0;
}

/* The state of particle `id` right after initialisation (for pins). */
void or_initial_velocity(double eps0_mean_eV, uint64_t seed, uint64_t id, double v[3])
{
    or_config c;
    memset(&c, 0, sizeof c);
    c.eps0_mean_eV = eps0_mean_eV;
    c.seed = seed;
    init_velocity(&c, id, v);
}

/* Vectorised helpers for the pins (plain loops over the scalar functions). */
void or_nu_many(const or_mixture *m, int64_t n, const double *eps, double *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = or_nu(m, eps[i]);
}

void or_sigma_many(const or_mixture *m, int c, int64_t n, const double *eps, double *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = or_sigma(m, c, eps[i]);
}

void or_initial_velocity_many(double eps0_mean_eV, uint64_t seed, uint64_t id0, int64_t n, double *v)
{
    for (int64_t i = 0; i < n; ++i) or_initial_velocity(eps0_mean_eV, seed, id0 + (uint64_t)i, v + 3 * i);
}
