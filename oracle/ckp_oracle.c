/*
 * ckp_oracle.c -- plain FP64 CPU oracle for the correntropy kernelized
 * periodogram (CKP / nCKP) of Protopapas et al., arXiv:1412.1840.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant with the CUDA implementation.
 *
 * Every function follows the paper's definitions literally, in double
 * precision, with libm exp/sin, no blocking and no reordering:
 *   - Gaussian kernel              Eq. (Gausskernel), Section 2
 *   - periodic kernel              Eq. (periodickernel), Section 2.1
 *   - information potential        Eq. (IP), Section 3
 *   - CKP                          Eq. (HP), Section 3 (ordered double loop
 *                                  over ALL i, j, the diagonal included)
 *   - normalized CKP               Eq. (CKP), Section 3
 *   - sigma_y = med(e)             Eq. (pavlosrule), Section 3
 *   - pSNR                         Eq. (pSNR), Section 5.2
 *   - sigma_t skewness rule        the Bowley-skewness rule that Section 3
 *                                  keeps in the LaTeX source as commented-out
 *                                  text (lambda = 0.1, mu = 12)
 *   - periodicity thresholds       Table "tab:th", Section 4.1
 *   - best period                  argmax over trial frequencies, Section 3
 *   - coarse-then-fine search      top-k local maxima of a coarse grid,
 *                                  each refined on a fine window
 *
 * Readings where the paper is silent:
 *   median of an even count = mean of the two middle values;
 *   iqr(y) for pSNR = Q3 - Q1 with quantiles by linear interpolation between
 *     order statistics (position q*(N-1));
 *   sigma_t rule quartiles = medians of the lower and upper halves of the
 *     sorted magnitudes (the rule's own footnote), the middle value excluded
 *     for odd N; S = 0 when Q3 == Q1;
 *   argmax ties go to the lowest frequency index;
 *   SNR bins are left-closed, pSNR >= 20 falls in the last bin;
 *   bands method: derivatives between consecutive samples as given (time
 *     order), d_i = 0 when t_{i+1} == t_i; d_i belongs to the band of its left
 *     sample; band k holds the samples of magnitude rank [floor(kN/10),
 *     floor((k+1)N/10)) (ties by sample index); bands ordered by D_j
 *     descending, ties to the lower band; one-day frequencies keep their
 *     values in the local-maximum test and are only skipped as candidates;
 *     a one-sample band's window is exactly 1; missing entries are -1;
 *   preprocessing: std(e) is the population standard deviation; the cut is
 *     strict (e_i < mean + 3 std); chi^2 weights 1/e_i^2; the correlation is
 *     the unweighted Pearson coefficient between the kept magnitudes and the
 *     fitted line; the whole fit a0 + a1 t (intercept included) is removed;
 *     the sample order of the kept points is preserved;
 *   spurious-period exclusion windows (Section 6.1; the paper's mask widths
 *     are not given, so the caller supplies closed frequency intervals):
 *     excluded frequencies are never the best period, nor a coarse peak of the
 *     coarse-then-fine search; the bands method's trial lists are unchanged
 *     (the paper filters at the choice of the best trial);
 *   whitening: phase = frac(t / P0); folded order by phase, equal phases by
 *     sample index; the moving average is circular over the folded curve
 *     (the fold is periodic), window of w = min(30, N) samples covering
 *     folded positions k - w/2 .. k - w/2 + w - 1.
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Threads the OpenMP loops of this file run on (reported beside timed runs). */
int orc_max_threads(void) { return omp_get_max_threads(); }

#define ORC_PI 3.14159265358979323846

/* Eq. (Gausskernel): G_sigma(x) = exp(-x^2 / (2 sigma^2)) / (sqrt(2 pi) sigma). */
double orc_gauss(double x, double sigma)
{
    return exp(-(x * x) / (2.0 * sigma * sigma)) / (sqrt(2.0 * ORC_PI) * sigma);
}

/* Eq. (periodickernel): G^P_sigma(f, dt) = exp(-2 sin^2(pi f dt) / sigma^2) / (sqrt(2 pi) sigma). */
double orc_periodic_kernel(double f, double dt, double sigma)
{
    double s = sin(ORC_PI * f * dt);
    return exp(-2.0 * s * s / (sigma * sigma)) / (sqrt(2.0 * ORC_PI) * sigma);
}

/* Eq. (IP): IP = (1/N^2) sum_i sum_j G_sigma_y(y_i - y_j). */
double orc_information_potential(const double *y, int64_t n, double sigma_y)
{
    double acc = 0.0;
    for (int64_t i = 0; i < n; i++)
        for (int64_t j = 0; j < n; j++)
            acc += orc_gauss(y[i] - y[j], sigma_y);
    return acc / ((double)n * (double)n);
}

/* Eq. (HP): CKP(f) = (1/N^2) sum_i sum_j (G_sy(dy_ij) - IP) G^P_st(f, dt_ij),
 * for each of nf trial frequencies. */
void orc_ckp(const double *t, const double *y, int64_t n, double sigma_y, double sigma_t,
             const double *freqs, int64_t nf, double *out)
{
    double ip = orc_information_potential(y, n, sigma_y);
    for (int64_t k = 0; k < nf; k++) {
        double acc = 0.0;
        for (int64_t i = 0; i < n; i++)
            for (int64_t j = 0; j < n; j++)
                acc += (orc_gauss(y[i] - y[j], sigma_y) - ip) *
                       orc_periodic_kernel(freqs[k], t[i] - t[j], sigma_t);
        out[k] = acc / ((double)n * (double)n);
    }
}

/* Eq. (CKP): nCKP(f) = sqrt(N sigma_t) / IP * CKP(f). */
void orc_nckp(const double *t, const double *y, int64_t n, double sigma_y, double sigma_t,
              const double *freqs, int64_t nf, double *out)
{
    double ip = orc_information_potential(y, n, sigma_y);
    orc_ckp(t, y, n, sigma_y, sigma_t, freqs, nf, out);
    double scale = sqrt((double)n * sigma_t) / ip;
    for (int64_t k = 0; k < nf; k++)
        out[k] *= scale;
}

/* ---------------------------------------------------------------------- */
/* Order statistics                                                        */
/* ---------------------------------------------------------------------- */

static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

static double *sorted_copy(const double *x, int64_t n)
{
    double *s = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    memcpy(s, x, (size_t)n * sizeof(double));
    qsort(s, (size_t)n, sizeof(double), cmp_double);
    return s;
}

static double median_sorted(const double *s, int64_t n)
{
    if (n % 2 == 1)
        return s[n / 2];
    return 0.5 * (s[n / 2 - 1] + s[n / 2]);
}

/* Median; an even count takes the mean of the two middle values. */
double orc_median(const double *x, int64_t n)
{
    double *s = sorted_copy(x, n);
    double m = median_sorted(s, n);
    free(s);
    return m;
}

/* Quantile q in [0, 1] by linear interpolation between order statistics at position q*(N-1). */
double orc_quantile(const double *x, int64_t n, double q)
{
    double *s = sorted_copy(x, n);
    double pos = q * (double)(n - 1);
    int64_t lo = (int64_t)floor(pos);
    int64_t hi = lo + 1 < n ? lo + 1 : n - 1;
    double v = s[lo] + (pos - (double)lo) * (s[hi] - s[lo]);
    free(s);
    return v;
}

/* Eq. (pSNR): pSNR = 0.7413 iqr(y) / (alpha med(e)). */
double orc_psnr(const double *y, const double *e, int64_t n, double alpha)
{
    double iqr = orc_quantile(y, n, 0.75) - orc_quantile(y, n, 0.25);
    return 0.7413 * iqr / (alpha * orc_median(e, n));
}

/* Bowley skewness with quartiles as medians of the lower / upper halves
 * (middle value excluded for odd N), and the commented-out sigma_t rule
 * sigma_t = lambda + 0.5 exp(-mu S^2) with lambda = 0.1, mu = 12. */
double orc_bowley_skewness(const double *y, int64_t n)
{
    double *s = sorted_copy(y, n);
    int64_t h = n / 2;
    double q1 = median_sorted(s, h);
    double q3 = median_sorted(s + (n - h), h);
    double q2 = median_sorted(s, n);
    free(s);
    if (q3 == q1)
        return 0.0;
    return (q3 + q1 - 2.0 * q2) / (q3 - q1);
}

double orc_sigma_t_rule(const double *y, int64_t n)
{
    double sk = orc_bowley_skewness(y, n);
    return 0.1 + 0.5 * exp(-12.0 * sk * sk);
}

/* Table "tab:th": SNR bins [0,1.5) [1.5,2) [2,2.5) [2.5,3.5) [3.5,5) [5,10) [10,20) [20,inf). */
static const double ORC_BIN_LO[8] = {0.0, 1.5, 2.0, 2.5, 3.5, 5.0, 10.0, 20.0};
static const double ORC_TH[8] = {0.4584, 0.4565, 0.4537, 0.4581, 0.5875, 1.1153, 1.6464, 2.4112};

int orc_snr_bin(double psnr)
{
    int b = 0;
    for (int k = 0; k < 8; k++)
        if (psnr >= ORC_BIN_LO[k])
            b = k;
    return b;
}

double orc_threshold(double psnr)
{
    return ORC_TH[orc_snr_bin(psnr)];
}

/* ---------------------------------------------------------------------- */
/* Best period                                                             */
/* ---------------------------------------------------------------------- */

/* argmax over v[0..n), ties to the lowest index. */
int64_t orc_argmax(const double *v, int64_t n)
{
    int64_t b = 0;
    for (int64_t k = 1; k < n; k++)
        if (v[k] > v[b])
            b = k;
    return b;
}

/* Local maxima of v: v[k] > v[k-1] and v[k] >= v[k+1]; an end point is
 * compared with its single neighbour.  The top_k largest are written to
 * peaks (value descending, ties to the lower index).  Returns their count. */
int64_t orc_top_local_maxima(const double *v, int64_t n, int64_t top_k, int64_t *peaks)
{
    int64_t cnt = 0;
    for (int64_t k = 0; k < n; k++) {
        int left_ok = (k == 0) || (v[k] > v[k - 1]);
        int right_ok = (k == n - 1) || (v[k] >= v[k + 1]);
        if (n == 1)
            left_ok = right_ok = 1;
        if (!(left_ok && right_ok))
            continue;
        /* insertion into the sorted top list */
        int64_t pos = cnt < top_k ? cnt : top_k;
        while (pos > 0 && v[k] > v[peaks[pos - 1]])
            pos--;
        if (pos >= top_k)
            continue;
        int64_t last = cnt < top_k ? cnt : top_k - 1;
        for (int64_t m = last; m > pos; m--)
            peaks[m] = peaks[m - 1];
        peaks[pos] = k;
        if (cnt < top_k)
            cnt++;
    }
    return cnt;
}

typedef struct {
    double f_min, df;
    int64_t n_freq;
    int hierarchical;
    double coarse_df;
    int64_t top_k;
    double fine_df, fine_halfwidth;
    int64_t n_bands, trials_per_band;   /* bands method (hierarchical == 2) */
    int64_t n_exclude;                  /* spurious-period exclusion windows, Section 6.1 */
    const double *exclude;              /* [2 n_exclude]: closed frequency intervals [lo, hi] */
} orc_grid;

/* Section 6.1: a frequency inside any caller-supplied window [lo, hi]
 * (closed, 1/day, compared in FP64) is never chosen as the best period; in
 * the coarse-then-fine search it is not a coarse peak candidate either (its
 * value still counts in its neighbours' local-maximum tests). */
int orc_is_excluded(double f, int64_t n_exclude, const double *exclude)
{
    for (int64_t q = 0; q < n_exclude; q++)
        if (f >= exclude[2 * q] && f <= exclude[2 * q + 1])
            return 1;
    return 0;
}

/* Local maxima as in orc_top_local_maxima, excluded frequencies f_min + k df
 * skipped as candidates (their values stay in the neighbour comparisons). */
int64_t orc_top_local_maxima_excl(const double *v, int64_t n, int64_t top_k, double f_min, double df,
                                  int64_t n_exclude, const double *exclude, int64_t *peaks)
{
    int64_t cnt = 0;
    for (int64_t k = 0; k < n; k++) {
        int left_ok = (k == 0) || (v[k] > v[k - 1]);
        int right_ok = (k == n - 1) || (v[k] >= v[k + 1]);
        if (n == 1)
            left_ok = right_ok = 1;
        if (!(left_ok && right_ok) || orc_is_excluded(f_min + (double)k * df, n_exclude, exclude))
            continue;
        int64_t pos = cnt < top_k ? cnt : top_k;
        while (pos > 0 && v[k] > v[peaks[pos - 1]])
            pos--;
        if (pos >= top_k)
            continue;
        int64_t last = cnt < top_k ? cnt : top_k - 1;
        for (int64_t m = last; m > pos; m--)
            peaks[m] = peaks[m - 1];
        peaks[pos] = k;
        if (cnt < top_k)
            cnt++;
    }
    return cnt;
}

/* argmax over the entries of v whose frequency fr[k] is not excluded, ties
 * to the lowest index; -1 when every entry is excluded. */
static int64_t argmax_allowed(const double *v, const double *fr, int64_t n, const orc_grid *g)
{
    int64_t b = -1;
    for (int64_t k = 0; k < n; k++) {
        if (orc_is_excluded(fr[k], g->n_exclude, g->exclude))
            continue;
        if (b < 0 || v[k] > v[b])
            b = k;
    }
    return b;
}

typedef struct {
    int sigma_t_mode;               /* 0 fixed, 1 per-curve array, 2 skewness rule */
    double sigma_t;
    const double *sigma_t_per_curve;
    double alpha;
} orc_options;

typedef struct {
    int64_t best_idx;
    double best_freq;
    double best_stat;
    int is_periodic;
    double psnr, sigma_y, sigma_t, ip;
} orc_result;

void orc_bands_trials(const double *t, const double *y, int64_t n, double f_min, double df, int64_t nk,
                      int64_t n_bands, int64_t n_t, int64_t *out_k);

static double curve_sigma_t(const orc_options *o, const double *y, int64_t n, int64_t c)
{
    if (o->sigma_t_mode == 1)
        return o->sigma_t_per_curve[c];
    if (o->sigma_t_mode == 2)
        return orc_sigma_t_rule(y, n);
    return o->sigma_t;
}

static int64_t n_coarse(const orc_grid *g)
{
    double f_max = g->f_min + (double)(g->n_freq - 1) * g->df;
    return (int64_t)floor((f_max - g->f_min) / g->coarse_df + 0.5) + 1;
}

/* One curve: sigma_y, sigma_t, pSNR, best frequency, discriminator.
 * Full grid: best = argmax over f_k = f_min + k df.
 * Hierarchical: coarse grid f_min + k coarse_df (within [f_min, f_max]),
 * top_k local maxima, each refined over f_peak + j fine_df, |j| <= J with
 * J = round(fine_halfwidth / fine_df), points outside [f_min, f_max]
 * skipped; best over (rank, j) by value, ties to the lower candidate
 * index rank*(2J+1) + (j+J), which is reported as best_idx.
 * Bands method (hierarchical == 2): the n_bands * trials_per_band trial grid
 * indices of Section 3.1; best over the trial list by value, ties to the
 * lower list position; best_idx is the winning grid index k.
 * Exclusion windows (Section 6.1, orc_is_excluded): excluded frequencies are
 * skipped by every argmax above (full grid, fine candidates, trial list) and
 * as coarse peaks; with no admissible candidate best_idx = -1 and the
 * frequency and statistic are NaN. */
void orc_curve_best(const double *t, const double *y, const double *e, int64_t n, int64_t c,
                    const orc_grid *g, const orc_options *o, orc_result *r)
{
    double sy = orc_median(e, n);
    double st = curve_sigma_t(o, y, n, c);
    r->sigma_y = sy;
    r->sigma_t = st;
    r->ip = orc_information_potential(y, n, sy);
    r->psnr = orc_psnr(y, e, n, o->alpha);
    double f_max = g->f_min + (double)(g->n_freq - 1) * g->df;
    if (g->hierarchical == 2) {
        int64_t L = g->n_bands * g->trials_per_band, m = 0;
        int64_t *ks = (int64_t *)malloc((size_t)(L > 0 ? L : 1) * sizeof(int64_t));
        double *fr = (double *)malloc((size_t)(L > 0 ? L : 1) * sizeof(double));
        double *v = (double *)malloc((size_t)(L > 0 ? L : 1) * sizeof(double));
        int64_t *kk = (int64_t *)malloc((size_t)(L > 0 ? L : 1) * sizeof(int64_t));
        orc_bands_trials(t, y, n, g->f_min, g->df, g->n_freq, g->n_bands, g->trials_per_band, ks);
        for (int64_t q = 0; q < L; q++)
            if (ks[q] >= 0) {
                kk[m] = ks[q];
                fr[m++] = g->f_min + (double)ks[q] * g->df;
            }
        orc_nckp(t, y, n, sy, st, fr, m, v);
        r->best_idx = -1;
        r->best_freq = NAN;
        r->best_stat = NAN;
        int64_t b = argmax_allowed(v, fr, m, g);
        if (b >= 0) {
            r->best_idx = kk[b];
            r->best_freq = fr[b];
            r->best_stat = v[b];
        }
        free(kk);
        free(v);
        free(fr);
        free(ks);
    } else if (!g->hierarchical) {
        double *fr = (double *)malloc((size_t)g->n_freq * sizeof(double));
        double *v = (double *)malloc((size_t)g->n_freq * sizeof(double));
        for (int64_t k = 0; k < g->n_freq; k++)
            fr[k] = g->f_min + (double)k * g->df;
        orc_nckp(t, y, n, sy, st, fr, g->n_freq, v);
        int64_t b = argmax_allowed(v, fr, g->n_freq, g);
        r->best_idx = b;
        r->best_freq = b >= 0 ? fr[b] : NAN;
        r->best_stat = b >= 0 ? v[b] : NAN;
        free(fr);
        free(v);
    } else {
        int64_t kc = n_coarse(g);
        double *fr = (double *)malloc((size_t)kc * sizeof(double));
        double *v = (double *)malloc((size_t)kc * sizeof(double));
        for (int64_t k = 0; k < kc; k++)
            fr[k] = g->f_min + (double)k * g->coarse_df;
        orc_nckp(t, y, n, sy, st, fr, kc, v);
        int64_t *peaks = (int64_t *)malloc((size_t)(g->top_k > 0 ? g->top_k : 1) * sizeof(int64_t));
        int64_t np = orc_top_local_maxima_excl(v, kc, g->top_k, g->f_min, g->coarse_df, g->n_exclude, g->exclude,
                                               peaks);
        int64_t J = (int64_t)floor(g->fine_halfwidth / g->fine_df + 0.5);
        int64_t w = 2 * J + 1;
        double best = -INFINITY, bestf = fr[0];
        int64_t bestc = -1;
        double *ff = (double *)malloc((size_t)w * sizeof(double));
        double *fv = (double *)malloc((size_t)w * sizeof(double));
        for (int64_t p = 0; p < np; p++) {
            double fp = g->f_min + (double)peaks[p] * g->coarse_df;
            int64_t m = 0;
            int64_t jj[4096];
            int64_t *jl = w <= 4096 ? jj : (int64_t *)malloc((size_t)w * sizeof(int64_t));
            for (int64_t j = -J; j <= J; j++) {
                double f = fp + (double)j * g->fine_df;
                if (f < g->f_min || f > f_max || orc_is_excluded(f, g->n_exclude, g->exclude))
                    continue;
                ff[m] = f;
                jl[m] = j;
                m++;
            }
            orc_nckp(t, y, n, sy, st, ff, m, fv);
            for (int64_t q = 0; q < m; q++) {
                int64_t cand = p * w + (jl[q] + J);
                if (fv[q] > best || (fv[q] == best && cand < bestc)) {
                    best = fv[q];
                    bestf = ff[q];
                    bestc = cand;
                }
            }
            if (jl != jj)
                free(jl);
        }
        r->best_idx = bestc;
        r->best_freq = bestc >= 0 ? bestf : NAN;
        r->best_stat = bestc >= 0 ? best : NAN;
        free(ff);
        free(fv);
        free(peaks);
        free(fr);
        free(v);
    }
    r->is_periodic = r->best_stat > orc_threshold(r->psnr);   /* false when no candidate (NaN) */
}

/* Batch driver over a CSR lightcurve set (times f64, mags/errs f32 as
 * stored; widened to f64 exactly), parallel over curves with OpenMP. */
void orc_batch_best(const double *times, const float *mags, const float *errs,
                    const int64_t *offsets, int64_t n_curves, const orc_grid *g,
                    const orc_options *o, orc_result *res)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t c = 0; c < n_curves; c++) {
        int64_t a = offsets[c], n = offsets[c + 1] - offsets[c];
        double *y = (double *)malloc((size_t)n * sizeof(double));
        double *e = (double *)malloc((size_t)n * sizeof(double));
        for (int64_t i = 0; i < n; i++) {
            y[i] = (double)mags[a + i];
            e[i] = (double)errs[a + i];
        }
        orc_curve_best(times + a, y, e, n, c, g, o, &res[c]);
        free(y);
        free(e);
    }
}

/* Batch nCKP on an explicit frequency list per curve (freqs[c*nf + k]),
 * parallel over (curve, frequency) with OpenMP.  sigma_t per curve. */
void orc_batch_nckp(const double *times, const float *mags, const float *errs,
                    const int64_t *offsets, int64_t n_curves, const double *sigma_t,
                    const double *freqs, int64_t nf, double *out)
{
    double *ips = (double *)malloc((size_t)(n_curves > 0 ? n_curves : 1) * sizeof(double));
    double *sys = (double *)malloc((size_t)(n_curves > 0 ? n_curves : 1) * sizeof(double));
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t c = 0; c < n_curves; c++) {
        int64_t a = offsets[c], n = offsets[c + 1] - offsets[c];
        double *y = (double *)malloc((size_t)n * sizeof(double));
        double *e = (double *)malloc((size_t)n * sizeof(double));
        for (int64_t i = 0; i < n; i++) {
            y[i] = (double)mags[a + i];
            e[i] = (double)errs[a + i];
        }
        sys[c] = orc_median(e, n);
        ips[c] = orc_information_potential(y, n, sys[c]);
        free(y);
        free(e);
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t w = 0; w < n_curves * nf; w++) {
        int64_t c = w / nf, k = w % nf;
        int64_t a = offsets[c], n = offsets[c + 1] - offsets[c];
        const double *t = times + a;
        double ip = ips[c], sy = sys[c], st = sigma_t[c], f = freqs[w];
        double acc = 0.0;
        for (int64_t i = 0; i < n; i++)
            for (int64_t j = 0; j < n; j++)
                acc += (orc_gauss((double)mags[a + i] - (double)mags[a + j], sy) - ip) *
                       orc_periodic_kernel(f, t[i] - t[j], st);
        out[w] = sqrt((double)n * st) / ip * (acc / ((double)n * (double)n));
    }
    free(ips);
    free(sys);
}

/* ---------------------------------------------------------------------- */
/* Bands method, Section 3.1                                               */
/* ---------------------------------------------------------------------- */

typedef struct { double y; int64_t i; } orc_rank_item;

static int cmp_rank_item(const void *a, const void *b)
{
    const orc_rank_item *x = (const orc_rank_item *)a, *z = (const orc_rank_item *)b;
    if (x->y < z->y) return -1;
    if (x->y > z->y) return 1;
    return (x->i > z->i) - (x->i < z->i);
}

/* Step 2: ten bands of equal sample count on the magnitude axis.  Band k
 * holds the samples of magnitude rank r with floor(kN/10) <= r < floor((k+1)N/10)
 * (rank 0 = smallest magnitude number, i.e. the brightest value; equal magnitudes
 * ranked by sample index). */
void orc_bands_of(const double *y, int64_t n, int32_t *band)
{
    orc_rank_item *r = (orc_rank_item *)malloc((size_t)(n > 0 ? n : 1) * sizeof(orc_rank_item));
    for (int64_t i = 0; i < n; i++) {
        r[i].y = y[i];
        r[i].i = i;
    }
    qsort(r, (size_t)n, sizeof(orc_rank_item), cmp_rank_item);
    for (int64_t rank = 0; rank < n; rank++) {
        int k = 0;
        while (k < 9 && rank >= ((int64_t)(k + 1) * n) / 10)
            k++;
        band[r[rank].i] = k;
    }
    free(r);
}

/* Steps 1 and 3: d_i = (x_{i+1} - x_i) / (t_{i+1} - t_i) for consecutive
 * samples (0 where the two times are equal); D_k = sum of |d_i| over the d_i
 * whose sample i lies in band k. */
void orc_band_derivative_sums(const double *t, const double *y, int64_t n, const int32_t *band, double *D)
{
    for (int k = 0; k < 10; k++)
        D[k] = 0.0;
    for (int64_t i = 0; i + 1 < n; i++) {
        double dt = t[i + 1] - t[i];
        double d = dt != 0.0 ? (y[i + 1] - y[i]) / dt : 0.0;
        D[band[i]] += fabs(d);
    }
}

/* Step 4: the ten bands in descending order of D (equal D: lower band first). */
void orc_band_order(const double *D, int32_t *order)
{
    for (int k = 0; k < 10; k++)
        order[k] = k;
    for (int a = 1; a < 10; a++) {
        int32_t v = order[a];
        int b = a;
        while (b > 0 && D[order[b - 1]] < D[v]) {
            order[b] = order[b - 1];
            b--;
        }
        order[b] = v;
    }
}

/* Step 5, Eq. (bands): S_j(f) = |sum_{i in B_j} exp(i 2 pi f t_i)|^2 on the
 * linear grid f_k = f_min + k df, k < nk.  A band of one sample has the
 * exact value |exp(i x)|^2 = 1 at every f (cos^2 + sin^2 would add rounding
 * noise that alone would decide its local maxima). */
void orc_spectral_window(const double *t, int64_t n, const int32_t *band, int32_t j, double f_min, double df,
                         int64_t nk, double *S)
{
    int64_t m = 0;
    for (int64_t i = 0; i < n; i++)
        m += band[i] == j;
    for (int64_t k = 0; k < nk; k++) {
        if (m <= 1) {
            S[k] = (double)m;
            continue;
        }
        double f = f_min + (double)k * df, re = 0.0, im = 0.0;
        for (int64_t i = 0; i < n; i++)
            if (band[i] == j) {
                re += cos(2.0 * ORC_PI * f * t[i]);
                im += sin(2.0 * ORC_PI * f * t[i]);
            }
        S[k] = re * re + im * im;
    }
}

/* The one-day pseudo-sampling period: periods with |P - 1| < 1e-4 day. */
int orc_is_one_day(double f)
{
    return f > 0.0 && fabs(1.0 / f - 1.0) < 1e-4;
}

/* Step 6 for one band: grid indices of the n_t highest local maxima of S
 * (local maximum as in orc_top_local_maxima; value descending, ties to the
 * lower index), the one-day frequencies left out before the choice.
 * Writes n_t entries, -1 after the last one found; returns the count. */
int64_t orc_window_trials(const double *S, int64_t nk, double f_min, double df, int64_t n_t, int64_t *out_k)
{
    int64_t *pk = (int64_t *)malloc((size_t)(n_t > 0 ? n_t : 1) * sizeof(int64_t));
    /* a one-day point keeps its value in its neighbours' comparisons; it is
     * only skipped as a candidate */
    int64_t cnt = 0;
    for (int64_t k = 0; k < nk; k++) {
        int left_ok = (k == 0) || (S[k] > S[k - 1]);
        int right_ok = (k == nk - 1) || (S[k] >= S[k + 1]);
        if (!(left_ok && right_ok) || orc_is_one_day(f_min + (double)k * df))
            continue;
        int64_t pos = cnt < n_t ? cnt : n_t;
        while (pos > 0 && S[k] > S[pk[pos - 1]])
            pos--;
        if (pos >= n_t)
            continue;
        int64_t last = cnt < n_t ? cnt : n_t - 1;
        for (int64_t m = last; m > pos; m--)
            pk[m] = pk[m - 1];
        pk[pos] = k;
        if (cnt < n_t)
            cnt++;
    }
    for (int64_t r = 0; r < n_t; r++)
        out_k[r] = r < cnt ? pk[r] : -1;
    free(pk);
    return cnt;
}

/* All six steps: n_bands * n_t trial grid indices, band-rank major
 * (out_k[b * n_t + r] = r-th trial of the b-th band in D order). */
void orc_bands_trials(const double *t, const double *y, int64_t n, double f_min, double df, int64_t nk,
                      int64_t n_bands, int64_t n_t, int64_t *out_k)
{
    int32_t *band = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    double D[10];
    int32_t order[10];
    orc_bands_of(y, n, band);
    orc_band_derivative_sums(t, y, n, band, D);
    orc_band_order(D, order);
    double *S = (double *)malloc((size_t)(nk > 0 ? nk : 1) * sizeof(double));
    for (int64_t b = 0; b < n_bands; b++) {
        orc_spectral_window(t, n, band, order[b], f_min, df, nk, S);
        orc_window_trials(S, nk, f_min, df, n_t, out_k + b * n_t);
    }
    free(S);
    free(band);
}

/* Trial lists of a CSR batch, parallel over curves: out_k[c * n_bands * n_t + ...]. */
void orc_batch_bands_trials(const double *times, const float *mags, const int64_t *offsets, int64_t n_curves,
                            double f_min, double df, int64_t nk, int64_t n_bands, int64_t n_t, int64_t *out_k)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t c = 0; c < n_curves; c++) {
        int64_t a = offsets[c], n = offsets[c + 1] - offsets[c];
        double *y = (double *)malloc((size_t)n * sizeof(double));
        for (int64_t i = 0; i < n; i++)
            y[i] = (double)mags[a + i];
        orc_bands_trials(times + a, y, n, f_min, df, nk, n_bands, n_t, out_k + c * n_bands * n_t);
        free(y);
    }
}

/* ---------------------------------------------------------------------- */
/* Preprocessing, Section 5.2                                              */
/* ---------------------------------------------------------------------- */

typedef struct {
    int64_t n_in, n_out;     /* samples before / after the error-bar cut          */
    int kept;                /* n_out >= 50                                       */
    int detrended;           /* fit removed (corr > 0.5)                          */
    double e_mean, e_std;    /* of the input error bars                           */
    double a0, a1, r;        /* chi^2 fit x = a0 + a1 t and its correlation        */
} orc_prep;

/* Eq. (chisquare): minimise sum (a0 + a1 t_i - x_i)^2 / e_i^2 by its normal
 * equations (derivatives wrt a0 and a1 set to zero), solved by Cramer's rule. */
void orc_chi2_line(const double *t, const double *x, const double *e, int64_t n, double *a0, double *a1)
{
    double S = 0, St = 0, Sx = 0, Stt = 0, Stx = 0;
    for (int64_t i = 0; i < n; i++) {
        double w = 1.0 / (e[i] * e[i]);
        S += w;
        St += w * t[i];
        Sx += w * x[i];
        Stt += w * t[i] * t[i];
        Stx += w * t[i] * x[i];
    }
    double det = S * Stt - St * St;
    *a1 = (S * Stx - St * Sx) / det;
    *a0 = (Stt * Sx - St * Stx) / det;
}

/* Pearson correlation coefficient of two sequences (0 when either is constant). */
double orc_pearson(const double *u, const double *v, int64_t n)
{
    double mu = 0, mv = 0;
    for (int64_t i = 0; i < n; i++) {
        mu += u[i];
        mv += v[i];
    }
    mu /= (double)n;
    mv /= (double)n;
    double suv = 0, suu = 0, svv = 0;
    for (int64_t i = 0; i < n; i++) {
        suv += (u[i] - mu) * (v[i] - mv);
        suu += (u[i] - mu) * (u[i] - mu);
        svv += (v[i] - mv) * (v[i] - mv);
    }
    if (suu == 0.0 || svv == 0.0)
        return 0.0;
    return suv / sqrt(suu * svv);
}

/* One curve: error-bar cut, size check, chi^2 detrend.  Writes the kept
 * samples (in their order) to out_t, out_x, out_e (detrended x when the fit
 * is removed) and returns the summary.  min_n = 50 in the paper. */
orc_prep orc_preprocess(const double *t, const double *x, const double *e, int64_t n, int64_t min_n,
                        double *out_t, double *out_x, double *out_e)
{
    orc_prep r;
    memset(&r, 0, sizeof(r));
    r.n_in = n;
    double m = 0;
    for (int64_t i = 0; i < n; i++)
        m += e[i];
    m /= (double)n;
    double v = 0;
    for (int64_t i = 0; i < n; i++)
        v += (e[i] - m) * (e[i] - m);
    r.e_mean = m;
    r.e_std = sqrt(v / (double)n);
    double cut = r.e_mean + 3.0 * r.e_std;
    int64_t k = 0;
    for (int64_t i = 0; i < n; i++)
        if (e[i] < cut) {
            out_t[k] = t[i];
            out_x[k] = x[i];
            out_e[k] = e[i];
            k++;
        }
    r.n_out = k;
    r.kept = k >= min_n;
    if (k < 2)
        return r;
    orc_chi2_line(out_t, out_x, out_e, k, &r.a0, &r.a1);
    double *fit = (double *)malloc((size_t)k * sizeof(double));
    for (int64_t i = 0; i < k; i++)
        fit[i] = r.a0 + r.a1 * out_t[i];
    r.r = orc_pearson(out_x, fit, k);
    if (r.r > 0.5) {
        r.detrended = 1;
        for (int64_t i = 0; i < k; i++)
            out_x[i] -= fit[i];
    }
    free(fit);
    return r;
}

/* Batch driver: CSR in (times f64, mags / errs f32 widened exactly), CSR out
 * of the kept curves' samples (out_offsets over the input curves: curve c's
 * kept samples at [out_offsets[c], out_offsets[c+1]) when kept, empty when
 * discarded), summaries per input curve. */
void orc_batch_preprocess(const double *times, const float *mags, const float *errs, const int64_t *offsets,
                          int64_t n_curves, int64_t min_n, double *out_t, double *out_x, double *out_e,
                          int64_t *out_offsets, orc_prep *res)
{
    out_offsets[0] = 0;
    for (int64_t c = 0; c < n_curves; c++) {
        int64_t a = offsets[c], n = offsets[c + 1] - offsets[c];
        double *x = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
        double *e = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
        for (int64_t i = 0; i < n; i++) {
            x[i] = (double)mags[a + i];
            e[i] = (double)errs[a + i];
        }
        int64_t o = out_offsets[c];
        res[c] = orc_preprocess(times + a, x, e, n, min_n, out_t + o, out_x + o, out_e + o);
        out_offsets[c + 1] = o + (res[c].kept ? res[c].n_out : 0);
        free(x);
        free(e);
    }
}

/* ---------------------------------------------------------------------- */
/* Whitening, Section 7.1                                                  */
/* ---------------------------------------------------------------------- */

typedef struct { double ph; int64_t i; } orc_phase_item;

static int cmp_phase_item(const void *a, const void *b)
{
    const orc_phase_item *x = (const orc_phase_item *)a, *z = (const orc_phase_item *)b;
    if (x->ph < z->ph) return -1;
    if (x->ph > z->ph) return 1;
    return (x->i > z->i) - (x->i < z->i);
}

/* Steps 1-4: fold at p0, template = moving average of w folded samples,
 * subtract it, samples back in time order (out[i] for input sample i). */
void orc_whiten(const double *t, const double *x, int64_t n, double p0, int64_t w, double *out)
{
    orc_phase_item *f = (orc_phase_item *)malloc((size_t)(n > 0 ? n : 1) * sizeof(orc_phase_item));
    for (int64_t i = 0; i < n; i++) {
        double q = t[i] / p0;
        f[i].ph = q - floor(q);
        f[i].i = i;
    }
    qsort(f, (size_t)n, sizeof(orc_phase_item), cmp_phase_item);
    if (w > n)
        w = n;
    for (int64_t k = 0; k < n; k++) {
        double acc = 0.0;
        for (int64_t j = 0; j < w; j++) {
            int64_t q = k - w / 2 + j;
            q = ((q % n) + n) % n;
            acc += x[f[q].i];
        }
        out[f[k].i] = x[f[k].i] - acc / (double)w;
    }
    free(f);
}

/* Batch driver: one period per curve (p0 <= 0 or non-finite: copied unchanged). */
void orc_batch_whiten(const double *times, const float *mags, const int64_t *offsets, int64_t n_curves,
                      const double *p0, int64_t w, double *out)
{
    for (int64_t c = 0; c < n_curves; c++) {
        int64_t a = offsets[c], n = offsets[c + 1] - offsets[c];
        double *x = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
        for (int64_t i = 0; i < n; i++)
            x[i] = (double)mags[a + i];
        if (p0[c] > 0.0 && isfinite(p0[c]))
            orc_whiten(times + a, x, n, p0[c], w, out + a);
        else
            for (int64_t i = 0; i < n; i++)
                out[a + i] = x[i];
        free(x);
    }
}
