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
 * Readings where the paper is silent (all also listed in the design doc):
 *   median of an even count = mean of the two middle values;
 *   iqr(y) for pSNR = Q3 - Q1 with quantiles by linear interpolation between
 *     order statistics (position q*(N-1));
 *   sigma_t rule quartiles = medians of the lower and upper halves of the
 *     sorted magnitudes (the rule's own footnote), the middle value excluded
 *     for odd N; S = 0 when Q3 == Q1;
 *   argmax ties go to the lowest frequency index;
 *   SNR bins are left-closed, pSNR >= 20 falls in the last bin.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

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
} orc_grid;

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
 * index rank*(2J+1) + (j+J), which is reported as best_idx. */
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
    if (!g->hierarchical) {
        double *fr = (double *)malloc((size_t)g->n_freq * sizeof(double));
        double *v = (double *)malloc((size_t)g->n_freq * sizeof(double));
        for (int64_t k = 0; k < g->n_freq; k++)
            fr[k] = g->f_min + (double)k * g->df;
        orc_nckp(t, y, n, sy, st, fr, g->n_freq, v);
        int64_t b = orc_argmax(v, g->n_freq);
        r->best_idx = b;
        r->best_freq = fr[b];
        r->best_stat = v[b];
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
        int64_t np = orc_top_local_maxima(v, kc, g->top_k, peaks);
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
                if (f < g->f_min || f > f_max)
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
        r->best_freq = bestf;
        r->best_stat = best;
        free(ff);
        free(fv);
        free(peaks);
        free(fr);
        free(v);
    }
    r->is_periodic = r->best_stat > orc_threshold(r->psnr);
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
