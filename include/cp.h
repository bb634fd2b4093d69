/*
 * cp.h -- C ABI of the GB300 (sm_103a) correntropy kernelized periodogram.
 *
 * The library evaluates, for a ragged batch of irregularly sampled
 * lightcurves, the normalized correntropy kernelized periodogram of
 * Protopapas et al., arXiv:1412.1840:
 *
 *   CKP(f)  = (1/N^2) sum_i sum_j (G_sy(y_i - y_j) - IP) G^P_st(f, t_i - t_j)   Eq. (HP)
 *   IP      = (1/N^2) sum_i sum_j G_sy(y_i - y_j)                               Eq. (IP)
 *   nCKP(f) = sqrt(N st) / IP * CKP(f)                                          Eq. (CKP)
 *
 * with the Gaussian kernel G_s(x) = exp(-x^2/(2 s^2)) / (sqrt(2 pi) s)
 * (Eq. (Gausskernel)) and the periodic kernel
 * G^P_s(f, dt) = exp(-2 sin^2(pi f dt) / s^2) / (sqrt(2 pi) s)
 * (Eq. (periodickernel)); sy = med(e) (Eq. (pavlosrule)); st fixed, per
 * curve, or from the Bowley-skewness rule of Section 3.  The best period is
 * the argmax of nCKP over the trial frequencies (Section 3), and a curve is
 * labelled periodic when nCKP(best) exceeds th(pSNR) of Table tab:th with
 * pSNR = 0.7413 iqr(y) / (alpha med(e)) (Eq. (pSNR), Section 5.2).
 *
 * All entry points return a cp_status and never throw.  On failure
 * cp_last_error() returns a thread-local message.  Every step of the method
 * runs in CUDA kernels on the plan's device; the host validates arguments,
 * schedules work units and launches (its one piece of arithmetic is the
 * table of sigma_t thresholds that picks the tensor form's harmonic count,
 * from the FP64 coefficients of cp_bessel_coefficients).  A missing or
 * unusable device is an error (CP_ECUDA).
 */
#ifndef CP_H
#define CP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CP_OK = 0,
    CP_EINVAL = 1,       /* invalid argument or input value (see cp_last_error)      */
    CP_ENOMEM = 2,       /* device or pinned host allocation failed                  */
    CP_ECUDA = 3,        /* CUDA runtime / driver error                              */
    CP_ETIMEOUT = 4,     /* a bounded device wait of a tensor-form kernel gave up     */
    CP_ESTATE = 5,       /* plan used in a state that does not allow the call        */
    CP_EUNSUPPORTED = 6  /* valid request the build does not support (e.g. N > max)  */
} cp_status;

typedef struct cp_plan_s *cp_plan_t;

/* Evaluation form. */
enum { CP_FORM_DIRECT = 0, /* FP32 pair sum, FP64-exact fixed-point phases          */
       CP_FORM_TENSOR = 1  /* Fourier/Bessel series, FP16/BF16 tcgen05 GEMMs        */ };
/* Operand type of the tensor form (FP32 accumulation in every case).
 * FP16: 11 significand bits; meets 1e-3 of the peak with single operands.
 * BF16: 8 bits; the magnitude-kernel operand W' is split into hi + lo BF16
 *       parts (two MMAs per K slice), the harmonic operand Z stays single:
 *       ~1e-3 to 1.5e-3 of the peak on harmonic-rich curves.
 * BF16_SPLIT: BF16 with both W' and Z split into hi + lo parts (the lo part
 *       of Z in the upper half of each unit's MMA columns, so a unit covers
 *       half the frequencies): meets 1e-3 in BF16 at about half BF16's rate;
 *       harmonic counts 4, 8, 16 and 32 (a curve that would take 12 takes 16,
 *       one that would take 48 runs in the direct form). */
enum { CP_DTYPE_FP16 = 0, CP_DTYPE_BF16 = 1, CP_DTYPE_BF16_SPLIT = 2 };
/* How sigma_t is chosen per curve. */
enum { CP_SIGMA_T_FIXED = 0,     /* options.sigma_t for every curve                    */
       CP_SIGMA_T_PER_CURVE = 1, /* options.sigma_t_per_curve[c] (host array)          */
       CP_SIGMA_T_RULE = 2       /* 0.1 + 0.5 exp(-12 S^2), S = Bowley skewness of y   */ };
/* Where times / mags / errs live. */
enum { CP_MEM_HOST = 0, CP_MEM_DEVICE = 1 };

/*
 * Trial frequencies (1/day).  The uniform grid is f_k = f_min + k*df,
 * k = 0..n_freq-1, each computed in FP64 (not accumulated); it spans
 * [f_min, f_max] with f_max = f_min + (n_freq-1)*df.
 *
 * hierarchical != 0 makes cp_best_period run the coarse-then-fine search:
 * coarse grid f_min + k*coarse_df over [f_min, f_max]; the top_k local
 * maxima (v[k] > v[k-1] and v[k] >= v[k+1], ends compared with their single
 * neighbour; ties to the lower k); each refined on f_peak + j*fine_df,
 * |j| <= J = round(fine_halfwidth / fine_df), points outside [f_min, f_max]
 * skipped; the best over all refined candidates by value, ties to the lower
 * candidate index rank*(2J+1) + (j+J).  cp_periodogram always evaluates the
 * uniform grid.
 *
 * hierarchical == CP_SEARCH_BANDS runs the trial-period extraction of
 * Section 3.1 (the bands method) on the device before the pair sums:
 *   1. d_i = (y_{i+1} - y_i) / (t_{i+1} - t_i) over consecutive samples in
 *      the order given (0 where the two times are equal);
 *   2. ten bands of equal count on the magnitude axis: band b holds the
 *      samples of magnitude rank r (ascending, equal values by sample index)
 *      with floor(bN/10) <= r < floor((b+1)N/10);
 *   3. D_b = sum of |d_i| over the d_i whose sample i is in band b (FP64);
 *   4. the n_bands bands of largest D (equal D: lower band first);
 *   5. for each, the spectral window S_b(f) = |sum_{i in b} exp(i 2 pi f t_i)|^2
 *      of Eq. (bands) on the uniform grid above;
 *   6. the trials_per_band highest local maxima of S_b (local maximum and
 *      tie rule as above), leaving out the one-day frequencies
 *      |1/f - 1| < 1e-4 (FP64).
 * The window is evaluated in FP32 over the grid; every local-maximum test
 * and every ordering that lies within the FP32 error bound is decided again
 * from FP64 window values (exact 64-bit phases), and a band whose candidate
 * set the bound cannot prove complete is scanned in FP64 over the whole grid,
 * so the lists are those of an FP64 evaluation (n_freq < 2^28).
 * nCKP is then evaluated at the n_bands * trials_per_band trial grid
 * frequencies only, and the best is the largest, ties to the lower
 * position in the band-major trial list.  best_idx is the winning grid
 * index k.  cp_trial_frequencies returns the list and its nCKP values.
 *
 * Spurious-period exclusion windows (Section 6.1, Filtering of spurious
 * periods; Table tab:spuriousperiods lists the periods -- the solar day, the
 * synodic month, the year, the time span and their aliases -- but not the
 * widths of the paper's masks, so the caller supplies them): n_exclude closed
 * frequency intervals exclude[2q] <= f <= exclude[2q+1] (1/day).  A frequency
 * f in any window (compared in FP64 with f computed as for best_freq) is
 * never returned as the best: the full-grid argmax and the choice among
 * the refined candidates and among the bands trials skip it, and the
 * coarse-then-fine search does not take it as a coarse peak (its value
 * still counts in its neighbours' local-maximum tests).  The bands trial
 * lists themselves are unchanged (the paper filters at the choice of the
 * best trial).  cp_periodogram is unaffected.  A curve left without any
 * admissible candidate reports best_idx -1, NaN frequency and statistic,
 * and is_periodic 0.
 */
enum { CP_SEARCH_FULL = 0, CP_SEARCH_COARSE_FINE = 1, CP_SEARCH_BANDS = 2 };
#define CP_BANDS_MAX_TRIALS 512
#define CP_MAX_EXCLUDE 64

typedef struct {
    double f_min;
    double df;
    int64_t n_freq;
    int32_t hierarchical;            /* CP_SEARCH_*                                    */
    int32_t top_k;                   /* coarse-then-fine: peaks refined                */
    double coarse_df;
    double fine_df;
    double fine_halfwidth;
    int32_t n_bands;                 /* bands method: N_b in [1, 10]                   */
    int32_t trials_per_band;         /* bands method: N_t in [1, CP_BANDS_MAX_TRIALS]  */
    int32_t n_exclude;               /* exclusion windows: 0..CP_MAX_EXCLUDE           */
    int32_t reserved0;
    const double *exclude;           /* host, 2 n_exclude values: [lo, hi] pairs with  */
                                     /* finite lo <= hi (1/day); copied by cp_plan     */
} cp_freq_grid;

/*
 * Tuned launch choices (written by the package's autotuner from timings on
 * the target GPU; not part of the method).  Curves are grouped in buckets by
 * N: bucket b holds bucket_max_n[b-1] < N <= bucket_max_n[b].  For a curve
 * in bucket b:
 *   direct_fc[b]       frequencies per work unit of the direct form (2, 4, 8
 *                      or 16; lowered to the largest that fits the kernel's
 *                      shared trig table for the curve's N);
 *   tensor_classes[b]  with n_max = 0, bit 0, 1, 2, 3, 4 set lets the harmonic
 *                      class 8, 16, 32, 12, 48 run in the tensor form; a curve
 *                      whose class bit is clear runs in the direct form.
 * Curves above the last bucket, and plans without tuning, use the built-in
 * choices (16 frequencies per unit where they fit; every class in the tensor
 * form).  Results never depend on the tuning beyond the form's own rounding.
 */
#define CP_TUNE_MAX_BUCKETS 16
typedef struct {
    int32_t n_buckets;                              /* 0..CP_TUNE_MAX_BUCKETS        */
    int32_t bucket_max_n[CP_TUNE_MAX_BUCKETS];      /* strictly ascending, >= 2      */
    int32_t direct_fc[CP_TUNE_MAX_BUCKETS];
    int32_t tensor_classes[CP_TUNE_MAX_BUCKETS];
} cp_tuning;

typedef struct {
    int32_t sigma_t_mode;            /* CP_SIGMA_T_*                                    */
    float sigma_t;                   /* fixed kernel size (mode FIXED)                  */
    const float *sigma_t_per_curve;  /* host, n_curves values (mode PER_CURVE); copied  */
    float alpha;                     /* error-bar correction factor of Eq. (pSNR), >0   */
    int32_t form;                    /* CP_FORM_*                                       */
    int32_t dtype;                   /* CP_DTYPE_* (tensor form only)                   */
    int32_t n_max;                   /* harmonics of the tensor form (4, 8, 12, 16, 32, */
                                     /* 48; 12 and 48 not with CP_DTYPE_BF16_SPLIT);    */
                                     /* 0 = per curve: the smallest of 8, 12, 16, 32, 48 */
                                     /* whose truncation tail is <= 1e-4 of the kernel  */
                                     /* peak for the curve's sigma_t (computed on the   */
                                     /* device at plan time; 48 covers sigma_t >= 0.1,  */
                                     /* the rule's smallest value); curves that need    */
                                     /* more (or 48 with split Z) run in the direct     */
                                     /* form.  Each call checks, on the device,         */
                                     /* that every curve's current sigma_t is still     */
                                     /* covered by its count; if one is not (the        */
                                     /* magnitudes changed, e.g. by cp_whiten), the     */
                                     /* call rebuilds the plan on the new sigma_t and   */
                                     /* runs again (cp_plan_info.replans counts this)   */
    int32_t input_memory;            /* CP_MEM_HOST or CP_MEM_DEVICE                    */
    int32_t use_graph;               /* capture cp_best_period's step in a CUDA graph   */
    int32_t device;                  /* CUDA device ordinal                             */
    const cp_tuning *tuning;         /* host, copied by cp_plan; NULL = built-in choices */
} cp_options;

/* Fills defaults: FIXED sigma_t = 0.3, alpha = 1, DIRECT form, FP16,
 * n_max = 0, HOST inputs, graphs on, device 0, no tuning. */
void cp_default_options(cp_options *opt);

/*
 * cp_plan -- validate a ragged lightcurve batch, allocate device buffers,
 * and bind the input arrays to a new plan.
 *
 *   times   FP64 observation times (days), sum N values, curve c occupies
 *           [offsets[c], offsets[c+1]); any order within a curve.
 *   mags    FP32 magnitudes, same layout.
 *   errs    FP32 error bars (> 0 median per curve), same layout.
 *   offsets HOST int64 array of n_curves+1 entries: offsets[0] = 0, each
 *           curve holds 2 <= N <= cp_max_points() samples.
 *   grid, opt  as above (opt NULL = defaults).
 *   cuda_stream  cudaStream_t the plan runs on (NULL = legacy default stream).
 *
 * times/mags/errs are host or device pointers as opt->input_memory says.
 * The plan keeps the POINTERS, not copies: every cp_periodogram /
 * cp_best_period call reads their current contents (host arrays are copied
 * to the device inside the call), so the caller keeps them alive and
 * unchanged in size until cp_destroy.  Non-finite values and a zero median
 * error are reported by the call that reads them (CP_EINVAL).
 * offsets, grid, options and sigma_t_per_curve are copied at plan time.
 * The plan owns its device memory until cp_destroy.  A plan is used by one
 * host thread at a time.
 */
cp_status cp_plan(const double *times, const float *mags, const float *errs,
                  const int64_t *offsets, int64_t n_curves, const cp_freq_grid *grid,
                  const cp_options *opt, void *cuda_stream, cp_plan_t *out_plan);

/*
 * cp_periodogram -- nCKP of every curve on the uniform grid, Eq. (CKP).
 *   out  DEVICE float array, n_curves x n_freq, row-major in the caller's
 *        curve order (row c = curve c); may be NULL to only run the pass.
 * Asynchronous on the plan's stream; cp_sync() reports input errors.
 */
cp_status cp_periodogram(cp_plan_t plan, float *out);

/*
 * cp_best_period -- best frequency, its nCKP and the discriminator of
 * Section 4.1 for every curve (full grid or coarse-then-fine per the grid).
 * All outputs are HOST arrays of n_curves entries in the caller's curve
 * order; any may be NULL.
 *   best_idx   full grid and bands method: k of the best frequency;
 *              coarse-then-fine: candidate index rank*(2J+1) + (j+J)
 *   best_freq  FP64 best frequency (1/day); best period = 1/best_freq
 *   best_stat  nCKP at the best frequency
 *   is_periodic  1 if best_stat > th(pSNR bin) of Table tab:th
 *   psnr       pSNR of Eq. (pSNR)
 * Synchronous: returns after the results are on the host.  With per-curve
 * harmonic counts (tensor form, n_max = 0) a call may rebuild the plan first
 * (see cp_options.n_max); the results are then those of the rebuilt plan.
 */
cp_status cp_best_period(cp_plan_t plan, int64_t *best_idx, double *best_freq, float *best_stat,
                         uint8_t *is_periodic, float *psnr);

/* Waits for the plan's stream and returns the device-side status of the
 * last call (CP_EINVAL for non-finite inputs or a zero median error).  If the
 * last call was a cp_periodogram whose per-curve harmonic counts no longer
 * cover a curve's sigma_t, it rebuilds the plan and runs that pass again
 * into the same output before returning. */
cp_status cp_sync(cp_plan_t plan);

/*
 * cp_curve_stats -- per-curve scalars of the last call, HOST arrays of
 * n_curves (any may be NULL): sigma_y = med(e) (Eq. (pavlosrule)), the
 * sigma_t used, IP of Eq. (IP), pSNR of Eq. (pSNR).  Synchronous.
 */
cp_status cp_curve_stats(cp_plan_t plan, float *sigma_y, float *sigma_t, double *ip, float *psnr);

/*
 * cp_trial_frequencies -- the trial list of the last cp_best_period of a
 * bands-method plan (Section 3.1), HOST arrays of n_curves x
 * (n_bands * trials_per_band), row-major in the caller's curve order, band
 * rank major (entry b * trials_per_band + r = the r-th highest admissible
 * local maximum of the b-th band in D order); either may be NULL.
 *   trial_idx   grid index k of the trial frequency, -1 where the band had
 *               fewer admissible local maxima
 *   trial_stat  nCKP at that frequency (NaN where trial_idx is -1)
 * CP_ESTATE for a plan without the bands method or before a search ran.
 * Synchronous.
 */
cp_status cp_trial_frequencies(cp_plan_t plan, int32_t *trial_idx, float *trial_stat);

/*
 * cp_preprocess -- the cleaning of Section 5.2 on the device, for a batch
 * before it is planned: samples whose error bar is not below
 * mean(e) + 3 std(e) (population std, per curve) are dropped; curves with
 * fewer than min_n samples left (50 in the paper) are discarded; the
 * weighted linear fit of Eq. (chisquare), x = a0 + a1 t with weights
 * 1/e^2, is subtracted (intercept included) when the Pearson correlation
 * of the kept magnitudes with the fit exceeds 0.5.  Kept samples keep
 * their order.  Statistics in FP64.
 *   times, mags, errs        DEVICE input CSR arrays (offsets[n_curves] samples)
 *   offsets                  HOST, n_curves + 1, offsets[0] = 0, curves of 1..cp_max_points()
 *   out_times, out_mags, out_errs  DEVICE, room for offsets[n_curves] samples;
 *                            the kept samples of the kept curves, curve by curve
 *   out_offsets              HOST, n_curves + 1: curve c's kept samples are at
 *                            [out_offsets[c], out_offsets[c+1]); empty when discarded
 *   flags                    HOST, n_curves or NULL: bit 0 kept, bit 1 fit removed
 *   fit                      HOST, 3 * n_curves or NULL: a0, a1, correlation
 * Synchronous on cuda_stream (the output offsets need the kept counts);
 * allocates and frees small temporaries.
 */
cp_status cp_preprocess(const double *times, const float *mags, const float *errs, const int64_t *offsets,
                        int64_t n_curves, int32_t min_n, double *out_times, float *out_mags, float *out_errs,
                        int64_t *out_offsets, uint8_t *flags, double *fit, void *cuda_stream);

/*
 * cp_whiten -- the whitening of Section 7.1 (multimodes) on the device: each
 * curve is folded at its period p0[c] (phase = frac(t / p0), equal phases in
 * sample order), a template is taken as the circular moving average of
 * w = min(window, N) folded samples (30 in the paper; folded positions
 * k - w/2 .. k - w/2 + w - 1), subtracted, and the samples are returned in
 * their original order.  A curve with p0[c] <= 0 or not finite is copied.
 *   times, mags, out_mags    DEVICE CSR arrays; out_mags may equal mags
 *   offsets, p0              HOST, n_curves + 1 and n_curves entries
 * Synchronous on cuda_stream.  Searching the whitened curves (a plan bound to
 * out_mags) gives the second mode P1.
 */
cp_status cp_whiten(const double *times, const float *mags, const int64_t *offsets, int64_t n_curves,
                    const double *p0, int32_t window, float *out_mags, void *cuda_stream);

/* Work and timing of the plan (for throughput and roofline reports). */
typedef struct {
    int64_t n_curves;
    int64_t n_points;             /* sum N                                             */
    double pair_freq_full;        /* sum_c N(N-1)/2 * n_freq: one uniform-grid pass     */
    double pair_freq_search;      /* pair-frequency evaluations of one cp_best_period   */
    int64_t launches_per_search;  /* kernels one cp_best_period launches                */
    float last_pair_kernel_ms;    /* device time of the pair-sum kernel(s), last call   */
    float last_step_ms;           /* device time of the whole last cp_best_period       */
    int32_t n_sm;                 /* SMs of the plan's device                           */
    int32_t max_n;                /* largest N in the batch                             */
    int64_t class_curves[7];      /* curves per evaluation class: direct form, then the */
                                  /* tensor form with 4, 8, 12, 16, 32, 48 harmonics    */
    float last_tensor_kernel_ms;  /* device time of the tensor-form launches, last call */
    float last_direct_kernel_ms;  /* device time of the direct-form launches, last call */
    double tensor_flops_search;   /* tensor-form GEMM flops of one cp_best_period:      */
                                  /* 2 N^2 n_max per curve and frequency (the upper     */
                                  /* block triangle of the 4 N^2 n_max dense product)   */
    double direct_pair_freq_search; /* pair-frequency evaluations of the direct curves  */
    float last_bands_kernel_ms;   /* device time of the bands-method kernels, last call */
    float reserved0;
    double window_terms_search;   /* bands method: spectral-window terms (band point x  */
                                  /* grid frequency) of one cp_best_period              */
    double w_bytes_direct;        /* bytes of the magnitude-kernel tiles one search     */
    double w_bytes_tensor;        /* builds for the direct / tensor-form curves         */
    int64_t replans;              /* plans rebuilt after a curve's sigma_t left the     */
                                  /* range of its harmonic count (see cp_options.n_max) */
    int64_t bands_exact_scans;    /* bands method, last search: (curve, band) lists     */
                                  /* chosen by a whole-grid FP64 scan because the FP32  */
                                  /* window bound could not prove the candidate set     */
                                  /* complete (peaks of nearly equal height)            */
} cp_plan_info;

cp_status cp_get_plan_info(cp_plan_t plan, cp_plan_info *info);

/* Releases the plan's device and pinned host memory (NULL is a no-op). */
void cp_destroy(cp_plan_t plan);

/* Largest N per curve the build supports. */
int64_t cp_max_points(void);

/*
 * cp_bessel_coefficients -- Fourier coefficients of the periodic kernel
 * used by the tensor form: exp(-2 sin^2(x)/s^2) = a_0 + sum_n a_n cos(2 n x)
 * with a_0 = e^-k I_0(k), a_n = 2 e^-k I_n(k), k = 1/s^2 (Eq. (taylor)
 * regrouped by harmonic).  Writes a_0..a_n_max to out (host, n_max+1).
 * Computed in FP64 by the trapezoid rule on (1/pi) int_0^pi e^{k(cos t - 1)} cos(n t) dt.
 */
cp_status cp_bessel_coefficients(double sigma_t, int32_t n_max, double *out);

/*
 * cp_best_period_noalloc -- the best-period search for callers that cannot
 * allocate device memory at the time of the call.  The paper has no
 * counterpart: this is an interface for hosts that reserve all device memory
 * for their own pools at start-up, latency-bounded pipelines that must not
 * enter the allocator, or plug-ins whose host owns the allocator.
 *
 * It runs the direct form (same kernels and results as cp_best_period with
 * CP_FORM_DIRECT, CP_SIGMA_T_FIXED, alpha = 1) and allocates nothing: every
 * intermediate buffer lives in one static device array of
 * CP_NOALLOC_SCRATCH_BYTES that each GPU loading the library holds until the
 * process exits.  Its first call on a device looks up that array's device
 * address (cudaGetSymbolAddress) with the device current.
 *
 *   times, mags, errs   DEVICE arrays, CSR layout as in cp_plan.
 *   offsets             HOST int64, n_curves+1 entries, offsets[0] = 0.
 *   n_curves            1 .. CP_NOALLOC_MAX_CURVES; the whole batch must fit
 *                       the scratch array (CP_EUNSUPPORTED otherwise).
 *   grid                as in cp_plan (full or coarse-then-fine, no exclusion
 *                       windows: CP_EUNSUPPORTED otherwise).
 *   sigma_t             fixed periodic-kernel size, > 0.
 *   cuda_stream         stream of the current device (NULL = legacy default).
 *   best_idx, best_freq, best_stat, is_periodic
 *                       DEVICE arrays of n_curves entries (any may be NULL),
 *                       meaning as in cp_best_period.
 *
 * Synchronous: returns after the results are written; CP_EINVAL then also
 * reports non-finite inputs or a zero median error bar.  Every call uses the
 * same scratch array, which keeps the last call's contents (the call clears
 * what must start at zero): calls that overlap on the GPU -- from several
 * host threads, or on several streams -- race and give wrong results.
 */
#define CP_NOALLOC_SCRATCH_BYTES (64u << 20)
#define CP_NOALLOC_MAX_CURVES 256
cp_status cp_best_period_noalloc(const double *times, const float *mags, const float *errs,
                                 const int64_t *offsets, int64_t n_curves, const cp_freq_grid *grid,
                                 float sigma_t, void *cuda_stream, int64_t *best_idx, double *best_freq,
                                 float *best_stat, uint8_t *is_periodic);

const char *cp_status_string(cp_status s);
const char *cp_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CP_H */
