// cp_internal.cuh -- device-side types and helpers shared by the CKP kernels.
//
// Notation follows arXiv:1412.1840, Section 3: a curve has N samples
// (t_i, y_i, e_i); sigma_y = med(e) (Eq. (pavlosrule)); the periodic kernel
// size is sigma_t; IP is the information potential of Eq. (IP).
//
// Normalised quantities used on the device (prefactors 1/(sqrt(2 pi) s) are
// folded into the per-curve normalisation):
//   g_ij = exp(-(y_i - y_j)^2 / (2 sigma_y^2))   = 2^-(y'_i - y'_j)^2,
//          y'_i = (y_i - y_ref) * gamma, gamma = sqrt(log2(e) / (2 sigma_y^2))
//   ip   = (1/N^2) sum_ij g_ij                   (IP = ip / (sqrt(2 pi) sigma_y))
//   w_ij = g_ij - ip
//   e_ij = exp(-2 sin^2(pi f dt_ij) / sigma_t^2) = 2^-(beta d_ij)^2,
//          d_ij = sin(pi phi_i) cos(pi phi_j) - cos(pi phi_i) sin(pi phi_j),
//          phi_i = frac(f t_i), beta = sqrt(2 log2(e)) / sigma_t
//   S(f) = sum_ij w_ij e_ij = N (1 - ip) + 2 sum_{i<j} w_ij e_ij
//   nCKP = sqrt(N sigma_t) / IP * CKP = S sqrt(N) / (N^2 ip sqrt(2 pi) sqrt(sigma_t))
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "cp.h"

namespace cpk {

constexpr int kMaxN = 4096;            // largest curve the kernels accept
constexpr int kTableBytes = 196608;    // shared trig table budget of the direct kernel (192 KB)
constexpr int kFcMax = 16;             // frequencies per work unit (direct form)

// Per-curve parameters, indexed by the caller's curve number.
struct CurveParams {
    int64_t off;      // first sample in the CSR arrays
    int32_t n;        // samples
    int32_t fc;       // frequencies per work unit for this curve (direct form)
    float sigma_y;    // med(e)
    float sigma_t;
    float psnr;
    float th;         // threshold of the curve's pSNR bin (Table tab:th)
    float ip_hi;      // ip split so that w = (g - ip_hi) - ip_lo keeps sum(w) ~ 0
    float ip_lo;
    float norm;       // sqrt(N) / (N^2 ip sqrt(2 pi) sqrt(sigma_t))
    float diag;       // N (1 - ip): the i == j terms of S(f)
    float tscale;     // sqrt(beta): trig table scale, so products carry beta
    float gamma;      // magnitude scale
    double ip;        // FP64 ip
    double t0;        // min t of the curve
    float st_floor;   // smallest sigma_t the curve's planned evaluation class covers
                      // (tensor form: its harmonic count's truncation target; else 0)
    float dwsum;      // tensor form: sum over all (i, j) of the 16-bit operand's rounding
                      // error of w_ij (the row sums per sample are in StatsArgs::wrho)
};

// sigma_t = 0.1 + 0.5 exp(-12 S^2), S the Bowley skewness of the magnitudes
// with quartiles = medians of the lower and upper halves of the sorted values
// (the middle value excluded for odd N), S = 0 when Q3 = Q1: the rule that
// Section 3 keeps in the paper's source as commented-out text.  `ys` holds
// the curve's n magnitudes in ascending order.
__device__ __forceinline__ double median_of_sorted(const float* s, int n)
{
    return (n & 1) ? (double)s[n >> 1] : 0.5 * ((double)s[(n >> 1) - 1] + (double)s[n >> 1]);
}
__device__ __forceinline__ double sigma_t_rule(const float* ys, int n)
{
    const int h = n >> 1;
    const double q2 = median_of_sorted(ys, n);
    const double lq = median_of_sorted(ys, h), uq = median_of_sorted(ys + (n - h), h);
    const double sk = (uq == lq) ? 0.0 : (uq + lq - 2.0 * q2) / (uq - lq);
    return 0.1 + 0.5 * exp(-12.0 * sk * sk);
}

// Search stages.
// kStageList evaluates an explicit per-curve list of grid indices (the trial
// frequencies of the bands method).
enum Stage : int { kStageFull = 0, kStageCoarse = 1, kStageFine = 2, kStageList = 3 };

// Direct-form pair tiling: a warp owns a 32 x 32 tile of (row i, col j)
// pairs of the upper block triangle; lane (a, b) = (lane / 8, lane % 8)
// holds rows i = I0 + a + 4k (k < 8) and columns j = J0 + b + 8m (m < 4).
constexpr int kTile = 32;
constexpr int kRowsPerLane = 8;
constexpr int kColsPerLane = 4;
constexpr int kTileFloats = kTile * kTile;   // w values per stored tile

__host__ __device__ inline int tiles_of(int n)
{
    const int nb = (n + kTile - 1) / kTile;
    return nb * (nb + 1) / 2;
}

// Spurious-period exclusion windows (Section 6.1): closed frequency intervals,
// as FP64 bounds (checked against a computed frequency) and as the index
// ranges [k_lo, k_hi] they cover on the uniform grid (full_k) and on the
// coarse grid (coarse_k).  n = 0: no windows.
struct Exclusion {
    int32_t n;
    const double* f;          // [2n] lo, hi
    const int32_t* full_k;    // [2n]
    const int32_t* coarse_k;  // [2n]
};

__device__ __forceinline__ bool excluded_k(const int32_t* r, int n, int64_t k)
{
    for (int q = 0; q < n; q++)
        if (k >= r[2 * q] && k <= r[2 * q + 1]) return true;
    return false;
}

__device__ __forceinline__ bool excluded_f(const Exclusion& e, double f)
{
    for (int q = 0; q < e.n; q++)
        if (f >= e.f[2 * q] && f <= e.f[2 * q + 1]) return true;
    return false;
}

// base + k * step in FP64 without contraction: the expression the search and
// its frequency outputs use everywhere.
__device__ __forceinline__ double grid_freq(double base, double k, double step)
{
    return __dadd_rn(base, __dmul_rn(k, step));
}

// Rounding error of the tensor form's 16-bit magnitude-kernel operand for one
// entry w: FP16 round(w) - w, or for BF16 (hi + lo) - w with hi = bf16(w),
// lo = bf16(w - hi) (the operand is stored as those two parts).  The tile
// builder stores exactly these values; the statistics kernel sums the errors.
__device__ __forceinline__ float w16_err(float w, bool bf)
{
    if (bf) {
        const float hi = __bfloat162float(__float2bfloat16_rn(w));
        const float lo = __bfloat162float(__float2bfloat16_rn(w - hi));
        return (hi + lo) - w;
    }
    return __half2float(__float2half_rn(w)) - w;
}

struct PairArgs {
    const CurveParams* cp;       // [n_curves]
    const int32_t* order;        // sorted slot -> curve (N descending)
    const int64_t* unit_start;   // [n_slots+1] first unit of each slot (this stage)
    const int64_t* wtile_start;  // [n_slots+1] first W tile of each slot
    const float* W;              // W tiles of the current wave
    const float* yp;             // y' per sample (unused by the pair kernel)
    const uint64_t* ph_base;     // frac(f_min * (t - t0)) in 2^-64 turns, per sample
    const uint64_t* ph_step;     // frac(step * (t - t0)) for this stage's step
    const uint64_t* ph_coarse;   // coarse step (fine stage: peak offsets)
    const int32_t* peaks;        // [n_curves * top_k] coarse peak indices (fine stage)
    const int32_t* n_peaks;      // [n_curves]
    int stage;
    int slot_begin, slot_end;    // slots of the current wave
    int64_t unit_begin, unit_end;// units of the current wave
    int64_t wtile_base;          // wtile_start[slot_begin]
    int64_t n_freq;              // grid points of this stage (full / coarse)
    int32_t top_k;
    int32_t fine_half;           // J
    double f_min, f_max, step, coarse_df;
    float* out;                  // full stage: periodogram rows (may be null)
    int64_t out_ld;
    float* coarse_out;           // coarse stage: [n_curves * n_freq]
    unsigned long long* best_key;// [n_curves]
    unsigned long long* queue;   // work counter of this (stage, wave)
    const int32_t* trials;       // list stage: [n_curves * n_trials] grid indices, -1 = none
    int32_t n_trials;
    float* trial_stat;           // list stage: nCKP per trial (may be null)
    Exclusion ex;                // spurious-period windows (Section 6.1)
};

struct StatsArgs {
    const double* times;
    const float* mags;
    const float* errs;
    CurveParams* cp;
    float* yp;
    uint64_t* ph_base;
    uint64_t* ph_full;
    uint64_t* ph_coarse;
    uint64_t* ph_fine;
    const float* sigma_t_per_curve;
    double f_min, df, coarse_df, fine_df;
    int hierarchical;
    int sigma_t_mode;
    float sigma_t;
    float alpha;
    int np2max;
    int* status;
    float* wrho;      // tensor form: per sample, sum_j of the 16-bit rounding error of w_ij (else null)
    int wrho_bf16;    // that operand is BF16 hi + lo (else FP16)
};

struct BuildWArgs {
    const CurveParams* cp;
    const int32_t* order;
    const int64_t* wtile_start;
    const float* yp;
    float* W;
    int slot_begin, slot_end;
    int64_t tile_begin, tile_end;
};

struct TopkArgs {
    const float* coarse;
    const int32_t* order;
    int slot_begin, slot_end;
    int64_t n_freq;
    int top_k;
    int32_t* peaks;
    int32_t* n_peaks;
    Exclusion ex;                 // excluded coarse points are not peak candidates
};

struct FinalArgs {
    const CurveParams* cp;
    const unsigned long long* best_key;
    const int32_t* peaks;
    int n_curves;
    int hierarchical;             // CP_SEARCH_*
    int top_k;
    int fine_half;
    double f_min, df, coarse_df, fine_df;
    const int32_t* trials;        // bands method: best key index -> grid index
    int32_t n_trials;
    int64_t* best_idx;
    double* best_freq;
    float* best_stat;
    uint8_t* is_periodic;
    float* psnr;
};

// Tensor form (cp_tensor.cu).
struct BuildW16Args {
    const CurveParams* cp;
    const int32_t* order;
    const int64_t* wtile_start;   // first W' tile of each slot (128 x 64 tiles)
    const float* yp;
    const float* wrho;            // per sample: row sums of the operand's rounding error
    void* W16;
    int slot_begin, slot_end;
    int64_t tile_begin, tile_end;
    int bf16;
};

struct TensorArgs {
    const CurveParams* cp;
    const int32_t* order;
    const int64_t* unit_start;
    const int64_t* wtile_start;
    const void* W16;
    const float* coef;            // [n_curves * coef_stride] a_1 .. a_nmax
    int32_t coef_stride;
    const uint64_t* ph_base;
    const uint64_t* ph_step;
    const uint64_t* ph_coarse;
    const int32_t* peaks;
    const int32_t* n_peaks;
    int stage;
    int slot_begin, slot_end;
    int64_t unit_begin, unit_end;
    int64_t wtile_base;
    int64_t n_freq;
    int32_t top_k;
    int32_t fine_half;
    int32_t n_max;
    int32_t bf16;
    int32_t zsplit;               // Z as hi + lo BF16 parts (BF16 only)
    int32_t ft;                   // frequencies per unit: (zsplit ? 64 : 128) / n_max
    double f_min, f_max, step, coarse_df;
    float* out;
    int64_t out_ld;
    float* coarse_out;
    unsigned long long* best_key;
    int* status;
    uint32_t wait_limit;          // polls before a wait gives up (CP_ETIMEOUT)
    int32_t ctas_per_unit;        // 1 (one CTA per unit)
    const int32_t* trials;        // list stage (as in PairArgs)
    int32_t n_trials;
    float* trial_stat;
    Exclusion ex;
};

// Bands method, Section 3.1 (cp_bands.cu).
constexpr int kBandsMaxTrials = CP_BANDS_MAX_TRIALS;

struct BandsArgs {
    const double* times;
    const float* mags;
    const CurveParams* cp;
    int8_t* band_of;              // [n_points] band 0..9 of every sample
    int32_t* kept;                // [n_curves * n_bands] bands in D order
    int n_bands;
    int np2max;
};

struct WindowArgs {
    const CurveParams* cp;
    const int8_t* band_of;
    const int32_t* kept;
    const uint64_t* ph_base;      // frac(f_min (t - t0)) in 2^-64 turns
    const uint64_t* ph_step;      // frac(df (t - t0))
    int32_t* trials;              // [n_curves * n_bands * n_t]
    unsigned long long* cand;     // [n_curves * n_bands * 2 n_t] FP32 candidates (window -> refine)
    int* exact_scans;             // lists chosen by a whole-grid FP64 scan (completeness unproven)
    int n_curves, n_bands, n_t;
    int n_freq;
    int ex_lo, ex_hi;             // one-day grid indices [ex_lo, ex_hi] (ex_lo > ex_hi: none)
    int max_band_points;
};

size_t bands_smem_bytes(int np2max);
size_t window_smem_bytes(int max_band_points, int n_t);
size_t refine_smem_bytes(int max_band_points, int n_t);
cudaError_t prepare_bands_kernels(int np2max, int max_band_points, int n_t);
cudaError_t launch_bands(const BandsArgs& a, int n_curves, cudaStream_t s);
cudaError_t launch_window(const WindowArgs& a, cudaStream_t s);

size_t tensor_smem_bytes(bool bf16);
size_t tensor_tile_bytes(bool bf16);   // bytes of one stored W' tile (BF16: hi and lo parts)
// Largest harmonic count of the tensor form (the coefficient arrays hold this many per curve).
constexpr int kTcMaxHarmonics = 48;
int tensor_tiles_of(int n);
int tensor_freqs_per_unit(int n_max, bool zsplit);
cudaError_t prepare_tensor_kernel(int n_max);
cudaError_t launch_build_w16(const BuildW16Args& a, cudaStream_t s);
cudaError_t launch_harmonic_coef(const CurveParams* cp, int n_curves, int n_max, int stride, float* coef,
                                 cudaStream_t s);
cudaError_t launch_pair_tensor(const TensorArgs& a, int grid, cudaStream_t s);

// Launchers (cp_kernels.cu); return the launch error.
cudaError_t launch_stats(const StatsArgs& a, int n_curves, cudaStream_t s);
cudaError_t launch_build_w(const BuildWArgs& a, cudaStream_t s);
cudaError_t launch_pair_direct(const PairArgs& a, int grid, size_t smem, cudaStream_t s);
cudaError_t launch_topk(const TopkArgs& a, cudaStream_t s);
cudaError_t launch_finalize(const FinalArgs& a, cudaStream_t s);
cudaError_t launch_zero_u64(unsigned long long* p, int64_t n, cudaStream_t s);
int pair_direct_threads();
cudaError_t pair_direct_occupancy(int* blocks_per_sm, size_t smem);
size_t stats_smem_bytes(int np2max);
cudaError_t prepare_kernels(int np2max, size_t pair_smem);
// sigma_t of the skewness rule for every curve (one CTA per curve), from
// device magnitudes and device CSR offsets: the plan uses it to choose the
// tensor form's harmonic count per curve.
cudaError_t launch_sigma_t_rule(const float* mags, const int64_t* offsets, int n_curves, int np2max, float* out,
                                cudaStream_t s);

// Raises a kernel's dynamic shared-memory limit on the current device to at
// least `bytes`; never lowers it.  The limit is process-wide per device, so
// a plan (or another entry point) that needs less must not shrink the limit
// that an earlier plan's launches rely on.
cudaError_t raise_dyn_smem(const void* func, size_t bytes);

// Thread-local message returned by cp_last_error() (fixed buffer, no heap).
cp_status set_error(cp_status s, const char* msg);
const char* last_error_buffer();

// ---------------------------------------------------------------------------
// FP64-exact phase in 64-bit fixed point: frac(a * b) * 2^64 (mod 2^64).
// p + e == a*b exactly (FMA error-free product); frac(p) is exact in FP64.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t fixfrac(double a, double b)
{
    double p = a * b;
    double e = fma(a, b, -p);
    double fr = p - floor(p);                    // [0, 1), exact
    uint64_t hi = __double2ull_rn(fr * 18446744073709551616.0);   // fr has <= 53 significant bits
    long long lo = __double2ll_rn(e * 18446744073709551616.0);
    return hi + (uint64_t)lo;
}

// sin(pi x), cos(pi x) for the phase x = U / 2^32 (turns of pi), up to a
// common sign, from the Taylor series of sin and cos about 0 on the reduced
// argument r in [-1/4, 1/4]: sin(pi r) = sum (-1)^k (pi r)^(2k+1)/(2k+1)!,
// cos(pi r) = sum (-1)^k (pi r)^(2k)/(2k)!, truncated after pi^9 r^9 and
// pi^10 r^10 (remainders below 2e-9 on |r| <= 1/4).
#define CP_PI 3.14159265358979323846
__device__ __forceinline__ void sincospi_turns(uint32_t U, float& s, float& c)
{
    const uint32_t n = (U + 0x40000000u) >> 31;            // nearest multiple of 1/2 (mod 1)
    const int32_t r = (int32_t)(U - (n << 31));             // [-2^30, 2^30)
    const float x = (float)r * 2.3283064365386963e-10f;    // r / 2^32
    const float x2 = x * x;
    const float s1 = (float)(CP_PI);
    const float s3 = (float)(-CP_PI * CP_PI * CP_PI / 6.0);
    const float s5 = (float)(CP_PI * CP_PI * CP_PI * CP_PI * CP_PI / 120.0);
    const float s7 = (float)(-CP_PI * CP_PI * CP_PI * CP_PI * CP_PI * CP_PI * CP_PI / 5040.0);
    const float s9 = (float)(CP_PI * CP_PI * CP_PI * CP_PI * CP_PI * CP_PI * CP_PI * CP_PI * CP_PI / 362880.0);
    const float c2 = (float)(-CP_PI * CP_PI / 2.0);
    const float c4 = (float)(CP_PI * CP_PI * CP_PI * CP_PI / 24.0);
    const float c6 = (float)(-CP_PI * CP_PI * CP_PI * CP_PI * CP_PI * CP_PI / 720.0);
    const float c8 = (float)(CP_PI * CP_PI * CP_PI * CP_PI * CP_PI * CP_PI * CP_PI * CP_PI / 40320.0);
    const float c10 = (float)(-CP_PI * CP_PI * CP_PI * CP_PI * CP_PI * CP_PI * CP_PI * CP_PI * CP_PI * CP_PI / 3628800.0);
    float ps = fmaf(x2, s9, s7);
    ps = fmaf(x2, ps, s5);
    ps = fmaf(x2, ps, s3);
    ps = fmaf(x2, ps, s1);
    const float sx = ps * x;
    float pc = fmaf(x2, c10, c8);
    pc = fmaf(x2, pc, c6);
    pc = fmaf(x2, pc, c4);
    pc = fmaf(x2, pc, c2);
    const float cx = fmaf(x2, pc, 1.0f);
    // x + 1/2: sin -> cos, cos -> -sin
    s = n ? cx : sx;
    c = n ? -sx : cx;
}

// sin(2 pi x), cos(2 pi x) for x = U / 2^32, exact quadrant handling.
__device__ __forceinline__ void sincos2pi_turns(uint32_t U, float& s, float& c)
{
    const uint32_t q = ((U + 0x20000000u) >> 30) & 3u;      // nearest quarter turn
    const int32_t r = (int32_t)(U - (q << 30));              // [-2^29, 2^29)
    // reuse the pi-polynomial on the doubled residual: sin(2 pi r') = sin(pi (2 r'))
    const uint32_t U2 = (uint32_t)(r * 2);                    // 2r' in turns of pi, |.| <= 1/4
    float sx, cx;
    sincospi_turns(U2, sx, cx);                               // n = 0 branch: exact for |x| <= 1/4
    switch (q) {
    case 0: s = sx; c = cx; break;
    case 1: s = cx; c = -sx; break;
    case 2: s = -sx; c = -cx; break;
    default: s = -cx; c = sx; break;
    }
}

// sin(2 pi x), cos(2 pi x) for x = U / 2^32 from the SFU approximations on
// the exactly reduced angle in [-pi, pi): absolute error below 1e-6, for
// operands that are rounded to 16-bit floats afterwards.
__device__ __forceinline__ void sincos2pi_turns_sfu(uint32_t U, float& s, float& c)
{
    const float x = (float)(int32_t)U * 1.4629180792671596e-09f;   // 2 pi / 2^32
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(s) : "f"(x));
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(c) : "f"(x));
}

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// g = exp(-(y_i - y_j)^2 / (2 sigma_y^2)) from the scaled magnitudes.
__device__ __forceinline__ float gauss_g(float ypi, float ypj)
{
    const float d = ypi - ypj;
    return ex2_approx(-(d * d));
}

// ---------------------------------------------------------------------------
// Packed FP32 pairs (sm_100+ f32x2 arithmetic): two lanes per instruction.
// ---------------------------------------------------------------------------
typedef unsigned long long f2;
__device__ __forceinline__ f2 pk(float lo, float hi)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk(f2 v, float& lo, float& hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b)
{
    f2 d;
    asm("mul.rn.ftz.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c)
{
    f2 d;
    asm("fma.rn.ftz.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2 add2(f2 a, f2 b)
{
    f2 d;
    asm("add.rn.ftz.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// ---------------------------------------------------------------------------
// Best-candidate keys: max over (value, -index) with one 64-bit atomicMax.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t orderable(float v)
{
    uint32_t u = __float_as_uint(v);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float from_orderable(uint32_t u)
{
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}
__device__ __forceinline__ unsigned long long make_key(float v, uint32_t idx)
{
    return ((unsigned long long)orderable(v) << 32) | (unsigned long long)(0xffffffffu - idx);
}

}  // namespace cpk
