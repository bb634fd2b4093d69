// cp_api.cu -- host side of the C ABI declared in include/cp.h.
//
// A plan binds a ragged CSR lightcurve batch (arXiv:1412.1840, Section 5.1:
// one file of (t, magnitude, error) per star) and a trial-frequency grid to
// device buffers, a longest-first work schedule and, optionally, a captured
// CUDA graph of one best-period search.  All arithmetic of the method runs in
// the kernels of cp_kernels.cu; this file only validates, schedules, allocates
// and launches.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "cp.h"
#include "cp_internal.cuh"

using namespace cpk;

namespace cpk {

namespace {
thread_local char g_last_error[512];
}

const char* last_error_buffer() { return g_last_error; }

cp_status set_error(cp_status s, const char* msg)
{
    std::strncpy(g_last_error, msg ? msg : "", sizeof(g_last_error) - 1);
    g_last_error[sizeof(g_last_error) - 1] = 0;
    return s;
}

}  // namespace cpk

namespace {

cp_status fail(cp_status s, const std::string& msg) { return cpk::set_error(s, msg.c_str()); }

// A failed runtime call also sets the runtime's per-thread last error; it is
// cleared here so that it cannot surface later in unrelated CUDA code.
#define CP_CUDA(call)                                                                   \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            cudaGetLastError();                                                         \
            return fail(e_ == cudaErrorMemoryAllocation ? CP_ENOMEM : CP_ECUDA,         \
                        std::string(#call) + ": " + cudaGetErrorString(e_));            \
        }                                                                               \
    } while (0)

// Entry-point epilogue: a pending runtime error that no CP_CUDA check saw is
// reported (and cleared) instead of being left behind.
static cp_status finish(cp_status st, const char* where)
{
    const cudaError_t e = cudaGetLastError();
    if (st == CP_OK && e != cudaSuccess)
        return fail(CP_ECUDA, std::string(where) + ": pending CUDA error " + cudaGetErrorString(e));
    return st;
}

struct Wave {
    int slot_begin, slot_end;
    int64_t tile_begin, tile_end;
    int cls;              // 0: direct form; else the tensor form with this many harmonics
};

struct PairLaunch {
    int stage;
    int wave;
};

}  // namespace

struct cp_plan_s {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;
    int n_sm = 0;

    const double* times = nullptr;
    const float* mags = nullptr;
    const float* errs = nullptr;
    bool host_inputs = true;
    bool host_pinned = false;

    int64_t n_curves = 0, n_points = 0;
    std::vector<int64_t> offsets;
    cp_freq_grid grid{};
    cp_options opt{};
    int max_n = 0, np2max = 1;
    int64_t kc = 0;   // coarse grid points
    int J = 0;        // fine half-width in steps
    bool bands = false;          // bands method (Section 3.1)
    int n_trials = 0;            // n_bands * trials_per_band
    int ex_lo = 1, ex_hi = 0;    // one-day grid indices (empty when ex_lo > ex_hi)
    std::vector<double> excl_f;          // spurious-period windows [lo, hi] (Section 6.1)
    std::vector<int32_t> excl_full, excl_coarse;   // their grid index ranges [k_lo, k_hi]
    int max_band_points = 0;
    double f_max = 0;

    std::vector<int32_t> order;          // slot -> curve
    std::vector<int32_t> fc;             // per curve
    std::vector<int32_t> cls;            // per curve: 0 direct, else tensor harmonics
    int64_t class_count[7] = {0, 0, 0, 0, 0, 0, 0};   // curves per class {direct, 4, 8, 12, 16, 32, 48}
    std::vector<int64_t> unit_full, unit_coarse, unit_fine, unit_list, wtile;
    std::vector<Wave> waves;
    size_t pair_smem = 0;
    int pair_grid = 0;
    bool tensor = false;               // CP_FORM_TENSOR
    uint32_t wait_limit = 1u << 26;    // polls per bounded device wait (tensor form)
    int n_max = 0;                     // harmonics of the tensor form
    void* d_W16 = nullptr;             // pre-swizzled W' tiles (tensor form)
    float* d_coef = nullptr;           // [n_curves * n_max]
    float* d_wrho = nullptr;           // tensor form: per sample, row sum of the 16-bit operand's rounding error

    // device buffers
    void* dblock = nullptr;              // one allocation for everything below
    double* d_times = nullptr;
    float* d_mags = nullptr;
    float* d_errs = nullptr;
    CurveParams* d_cp = nullptr;
    float* d_yp = nullptr;
    uint64_t *d_ph_base = nullptr, *d_ph_full = nullptr, *d_ph_coarse = nullptr, *d_ph_fine = nullptr;
    float* d_stpc = nullptr;
    int32_t* d_order = nullptr;
    int64_t *d_unit_full = nullptr, *d_unit_coarse = nullptr, *d_unit_fine = nullptr, *d_wtile = nullptr;
    int64_t* d_unit_list = nullptr;
    int8_t* d_band_of = nullptr;         // bands method
    int32_t* d_kept = nullptr;
    int32_t* d_trials = nullptr;
    unsigned long long* d_wcand = nullptr;   // bands: FP32 window candidates per (curve, band)
    float* d_trial_stat = nullptr;
    double* d_excl_f = nullptr;
    int32_t *d_excl_full = nullptr, *d_excl_coarse = nullptr;
    float* d_W = nullptr;
    float* d_coarse = nullptr;
    int32_t *d_peaks = nullptr, *d_npeaks = nullptr;
    unsigned long long* d_u64 = nullptr;  // [status | best_key (n_curves) | queues]
    int64_t n_u64 = 0;
    int64_t* d_res_idx = nullptr;
    double* d_res_freq = nullptr;
    float* d_res_stat = nullptr;
    uint8_t* d_res_per = nullptr;
    float* d_res_psnr = nullptr;

    // pinned host
    void* hblock = nullptr;
    int64_t* h_res_idx = nullptr;
    double* h_res_freq = nullptr;
    float* h_res_stat = nullptr;
    uint8_t* h_res_per = nullptr;
    float* h_res_psnr = nullptr;
    unsigned long long* h_status = nullptr;
    double* h_times = nullptr;             // pinned staging for pageable host inputs
    float* h_mags = nullptr;
    float* h_errs = nullptr;

    // graph and timing
    cudaGraphExec_t exec = nullptr;
    bool graph_ready = false;
    std::vector<cudaEvent_t> ev_pair;      // 2 per pair launch of a search
    cudaEvent_t ev_step0 = nullptr, ev_step1 = nullptr;
    cudaEvent_t ev_bands0 = nullptr, ev_bands1 = nullptr;
    float last_pair_ms = 0.f, last_step_ms = 0.f, last_tensor_ms = 0.f, last_direct_ms = 0.f, last_bands_ms = 0.f;
    double window_terms = 0;
    std::vector<int> ev_cls;               // class of each pair launch (0 direct)
    double tensor_flops = 0, direct_pf = 0;
    int64_t launches_per_search = 0;
    double pf_full = 0, pf_search = 0;
    bool ran = false;
    bool searched = false;    // a best-period search completed (trial list valid)
    bool capturing = false;   // inside build_graph's stream capture
    cp_tuning tune{};         // copy of the caller's tuning table (has_tune)
    bool has_tune = false;
    int64_t replans = 0;      // plans rebuilt because a curve's sigma_t left its class
    float* last_out = nullptr;   // output of the last cp_periodogram (re-run after a re-plan)
};

namespace {

inline unsigned long long* status_word(cp_plan_t p) { return p->d_u64; }
inline unsigned long long* best_keys(cp_plan_t p) { return p->d_u64 + 1; }
inline unsigned long long* queue_word(cp_plan_t p, int i) { return p->d_u64 + 1 + p->n_curves + i; }
constexpr int kQueuesPerWave = 4;   // one work counter per (wave, stage)

constexpr int kCoefStride = kTcMaxHarmonics;   // a_1..a_48 stored per curve (largest class)

int class_rank(int cls)
{
    switch (cls) {
    case 4: return 1;
    case 8: return 2;
    case 12: return 3;
    case 16: return 4;
    case 32: return 5;
    case 48: return 6;
    }
    return 0;   // direct form
}

// Truncation tail 1 - (a_0 + ... + a_n) of the periodic kernel's harmonic
// series, relative to its peak value 1.
double harmonic_tail(double sigma_t, int n)
{
    double a[kTcMaxHarmonics + 1];
    if (n > kTcMaxHarmonics || cp_bessel_coefficients(sigma_t, n, a) != CP_OK) return 1.0;
    double s = 0.0;
    for (int k = 0; k <= n; k++) s += a[k];
    return 1.0 - s;
}

// Smallest harmonic count of the tensor form (8, 12, 16, 32, 48) whose
// truncation tail stays below 1e-4 of the kernel peak; 0 (direct form) when even
// 48 harmonics do not reach it (sigma_t below about 0.09, which the sigma_t rule
// never gives).  The tail falls as sigma_t grows, so each class is a threshold
// on sigma_t, found once by bisection.
const std::vector<double>& harmonic_thresholds()
{
    static const std::vector<double> thr = [] {
        std::vector<double> t;
        for (int n : {8, 12, 16, 32, 48}) {
            double lo = 0.02, hi = 4.0;
            for (int it = 0; it < 40; it++) {
                const double mid = 0.5 * (lo + hi);
                if (harmonic_tail(mid, n) <= 1e-4) hi = mid; else lo = mid;
            }
            t.push_back(hi);
        }
        return t;
    }();
    return thr;
}

// W' is stored as hi + lo BF16 parts for both BF16 operand types.
static bool w_bf16(int dtype) { return dtype == CP_DTYPE_BF16 || dtype == CP_DTYPE_BF16_SPLIT; }

int harmonics_for(float sigma_t)
{
    const std::vector<double>& thr = harmonic_thresholds();
    const int cls[5] = {8, 12, 16, 32, 48};
    for (int k = 0; k < 5; k++)
        if ((double)sigma_t >= thr[k]) return cls[k];
    return 0;
}

// Smallest sigma_t (as the FP32 value the kernels use) that harmonic class cls
// covers; 0 for the direct form.
float sigma_t_floor(int cls)
{
    const std::vector<double>& thr = harmonic_thresholds();
    const int k = cls == 8 ? 0 : cls == 12 ? 1 : cls == 16 ? 2 : cls == 32 ? 3 : cls == 48 ? 4 : -1;
    if (k < 0) return 0.f;
    float f = (float)thr[k];
    if ((double)f < thr[k]) f = std::nextafter(f, INFINITY);   // the first FP32 value harmonics_for accepts
    return f;
}

// sigma_t of every curve as the plan sees it at creation time (to choose the
// tensor form's harmonic count per curve).  The rule mode evaluates the rule
// on the device from the current magnitudes (one kernel; only the n_curves
// results come back to the host).
cp_status plan_sigma_t(cp_plan_t p, const cp_options& opt, std::vector<float>& st)
{
    const int64_t nc = p->n_curves;
    if (opt.sigma_t_mode == CP_SIGMA_T_FIXED) {
        std::fill(st.begin(), st.end(), opt.sigma_t);
        return CP_OK;
    }
    if (opt.sigma_t_mode == CP_SIGMA_T_PER_CURVE) {
        for (int64_t c = 0; c < nc; c++) st[c] = opt.sigma_t_per_curve[c];
        return CP_OK;
    }
    const size_t npb = (size_t)p->n_points * sizeof(float);
    const size_t ob = (size_t)(nc + 1) * sizeof(int64_t), sb = (size_t)nc * sizeof(float);
    char* tmp = nullptr;
    const size_t mb = p->host_inputs ? (npb + 255) / 256 * 256 : 0;
    CP_CUDA(cudaMalloc(&tmp, mb + (ob + 255) / 256 * 256 + sb));
    float* d_m = p->host_inputs ? reinterpret_cast<float*>(tmp) : const_cast<float*>(p->mags);
    int64_t* d_off = reinterpret_cast<int64_t*>(tmp + mb);
    float* d_st = reinterpret_cast<float*>(tmp + mb + (ob + 255) / 256 * 256);
    cudaError_t e = cudaSuccess;
    if (p->host_inputs) e = cudaMemcpyAsync(d_m, p->mags, npb, cudaMemcpyHostToDevice, p->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_off, p->offsets.data(), ob, cudaMemcpyHostToDevice, p->stream);
    if (e == cudaSuccess) e = launch_sigma_t_rule(d_m, d_off, (int)nc, p->np2max, d_st, p->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(st.data(), d_st, sb, cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    cudaFree(tmp);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(CP_ECUDA, std::string("cp_plan: sigma_t rule on the device: ") + cudaGetErrorString(e));
    }
    return CP_OK;
}

// Grid indices k in [0, n) with lo <= base + k * step <= hi, the frequency
// evaluated in FP64 exactly as the search evaluates it (base + k*step, no
// contraction); the frequency is non-decreasing in k, so the set is the range
// [first, last] found by two bisections (empty when first > last).
void grid_index_range(double base, double step, int64_t n, double lo, double hi, int32_t* out)
{
    auto f = [&](int64_t k) { return base + (double)k * step; };
    int64_t a = 0, b = n;
    while (a < b) {
        const int64_t m = a + (b - a) / 2;
        if (f(m) >= lo) b = m; else a = m + 1;
    }
    const int64_t first = a;
    a = 0;
    b = n;
    while (a < b) {
        const int64_t m = a + (b - a) / 2;
        if (f(m) > hi) b = m; else a = m + 1;
    }
    const int64_t last = a - 1;
    out[0] = (int32_t)std::min<int64_t>(first, INT32_MAX);
    out[1] = (int32_t)std::max<int64_t>(last, -1);
}

Exclusion exclusion_of(cp_plan_t p)
{
    Exclusion e{};
    e.n = (int32_t)(p->excl_f.size() / 2);
    e.f = p->d_excl_f;
    e.full_k = p->d_excl_full;
    e.coarse_k = p->d_excl_coarse;
    return e;
}

// Events recorded during capture must be external nodes to stay timeable;
// outside capture the flag is not allowed.
unsigned rec_flags(cp_plan_t p) { return p->capturing ? cudaEventRecordExternal : cudaEventRecordDefault; }

// Frequencies per direct-form unit: the requested count (16 by default),
// halved until the unit's trig table fits the kernel's shared-memory budget.
int fc_for(int n, int want = kFcMax)
{
    const int npad = (n + kTile - 1) / kTile * kTile;
    int f = want;
    while (f > 2 && (size_t)npad * f * 12 > (size_t)kTableBytes) f >>= 1;
    return f;
}

// Tuning bucket of a curve of n samples, or -1 (built-in choices).
int tune_bucket(const cp_tuning& t, int n)
{
    for (int b = 0; b < t.n_buckets; b++)
        if (n <= t.bucket_max_n[b]) return b;
    return -1;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Failure-injection hook for tests: with CP_FAIL_ALLOC=k in the environment,
// the k-th allocation (device or pinned host, counted from 1) of one cp_plan
// call reports cudaErrorMemoryAllocation without allocating.  The plan must
// then return CP_ENOMEM and release everything it allocated before.
struct AllocHook {
    int target = 0, count = 0;
    AllocHook()
    {
        if (const char* env = std::getenv("CP_FAIL_ALLOC")) target = std::atoi(env);
    }
    cudaError_t device(void** p, size_t bytes)
    {
        if (++count == target) return cudaErrorMemoryAllocation;
        return cudaMalloc(p, bytes);
    }
    cudaError_t pinned(void** p, size_t bytes)
    {
        if (++count == target) return cudaErrorMemoryAllocation;
        return cudaMallocHost(p, bytes);
    }
};

// Copies host inputs (pageable case) into the pinned staging buffers.
void stage_host_inputs(cp_plan_t p)
{
    if (p->host_inputs && !p->host_pinned) {
        std::memcpy(p->h_times, p->times, (size_t)p->n_points * sizeof(double));
        std::memcpy(p->h_mags, p->mags, (size_t)p->n_points * sizeof(float));
        std::memcpy(p->h_errs, p->errs, (size_t)p->n_points * sizeof(float));
    }
}

cp_status enqueue_inputs(cp_plan_t p, cudaStream_t s)
{
    if (!p->host_inputs) return CP_OK;
    const double* st = p->host_pinned ? p->times : p->h_times;
    const float* sm = p->host_pinned ? p->mags : p->h_mags;
    const float* se = p->host_pinned ? p->errs : p->h_errs;
    CP_CUDA(cudaMemcpyAsync(p->d_times, st, (size_t)p->n_points * sizeof(double), cudaMemcpyHostToDevice, s));
    CP_CUDA(cudaMemcpyAsync(p->d_mags, sm, (size_t)p->n_points * sizeof(float), cudaMemcpyHostToDevice, s));
    CP_CUDA(cudaMemcpyAsync(p->d_errs, se, (size_t)p->n_points * sizeof(float), cudaMemcpyHostToDevice, s));
    return CP_OK;
}

cp_status enqueue_stats(cp_plan_t p, cudaStream_t s)
{
    CP_CUDA(launch_zero_u64(p->d_u64, p->n_u64, s));
    StatsArgs a{};
    a.times = p->host_inputs ? p->d_times : p->times;
    a.mags = p->host_inputs ? p->d_mags : p->mags;
    a.errs = p->host_inputs ? p->d_errs : p->errs;
    a.cp = p->d_cp;
    a.yp = p->d_yp;
    a.ph_base = p->d_ph_base;
    a.ph_full = p->d_ph_full;
    a.ph_coarse = p->d_ph_coarse;
    a.ph_fine = p->d_ph_fine;
    a.sigma_t_per_curve = p->d_stpc;
    a.f_min = p->grid.f_min;
    a.df = p->grid.df;
    a.coarse_df = p->grid.coarse_df;
    a.fine_df = p->grid.fine_df;
    a.hierarchical = p->grid.hierarchical == CP_SEARCH_COARSE_FINE ? 1 : 0;   // coarse / fine phase steps
    a.sigma_t_mode = p->opt.sigma_t_mode;
    a.sigma_t = p->opt.sigma_t;
    a.alpha = p->opt.alpha;
    a.np2max = p->np2max;
    a.status = reinterpret_cast<int*>(status_word(p));
    a.wrho = p->tensor ? p->d_wrho : nullptr;
    a.wrho_bf16 = w_bf16(p->opt.dtype) ? 1 : 0;
    CP_CUDA(launch_stats(a, (int)p->n_curves, s));
    if (p->tensor) {
        // coefficients up to the plan's largest class (the quadrature size follows the count)
        const int count = p->class_count[class_rank(48)] ? 48 : 32;
        CP_CUDA(launch_harmonic_coef(p->d_cp, (int)p->n_curves, count, kCoefStride, p->d_coef, s));
    }
    return CP_OK;
}

PairArgs pair_args(cp_plan_t p, int stage, int w, float* out)
{
    const Wave& wv = p->waves[w];
    PairArgs a{};
    a.cp = p->d_cp;
    a.order = p->d_order;
    a.wtile_start = p->d_wtile;
    a.W = p->d_W;
    a.yp = p->d_yp;
    a.ph_base = p->d_ph_base;
    a.ph_coarse = p->d_ph_coarse;
    a.peaks = p->d_peaks;
    a.n_peaks = p->d_npeaks;
    a.stage = stage;
    a.slot_begin = wv.slot_begin;
    a.slot_end = wv.slot_end;
    a.wtile_base = wv.tile_begin;
    a.top_k = p->grid.top_k;
    a.fine_half = p->J;
    a.f_min = p->grid.f_min;
    a.f_max = p->f_max;
    a.coarse_df = p->grid.coarse_df;
    a.out = out;
    a.out_ld = p->grid.n_freq;
    a.coarse_out = p->d_coarse;
    a.best_key = best_keys(p);
    a.queue = queue_word(p, kQueuesPerWave * w + stage);
    a.ex = exclusion_of(p);
    const std::vector<int64_t>* us;
    if (stage == kStageList) {
        a.unit_start = p->d_unit_list;
        a.ph_step = p->d_ph_full;
        a.n_freq = p->grid.n_freq;
        a.step = p->grid.df;
        a.trials = p->d_trials;
        a.n_trials = p->n_trials;
        a.trial_stat = p->d_trial_stat;
        us = &p->unit_list;
    } else if (stage == kStageFull) {
        a.unit_start = p->d_unit_full;
        a.ph_step = p->d_ph_full;
        a.n_freq = p->grid.n_freq;
        a.step = p->grid.df;
        us = &p->unit_full;
    } else if (stage == kStageCoarse) {
        a.unit_start = p->d_unit_coarse;
        a.ph_step = p->d_ph_coarse;
        a.n_freq = p->kc;
        a.step = p->grid.coarse_df;
        us = &p->unit_coarse;
    } else {
        a.unit_start = p->d_unit_fine;
        a.ph_step = p->d_ph_fine;
        a.n_freq = p->kc;
        a.step = p->grid.fine_df;
        us = &p->unit_fine;
    }
    a.unit_begin = (*us)[wv.slot_begin];
    a.unit_end = (*us)[wv.slot_end];
    return a;
}

cp_status enqueue_wave_w(cp_plan_t p, int w, cudaStream_t s)
{
    const Wave& wv = p->waves[w];
    if (wv.cls != 0) {
        BuildW16Args b{};
        b.cp = p->d_cp;
        b.order = p->d_order;
        b.wtile_start = p->d_wtile;
        b.yp = p->d_yp;
        b.wrho = p->d_wrho;
        b.W16 = p->d_W16;
        b.slot_begin = wv.slot_begin;
        b.slot_end = wv.slot_end;
        b.tile_begin = wv.tile_begin;
        b.tile_end = wv.tile_end;
        b.bf16 = w_bf16(p->opt.dtype) ? 1 : 0;
        CP_CUDA(launch_build_w16(b, s));
        return CP_OK;
    }
    BuildWArgs b{};
    b.cp = p->d_cp;
    b.order = p->d_order;
    b.wtile_start = p->d_wtile;
    b.yp = p->d_yp;
    b.W = p->d_W;
    b.slot_begin = wv.slot_begin;
    b.slot_end = wv.slot_end;
    b.tile_begin = wv.tile_begin;
    b.tile_end = wv.tile_end;
    CP_CUDA(launch_build_w(b, s));
    return CP_OK;
}

TensorArgs tensor_args(const PairArgs& d, cp_plan_t p)
{
    TensorArgs t{};
    t.cp = d.cp;
    t.order = d.order;
    t.unit_start = d.unit_start;
    t.wtile_start = d.wtile_start;
    t.W16 = p->d_W16;
    t.coef = p->d_coef;
    t.coef_stride = kCoefStride;
    t.ph_base = d.ph_base;
    t.ph_step = d.ph_step;
    t.ph_coarse = d.ph_coarse;
    t.peaks = d.peaks;
    t.n_peaks = d.n_peaks;
    t.stage = d.stage;
    t.slot_begin = d.slot_begin;
    t.slot_end = d.slot_end;
    t.unit_begin = d.unit_begin;
    t.unit_end = d.unit_end;
    t.wtile_base = d.wtile_base;
    t.n_freq = d.n_freq;
    t.top_k = d.top_k;
    t.fine_half = d.fine_half;
    t.n_max = p->n_max;
    t.bf16 = w_bf16(p->opt.dtype) ? 1 : 0;
    t.zsplit = p->opt.dtype == CP_DTYPE_BF16_SPLIT ? 1 : 0;
    t.f_min = d.f_min;
    t.f_max = d.f_max;
    t.step = d.step;
    t.coarse_df = d.coarse_df;
    t.out = d.out;
    t.out_ld = d.out_ld;
    t.coarse_out = d.coarse_out;
    t.best_key = d.best_key;
    t.status = reinterpret_cast<int*>(status_word(p));
    t.wait_limit = p->wait_limit;
    t.ctas_per_unit = 1;
    t.trials = d.trials;
    t.n_trials = d.n_trials;
    t.trial_stat = d.trial_stat;
    t.ex = d.ex;
    return t;
}

cp_status enqueue_pair(cp_plan_t p, int stage, int w, float* out, cudaStream_t s, int* ev_idx)
{
    const PairArgs a = pair_args(p, stage, w, out);
    if (ev_idx) {
        CP_CUDA(cudaEventRecordWithFlags(p->ev_pair[2 * (*ev_idx)], s, rec_flags(p)));
        p->ev_cls[*ev_idx] = p->waves[w].cls;
    }
    if (p->waves[w].cls != 0) {
        TensorArgs t = tensor_args(a, p);
        t.n_max = p->waves[w].cls;
        t.ft = tensor_freqs_per_unit(t.n_max, t.zsplit != 0);
        CP_CUDA(launch_pair_tensor(t, p->n_sm, s));
    } else {
        CP_CUDA(launch_pair_direct(a, p->pair_grid, p->pair_smem, s));
    }
    if (ev_idx) {
        CP_CUDA(cudaEventRecordWithFlags(p->ev_pair[2 * (*ev_idx) + 1], s, rec_flags(p)));
        (*ev_idx)++;
    }
    return CP_OK;
}

cp_status enqueue_search(cp_plan_t p, cudaStream_t s)
{
    cp_status st;
    CP_CUDA(cudaEventRecordWithFlags(p->ev_step0, s, rec_flags(p)));
    if ((st = enqueue_inputs(p, s)) != CP_OK) return st;
    if ((st = enqueue_stats(p, s)) != CP_OK) return st;
    if (p->bands) {
        CP_CUDA(cudaEventRecordWithFlags(p->ev_bands0, s, rec_flags(p)));
        BandsArgs b{};
        b.times = p->host_inputs ? p->d_times : p->times;
        b.mags = p->host_inputs ? p->d_mags : p->mags;
        b.cp = p->d_cp;
        b.band_of = p->d_band_of;
        b.kept = p->d_kept;
        b.n_bands = p->grid.n_bands;
        b.np2max = p->np2max;
        CP_CUDA(launch_bands(b, (int)p->n_curves, s));
        WindowArgs wa{};
        wa.cp = p->d_cp;
        wa.band_of = p->d_band_of;
        wa.kept = p->d_kept;
        wa.ph_base = p->d_ph_base;
        wa.ph_step = p->d_ph_full;
        wa.trials = p->d_trials;
        wa.cand = p->d_wcand;
        wa.exact_scans = reinterpret_cast<int*>(status_word(p)) + 1;   // high half of the status word
        wa.n_curves = (int)p->n_curves;
        wa.n_bands = p->grid.n_bands;
        wa.n_t = p->grid.trials_per_band;
        wa.n_freq = (int)p->grid.n_freq;
        wa.ex_lo = p->ex_lo;
        wa.ex_hi = p->ex_hi;
        wa.max_band_points = p->max_band_points;
        CP_CUDA(launch_window(wa, s));
        CP_CUDA(cudaEventRecordWithFlags(p->ev_bands1, s, rec_flags(p)));
    }
    int ev = 0;
    for (int w = 0; w < (int)p->waves.size(); w++) {
        if ((st = enqueue_wave_w(p, w, s)) != CP_OK) return st;
        if (p->bands) {
            if ((st = enqueue_pair(p, kStageList, w, nullptr, s, &ev)) != CP_OK) return st;
        } else if (!p->grid.hierarchical) {
            if ((st = enqueue_pair(p, kStageFull, w, nullptr, s, &ev)) != CP_OK) return st;
        } else {
            if ((st = enqueue_pair(p, kStageCoarse, w, nullptr, s, &ev)) != CP_OK) return st;
            TopkArgs t{};
            t.coarse = p->d_coarse;
            t.order = p->d_order;
            t.slot_begin = p->waves[w].slot_begin;
            t.slot_end = p->waves[w].slot_end;
            t.n_freq = p->kc;
            t.top_k = p->grid.top_k;
            t.peaks = p->d_peaks;
            t.n_peaks = p->d_npeaks;
            t.ex = exclusion_of(p);
            CP_CUDA(launch_topk(t, s));
            if ((st = enqueue_pair(p, kStageFine, w, nullptr, s, &ev)) != CP_OK) return st;
        }
    }
    FinalArgs f{};
    f.cp = p->d_cp;
    f.best_key = best_keys(p);
    f.peaks = p->d_peaks;
    f.n_curves = (int)p->n_curves;
    f.hierarchical = p->grid.hierarchical;
    f.top_k = p->grid.top_k;
    f.trials = p->d_trials;
    f.n_trials = p->n_trials;
    f.fine_half = p->J;
    f.f_min = p->grid.f_min;
    f.df = p->grid.df;
    f.coarse_df = p->grid.coarse_df;
    f.fine_df = p->grid.fine_df;
    f.best_idx = p->d_res_idx;
    f.best_freq = p->d_res_freq;
    f.best_stat = p->d_res_stat;
    f.is_periodic = p->d_res_per;
    f.psnr = p->d_res_psnr;
    CP_CUDA(launch_finalize(f, s));
    const size_t nc = (size_t)p->n_curves;
    CP_CUDA(cudaMemcpyAsync(p->h_res_idx, p->d_res_idx, nc * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CP_CUDA(cudaMemcpyAsync(p->h_res_freq, p->d_res_freq, nc * sizeof(double), cudaMemcpyDeviceToHost, s));
    CP_CUDA(cudaMemcpyAsync(p->h_res_stat, p->d_res_stat, nc * sizeof(float), cudaMemcpyDeviceToHost, s));
    CP_CUDA(cudaMemcpyAsync(p->h_res_per, p->d_res_per, nc, cudaMemcpyDeviceToHost, s));
    CP_CUDA(cudaMemcpyAsync(p->h_res_psnr, p->d_res_psnr, nc * sizeof(float), cudaMemcpyDeviceToHost, s));
    CP_CUDA(cudaMemcpyAsync(p->h_status, p->d_u64, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    CP_CUDA(cudaEventRecordWithFlags(p->ev_step1, s, rec_flags(p)));
    return CP_OK;
}

cp_status build_graph(cp_plan_t p)
{
    CP_CUDA(cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal));
    p->capturing = true;
    cp_status st = enqueue_search(p, p->cap);
    p->capturing = false;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(p->cap, &g);
    if (st != CP_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return fail(CP_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&p->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(CP_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    p->graph_ready = true;
    return CP_OK;
}

cp_status read_timings(cp_plan_t p)
{
    float total = 0.f, tens = 0.f, dir = 0.f;
    const int npl = (int)p->ev_pair.size() / 2;
    for (int i = 0; i < npl; i++) {
        float ms = 0.f;
        CP_CUDA(cudaEventElapsedTime(&ms, p->ev_pair[2 * i], p->ev_pair[2 * i + 1]));
        total += ms;
        (p->ev_cls[i] ? tens : dir) += ms;
    }
    p->last_pair_ms = total;
    p->last_tensor_ms = tens;
    p->last_direct_ms = dir;
    float ms = 0.f;
    CP_CUDA(cudaEventElapsedTime(&ms, p->ev_step0, p->ev_step1));
    p->last_step_ms = ms;
    if (p->bands) {
        CP_CUDA(cudaEventElapsedTime(&ms, p->ev_bands0, p->ev_bands1));
        p->last_bands_ms = ms;
    }
    return CP_OK;
}

}  // namespace

extern "C" {

void cp_default_options(cp_options* o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->sigma_t_mode = CP_SIGMA_T_FIXED;
    o->sigma_t = 0.3f;
    o->sigma_t_per_curve = nullptr;
    o->alpha = 1.0f;
    o->form = CP_FORM_DIRECT;
    o->dtype = CP_DTYPE_FP16;
    o->n_max = 0;
    o->input_memory = CP_MEM_HOST;
    o->use_graph = 1;
    o->device = 0;
    o->tuning = nullptr;
}

int64_t cp_max_points(void) { return kMaxN; }

const char* cp_status_string(cp_status s)
{
    switch (s) {
    case CP_OK: return "ok";
    case CP_EINVAL: return "invalid argument";
    case CP_ENOMEM: return "out of memory";
    case CP_ECUDA: return "CUDA error";
    case CP_ETIMEOUT: return "device wait timed out";
    case CP_ESTATE: return "invalid plan state";
    case CP_EUNSUPPORTED: return "unsupported request";
    }
    return "unknown status";
}

const char* cp_last_error(void) { return cpk::last_error_buffer(); }

void cp_destroy(cp_plan_t p)
{
    if (!p) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(p->device);
    if (p->stream) cudaStreamSynchronize(p->stream);
    if (p->exec) cudaGraphExecDestroy(p->exec);
    for (cudaEvent_t e : p->ev_pair) cudaEventDestroy(e);
    if (p->ev_step0) cudaEventDestroy(p->ev_step0);
    if (p->ev_step1) cudaEventDestroy(p->ev_step1);
    if (p->ev_bands0) cudaEventDestroy(p->ev_bands0);
    if (p->ev_bands1) cudaEventDestroy(p->ev_bands1);
    if (p->cap) cudaStreamDestroy(p->cap);
    if (p->dblock) cudaFree(p->dblock);
    if (p->hblock) cudaFreeHost(p->hblock);
    cudaSetDevice(prev);
    cudaGetLastError();
    delete p;
}

static cp_status plan_impl(const double* times, const float* mags, const float* errs,
                           const int64_t* offsets, int64_t n_curves, const cp_freq_grid* grid,
                           const cp_options* opt_in, void* stream, cp_plan_s* p)
{
    if (!times || !mags || !errs || !offsets || !grid)
        return fail(CP_EINVAL, "cp_plan: null argument");
    if (n_curves < 1 || n_curves > (int64_t)1 << 30)
        return fail(CP_EINVAL, "cp_plan: n_curves must be in [1, 2^30]");
    cp_options opt;
    if (opt_in) opt = *opt_in; else cp_default_options(&opt);
    if (opt.form != CP_FORM_DIRECT && opt.form != CP_FORM_TENSOR)
        return fail(CP_EINVAL, "cp_plan: form must be CP_FORM_DIRECT or CP_FORM_TENSOR");
    if (opt.form == CP_FORM_TENSOR) {
        if (opt.dtype != CP_DTYPE_FP16 && opt.dtype != CP_DTYPE_BF16 && opt.dtype != CP_DTYPE_BF16_SPLIT)
            return fail(CP_EINVAL, "cp_plan: dtype must be CP_DTYPE_FP16, CP_DTYPE_BF16 or CP_DTYPE_BF16_SPLIT");
        if (opt.n_max != 0 && opt.n_max != 4 && opt.n_max != 8 && opt.n_max != 12 && opt.n_max != 16 &&
            opt.n_max != 32 && opt.n_max != 48)
            return fail(CP_EINVAL, "cp_plan: n_max must be 0 (per curve), 4, 8, 12, 16, 32 or 48");
        if (opt.dtype == CP_DTYPE_BF16_SPLIT && (opt.n_max == 12 || opt.n_max == 48))
            return fail(CP_EINVAL, "cp_plan: n_max 12 and 48 are not available with CP_DTYPE_BF16_SPLIT (4, 8, 16 or 32)");
        p->tensor = true;
        p->n_max = opt.n_max;
        // test hook: shorter bounded waits, to exercise the timeout path
        if (const char* env = std::getenv("CP_WAIT_LIMIT")) p->wait_limit = (uint32_t)std::strtoul(env, nullptr, 10);
    }
    if (opt.sigma_t_mode < 0 || opt.sigma_t_mode > 2)
        return fail(CP_EINVAL, "cp_plan: sigma_t_mode must be 0, 1 or 2");
    if (opt.sigma_t_mode == CP_SIGMA_T_FIXED && !(opt.sigma_t > 0.f && std::isfinite(opt.sigma_t)))
        return fail(CP_EINVAL, "cp_plan: sigma_t must be finite and > 0");
    if (opt.sigma_t_mode == CP_SIGMA_T_PER_CURVE && !opt.sigma_t_per_curve)
        return fail(CP_EINVAL, "cp_plan: sigma_t_per_curve is NULL");
    if (!(opt.alpha > 0.f && std::isfinite(opt.alpha)))
        return fail(CP_EINVAL, "cp_plan: alpha must be finite and > 0");
    if (opt.input_memory != CP_MEM_HOST && opt.input_memory != CP_MEM_DEVICE)
        return fail(CP_EINVAL, "cp_plan: input_memory must be CP_MEM_HOST or CP_MEM_DEVICE");
    cp_tuning tune{};
    if (opt.tuning) {
        tune = *opt.tuning;
        if (tune.n_buckets < 0 || tune.n_buckets > CP_TUNE_MAX_BUCKETS)
            return fail(CP_EINVAL, "cp_plan: tuning.n_buckets must be in [0, CP_TUNE_MAX_BUCKETS]");
        for (int b = 0; b < tune.n_buckets; b++) {
            const int fc = tune.direct_fc[b];
            if (tune.bucket_max_n[b] < 2 || (b > 0 && tune.bucket_max_n[b] <= tune.bucket_max_n[b - 1]))
                return fail(CP_EINVAL, "cp_plan: tuning.bucket_max_n must be >= 2 and strictly ascending");
            if (fc != 2 && fc != 4 && fc != 8 && fc != 16)
                return fail(CP_EINVAL, "cp_plan: tuning.direct_fc must be 2, 4, 8 or 16");
            if (tune.tensor_classes[b] < 0 || tune.tensor_classes[b] > 31)
                return fail(CP_EINVAL, "cp_plan: tuning.tensor_classes must be a 5-bit mask");
        }
        opt.tuning = nullptr;   // copied; the caller's struct is not kept
        p->tune = tune;
        p->has_tune = true;
    }
    const cp_freq_grid g = *grid;
    if (!(std::isfinite(g.f_min) && g.f_min >= 0.0 && std::isfinite(g.df) && g.df > 0.0))
        return fail(CP_EINVAL, "cp_plan: need finite f_min >= 0 and df > 0");
    if (g.n_freq < 1 || g.n_freq > ((int64_t)1 << 31) - 1)
        return fail(CP_EINVAL, "cp_plan: n_freq must be in [1, 2^31)");
    p->f_max = g.f_min + (double)(g.n_freq - 1) * g.df;
    if (g.hierarchical < CP_SEARCH_FULL || g.hierarchical > CP_SEARCH_BANDS)
        return fail(CP_EINVAL, "cp_plan: hierarchical must be CP_SEARCH_FULL, _COARSE_FINE or _BANDS");
    if (g.hierarchical == CP_SEARCH_BANDS) {
        if (g.n_bands < 1 || g.n_bands > 10)
            return fail(CP_EINVAL, "cp_plan: n_bands must be in [1, 10]");
        if (g.trials_per_band < 1 || g.trials_per_band > kBandsMaxTrials)
            return fail(CP_EINVAL, "cp_plan: trials_per_band must be in [1, " + std::to_string(kBandsMaxTrials) + "]");
        if (g.n_freq >= ((int64_t)1 << 28))
            return fail(CP_EUNSUPPORTED, "cp_plan: the bands method supports grids of fewer than 2^28 points");
        p->bands = true;
        p->n_trials = g.n_bands * g.trials_per_band;
        // grid indices of the one-day frequencies |1/f - 1| < 1e-4 (a contiguous range; the
        // test is evaluated per index with the FP64 expressions of the search itself)
        const double klo = std::floor((1.0 / 1.0001 - g.f_min) / g.df) - 2.0;
        const double khi = std::ceil((1.0 / 0.9999 - g.f_min) / g.df) + 2.0;
        if (khi >= 0.0 && klo <= (double)(g.n_freq - 1)) {
            const int64_t a0 = std::max<int64_t>(0, (int64_t)klo), a1 = std::min<int64_t>(g.n_freq - 1, (int64_t)khi);
            for (int64_t k = a0; k <= a1; k++) {
                const double prod = (double)k * g.df;
                const double f = g.f_min + prod;
                if (f > 0.0 && std::fabs(1.0 / f - 1.0) < 1e-4) {
                    if (p->ex_lo > p->ex_hi) p->ex_lo = p->ex_hi = (int)k;
                    p->ex_lo = std::min(p->ex_lo, (int)k);
                    p->ex_hi = std::max(p->ex_hi, (int)k);
                }
            }
        }
    } else if (g.hierarchical) {
        if (!(g.coarse_df > 0.0 && std::isfinite(g.coarse_df) && g.fine_df > 0.0 && std::isfinite(g.fine_df) &&
              g.fine_halfwidth >= 0.0 && std::isfinite(g.fine_halfwidth)))
            return fail(CP_EINVAL, "cp_plan: hierarchical grid needs coarse_df > 0, fine_df > 0, fine_halfwidth >= 0");
        if (g.top_k < 1 || g.top_k > 1024)
            return fail(CP_EINVAL, "cp_plan: top_k must be in [1, 1024]");
        p->kc = (int64_t)std::floor((p->f_max - g.f_min) / g.coarse_df + 0.5) + 1;
        const double jd = std::floor(g.fine_halfwidth / g.fine_df + 0.5);
        if (jd > 1e6 || (2.0 * jd + 1.0) * g.top_k > 2e9 || p->kc > ((int64_t)1 << 31) - 1)
            return fail(CP_EINVAL, "cp_plan: hierarchical grid too large");
        p->J = (int)jd;
    }

    // spurious-period exclusion windows (Section 6.1), copied; their index ranges on
    // the uniform grid and (coarse-then-fine) on the coarse grid
    if (g.n_exclude < 0 || g.n_exclude > CP_MAX_EXCLUDE)
        return fail(CP_EINVAL, "cp_plan: n_exclude must be in [0, CP_MAX_EXCLUDE]");
    if (g.n_exclude > 0 && !g.exclude) return fail(CP_EINVAL, "cp_plan: exclude is NULL");
    for (int q = 0; q < g.n_exclude; q++) {
        const double lo = g.exclude[2 * q], hi = g.exclude[2 * q + 1];
        if (!(std::isfinite(lo) && std::isfinite(hi) && lo <= hi))
            return fail(CP_EINVAL, "cp_plan: exclusion windows need finite lo <= hi");
        p->excl_f.push_back(lo);
        p->excl_f.push_back(hi);
        int32_t r[2];
        grid_index_range(g.f_min, g.df, g.n_freq, lo, hi, r);
        p->excl_full.insert(p->excl_full.end(), r, r + 2);
        grid_index_range(g.f_min, g.coarse_df, g.hierarchical == CP_SEARCH_COARSE_FINE ? p->kc : 0, lo, hi, r);
        p->excl_coarse.insert(p->excl_coarse.end(), r, r + 2);
    }

    // curve sizes
    if (offsets[0] != 0) return fail(CP_EINVAL, "cp_plan: offsets[0] must be 0");
    p->offsets.assign(offsets, offsets + n_curves + 1);
    p->n_curves = n_curves;
    p->fc.resize(n_curves);
    int max_n = 0;
    for (int64_t c = 0; c < n_curves; c++) {
        const int64_t n = offsets[c + 1] - offsets[c];
        if (n < 2) return fail(CP_EINVAL, "cp_plan: curve " + std::to_string(c) + " has fewer than 2 samples");
        if (n > kMaxN)
            return fail(CP_EUNSUPPORTED, "cp_plan: curve " + std::to_string(c) + " has " + std::to_string(n) +
                                             " samples; the maximum is " + std::to_string(kMaxN));
        max_n = std::max(max_n, (int)n);
        const int tb = tune_bucket(tune, (int)n);
        p->fc[c] = fc_for((int)n, tb >= 0 ? tune.direct_fc[tb] : kFcMax);
    }
    p->max_band_points = (max_n + 9) / 10;   // a band holds at most ceil(N/10) samples
    p->n_points = offsets[n_curves];
    p->max_n = max_n;
    while (p->np2max < max_n) p->np2max <<= 1;
    p->grid = g;
    p->grid.exclude = nullptr;   // copied above; the caller's array is not kept
    p->opt = opt;
    p->times = times;
    p->mags = mags;
    p->errs = errs;
    p->host_inputs = opt.input_memory == CP_MEM_HOST;

    // device, stream
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1)
        return fail(CP_ECUDA, "cp_plan: no CUDA device available");
    if (opt.device < 0 || opt.device >= ndev) return fail(CP_EINVAL, "cp_plan: bad device ordinal");
    p->device = opt.device;
    CP_CUDA(cudaSetDevice(p->device));
    CP_CUDA(cudaDeviceGetAttribute(&p->n_sm, cudaDevAttrMultiProcessorCount, p->device));
    p->stream = (cudaStream_t)stream;
    CP_CUDA(cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking));

    // pointer kinds
    auto kind = [](const void* ptr) {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
            cudaGetLastError();
            return cudaMemoryTypeUnregistered;
        }
        return at.type;
    };
    if (p->host_inputs) {
        const bool pt = kind(times) == cudaMemoryTypeHost, pm = kind(mags) == cudaMemoryTypeHost,
                   pe = kind(errs) == cudaMemoryTypeHost;
        p->host_pinned = pt && pm && pe;
    } else {
        for (const void* q : {(const void*)times, (const void*)mags, (const void*)errs}) {
            const cudaMemoryType k = kind(q);
            if (k != cudaMemoryTypeDevice && k != cudaMemoryTypeManaged)
                return fail(CP_EINVAL, "cp_plan: input_memory is CP_MEM_DEVICE but an input is not device memory");
        }
    }

    // per-curve evaluation class: 0 = direct form, else tensor form with cls harmonics
    p->cls.assign(n_curves, 0);
    if (p->tensor) {
        if (opt.n_max != 0) {
            std::fill(p->cls.begin(), p->cls.end(), opt.n_max);
        } else {
            std::vector<float> st((size_t)n_curves);
            cp_status s2 = plan_sigma_t(p, opt, st);
            if (s2 != CP_OK) return s2;
            for (int64_t c = 0; c < n_curves; c++) {
                int cl = harmonics_for(st[c]);
                if (cl == 12 && opt.dtype == CP_DTYPE_BF16_SPLIT) cl = 16;   // no 12-harmonic split-Z class
                if (cl == 48 && opt.dtype == CP_DTYPE_BF16_SPLIT) cl = 0;    // nor a 48-harmonic one
                const int tb = tune_bucket(tune, (int)(offsets[c + 1] - offsets[c]));
                const int bit = cl == 8 ? 1 : cl == 16 ? 2 : cl == 32 ? 4 : cl == 12 ? 8 : cl == 48 ? 16 : 0;
                if (tb >= 0 && bit && !(tune.tensor_classes[tb] & bit)) cl = 0;   // tuned: direct form is faster here
                p->cls[c] = cl;
            }
        }
    }
    for (int64_t c = 0; c < n_curves; c++) p->class_count[class_rank(p->cls[c])]++;

    // schedule: slots grouped by class, N descending within a class (stable)
    p->order.resize(n_curves);
    std::iota(p->order.begin(), p->order.end(), 0);
    std::stable_sort(p->order.begin(), p->order.end(), [&](int32_t a, int32_t b) {
        const int ra = class_rank(p->cls[a]), rb = class_rank(p->cls[b]);
        if (ra != rb) return ra < rb;
        return (offsets[a + 1] - offsets[a]) > (offsets[b + 1] - offsets[b]);
    });
    p->unit_full.assign(n_curves + 1, 0);
    p->unit_coarse.assign(n_curves + 1, 0);
    p->unit_fine.assign(n_curves + 1, 0);
    p->unit_list.assign(n_curves + 1, 0);
    p->wtile.assign(n_curves + 1, 0);
    double pf_full = 0, pf_search = 0;
    size_t smem = 0;
    for (int64_t s = 0; s < n_curves; s++) {
        const int c = p->order[s];
        const int n = (int)(offsets[c + 1] - offsets[c]);
        const int f = p->cls[c] ? tensor_freqs_per_unit(p->cls[c], opt.dtype == CP_DTYPE_BF16_SPLIT) : p->fc[c];
        const double pairs = 0.5 * (double)n * (double)(n - 1);
        p->unit_full[s + 1] = p->unit_full[s] + (g.n_freq + f - 1) / f;
        p->unit_list[s + 1] = p->unit_list[s] + (p->n_trials + f - 1) / f;
        if (p->bands) {
            pf_search += pairs * (double)p->n_trials;
            p->window_terms += (double)n * (double)g.n_freq * (double)g.n_bands / 10.0;
        } else if (g.hierarchical) {
            p->unit_coarse[s + 1] = p->unit_coarse[s] + (p->kc + f - 1) / f;
            p->unit_fine[s + 1] = p->unit_fine[s] + (int64_t)g.top_k * ((2 * p->J + 1 + f - 1) / f);
            pf_search += pairs * (double)(p->kc + (int64_t)g.top_k * (2 * p->J + 1));
        } else {
            pf_search += pairs * (double)g.n_freq;
        }
        pf_full += pairs * (double)g.n_freq;
        {
            const double kk = p->bands ? (double)p->n_trials
                              : g.hierarchical ? (double)(p->kc + (int64_t)g.top_k * (2 * p->J + 1))
                                               : (double)g.n_freq;
            if (p->cls[c]) p->tensor_flops += 2.0 * (double)n * (double)n * (double)p->cls[c] * kk;
            else p->direct_pf += pairs * kk;
        }
        // tile counts in the unit of the curve's form (a wave never mixes forms)
        p->wtile[s + 1] = p->wtile[s] + (p->cls[c] ? tensor_tiles_of(n) : tiles_of(n));
        const size_t npad = (size_t)((n + kTile - 1) / kTile * kTile);
        if (!p->cls[c]) smem = std::max(smem, npad * (size_t)p->fc[c] * 12);   // direct-form trig table
    }
    p->pf_full = pf_full;
    p->pf_search = pf_search;
    p->pair_smem = std::max<size_t>(smem, 1024);

    // waves: contiguous slots of one class, bounded by the W buffer budget
    size_t free_b = 0, total_b = 0;
    CP_CUDA(cudaMemGetInfo(&free_b, &total_b));
    size_t budget = std::min<size_t>((size_t)8 << 30, free_b / 3);
    if (const char* env = std::getenv("CP_W_BUDGET_KB")) budget = (size_t)std::atoll(env) << 10;
    const size_t tile16_bytes = tensor_tile_bytes(w_bf16(opt.dtype)), tile32_bytes = kTileFloats * sizeof(float);
    int64_t max_tiles32 = 0, max_tiles16 = 0;
    {
        auto close_wave = [&](int sb, int se) {
            const int cl = p->cls[p->order[sb]];
            const int64_t nt = p->wtile[se] - p->wtile[sb];
            p->waves.push_back({sb, se, p->wtile[sb], p->wtile[se], cl});
            if (cl) max_tiles16 = std::max(max_tiles16, nt); else max_tiles32 = std::max(max_tiles32, nt);
        };
        int sb = 0;
        for (int s = 0; s < (int)n_curves; s++) {
            const int cl = p->cls[p->order[s]];
            const int64_t tile_budget =
                std::max<int64_t>(1, (int64_t)(budget / (cl ? tile16_bytes : tile32_bytes)));
            const bool new_class = s > sb && cl != p->cls[p->order[sb]];
            const bool over = s > sb && p->wtile[s + 1] - p->wtile[sb] > tile_budget;
            if (new_class || over) {
                close_wave(sb, s);
                sb = s;
            }
        }
        close_wave(sb, (int)n_curves);
    }

    // device allocation (one block)
    const int64_t np = p->n_points, nc = n_curves;
    const int nq = kQueuesPerWave * (int)p->waves.size();
    p->n_u64 = 1 + nc + nq;
    struct Part { void** dst; size_t bytes; };
    const bool hier = g.hierarchical == CP_SEARCH_COARSE_FINE;
    const bool bnd = p->bands;
    std::vector<Part> parts = {
        {(void**)&p->d_times, p->host_inputs ? np * sizeof(double) : 0},
        {(void**)&p->d_mags, p->host_inputs ? np * sizeof(float) : 0},
        {(void**)&p->d_errs, p->host_inputs ? np * sizeof(float) : 0},
        {(void**)&p->d_cp, nc * sizeof(CurveParams)},
        {(void**)&p->d_yp, np * sizeof(float)},
        {(void**)&p->d_ph_base, np * sizeof(uint64_t)},
        {(void**)&p->d_ph_full, np * sizeof(uint64_t)},
        {(void**)&p->d_ph_coarse, hier ? np * sizeof(uint64_t) : 0},
        {(void**)&p->d_ph_fine, hier ? np * sizeof(uint64_t) : 0},
        {(void**)&p->d_stpc, opt.sigma_t_mode == CP_SIGMA_T_PER_CURVE ? nc * sizeof(float) : 0},
        {(void**)&p->d_order, nc * sizeof(int32_t)},
        {(void**)&p->d_unit_full, (nc + 1) * sizeof(int64_t)},
        {(void**)&p->d_unit_coarse, (nc + 1) * sizeof(int64_t)},
        {(void**)&p->d_unit_fine, (nc + 1) * sizeof(int64_t)},
        {(void**)&p->d_wtile, (nc + 1) * sizeof(int64_t)},
        {(void**)&p->d_unit_list, bnd ? (nc + 1) * sizeof(int64_t) : 0},
        {(void**)&p->d_band_of, bnd ? (size_t)np : 0},
        {(void**)&p->d_kept, bnd ? (size_t)nc * g.n_bands * sizeof(int32_t) : 0},
        {(void**)&p->d_trials, bnd ? (size_t)nc * p->n_trials * sizeof(int32_t) : 0},
        {(void**)&p->d_wcand, bnd ? (size_t)nc * 2 * p->n_trials * sizeof(unsigned long long) : 0},
        {(void**)&p->d_trial_stat, bnd ? (size_t)nc * p->n_trials * sizeof(float) : 0},
        {(void**)&p->d_excl_f, p->excl_f.size() * sizeof(double)},
        {(void**)&p->d_excl_full, p->excl_full.size() * sizeof(int32_t)},
        {(void**)&p->d_excl_coarse, p->excl_coarse.size() * sizeof(int32_t)},
        {(void**)&p->d_W, (size_t)max_tiles32 * tile32_bytes},
        {(void**)&p->d_W16, (size_t)max_tiles16 * tile16_bytes},
        {(void**)&p->d_coef, p->tensor ? (size_t)nc * kCoefStride * sizeof(float) : 0},
        {(void**)&p->d_wrho, p->tensor ? np * sizeof(float) : 0},
        {(void**)&p->d_coarse, hier ? (size_t)nc * p->kc * sizeof(float) : 0},
        {(void**)&p->d_peaks, hier ? (size_t)nc * g.top_k * sizeof(int32_t) : 0},
        {(void**)&p->d_npeaks, hier ? nc * sizeof(int32_t) : 0},
        {(void**)&p->d_u64, (size_t)p->n_u64 * sizeof(unsigned long long)},
        {(void**)&p->d_res_idx, nc * sizeof(int64_t)},
        {(void**)&p->d_res_freq, nc * sizeof(double)},
        {(void**)&p->d_res_stat, nc * sizeof(float)},
        {(void**)&p->d_res_per, (size_t)nc},
        {(void**)&p->d_res_psnr, nc * sizeof(float)},
    };
    size_t total = 0;
    for (auto& q : parts) total = align_up(total, 256) + q.bytes;
    AllocHook alloc;
    CP_CUDA(alloc.device(&p->dblock, std::max<size_t>(total, 256)));
    {
        size_t o = 0;
        for (auto& q : parts) {
            o = align_up(o, 256);
            *q.dst = q.bytes ? (void*)((char*)p->dblock + o) : nullptr;
            o += q.bytes;
        }
    }
    // pinned host block
    std::vector<Part> hparts = {
        {(void**)&p->h_res_idx, nc * sizeof(int64_t)},
        {(void**)&p->h_res_freq, nc * sizeof(double)},
        {(void**)&p->h_res_stat, nc * sizeof(float)},
        {(void**)&p->h_res_per, (size_t)nc},
        {(void**)&p->h_res_psnr, nc * sizeof(float)},
        {(void**)&p->h_status, sizeof(unsigned long long)},
        {(void**)&p->h_times, p->host_inputs && !p->host_pinned ? np * sizeof(double) : 0},
        {(void**)&p->h_mags, p->host_inputs && !p->host_pinned ? np * sizeof(float) : 0},
        {(void**)&p->h_errs, p->host_inputs && !p->host_pinned ? np * sizeof(float) : 0},
    };
    size_t htotal = 0;
    for (auto& q : hparts) htotal = align_up(htotal, 64) + q.bytes;
    CP_CUDA(alloc.pinned(&p->hblock, std::max<size_t>(htotal, 64)));
    {
        size_t o = 0;
        for (auto& q : hparts) {
            o = align_up(o, 64);
            *q.dst = q.bytes ? (void*)((char*)p->hblock + o) : nullptr;
            o += q.bytes;
        }
    }

    // per-curve constants and schedule tables
    std::vector<CurveParams> cps(nc);
    for (int64_t c = 0; c < nc; c++) {
        std::memset(&cps[c], 0, sizeof(CurveParams));
        cps[c].off = offsets[c];
        cps[c].n = (int32_t)(offsets[c + 1] - offsets[c]);
        cps[c].fc = p->fc[c];
        // per-curve classes follow sigma_t: a later sigma_t below the class's floor re-plans
        cps[c].st_floor = (p->tensor && opt.n_max == 0) ? sigma_t_floor(p->cls[c]) : 0.f;
    }
    CP_CUDA(cudaMemcpy(p->d_cp, cps.data(), nc * sizeof(CurveParams), cudaMemcpyHostToDevice));
    CP_CUDA(cudaMemcpy(p->d_order, p->order.data(), nc * sizeof(int32_t), cudaMemcpyHostToDevice));
    CP_CUDA(cudaMemcpy(p->d_unit_full, p->unit_full.data(), (nc + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
    CP_CUDA(cudaMemcpy(p->d_unit_coarse, p->unit_coarse.data(), (nc + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
    CP_CUDA(cudaMemcpy(p->d_unit_fine, p->unit_fine.data(), (nc + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
    CP_CUDA(cudaMemcpy(p->d_wtile, p->wtile.data(), (nc + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
    if (bnd)
        CP_CUDA(cudaMemcpy(p->d_unit_list, p->unit_list.data(), (nc + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
    if (!p->excl_f.empty()) {
        CP_CUDA(cudaMemcpy(p->d_excl_f, p->excl_f.data(), p->excl_f.size() * sizeof(double), cudaMemcpyHostToDevice));
        CP_CUDA(cudaMemcpy(p->d_excl_full, p->excl_full.data(), p->excl_full.size() * sizeof(int32_t),
                           cudaMemcpyHostToDevice));
        CP_CUDA(cudaMemcpy(p->d_excl_coarse, p->excl_coarse.data(), p->excl_coarse.size() * sizeof(int32_t),
                           cudaMemcpyHostToDevice));
    }
    if (opt.sigma_t_mode == CP_SIGMA_T_PER_CURVE) {
        for (int64_t c = 0; c < nc; c++)
            if (!(opt.sigma_t_per_curve[c] > 0.f && std::isfinite(opt.sigma_t_per_curve[c])))
                return fail(CP_EINVAL, "cp_plan: sigma_t_per_curve values must be finite and > 0");
        CP_CUDA(cudaMemcpy(p->d_stpc, opt.sigma_t_per_curve, nc * sizeof(float), cudaMemcpyHostToDevice));
    }
    p->opt.sigma_t_per_curve = nullptr;

    // launch geometry of the persistent pair kernel
    CP_CUDA(prepare_kernels(p->np2max, p->pair_smem));
    if (bnd) {
        int optin = 0;
        CP_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device));
        if (window_smem_bytes(p->max_band_points, g.trials_per_band) + 4096 > (size_t)optin ||
            refine_smem_bytes(p->max_band_points, g.trials_per_band) > (size_t)optin)
            return fail(CP_EUNSUPPORTED, "cp_plan: spectral-window buffers do not fit in shared memory");
        CP_CUDA(prepare_bands_kernels(p->np2max, p->max_band_points, g.trials_per_band));
    }
    for (int nm : {4, 8, 12, 16, 32, 48})
        if (p->class_count[class_rank(nm)]) CP_CUDA(prepare_tensor_kernel(nm));   // one CTA per SM
    {
        int occ = 1;
        CP_CUDA(pair_direct_occupancy(&occ, p->pair_smem));
        p->pair_grid = p->n_sm * std::max(occ, 1);
    }

    // events
    const int pair_launches = (int)p->waves.size() * (hier ? 2 : 1);
    p->ev_pair.resize(2 * pair_launches);
    p->ev_cls.assign(pair_launches, 0);
    for (auto& e : p->ev_pair) CP_CUDA(cudaEventCreate(&e));
    CP_CUDA(cudaEventCreate(&p->ev_step0));
    CP_CUDA(cudaEventCreate(&p->ev_step1));
    if (bnd) {
        CP_CUDA(cudaEventCreate(&p->ev_bands0));
        CP_CUDA(cudaEventCreate(&p->ev_bands1));
    }
    p->launches_per_search =
        2 /* zero, stats */ + (p->tensor ? 1 : 0) /* harmonic coefficients */ + (bnd ? 2 : 0) /* bands, window */ +
        (int64_t)p->waves.size() * (hier ? 4 : 2) + 1 /* finalize */;
    return CP_OK;
}

cp_status cp_plan(const double* times, const float* mags, const float* errs, const int64_t* offsets,
                  int64_t n_curves, const cp_freq_grid* grid, const cp_options* opt, void* stream,
                  cp_plan_t* out_plan)
{
    if (!out_plan) return fail(CP_EINVAL, "cp_plan: out_plan is NULL");
    *out_plan = nullptr;
    cp_plan_s* p = new (std::nothrow) cp_plan_s();
    if (!p) return fail(CP_ENOMEM, "cp_plan: host allocation failed");
    int prev = 0;
    cudaGetDevice(&prev);
    cp_status st = plan_impl(times, mags, errs, offsets, n_curves, grid, opt, stream, p);
    cudaSetDevice(prev);
    if (st != CP_OK) {
        char msg[512];
        std::strncpy(msg, cpk::last_error_buffer(), sizeof(msg) - 1);
        msg[sizeof(msg) - 1] = 0;
        cp_destroy(p);
        cpk::set_error(st, msg);
        return st;
    }
    *out_plan = p;
    return finish(CP_OK, "cp_plan");
}

// A call found a curve whose sigma_t (skewness rule on the current
// magnitudes) lies below the floor of its planned harmonic class: the plan is
// rebuilt on the device-computed sigma_t of the same inputs (schedule, buffers,
// graph), and the caller repeats the call.
static cp_status replan(cp_plan_t p)
{
    cp_plan_s* q = new (std::nothrow) cp_plan_s();
    if (!q) return fail(CP_ENOMEM, "re-plan: host allocation failed");
    cp_options o = p->opt;
    o.tuning = p->has_tune ? &p->tune : nullptr;
    cp_freq_grid g = p->grid;
    g.exclude = p->excl_f.empty() ? nullptr : p->excl_f.data();
    const std::vector<int64_t> off = p->offsets;
    int prev = 0;
    cudaGetDevice(&prev);
    cp_status st = plan_impl(p->times, p->mags, p->errs, off.data(), p->n_curves, &g, &o, p->stream, q);
    cudaSetDevice(prev);
    if (st != CP_OK) {
        char msg[512];
        std::strncpy(msg, cpk::last_error_buffer(), sizeof(msg) - 1);
        msg[sizeof(msg) - 1] = 0;
        cp_destroy(q);
        return cpk::set_error(st, msg);
    }
    q->replans = p->replans + 1;
    q->last_out = p->last_out;
    std::swap(*p, *q);
    cp_destroy(q);   // the previous plan's resources
    return CP_OK;
}

static cp_status periodogram_impl(cp_plan_t p, float* out)
{
    if (!p) return fail(CP_EINVAL, "cp_periodogram: NULL plan");
    int prev = 0;
    cudaGetDevice(&prev);
    CP_CUDA(cudaSetDevice(p->device));
    cp_status st = CP_OK;
    // the pinned staging copy must not overwrite data a previous call still reads
    if (p->host_inputs && !p->host_pinned) CP_CUDA(cudaStreamSynchronize(p->stream));
    stage_host_inputs(p);
    if ((st = enqueue_inputs(p, p->stream)) == CP_OK && (st = enqueue_stats(p, p->stream)) == CP_OK) {
        for (int w = 0; w < (int)p->waves.size() && st == CP_OK; w++) {
            st = enqueue_wave_w(p, w, p->stream);
            if (st == CP_OK) st = enqueue_pair(p, kStageFull, w, out, p->stream, nullptr);
        }
    }
    if (st == CP_OK)
        CP_CUDA(cudaMemcpyAsync(p->h_status, p->d_u64, sizeof(unsigned long long), cudaMemcpyDeviceToHost, p->stream));
    p->ran = true;
    p->last_out = out;
    cudaSetDevice(prev);
    return st;
}

static cp_status sync_impl(cp_plan_t p)
{
    if (!p) return fail(CP_EINVAL, "cp_sync: NULL plan");
    CP_CUDA(cudaSetDevice(p->device));
    CP_CUDA(cudaStreamSynchronize(p->stream));
    if (p->ran && (*p->h_status & 4) && !(*p->h_status & 3)) {
        // the last periodogram used a harmonic count too small for a curve's new sigma_t
        cp_status st = replan(p);
        if (st == CP_OK) st = periodogram_impl(p, p->last_out);
        if (st != CP_OK) return st;
        CP_CUDA(cudaStreamSynchronize(p->stream));
    }
    if (p->ran && (*p->h_status & 2))
        return fail(CP_ETIMEOUT, "a bounded device wait of the tensor-core kernel gave up");
    if (p->ran && (*p->h_status & 1))
        return fail(CP_EINVAL, "input contains a non-finite value, a zero median error bar or a bad sigma_t");
    return CP_OK;
}

static cp_status search_once(cp_plan_t p, int64_t* best_idx, double* best_freq, float* best_stat,
                             uint8_t* is_periodic, float* psnr);

static cp_status best_period_impl(cp_plan_t p, int64_t* best_idx, double* best_freq, float* best_stat,
                                  uint8_t* is_periodic, float* psnr)
{
    cp_status st = search_once(p, best_idx, best_freq, best_stat, is_periodic, psnr);
    // a curve's sigma_t left the range its planned harmonic count covers: re-plan
    // on the device-computed sigma_t and search again (the inputs are unchanged,
    // so the new plan's classes cover every curve)
    if (st == CP_OK && p && (*p->h_status & 4)) {
        if ((st = replan(p)) == CP_OK) st = search_once(p, best_idx, best_freq, best_stat, is_periodic, psnr);
        if (st == CP_OK && (*p->h_status & 4))
            return fail(CP_ESTATE, "cp_best_period: the magnitudes changed during the call");
    }
    return st;
}

static cp_status search_once(cp_plan_t p, int64_t* best_idx, double* best_freq, float* best_stat,
                             uint8_t* is_periodic, float* psnr)
{
    if (!p) return fail(CP_EINVAL, "cp_best_period: NULL plan");
    int prev = 0;
    cudaGetDevice(&prev);
    CP_CUDA(cudaSetDevice(p->device));
    cp_status st = CP_OK;
    // the pinned staging copy must not overwrite data a previous call still reads
    if (p->host_inputs && !p->host_pinned) CP_CUDA(cudaStreamSynchronize(p->stream));
    stage_host_inputs(p);
    if (p->opt.use_graph) {
        if (!p->graph_ready) st = build_graph(p);
        if (st == CP_OK) CP_CUDA(cudaGraphLaunch(p->exec, p->stream));
    } else {
        st = enqueue_search(p, p->stream);
    }
    if (st != CP_OK) {
        cudaSetDevice(prev);
        return st;
    }
    CP_CUDA(cudaStreamSynchronize(p->stream));
    p->ran = true;
    p->searched = true;
    if ((st = read_timings(p)) != CP_OK) {
        cudaSetDevice(prev);
        return st;
    }
    const size_t nc = (size_t)p->n_curves;
    if (best_idx) std::memcpy(best_idx, p->h_res_idx, nc * sizeof(int64_t));
    if (best_freq) std::memcpy(best_freq, p->h_res_freq, nc * sizeof(double));
    if (best_stat) std::memcpy(best_stat, p->h_res_stat, nc * sizeof(float));
    if (is_periodic) std::memcpy(is_periodic, p->h_res_per, nc);
    if (psnr) std::memcpy(psnr, p->h_res_psnr, nc * sizeof(float));
    cudaSetDevice(prev);
    if (*p->h_status & 2) return fail(CP_ETIMEOUT, "a bounded device wait of the tensor-core kernel gave up");
    if (*p->h_status & 1)
        return fail(CP_EINVAL, "input contains a non-finite value, a zero median error bar or a bad sigma_t");
    return CP_OK;
}

static cp_status curve_stats_impl(cp_plan_t p, float* sigma_y, float* sigma_t, double* ip, float* psnr)
{
    if (!p) return fail(CP_EINVAL, "cp_curve_stats: NULL plan");
    if (!p->ran) return fail(CP_ESTATE, "cp_curve_stats: no call has run on this plan yet");
    CP_CUDA(cudaSetDevice(p->device));
    CP_CUDA(cudaStreamSynchronize(p->stream));
    std::vector<CurveParams> cps((size_t)p->n_curves);
    CP_CUDA(cudaMemcpy(cps.data(), p->d_cp, cps.size() * sizeof(CurveParams), cudaMemcpyDeviceToHost));
    for (size_t c = 0; c < cps.size(); c++) {
        if (sigma_y) sigma_y[c] = cps[c].sigma_y;
        if (sigma_t) sigma_t[c] = cps[c].sigma_t;
        if (ip) ip[c] = cps[c].ip / (std::sqrt(2.0 * M_PI) * (double)cps[c].sigma_y);
        if (psnr) psnr[c] = cps[c].psnr;
    }
    return CP_OK;
}

static cp_status trials_impl(cp_plan_t p, int32_t* trial_idx, float* trial_stat)
{
    if (!p) return fail(CP_EINVAL, "cp_trial_frequencies: NULL plan");
    if (!p->bands) return fail(CP_ESTATE, "cp_trial_frequencies: the plan does not use the bands method");
    if (!p->searched) return fail(CP_ESTATE, "cp_trial_frequencies: no best-period search has run on this plan");
    int prev = 0;
    cudaGetDevice(&prev);
    CP_CUDA(cudaSetDevice(p->device));
    CP_CUDA(cudaStreamSynchronize(p->stream));
    const size_t cnt = (size_t)p->n_curves * (size_t)p->n_trials;
    if (trial_idx) CP_CUDA(cudaMemcpy(trial_idx, p->d_trials, cnt * sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (trial_stat) CP_CUDA(cudaMemcpy(trial_stat, p->d_trial_stat, cnt * sizeof(float), cudaMemcpyDeviceToHost));
    cudaSetDevice(prev);
    return CP_OK;
}

cp_status cp_trial_frequencies(cp_plan_t p, int32_t* trial_idx, float* trial_stat)
{
    return finish(trials_impl(p, trial_idx, trial_stat), "cp_trial_frequencies");
}

cp_status cp_periodogram(cp_plan_t p, float* out) { return finish(periodogram_impl(p, out), "cp_periodogram"); }

cp_status cp_sync(cp_plan_t p) { return finish(sync_impl(p), "cp_sync"); }

cp_status cp_best_period(cp_plan_t p, int64_t* best_idx, double* best_freq, float* best_stat,
                         uint8_t* is_periodic, float* psnr)
{
    return finish(best_period_impl(p, best_idx, best_freq, best_stat, is_periodic, psnr), "cp_best_period");
}

cp_status cp_curve_stats(cp_plan_t p, float* sigma_y, float* sigma_t, double* ip, float* psnr)
{
    return finish(curve_stats_impl(p, sigma_y, sigma_t, ip, psnr), "cp_curve_stats");
}

cp_status cp_get_plan_info(cp_plan_t p, cp_plan_info* info)
{
    if (!p || !info) return fail(CP_EINVAL, "cp_get_plan_info: NULL argument");
    info->n_curves = p->n_curves;
    info->n_points = p->n_points;
    info->pair_freq_full = p->pf_full;
    info->pair_freq_search = p->pf_search;
    info->launches_per_search = p->launches_per_search;
    info->last_pair_kernel_ms = p->last_pair_ms;
    info->last_step_ms = p->last_step_ms;
    info->n_sm = p->n_sm;
    info->max_n = p->max_n;
    for (int k = 0; k < 7; k++) info->class_curves[k] = p->class_count[k];
    info->last_tensor_kernel_ms = p->last_tensor_ms;
    info->last_direct_kernel_ms = p->last_direct_ms;
    info->tensor_flops_search = p->tensor_flops;
    info->direct_pair_freq_search = p->direct_pf;
    info->last_bands_kernel_ms = p->last_bands_ms;
    info->reserved0 = 0.f;
    info->window_terms_search = p->window_terms;
    double wd = 0, wt = 0;
    for (const Wave& w : p->waves)
        (w.cls ? wt : wd) += (double)(w.tile_end - w.tile_begin) *
                             (w.cls ? (double)tensor_tile_bytes(w_bf16(p->opt.dtype)) : (double)kTileFloats * 4);
    info->w_bytes_direct = wd;
    info->w_bytes_tensor = wt;
    info->replans = p->replans;
    info->bands_exact_scans = p->bands ? (int64_t)(*p->h_status >> 32) : 0;
    return CP_OK;
}

cp_status cp_bessel_coefficients(double sigma_t, int32_t n_max, double* out)
{
    if (!out || n_max < 0 || n_max > 100000 || !(sigma_t > 0.0) || !std::isfinite(sigma_t))
        return fail(CP_EINVAL, "cp_bessel_coefficients: bad argument");
    const double kappa = 1.0 / (sigma_t * sigma_t);
    // trapezoid rule on [0, pi] for the even periodic integrand (exponentially convergent)
    const int M = std::max(2048, 8 * (int)(kappa + n_max) + 64);
    for (int n = 0; n <= n_max; n++) {
        double acc = 0.0;
        for (int k = 0; k <= M; k++) {
            const double th = M_PI * (double)k / (double)M;
            const double wgt = (k == 0 || k == M) ? 0.5 : 1.0;
            acc += wgt * std::exp(kappa * (std::cos(th) - 1.0)) * std::cos((double)n * th);
        }
        acc /= (double)M;                 // (1/pi) * (pi/M) * sum
        out[n] = (n == 0) ? acc : 2.0 * acc;
    }
    return CP_OK;
}

}  // extern "C"
