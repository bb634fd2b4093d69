// cp_noalloc.cu -- best-period search that allocates no memory.
//
// Some callers cannot allocate device memory when they want a result: a host
// application that reserves all device memory at start-up for its own pool,
// a latency-bounded pipeline that must not enter the allocator, or a plug-in
// whose host owns the device allocator.  cp_best_period_noalloc serves them.
// It runs the same kernels as cp_best_period (direct form), but every buffer
// the search needs beyond the caller's inputs and outputs lives in one
// file-scope static device array, g_noalloc_scratch, of
// CP_NOALLOC_SCRATCH_BYTES.  Each GPU that loads the library holds that array
// until the process exits.  No cudaMalloc, cudaFree or allocating library
// routine is called on this path.
#include <cmath>
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "cp.h"
#include "cp_internal.cuh"

using namespace cpk;

namespace {

constexpr size_t kScratchBytes = (size_t)CP_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxCurves = CP_NOALLOC_MAX_CURVES;
constexpr int kMaxDevices = 64;

// The scratch array.  In host code this name is only a host-side stand-in:
// its device address comes from cudaGetSymbolAddress (see scratch_base).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

cp_status nfail(cp_status s, const char* msg) { return set_error(s, msg); }

#define NA_CUDA(call)                                                 \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) {                                      \
            cudaGetLastError();                                       \
            return nfail(CP_ECUDA, #call " failed");                  \
        }                                                             \
    } while (0)

// Device address of the scratch array on the current device, looked up once
// per device with that device current.
cp_status scratch_base(int dev, void** out)
{
    if (dev < 0 || dev >= kMaxDevices) return nfail(CP_EINVAL, "cp_best_period_noalloc: device ordinal too large");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return nfail(CP_ECUDA, "cp_best_period_noalloc: cudaGetSymbolAddress of the scratch array failed");
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return CP_OK;
}

// Waits for the stream when a call fails after it has queued work: the
// kernels already in flight write to the shared scratch array, and a retry
// (or the next call, on any stream) must not start while they run.
struct SyncOnError {
    cudaStream_t s;
    bool armed;
    ~SyncOnError()
    {
        if (armed) {
            cudaStreamSynchronize(s);
            cudaGetLastError();
        }
    }
};

struct Carve {
    char* base;
    size_t used;
    template <typename T>
    T* take(size_t count)
    {
        used = (used + 255) & ~(size_t)255;
        T* p = reinterpret_cast<T*>(base + used);
        used += count * sizeof(T);
        return p;
    }
};

}  // namespace

extern "C" cp_status cp_best_period_noalloc(const double* times, const float* mags, const float* errs,
                                            const int64_t* offsets, int64_t n_curves, const cp_freq_grid* grid,
                                            float sigma_t, void* cuda_stream, int64_t* best_idx,
                                            double* best_freq, float* best_stat, uint8_t* is_periodic)
{
    if (!times || !mags || !errs || !offsets || !grid)
        return nfail(CP_EINVAL, "cp_best_period_noalloc: null argument");
    if (n_curves < 1 || n_curves > kMaxCurves)
        return nfail(CP_EUNSUPPORTED, "cp_best_period_noalloc: n_curves must be in [1, CP_NOALLOC_MAX_CURVES]");
    if (!(sigma_t > 0.f) || !std::isfinite(sigma_t)) return nfail(CP_EINVAL, "cp_best_period_noalloc: bad sigma_t");
    const cp_freq_grid g = *grid;
    if (!(g.f_min >= 0.0 && std::isfinite(g.f_min) && g.df > 0.0 && std::isfinite(g.df)) || g.n_freq < 1 ||
        g.n_freq > ((int64_t)1 << 31) - 1)
        return nfail(CP_EINVAL, "cp_best_period_noalloc: bad frequency grid");
    const double f_max = g.f_min + (double)(g.n_freq - 1) * g.df;
    int64_t kc = 0;
    int J = 0;
    if (g.hierarchical == CP_SEARCH_BANDS)
        return nfail(CP_EUNSUPPORTED, "cp_best_period_noalloc: the bands method needs a plan (cp_plan)");
    if (g.n_exclude != 0)
        return nfail(CP_EUNSUPPORTED, "cp_best_period_noalloc: exclusion windows need a plan (cp_plan)");
    if (g.hierarchical != CP_SEARCH_FULL && g.hierarchical != CP_SEARCH_COARSE_FINE)
        return nfail(CP_EINVAL, "cp_best_period_noalloc: bad search mode");
    if (g.hierarchical) {
        if (!(g.coarse_df > 0.0 && std::isfinite(g.coarse_df) && g.fine_df > 0.0 && std::isfinite(g.fine_df) &&
              g.fine_halfwidth >= 0.0 && std::isfinite(g.fine_halfwidth)) ||
            g.top_k < 1 || g.top_k > 1024)
            return nfail(CP_EINVAL, "cp_best_period_noalloc: bad hierarchical grid");
        // range checks on the doubles, before any conversion to an integer type
        const double kcd = std::floor((f_max - g.f_min) / g.coarse_df + 0.5) + 1.0;
        const double jd = std::floor(g.fine_halfwidth / g.fine_df + 0.5);
        if (!(jd <= 1e6) || (2.0 * jd + 1.0) * g.top_k > 2e9 || !(kcd <= (double)(((int64_t)1 << 31) - 1)))
            return nfail(CP_EINVAL, "cp_best_period_noalloc: hierarchical grid too large");
        kc = (int64_t)kcd;
        J = (int)jd;
    }
    if (offsets[0] != 0) return nfail(CP_EINVAL, "cp_best_period_noalloc: offsets[0] must be 0");
    // inputs and outputs must be device memory of the current device (a host
    // pointer or a short buffer would otherwise be read or written by the kernels)
    {
        int cur = 0;
        NA_CUDA(cudaGetDevice(&cur));
        const void* ins[3] = {times, mags, errs};
        const void* outs[4] = {best_idx, best_freq, best_stat, is_periodic};
        for (int k = 0; k < 7; k++) {
            const void* q = k < 3 ? ins[k] : outs[k - 3];
            if (k >= 3 && !q) continue;
            cudaPointerAttributes at{};
            if (cudaPointerGetAttributes(&at, q) != cudaSuccess) {
                cudaGetLastError();
                return nfail(CP_EINVAL, "cp_best_period_noalloc: an input or output is not device memory");
            }
            if ((at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) ||
                (at.type == cudaMemoryTypeDevice && at.device != cur))
                return nfail(CP_EINVAL,
                             "cp_best_period_noalloc: inputs and outputs must be device memory of the current device");
        }
    }

    // schedule on the stack: slots by N descending (stable), unit and tile prefix sums
    int32_t order[kMaxCurves];
    int64_t unit_full[kMaxCurves + 1], unit_coarse[kMaxCurves + 1], unit_fine[kMaxCurves + 1], wtile[kMaxCurves + 1];
    CurveParams cps[kMaxCurves];
    int max_n = 0;
    for (int c = 0; c < n_curves; c++) {
        const int64_t n = offsets[c + 1] - offsets[c];
        if (n < 2) return nfail(CP_EINVAL, "cp_best_period_noalloc: a curve has fewer than 2 samples");
        if (n > kMaxN) return nfail(CP_EUNSUPPORTED, "cp_best_period_noalloc: a curve exceeds cp_max_points()");
        max_n = n > max_n ? (int)n : max_n;
        int pos = c;   // insertion sort keeps equal sizes in input order
        while (pos > 0 && offsets[order[pos - 1] + 1] - offsets[order[pos - 1]] < n) {
            order[pos] = order[pos - 1];
            pos--;
        }
        order[pos] = c;
    }
    const int64_t n_points = offsets[n_curves];
    int np2max = 1;
    while (np2max < max_n) np2max <<= 1;
    unit_full[0] = unit_coarse[0] = unit_fine[0] = wtile[0] = 0;
    size_t pair_smem = 0;
    for (int s = 0; s < n_curves; s++) {
        const int c = order[s];
        const int n = (int)(offsets[c + 1] - offsets[c]);
        const int npad = (n + kTile - 1) / kTile * kTile;
        int fc = kFcMax;
        while (fc > 2 && (size_t)npad * fc * 12 > (size_t)kTableBytes) fc >>= 1;
        unit_full[s + 1] = unit_full[s] + (g.n_freq + fc - 1) / fc;
        unit_coarse[s + 1] = unit_coarse[s] + (g.hierarchical ? (kc + fc - 1) / fc : 0);
        unit_fine[s + 1] = unit_fine[s] + (g.hierarchical ? (int64_t)g.top_k * ((2 * J + 1 + fc - 1) / fc) : 0);
        wtile[s + 1] = wtile[s] + tiles_of(n);
        pair_smem = (size_t)npad * fc * 12 > pair_smem ? (size_t)npad * fc * 12 : pair_smem;
    }
    for (int c = 0; c < n_curves; c++) {
        std::memset(&cps[c], 0, sizeof(CurveParams));
        cps[c].off = offsets[c];
        cps[c].n = (int32_t)(offsets[c + 1] - offsets[c]);
        const int npad = (cps[c].n + kTile - 1) / kTile * kTile;
        int fc = kFcMax;
        while (fc > 2 && (size_t)npad * fc * 12 > (size_t)kTableBytes) fc >>= 1;
        cps[c].fc = fc;
    }

    int dev = 0;
    NA_CUDA(cudaGetDevice(&dev));
    void* base = nullptr;
    cp_status st = scratch_base(dev, &base);
    if (st != CP_OK) return st;

    // carve the scratch array (one wave: all W tiles must fit)
    Carve cv{static_cast<char*>(base), 0};
    const int nc = (int)n_curves;
    CurveParams* d_cp = cv.take<CurveParams>(nc);
    float* d_yp = cv.take<float>(n_points);
    uint64_t* d_ph_base = cv.take<uint64_t>(n_points);
    uint64_t* d_ph_full = cv.take<uint64_t>(n_points);
    uint64_t* d_ph_coarse = g.hierarchical ? cv.take<uint64_t>(n_points) : nullptr;
    uint64_t* d_ph_fine = g.hierarchical ? cv.take<uint64_t>(n_points) : nullptr;
    int32_t* d_order = cv.take<int32_t>(nc);
    int64_t* d_unit_full = cv.take<int64_t>(nc + 1);
    int64_t* d_unit_coarse = cv.take<int64_t>(nc + 1);
    int64_t* d_unit_fine = cv.take<int64_t>(nc + 1);
    int64_t* d_wtile = cv.take<int64_t>(nc + 1);
    float* d_W = cv.take<float>((size_t)wtile[nc] * kTileFloats);
    float* d_coarse = g.hierarchical ? cv.take<float>((size_t)nc * kc) : nullptr;
    int32_t* d_peaks = g.hierarchical ? cv.take<int32_t>((size_t)nc * g.top_k) : nullptr;
    int32_t* d_npeaks = g.hierarchical ? cv.take<int32_t>(nc) : nullptr;
    const int64_t n_u64 = 1 + nc + 3;
    unsigned long long* d_u64 = cv.take<unsigned long long>(n_u64);
    int64_t* d_idx = cv.take<int64_t>(nc);
    double* d_freq = cv.take<double>(nc);
    float* d_stat = cv.take<float>(nc);
    uint8_t* d_per = cv.take<uint8_t>(nc);
    float* d_psnr = cv.take<float>(nc);
    if (cv.used > kScratchBytes)
        return nfail(CP_EUNSUPPORTED, "cp_best_period_noalloc: batch needs more than CP_NOALLOC_SCRATCH_BYTES");

    cudaStream_t s = (cudaStream_t)cuda_stream;
    SyncOnError guard{s, true};
    NA_CUDA(cudaMemcpyAsync(d_cp, cps, nc * sizeof(CurveParams), cudaMemcpyHostToDevice, s));
    NA_CUDA(cudaMemcpyAsync(d_order, order, nc * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    NA_CUDA(cudaMemcpyAsync(d_unit_full, unit_full, (nc + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    NA_CUDA(cudaMemcpyAsync(d_unit_coarse, unit_coarse, (nc + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    NA_CUDA(cudaMemcpyAsync(d_unit_fine, unit_fine, (nc + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    NA_CUDA(cudaMemcpyAsync(d_wtile, wtile, (nc + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    NA_CUDA(launch_zero_u64(d_u64, n_u64, s));   // status, best keys and work counters start at zero

    StatsArgs sa{};
    sa.times = times;
    sa.mags = mags;
    sa.errs = errs;
    sa.cp = d_cp;
    sa.yp = d_yp;
    sa.ph_base = d_ph_base;
    sa.ph_full = d_ph_full;
    sa.ph_coarse = d_ph_coarse;
    sa.ph_fine = d_ph_fine;
    sa.f_min = g.f_min;
    sa.df = g.df;
    sa.coarse_df = g.coarse_df;
    sa.fine_df = g.fine_df;
    sa.hierarchical = g.hierarchical ? 1 : 0;
    sa.sigma_t_mode = CP_SIGMA_T_FIXED;
    sa.sigma_t = sigma_t;
    sa.alpha = 1.0f;
    sa.np2max = np2max;
    sa.status = reinterpret_cast<int*>(d_u64);
    NA_CUDA(prepare_kernels(np2max, pair_smem));
    NA_CUDA(launch_stats(sa, nc, s));

    BuildWArgs bw{};
    bw.cp = d_cp;
    bw.order = d_order;
    bw.wtile_start = d_wtile;
    bw.yp = d_yp;
    bw.W = d_W;
    bw.slot_begin = 0;
    bw.slot_end = nc;
    bw.tile_begin = 0;
    bw.tile_end = wtile[nc];
    NA_CUDA(launch_build_w(bw, s));

    int occ = 1, nsm = 1;
    NA_CUDA(pair_direct_occupancy(&occ, pair_smem));
    NA_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    PairArgs pa{};
    pa.cp = d_cp;
    pa.order = d_order;
    pa.wtile_start = d_wtile;
    pa.W = d_W;
    pa.yp = d_yp;
    pa.ph_base = d_ph_base;
    pa.ph_coarse = d_ph_coarse;
    pa.peaks = d_peaks;
    pa.n_peaks = d_npeaks;
    pa.slot_begin = 0;
    pa.slot_end = nc;
    pa.wtile_base = 0;
    pa.top_k = g.top_k;
    pa.fine_half = J;
    pa.f_min = g.f_min;
    pa.f_max = f_max;
    pa.coarse_df = g.coarse_df;
    pa.out = nullptr;
    pa.out_ld = g.n_freq;
    pa.coarse_out = d_coarse;
    pa.best_key = d_u64 + 1;
    if (!g.hierarchical) {
        pa.stage = kStageFull;
        pa.unit_start = d_unit_full;
        pa.ph_step = d_ph_full;
        pa.n_freq = g.n_freq;
        pa.step = g.df;
        pa.unit_begin = 0;
        pa.unit_end = unit_full[nc];
        pa.queue = d_u64 + 1 + nc;
        NA_CUDA(launch_pair_direct(pa, nsm * (occ > 0 ? occ : 1), pair_smem, s));
    } else {
        pa.stage = kStageCoarse;
        pa.unit_start = d_unit_coarse;
        pa.ph_step = d_ph_coarse;
        pa.n_freq = kc;
        pa.step = g.coarse_df;
        pa.unit_begin = 0;
        pa.unit_end = unit_coarse[nc];
        pa.queue = d_u64 + 1 + nc + 1;
        NA_CUDA(launch_pair_direct(pa, nsm * (occ > 0 ? occ : 1), pair_smem, s));
        TopkArgs ta{};
        ta.coarse = d_coarse;
        ta.order = d_order;
        ta.slot_begin = 0;
        ta.slot_end = nc;
        ta.n_freq = kc;
        ta.top_k = g.top_k;
        ta.peaks = d_peaks;
        ta.n_peaks = d_npeaks;
        NA_CUDA(launch_topk(ta, s));
        pa.stage = kStageFine;
        pa.unit_start = d_unit_fine;
        pa.ph_step = d_ph_fine;
        pa.step = g.fine_df;
        pa.unit_end = unit_fine[nc];
        pa.queue = d_u64 + 1 + nc + 2;
        NA_CUDA(launch_pair_direct(pa, nsm * (occ > 0 ? occ : 1), pair_smem, s));
    }
    FinalArgs fa{};
    fa.cp = d_cp;
    fa.best_key = d_u64 + 1;
    fa.peaks = d_peaks;
    fa.n_curves = nc;
    fa.hierarchical = g.hierarchical ? 1 : 0;
    fa.top_k = g.top_k;
    fa.fine_half = J;
    fa.f_min = g.f_min;
    fa.df = g.df;
    fa.coarse_df = g.coarse_df;
    fa.fine_df = g.fine_df;
    fa.best_idx = d_idx;
    fa.best_freq = d_freq;
    fa.best_stat = d_stat;
    fa.is_periodic = d_per;
    fa.psnr = d_psnr;
    NA_CUDA(launch_finalize(fa, s));
    if (best_idx) NA_CUDA(cudaMemcpyAsync(best_idx, d_idx, nc * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    if (best_freq) NA_CUDA(cudaMemcpyAsync(best_freq, d_freq, nc * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (best_stat) NA_CUDA(cudaMemcpyAsync(best_stat, d_stat, nc * sizeof(float), cudaMemcpyDeviceToDevice, s));
    if (is_periodic) NA_CUDA(cudaMemcpyAsync(is_periodic, d_per, nc, cudaMemcpyDeviceToDevice, s));
    unsigned long long status = 0;
    NA_CUDA(cudaMemcpyAsync(&status, d_u64, sizeof(status), cudaMemcpyDeviceToHost, s));
    NA_CUDA(cudaStreamSynchronize(s));
    guard.armed = false;
    if (status) return nfail(CP_EINVAL, "cp_best_period_noalloc: non-finite input, zero median error bar or bad sigma_t");
    return CP_OK;
}
