// cp_bands.cu -- trial-period extraction of arXiv:1412.1840, Section 3.1
// (the bands method), on the device.
//
//   k_bands   one CTA per curve: magnitude ranks (bitonic sort of
//             (magnitude, sample) keys), the ten equal-count bands, the FP64
//             sums D_b of |d_i|, d_i = (y_{i+1} - y_i) / (t_{i+1} - t_i), and
//             the bands in descending order of D (equal D: lower band first)
//   k_window  one CTA per (curve, kept band): the spectral window of
//             Eq. (bands), S(f_k) = |sum_{i in band} exp(i 2 pi f_k t_i)|^2,
//             on the uniform grid f_k = f_min + k df, held whole in shared
//             memory; then the n_t highest local maxima (one-day frequencies
//             left out) by a four-pass radix select on the value bits.
//
// Phases: exp(i 2 pi f_k t_i) with t_i - t0 (the window is invariant to a
// common time shift) from the exact 64-bit fixed-point phases
// base_i = frac(f_min (t_i - t0)) and step_i = frac(df (t_i - t0)) of the
// curve statistics pass: thread t evaluates k = k0 + t + 512 q (q < 16) by
// one sincos at k0 + t and fifteen FP32 rotations by exp(i 2 pi 512 step_i),
// whose angle is also taken exactly from 512 step_i mod 1.
#include <cstdint>
#include <cuda_runtime.h>

#include "cp_internal.cuh"

namespace cpk {

constexpr int kBandsThreads = 256;
constexpr int kWinThreads = 512;
constexpr int kWinRun = 16;                    // frequencies per thread per pass (stride kWinThreads)

// ===========================================================================
// k_bands
// ===========================================================================
__global__ void __launch_bounds__(kBandsThreads) k_bands(const BandsArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long* keys = reinterpret_cast<unsigned long long*>(smem);
    int8_t* bnd = reinterpret_cast<int8_t*>(keys + a.np2max);
    __shared__ double s_D[kBandsThreads / 32][10];

    const int c = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t off = a.cp[c].off;
    const int n = a.cp[c].n;
    int np2 = 1;
    while (np2 < n) np2 <<= 1;

    // (magnitude, sample index) keys; -0 ranks with +0
    for (int i = tid; i < np2; i += kBandsThreads) {
        unsigned long long k = ~0ull;
        if (i < n) {
            uint32_t u = __float_as_uint(a.mags[off + i]);
            if (u == 0x80000000u) u = 0u;
            k = ((unsigned long long)orderable(__uint_as_float(u)) << 32) | (unsigned long long)i;
        }
        keys[i] = k;
    }
    for (int k = 2; k <= np2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            __syncthreads();
            for (int i = tid; i < np2; i += kBandsThreads) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const bool up = (i & k) == 0;
                    const unsigned long long u = keys[i], v = keys[ixj];
                    if ((u > v) == up) { keys[i] = v; keys[ixj] = u; }
                }
            }
        }
    }
    __syncthreads();

    // rank r lies in band b iff floor(bN/10) <= r < floor((b+1)N/10), i.e. b = ceil(10(r+1)/N) - 1
    for (int r = tid; r < n; r += kBandsThreads) {
        const int i = (int)(keys[r] & 0xffffffffu);
        const int8_t b = (int8_t)((10 * (r + 1) - 1) / n);
        bnd[i] = b;
        a.band_of[off + i] = b;
    }
    __syncthreads();

    // D_b = sum |d_i| over the derivatives whose left sample is in band b (FP64, fixed order)
    double acc[10];
#pragma unroll
    for (int b = 0; b < 10; b++) acc[b] = 0.0;
    for (int i = tid; i + 1 < n; i += kBandsThreads) {
        const double dt = a.times[off + i + 1] - a.times[off + i];
        const double d = dt != 0.0 ? ((double)a.mags[off + i + 1] - (double)a.mags[off + i]) / dt : 0.0;
        const double ad = fabs(d);
        const int bi = bnd[i];
#pragma unroll
        for (int b = 0; b < 10; b++) acc[b] += (bi == b) ? ad : 0.0;
    }
#pragma unroll
    for (int b = 0; b < 10; b++) {
        double v = acc[b];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) s_D[warp][b] = v;
    }
    __syncthreads();
    if (tid == 0) {
        double D[10];
        int order[10];
        for (int b = 0; b < 10; b++) {
            double s = 0.0;
            for (int w = 0; w < kBandsThreads / 32; w++) s += s_D[w][b];
            D[b] = s;
            order[b] = b;
        }
        for (int x = 1; x < 10; x++) {           // stable: descending D, equal D keeps the lower band first
            const int v = order[x];
            int y = x;
            while (y > 0 && D[order[y - 1]] < D[v]) {
                order[y] = order[y - 1];
                y--;
            }
            order[y] = v;
        }
        for (int b = 0; b < a.n_bands; b++) a.kept[(int64_t)c * a.n_bands + b] = order[b];
    }
}

// ===========================================================================
// k_window
// ===========================================================================

// Shared-memory layout of k_window (bytes from the dynamic base).
struct WinLayout {
    size_t s, mask, pts, rot, sel, total;
};

__host__ __device__ inline WinLayout win_layout(int n_freq, int max_band_points)
{
    WinLayout L;
    const size_t kpad = ((size_t)n_freq + 3) & ~(size_t)3;
    const size_t words = (((size_t)n_freq + 31) / 32 + 3) & ~(size_t)3;
    L.s = 0;
    L.mask = L.s + kpad * sizeof(float);
    L.pts = L.mask + words * sizeof(uint32_t);
    L.rot = L.pts + (size_t)max_band_points * 2 * sizeof(uint64_t);
    L.sel = L.rot + (size_t)max_band_points * 2 * sizeof(float);
    L.total = L.sel + (size_t)kBandsMaxTrials * sizeof(unsigned long long);
    return L;
}

__device__ __forceinline__ bool win_cand(const uint32_t* mask, int k)
{
    return (mask[k >> 5] >> (k & 31)) & 1u;
}

__global__ void __launch_bounds__(kWinThreads, 1) k_window(const WindowArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const WinLayout Lo = win_layout(a.n_freq, a.max_band_points);
    float* S = reinterpret_cast<float*>(smem + Lo.s);
    uint32_t* mask = reinterpret_cast<uint32_t*>(smem + Lo.mask);
    ulonglong2* pts = reinterpret_cast<ulonglong2*>(smem + Lo.pts);
    float2* rot = reinterpret_cast<float2*>(smem + Lo.rot);
    unsigned long long* sel = reinterpret_cast<unsigned long long*>(smem + Lo.sel);
    __shared__ uint32_t hist[256];
    __shared__ int s_wsum[kWinThreads / 32];
    __shared__ int s_total, s_nsel, s_m;
    __shared__ uint32_t s_prefix;
    __shared__ int s_need, s_eq;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = kWinThreads / 32;
    const int c = blockIdx.x / a.n_bands, b = blockIdx.x - c * a.n_bands;
    const int K = a.n_freq, n_t = a.n_t;
    const int64_t off = a.cp[c].off;
    const int n = a.cp[c].n;
    const int band = a.kept[(int64_t)c * a.n_bands + b];

    // 1. the band's samples, in sample order: (base, step) phases and the rotation exp(i 2 pi 512 step)
    if (tid == 0) s_m = 0;
    __syncthreads();
    for (int i0 = 0; i0 < n; i0 += kWinThreads) {
        const int i = i0 + tid;
        const bool in = i < n && a.band_of[off + i] == band;
        const uint32_t bal = __ballot_sync(0xffffffffu, in);
        if (lane == 0) s_wsum[warp] = __popc(bal);
        __syncthreads();
        int before = s_m;
        for (int w = 0; w < warp; w++) before += s_wsum[w];
        const int pos = before + __popc(bal & ((1u << lane) - 1u));
        if (in && pos < a.max_band_points) {   // a band never exceeds ceil(N/10) samples
            const uint64_t st = a.ph_step[off + i];
            pts[pos] = make_ulonglong2(a.ph_base[off + i], st);
            float sr, cr;
            sincos2pi_turns((uint32_t)((st * (uint64_t)kWinThreads) >> 32), sr, cr);
            rot[pos] = make_float2(cr, sr);
        }
        __syncthreads();
        if (tid == 0) {
            int t = s_m;
            for (int w = 0; w < NW; w++) t += s_wsum[w];
            s_m = t;
        }
        __syncthreads();
    }
    const int m = s_m;

    // 2. spectral window, Eq. (bands): thread tid covers k = k0 + tid + 512 q
    for (int k0 = 0; k0 < K; k0 += kWinThreads * kWinRun) {
        const int kb = k0 + tid;
        float re[kWinRun], im[kWinRun];
#pragma unroll
        for (int q = 0; q < kWinRun; q++) { re[q] = 0.f; im[q] = 0.f; }
        if (kb < K) {
            for (int p = 0; p < m; p++) {
                const ulonglong2 e = pts[p];
                const float2 r = rot[p];
                float zi, zr;
                sincos2pi_turns((uint32_t)((e.x + (uint64_t)kb * e.y) >> 32), zi, zr);
#pragma unroll
                for (int q = 0; q < kWinRun; q++) {
                    re[q] += zr;
                    im[q] += zi;
                    const float nr = fmaf(zr, r.x, -zi * r.y);
                    const float ni = fmaf(zr, r.y, zi * r.x);
                    zr = nr;
                    zi = ni;
                }
            }
        }
#pragma unroll
        for (int q = 0; q < kWinRun; q++) {
            const int k = kb + q * kWinThreads;
            // a one-sample band is exactly 1 (|exp(i x)|^2), not cos^2 + sin^2 with rounding noise
            if (k < K) S[k] = m <= 1 ? (float)m : fmaf(re[q], re[q], im[q] * im[q]);
        }
    }
    if (tid == 0) { s_total = 0; s_nsel = 0; }
    __syncthreads();

    // 3. admissible local maxima: S[k] > S[k-1], S[k] >= S[k+1] (ends: one neighbour), not one-day
    const int words = (K + 31) >> 5;
    int local = 0;
    for (int w = warp; w < words; w += NW) {
        const int k = (w << 5) + lane;
        bool ok = false;
        if (k < K) {
            const float v = S[k];
            ok = (k == 0 || v > S[k - 1]) && (k == K - 1 || v >= S[k + 1]) && !(k >= a.ex_lo && k <= a.ex_hi);
        }
        const uint32_t bal = __ballot_sync(0xffffffffu, ok);
        if (lane == 0) {
            mask[w] = bal;
            local += __popc(bal);
        }
    }
    if (lane == 0) atomicAdd(&s_total, local);
    __syncthreads();
    const int total = s_total;

    // 4. threshold: the n_t-th largest value among the candidates (radix select on orderable bits)
    uint32_t T = 0u;        // select keys > T, plus `need` of the keys == T (lowest k first)
    int need = 0;
    bool take_all_eq = true;
    if (total > n_t) {
        if (tid == 0) { s_prefix = 0u; s_need = n_t; }
        for (int pass = 0; pass < 4; pass++) {
            const int shift = 24 - 8 * pass;
            for (int i = tid; i < 256; i += kWinThreads) hist[i] = 0u;
            __syncthreads();
            const uint32_t prefix = s_prefix;
            for (int k = tid; k < K; k += kWinThreads) {
                if (!win_cand(mask, k)) continue;
                const uint32_t key = orderable(S[k]);
                if (pass == 0 || (key >> (shift + 8)) == prefix) atomicAdd(&hist[(key >> shift) & 255u], 1u);
            }
            __syncthreads();
            if (warp == 0) {
                // lane l owns digits 255-8l-7 .. 255-8l; find the digit holding the need-th largest
                const int nd = s_need;
                uint32_t h[8];
                uint32_t sum = 0;
#pragma unroll
                for (int x = 0; x < 8; x++) {
                    h[x] = hist[255 - 8 * lane - x];
                    sum += h[x];
                }
                uint32_t incl = sum;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                const uint32_t excl = incl - sum;
                if (excl < (uint32_t)nd && (uint32_t)nd <= incl) {
                    uint32_t cum = excl;
#pragma unroll
                    for (int x = 0; x < 8; x++) {
                        if (cum + h[x] >= (uint32_t)nd) {
                            const uint32_t d = 255u - 8u * lane - x;
                            s_prefix = (prefix << 8) | d;
                            s_need = nd - (int)cum;
                            s_eq = (int)h[x];
                            break;
                        }
                        cum += h[x];
                    }
                }
            }
            __syncthreads();
        }
        T = s_prefix;
        need = s_need;
        take_all_eq = s_eq == need;
    }

    // 5. collect: keys > T (and == T when all of them are taken), unordered
    for (int k = tid; k < K; k += kWinThreads) {
        if (!win_cand(mask, k)) continue;
        const uint32_t key = orderable(S[k]);
        if (key > T || (key == T && take_all_eq && total > n_t)) {
            const int pos = atomicAdd(&s_nsel, 1);
            if (pos < kBandsMaxTrials) sel[pos] = ((unsigned long long)key << 32) | (0xffffffffu - (uint32_t)k);
        }
    }
    __syncthreads();
    if (!take_all_eq) {
        // ties at the threshold: the `need` lowest k, by an ordered scan
        int taken = 0;
        for (int k0 = 0; k0 < K && taken < need; k0 += kWinThreads) {
            const int k = k0 + tid;
            const bool eq = k < K && win_cand(mask, k) && orderable(S[k]) == T;
            const uint32_t bal = __ballot_sync(0xffffffffu, eq);
            if (lane == 0) s_wsum[warp] = __popc(bal);
            __syncthreads();
            int before = taken, chunk = 0;
            for (int w = 0; w < NW; w++) {
                if (w < warp) before += s_wsum[w];
                chunk += s_wsum[w];
            }
            if (eq) {
                const int rank = before + __popc(bal & ((1u << lane) - 1u));
                if (rank < need) {
                    const int pos = atomicAdd(&s_nsel, 1);
                    if (pos < kBandsMaxTrials) sel[pos] = ((unsigned long long)T << 32) | (0xffffffffu - (uint32_t)k);
                }
            }
            taken += chunk;
            __syncthreads();
        }
    }
    __syncthreads();
    const int nsel = min(s_nsel, n_t);

    // 6. order: value descending, ties to the lower k (bitonic sort of the keys, descending)
    int np2 = 1;
    while (np2 < nsel) np2 <<= 1;
    for (int i = nsel + tid; i < np2; i += kWinThreads) sel[i] = 0ull;
    for (int k = 2; k <= np2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            __syncthreads();
            for (int i = tid; i < np2; i += kWinThreads) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const bool down = (i & k) == 0;
                    const unsigned long long u = sel[i], v = sel[ixj];
                    if ((u < v) == down) { sel[i] = v; sel[ixj] = u; }
                }
            }
        }
    }
    __syncthreads();
    int32_t* out = a.trials + ((int64_t)c * a.n_bands + b) * n_t;
    for (int r = tid; r < n_t; r += kWinThreads)
        out[r] = r < nsel ? (int32_t)(0xffffffffu - (uint32_t)(sel[r] & 0xffffffffu)) : -1;
}

// ---------------------------------------------------------------------------
size_t bands_smem_bytes(int np2max) { return (size_t)np2max * (sizeof(unsigned long long) + 1); }

size_t window_smem_bytes(int n_freq, int max_band_points) { return win_layout(n_freq, max_band_points).total; }

cudaError_t prepare_bands_kernels(int np2max, int n_freq, int max_band_points)
{
    cudaError_t e = cudaFuncSetAttribute(k_bands, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)bands_smem_bytes(np2max));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_window, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)window_smem_bytes(n_freq, max_band_points));
}

cudaError_t launch_bands(const BandsArgs& a, int n_curves, cudaStream_t s)
{
    k_bands<<<n_curves, kBandsThreads, bands_smem_bytes(a.np2max), s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_window(const WindowArgs& a, cudaStream_t s)
{
    const int64_t ctas = (int64_t)a.n_curves * a.n_bands;
    if (ctas <= 0) return cudaSuccess;
    k_window<<<(unsigned)ctas, kWinThreads, window_smem_bytes(a.n_freq, a.max_band_points), s>>>(a);
    return cudaGetLastError();
}

}  // namespace cpk
