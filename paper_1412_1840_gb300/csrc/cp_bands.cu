// cp_bands.cu -- trial-period extraction of arXiv:1412.1840, Section 3.1
// (the bands method), on the device.
//
//   k_bands   one CTA per curve: magnitude ranks (bitonic sort of
//             (magnitude, sample) keys), the ten equal-count bands, the FP64
//             sums D_b of |d_i|, d_i = (y_{i+1} - y_i) / (t_{i+1} - t_i), and
//             the bands in descending order of D (equal D: lower band first)
//   k_window  one CTA per (curve, kept band): the spectral window of
//             Eq. (bands), S(f_k) = |sum_{i in band} exp(i 2 pi f_k t_i)|^2,
//             on the uniform grid f_k = f_min + k df in FP32, one segment of
//             the grid at a time in shared memory; the 2 n_t highest points
//             that may be local maxima within the FP32 error bound (one-day
//             frequencies left out): a histogram of the candidates' value
//             bits gives the bin of the segment's 2 n_t-th highest, the
//             candidates at or above it are sorted and merged into a running
//             sorted candidate list (an exact radix select on the value bits
//             when that bin holds too many), each candidate marked when its
//             local-maximum test is certain.
//   k_window_refine  one warp per (curve, kept band): the exact choice.  Every
//             candidate that can still reach the trials and whose
//             local-maximum test, or whose order against another candidate,
//             lies within the error bound gets its window value(s) again,
//             first in an accurate FP32 form, then in FP64 from the exact
//             phases; the n_t highest true local maxima (value descending,
//             ties to the lower k) are the trials, identical to an FP64
//             evaluation.
//
// Phases: exp(i 2 pi f_k t_i) with t_i - t0 (the window is invariant to a
// common time shift) from the exact 64-bit fixed-point phases
// base_i = frac(f_min (t_i - t0)) and step_i = frac(df (t_i - t0)) of the
// curve statistics pass: thread t evaluates k = k0 + t + 256 q (q < 16) by
// one sincos at k0 + t, one complex product for q = 8, and seven packed
// f32x2 rotations by exp(i 2 pi 256 step_i); both rotation angles are taken
// exactly from 256 step_i and 2048 step_i mod 1.
#include <cstdint>
#include <cuda_runtime.h>

#include "cp_internal.cuh"

namespace cpk {

constexpr int kBandsThreads = 256;
constexpr int kWinThreads = 256;
constexpr int kWinRun = 16;                    // frequencies per thread per pass (stride kWinThreads)
constexpr int kWinHalf = kWinRun / 2;          // q and q + kWinHalf share an f32x2 register
constexpr int kWinSeg = 2 * kWinThreads * kWinRun - 2;   // grid points per segment (two passes with neighbours)
// Error bound of an FP32 window value S of a band of m > 1 samples: each term
// exp(i x) carries at most kWinTermErr absolute error (SFU sin/cos below
// 2^-20.5 on an FP32 argument, plus up to 15 FP32 rotations of ~2^-22 each,
// about 4e-6 together, taken with a margin) and the m-term sums add
// at most m 2^-24 each, so |Z_fp32 - Z| <= e = m (kWinTermErr + m 2^-24) and
// |S_fp32 - S| <= 2 (sqrt(S_fp32) + e) e + e^2, plus the rounding of |Z|^2.
// The bound grows with the value: small side lobes are decided far more tightly
// than a bound on the band's largest possible value m^2.  Bands of one sample
// are exact (S = 1).
constexpr float kWinTermErr = 6e-6f;
__device__ __forceinline__ float win_err(float v, float e)
{
    if (e <= 0.f) return 0.f;
    const float z = sqrtf(fmaxf(v, 0.f)) + e;
    return fmaf(2.f * z, e, e * e) + fabsf(v) * 2.4e-7f;
}
__device__ __forceinline__ float win_term_err(int m)
{
    return m <= 1 ? 0.f : (float)m * (kWinTermErr + (float)m * 5.96e-8f);
}
__host__ __device__ constexpr int win_candidates(int n_t) { return 2 * n_t; }

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
// k_window: one CTA per (curve, kept band).  The grid is walked in segments
// of kWinSeg points; for each, S is computed (plus one neighbour on each
// side for the local-maximum test), the segment's n_t highest admissible
// maxima are selected and sorted, and merged into the running sorted list.
// The n_t highest of the whole grid are among the union of the per-segment
// n_t highest, so the result is exact.
// ===========================================================================

__host__ __device__ inline int pow2_at_least(int x)
{
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

// Shared-memory layout of k_window (bytes from the dynamic base).
struct WinLayout {
    size_t s, mask, pts, rot, lists, total;
};

__host__ __device__ inline WinLayout win_layout(int max_band_points, int n_t)
{
    WinLayout L;
    L.s = 0;
    L.mask = L.s + (size_t)(kWinSeg + 2 + 2) * sizeof(float);
    L.pts = L.mask + (size_t)((kWinSeg + 31) / 32 + 2) * sizeof(uint32_t);
    L.pts = (L.pts + 15) & ~(size_t)15;
    L.rot = L.pts + (size_t)max_band_points * sizeof(ulonglong2);
    L.lists = L.rot + (size_t)max_band_points * sizeof(float4);
    L.total = L.lists + 3 * (size_t)pow2_at_least(win_candidates(n_t)) * sizeof(unsigned long long);
    return L;
}

// Candidate key: the FP32 window value, then bit 31 set when the point's
// local-maximum test is certain (both comparisons decided by more than the two
// values' error bounds), then the lower grid index k.
__device__ __forceinline__ unsigned long long win_key(const float* S, int x, int k, int K, float e)
{
    const float v = S[x], ev = win_err(v, e);
    const bool sure = (k == 0 || v - S[x - 1] > ev + win_err(S[x - 1], e)) &&
                      (k == K - 1 || v - S[x + 1] > ev + win_err(S[x + 1], e));
    return ((unsigned long long)orderable(v) << 32) | (sure ? 0x80000000ull : 0ull) |
           (unsigned long long)(0x7fffffffu - (uint32_t)k);
}

__device__ __forceinline__ unsigned long long win_key_of(float v, bool sure, int k)
{
    return ((unsigned long long)orderable(v) << 32) | (sure ? 0x80000000ull : 0ull) |
           (unsigned long long)(0x7fffffffu - (uint32_t)k);
}

// Histogram bin of a value S >= 0: the bits below the orderable form's top bit
// (always set for S >= 0), as many as the bin count has.
__device__ __forceinline__ int win_digit(float v, int shift, int bins)
{
    return (int)((orderable(v) >> shift) & (uint32_t)(bins - 1));
}

__device__ __forceinline__ bool win_cand(const uint32_t* mask, int j)
{
    return (mask[j >> 5] >> (j & 31)) & 1u;
}

// Descending bitonic sort of n (a power of two) 64-bit keys in shared memory.
__device__ __forceinline__ void sort_desc(unsigned long long* v, int n, int tid)
{
    for (int k = 2; k <= n; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            __syncthreads();
            for (int i = tid; i < n; i += kWinThreads) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const bool down = (i & k) == 0;
                    const unsigned long long u = v[i], w = v[ixj];
                    if ((u < w) == down) { v[i] = w; v[ixj] = u; }
                }
            }
        }
    }
    __syncthreads();
}

// Number of entries of the descending list v[0..n) greater than x.
__device__ __forceinline__ int count_greater(const unsigned long long* v, int n, unsigned long long x)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (v[mid] > x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(kWinThreads) k_window(const WindowArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const WinLayout Lo = win_layout(a.max_band_points, a.n_t);
    float* S = reinterpret_cast<float*>(smem + Lo.s);
    uint32_t* mask = reinterpret_cast<uint32_t*>(smem + Lo.mask);
    ulonglong2* pts = reinterpret_cast<ulonglong2*>(smem + Lo.pts);
    float4* rot = reinterpret_cast<float4*>(smem + Lo.rot);
    const int cap = pow2_at_least(win_candidates(a.n_t));
    // lists: R0 R1 (the buffer of the fast path, the histogram before it; the
    // fallback's selection and merge output), R2 (the running list)
    unsigned long long* buf = reinterpret_cast<unsigned long long*>(smem + Lo.lists);
    unsigned long long* sel = buf;
    unsigned long long* nxt = buf + cap;
    unsigned long long* run = buf + 2 * cap;
    uint32_t* hist4 = reinterpret_cast<uint32_t*>(buf);   // 4 cap bins over R0 R1
    const int hbins = 4 * cap;
    int hshift = 31;                                       // digit = value bits 30 .. 31 - log2(hbins)
    for (int b = hbins; b > 1; b >>= 1) hshift--;
    __shared__ uint32_t hist[256];
    __shared__ int s_wsum[kWinThreads / 32];
    __shared__ int s_total, s_nsel, s_m;
    __shared__ uint32_t s_prefix;
    __shared__ int s_need, s_eq, s_d0, s_fast;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = kWinThreads / 32;
    const int c = blockIdx.x / a.n_bands, b = blockIdx.x - c * a.n_bands;
    const int K = a.n_freq, n_t = win_candidates(a.n_t);   // candidates kept per band
    const int64_t off = a.cp[c].off;
    const int n = a.cp[c].n;
    const int band = a.kept[(int64_t)c * a.n_bands + b];

    // 1. the band's samples, in sample order: phases (base, step) and the rotations
    //    exp(i 2 pi 256 step), exp(i 2 pi 2048 step)
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
            float sr, cr, s8, c8;
            sincos2pi_turns((uint32_t)((st * (uint64_t)kWinThreads) >> 32), sr, cr);
            sincos2pi_turns((uint32_t)((st * (uint64_t)(kWinThreads * kWinHalf)) >> 32), s8, c8);
            rot[pos] = make_float4(cr, sr, c8, s8);
        }
        __syncthreads();
        if (tid == 0) {
            int t = s_m;
            for (int w = 0; w < NW; w++) t += s_wsum[w];
            s_m = t;
        }
        __syncthreads();
    }
    const int m = min(s_m, a.max_band_points);
    const float e2 = win_term_err(m);   // per-term error scale of the band's window values

    int rc = 0;                       // running list: the n_t highest so far, descending
    for (int lo = 0; lo < K; lo += kWinSeg) {
        const int hi = min(K, lo + kWinSeg);
        const int v0 = max(lo - 1, 0), v1 = min(hi + 1, K);   // S[k - v0] holds k in [v0, v1)
        const int nv = v1 - v0;

        // 2. spectral window, Eq. (bands): thread tid covers k = v0 + p0 + tid + 256 q, q < 16, with
        //    q and q + 8 in the two lanes of an f32x2 register, rotated by exp(i 2 pi 256 step)
        for (int p0 = 0; p0 < nv; p0 += kWinThreads * kWinRun) {
            const int j0 = p0 + tid;
            f2 re2[kWinHalf], im2[kWinHalf];
#pragma unroll
            for (int q = 0; q < kWinHalf; q++) { re2[q] = 0ull; im2[q] = 0ull; }
            if (j0 < nv) {
                const uint64_t kb = (uint64_t)(v0 + j0);
                ulonglong2 en = pts[0];
                float4 rn = rot[0];
                for (int p = 0; p < m; p++) {
                    const ulonglong2 e = en;       // this point; the next one's loads are in flight
                    const float4 r = rn;
                    const int pn = p + 1 < m ? p + 1 : p;
                    en = pts[pn];
                    rn = rot[pn];
                    float zi, zr;
                    sincos2pi_turns_sfu((uint32_t)((e.x + kb * e.y) >> 32), zi, zr);
                    const float zr8 = fmaf(zr, r.z, -zi * r.w), zi8 = fmaf(zr, r.w, zi * r.z);
                    f2 ZR = pk(zr, zr8), ZI = pk(zi, zi8);
                    const f2 CR = pk(r.x, r.x), SR = pk(r.y, r.y), NSR = pk(-r.y, -r.y);
#pragma unroll
                    for (int q = 0; q < kWinHalf; q++) {
                        re2[q] = add2(re2[q], ZR);
                        im2[q] = add2(im2[q], ZI);
                        const f2 nr = fma2(ZR, CR, mul2(ZI, NSR));
                        const f2 ni = fma2(ZR, SR, mul2(ZI, CR));
                        ZR = nr;
                        ZI = ni;
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < kWinHalf; q++) {
                float rl, rh, il, ih;
                upk(re2[q], rl, rh);
                upk(im2[q], il, ih);
                const int ja = j0 + q * kWinThreads, jb = ja + kWinHalf * kWinThreads;
                // a one-sample band is exactly 1 (|exp(i x)|^2), not cos^2 + sin^2 with rounding noise
                if (ja < nv) S[ja] = m <= 1 ? (float)m : fmaf(rl, rl, il * il);
                if (jb < nv) S[jb] = m <= 1 ? (float)m : fmaf(rh, rh, ih * ih);
            }
        }
        if (tid == 0) { s_total = 0; s_nsel = 0; s_d0 = 0; s_fast = 1; }
        for (int i = tid; i < hbins; i += kWinThreads) hist4[i] = 0u;
        __syncthreads();

        // 3. candidates of the segment: points that can be local maxima S[k] > S[k-1],
        //    S[k] >= S[k+1] (grid ends: one neighbour) within the error bound, one-day
        //    frequencies left out; once the running list is full, only keys above its
        //    last entry can still enter it.  Each value's bound is computed once (the
        //    neighbours' come from the adjacent lanes), and a histogram of the
        //    candidates' value bits is kept for the threshold of step 4.
        const unsigned long long floor_key = rc == n_t ? run[n_t - 1] : 0ull;
        const int len = hi - lo;
        const int words = (len + 31) >> 5;
        int local = 0;
#pragma unroll 2
        for (int w = warp; w < words; w += NW) {   // warp-uniform: every lane takes the shuffles
            const int j = (w << 5) + lane;      // segment position, k = lo + j
            const int k = lo + j;
            const int x = k - v0;
            const bool in = j < len;
            const float v = in ? S[x] : 0.f;
            const float ev = in ? win_err(v, e2) : 0.f;
            float vl = __shfl_up_sync(0xffffffffu, v, 1), el = __shfl_up_sync(0xffffffffu, ev, 1);
            float vr = __shfl_down_sync(0xffffffffu, v, 1), er = __shfl_down_sync(0xffffffffu, ev, 1);
            if (in && lane == 0 && k > 0) { vl = S[x - 1]; el = win_err(vl, e2); }
            if (in && (lane == 31 || j + 1 >= len) && k < K - 1) { vr = S[x + 1]; er = win_err(vr, e2); }
            bool ok = false;
            if (in) {
                // may be a local maximum in exact values: not decided against it by more
                // than the two values' error bounds (exact bands: the exact test)
                const bool lok = k == 0 || (e2 > 0.f ? v >= vl - ev - el : v > vl);
                const bool rok = k == K - 1 || v >= vr - ev - er;
                if (lok && rok && !(k >= a.ex_lo && k <= a.ex_hi)) {
                    const bool sure = (k == 0 || v - vl > ev + el) && (k == K - 1 || v - vr > ev + er);
                    ok = win_key_of(v, sure, k) > floor_key;
                }
            }
            if (ok) atomicAdd(&hist4[win_digit(v, hshift, hbins)], 1u);
            const uint32_t bal = __ballot_sync(0xffffffffu, ok);
            if (lane == 0) {
                mask[w] = bal;
                local += __popc(bal);
            }
        }
        if (lane == 0 && local) atomicAdd(&s_total, local);
        __syncthreads();
        const int total = s_total;

        // 4. fast path: the buffer (2 cap) takes the running list and the candidates
        //    whose histogram bin is at or above the bin of the segment's n_t-th
        //    largest (all of them when they fit); one sort keeps the n_t highest.
        if (rc + total > 2 * cap && warp == 0) {
            const int G = (hbins + 31) / 32;   // lane l owns bins hbins-1-lG down to hbins-(l+1)G
            uint32_t sum = 0;
            for (int y = 0; y < G; y++) {
                const int d = hbins - 1 - lane * G - y;
                if (d >= 0) sum += hist4[d];
            }
            uint32_t incl = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            const uint32_t excl = incl - sum;
            if (excl < (uint32_t)n_t && (uint32_t)n_t <= incl) {   // one lane: total > n_t here
                uint32_t cum = excl;
                for (int y = 0; y < G; y++) {
                    const int d = hbins - 1 - lane * G - y;
                    cum += hist4[d];
                    if (cum >= (uint32_t)n_t) {
                        s_d0 = d;
                        s_fast = rc + (int)cum <= 2 * cap;
                        break;
                    }
                }
            }
        }
        __syncthreads();
        if (s_fast) {
            // the candidates in bins >= d0 into the buffer, in segment order: each warp
            // counts its own, then writes at its offset (no atomics on the path)
            const int d0 = s_d0;
            int mine = 0;
            for (int w = warp; w < words; w += NW) {
                const uint32_t bits = mask[w];
                bool take = false;
                if ((bits >> lane) & 1u) take = win_digit(S[lo + (w << 5) + lane - v0], hshift, hbins) >= d0;
                mine += __popc(__ballot_sync(0xffffffffu, take));
            }
            if (lane == 0) s_wsum[warp] = mine;
            __syncthreads();
            int off = 0, nsel = 0;
            for (int w = 0; w < NW; w++) {
                if (w < warp) off += s_wsum[w];
                nsel += s_wsum[w];
            }
            for (int w = warp; w < words; w += NW) {
                const uint32_t bits = mask[w];
                const int j = (w << 5) + lane;
                bool take = false;
                if ((bits >> lane) & 1u) take = win_digit(S[lo + j - v0], hshift, hbins) >= d0;
                const uint32_t tb = __ballot_sync(0xffffffffu, take);
                if (take) buf[off + __popc(tb & ((1u << lane) - 1u))] = win_key(S, lo + j - v0, lo + j, K, e2);
                off += __popc(tb);
            }
            // sort the new keys; merge their first n_t with the running list into R1
            // (R1 is free, or holds sorted keys ranked below n_t)
            const int np2 = pow2_at_least(nsel);
            for (int i = nsel + tid; i < np2; i += kWinThreads) buf[i] = 0ull;
            sort_desc(buf, np2, tid);
            const int ns = min(nsel, n_t);
            for (int i = tid; i < rc; i += kWinThreads) {
                const int r = i + count_greater(buf, ns, run[i]);
                if (r < n_t) nxt[r] = run[i];
            }
            for (int i = tid; i < ns; i += kWinThreads) {
                const int r = i + count_greater(run, rc, buf[i]);
                if (r < n_t) nxt[r] = buf[i];
            }
            rc = min(rc + ns, n_t);
            __syncthreads();
            for (int i = tid; i < rc; i += kWinThreads) run[i] = nxt[i];
            __syncthreads();
            continue;
        }

        // Fallback (the buffer would overflow: many candidates within one bin, such
        // as the equal maxima of a two-sample band): the exact selection of the
        // segment's n_t highest by a radix select on the value bits, then a merge.
        // 4. the segment's threshold: its n_t-th largest candidate value (radix select on the
        //    orderable bits, warp-aggregated histogram updates)
        uint32_t T = 0u;        // take keys > T, plus `need` keys == T (lowest k first)
        int need = 0;
        bool take_all_eq = true;
        if (total > n_t) {
            if (tid == 0) { s_prefix = 0u; s_need = n_t; }
            for (int pass = 0; pass < 4; pass++) {
                const int shift = 24 - 8 * pass;
                for (int i = tid; i < 256; i += kWinThreads) hist[i] = 0u;
                __syncthreads();
                const uint32_t prefix = s_prefix;
                for (int j0 = 0; j0 < len; j0 += kWinThreads) {
                    const int j = j0 + tid;
                    bool take = false;
                    uint32_t d = 0u;
                    if (j < len && win_cand(mask, j)) {
                        const uint32_t key = orderable(S[lo + j - v0]);
                        take = pass == 0 || (key >> (shift + 8)) == prefix;
                        d = (key >> shift) & 255u;
                    }
                    const uint32_t peers = __match_any_sync(0xffffffffu, take ? d : 256u + (uint32_t)lane);
                    if (take && lane == __ffs(peers) - 1) atomicAdd(&hist[d], (uint32_t)__popc(peers));
                }
                __syncthreads();
                if (warp == 0) {
                    // lane l owns digits 255-8l .. 248-8l; find the digit holding the need-th largest
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
                                s_prefix = (prefix << 8) | (255u - 8u * lane - x);
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
        for (int j0 = 0; j0 < len; j0 += kWinThreads) {
            const int j = j0 + tid;
            if (j < len && win_cand(mask, j)) {
                const uint32_t key = orderable(S[lo + j - v0]);
                if (key > T || (key == T && take_all_eq && total > n_t)) {
                    const int pos = atomicAdd(&s_nsel, 1);
                    if (pos < n_t) sel[pos] = win_key(S, lo + j - v0, lo + j, K, e2);
                }
            }
        }
        __syncthreads();
        if (!take_all_eq) {
            // ties at the threshold: the `need` lowest k, by an ordered scan
            int taken = 0;
            for (int j0 = 0; j0 < len && taken < need; j0 += kWinThreads) {
                const int j = j0 + tid;
                const bool eq = j < len && win_cand(mask, j) && orderable(S[lo + j - v0]) == T;
                const uint32_t bal = __ballot_sync(0xffffffffu, eq);
                if (lane == 0) s_wsum[warp] = __popc(bal);
                __syncthreads();
                int before = taken, chunk = 0;
                for (int w = 0; w < NW; w++) {
                    if (w < warp) before += s_wsum[w];
                    chunk += s_wsum[w];
                }
                if (eq) {
                    const int r = before + __popc(bal & ((1u << lane) - 1u));
                    if (r < need) {
                        const int pos = atomicAdd(&s_nsel, 1);
                        if (pos < n_t) sel[pos] = win_key(S, lo + j - v0, lo + j, K, e2);
                    }
                }
                taken += chunk;
                __syncthreads();
            }
        }
        __syncthreads();
        const int nsel = min(s_nsel, n_t);
        const int np2 = pow2_at_least(nsel);
        for (int i = nsel + tid; i < np2; i += kWinThreads) sel[i] = 0ull;
        sort_desc(sel, np2, tid);

        // 6. merge the sorted segment list into the running list (keys are unique: rank by counting)
        for (int i = tid; i < rc; i += kWinThreads) {
            const int r = i + count_greater(sel, nsel, run[i]);
            if (r < n_t) nxt[r] = run[i];
        }
        for (int i = tid; i < nsel; i += kWinThreads) {
            const int r = i + count_greater(run, rc, sel[i]);
            if (r < n_t) nxt[r] = sel[i];
        }
        rc = min(rc + nsel, n_t);
        __syncthreads();
        for (int i = tid; i < rc; i += kWinThreads) run[i] = nxt[i];
        __syncthreads();
    }

    unsigned long long* out = a.cand + ((int64_t)c * a.n_bands + b) * n_t;
    for (int r = tid; r < n_t; r += kWinThreads) out[r] = r < rc ? run[r] : 0ull;
}

// ===========================================================================
// k_window_refine: one warp per (curve, kept band), see the file header.
// ===========================================================================
constexpr int kRefineWarps = 8;

// Exact window value at grid index k from the band's 64-bit fixed-point phases
// (lanes split the points; FP64 sincospi of the exactly reduced angle).
__device__ double window_fp64(const ulonglong2* pts, int m, uint64_t k, int lane)
{
    if (m <= 1) return (double)m;
    double re = 0.0, im = 0.0;
    for (int p = lane; p < m; p += 32) {
        const uint64_t U = pts[p].x + k * pts[p].y;              // frac(f_k (t - t0)) in 2^-64 turns
        double sv, cv;
        sincospi((double)(int64_t)U * 0x1p-63, &sv, &cv);        // angle 2 pi U / 2^64 in (-pi, pi]
        re += cv;
        im += sv;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    return re * re + im * im;
}

// A tighter, still cheap evaluation (FP32): cos and sin of each term from the
// Taylor polynomials on the exactly reduced angle (each below 2.5e-7 absolute
// error with the FP32 rounding of the evaluation and of the angle), compensated
// (Kahan) sums per lane (below 2 2^-24 per term), lanes combined in FP64.  So
// |Z_acc - Z| <= e1 = m kAccTermErr, taken with a margin, and
// |S_acc - S| <= 2 (|Z_acc| + e1) e1 + e1^2.
constexpr float kAccTermErr = 1e-6f;
__device__ double window_acc(const ulonglong2* pts, int m, uint64_t k, int lane, float& bound)
{
    bound = 0.f;
    if (m <= 1) return (double)m;
    float re = 0.f, im = 0.f, cr = 0.f, ci = 0.f;
    for (int p = lane; p < m; p += 32) {
        const uint64_t U = pts[p].x + k * pts[p].y;
        float sv, cv;
        sincos2pi_turns((uint32_t)(U >> 32), sv, cv);
        float y = cv - cr, t = re + y;
        cr = (t - re) - y;
        re = t;
        y = sv - ci;
        t = im + y;
        ci = (t - im) - y;
        im = t;
    }
    double R = (double)re - (double)cr, I = (double)im - (double)ci;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        R += __shfl_xor_sync(0xffffffffu, R, o);
        I += __shfl_xor_sync(0xffffffffu, I, o);
    }
    const double S = R * R + I * I;
    const float e1 = (float)m * kAccTermErr;
    const float z = sqrtf((float)S) + e1;
    bound = fmaf(2.f * z, e1, e1 * e1);
    return S;
}

// The same value computed by one lane alone (points in sample order).
__device__ double window_fp64_lane(const ulonglong2* pts, int m, uint64_t k)
{
    if (m <= 1) return (double)m;
    double re = 0.0, im = 0.0;
    for (int p = 0; p < m; p++) {
        const uint64_t U = pts[p].x + k * pts[p].y;
        double sv, cv;
        sincospi((double)(int64_t)U * 0x1p-63, &sv, &cv);
        re += cv;
        im += sv;
    }
    return re * re + im * im;
}

// Lane 0 keeps the n_t best (value descending, ties to the lower k) in val/kk;
// candidates arrive in ascending k, so an equal value goes after the others.
__device__ __forceinline__ void list_insert(double* val, int32_t* kk, int& cnt, int n_t, double v, int k)
{
    if (cnt == n_t && !(v > val[n_t - 1])) return;
    int q = cnt < n_t ? cnt : n_t - 1;
    while (q > 0 && val[q - 1] < v) {
        val[q] = val[q - 1];
        kk[q] = kk[q - 1];
        q--;
    }
    val[q] = v;
    kk[q] = k;
    if (cnt < n_t) cnt++;
}

__global__ void __launch_bounds__(32 * kRefineWarps, 2) k_window_refine(const WindowArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int job = blockIdx.x * kRefineWarps + warp;       // (curve, kept band)
    if (job >= a.n_curves * a.n_bands) return;
    const int c = job / a.n_bands, b = job - c * a.n_bands;
    const int K = a.n_freq, n_t = a.n_t, nc = win_candidates(n_t);
    ulonglong2* pts = reinterpret_cast<ulonglong2*>(smem) + (size_t)warp * a.max_band_points;
    // per candidate: value (FP32 from the window, accurate FP32 or FP64 where
    // recomputed), its error bound, and the grid index (bits 0-27) with flags:
    // bit 30 local-maximum test uncertain, bit 29 open, bit 28 the value is exact
    unsigned char* vbase = smem + (size_t)kRefineWarps * a.max_band_points * sizeof(ulonglong2);
    double* val = reinterpret_cast<double*>(vbase) + (size_t)warp * nc;
    int32_t* kk = reinterpret_cast<int32_t*>(vbase + (size_t)kRefineWarps * nc * sizeof(double)) + (size_t)warp * nc;
    float* eb = reinterpret_cast<float*>(vbase + (size_t)kRefineWarps * nc * (sizeof(double) + sizeof(int32_t))) +
                (size_t)warp * nc;   // error bound of each value (0 once exact)
    float* fv = eb + (size_t)kRefineWarps * nc;   // each value rounded to FP32 (FP64 arithmetic is slow here)
    const int64_t off = a.cp[c].off;
    const int n = a.cp[c].n;
    const int band = a.kept[(int64_t)c * a.n_bands + b];

    // the band's exact phases, in sample order
    int m = 0;
    for (int i0 = 0; i0 < n; i0 += 32) {
        const int i = i0 + lane;
        const bool in = i < n && a.band_of[off + i] == band;
        const uint32_t bal = __ballot_sync(0xffffffffu, in);
        const int pos = m + __popc(bal & ((1u << lane) - 1u));
        if (in && pos < a.max_band_points) pts[pos] = make_ulonglong2(a.ph_base[off + i], a.ph_step[off + i]);
        m += __popc(bal);
    }
    m = min(m, a.max_band_points);
    __syncwarp();
    const float e = win_term_err(m);               // per-term error scale: win_err(v, e) bounds |S_fp32 - S|

    // candidates (descending FP32 value, then sure-first, then lower k)
    const unsigned long long* cand = a.cand + (int64_t)job * nc;
    int cnt = 0;
    for (int r0 = 0; r0 < nc; r0 += 32) {          // every lane takes every trip (the ballot needs all 32)
        const int r = r0 + lane;
        const unsigned long long key = r < nc ? cand[r] : 0ull;
        if (key) {
            fv[r] = from_orderable((uint32_t)(key >> 32));
            val[r] = (double)fv[r];
            kk[r] = (int32_t)(0x7fffffffu - (uint32_t)(key & 0x7fffffffu)) | (int32_t)((key & 0x80000000ull) ? 0 : 0x40000000);
        }
        const uint32_t bal = __ballot_sync(0xffffffffu, key != 0ull);
        cnt += __popc(bal);
    }
    __syncwarp();
    const float last32 = cnt > 0 ? fv[cnt - 1] : 0.f;
    const bool full = cnt == nc;

    // Only candidates that can still reach the first n_t trials matter: with the n_t
    // certain maxima of the list bounding the n_t-th trial's value from below by L,
    // a candidate whose value is below L by more than its error bound cannot.
    int rel = cnt;
    if (lane == 0) {                               // FP32 with directed rounding: the cut errs on the safe side
        int secured = 0;
        float L = INFINITY;
        for (int r = 0; r < cnt; r++) {
            const float v = fv[r], er = win_err(v, e);
            if (secured >= n_t && __fadd_ru(v, er) < L) { rel = r; break; }
            if (!(kk[r] & 0x40000000) && secured < n_t) {
                secured++;
                L = fminf(L, __fsub_rd(v, er));
            }
        }
    }
    rel = __shfl_sync(0xffffffffu, rel, 0);

    // Decide what the FP32 bounds leave open: first with the accurate FP32 value
    // (a bound about ten times tighter), then in FP64, repeated until nothing is
    // open.  Each round sorts the live entries (value descending, ties to the
    // lower k) and opens an entry whose local-maximum test is uncertain, or whose
    // interval value +- bound meets that of another entry when one of the two
    // sits in the first n_t places (their order, or which of them is a trial, is
    // undecided).  With nothing open, every entry outside the first n_t lies
    // below each of them and the first n_t are in their true order.
    for (int r = lane; r < rel; r += 32) eb[r] = win_err(fv[r], e);
    __syncwarp();
    for (int tier = 1;; tier = 2) {
        if (lane == 0) {                           // drop the rejected entries, sort the rest
            int kept = 0;                          // (values >= 0: their bit patterns order as integers)
            for (int r = 0; r < rel; r++) {
                const int t = kk[r];
                if (t < 0) continue;
                const double v = val[r];
                const long long vb = __double_as_longlong(v);
                const float bv = eb[r], f = fv[r];
                const int k = t & 0x0fffffff;
                int q = kept;
                while (q > 0) {
                    const long long pb = __double_as_longlong(val[q - 1]);
                    if (!(pb < vb || (pb == vb && (kk[q - 1] & 0x0fffffff) > k))) break;
                    val[q] = val[q - 1];
                    eb[q] = eb[q - 1];
                    fv[q] = fv[q - 1];
                    kk[q] = kk[q - 1];
                    q--;
                }
                val[q] = v;
                eb[q] = bv;
                fv[q] = f;
                kk[q] = t;
                kept++;
            }
            rel = kept;
        }
        rel = __shfl_sync(0xffffffffu, rel, 0);
        __syncwarp();
        float ebmax = 0.f;
        for (int r = lane; r < rel; r += 32) ebmax = fmaxf(ebmax, eb[r]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ebmax = fmaxf(ebmax, __shfl_xor_sync(0xffffffffu, ebmax, o));
        // two intervals meet when |v_r - v_q| <= b_r + b_q; compared in FP32 with a
        // slack above the rounding of the values and of their difference, so a pair
        // is never taken as apart when it is not.  The list is sorted, so each walk
        // from r ends at the first entry beyond b_r + max b.
        int open = 0;
        for (int r0 = 0; r0 < rel; r0 += 32) {
            const int r = r0 + lane;
            bool o = false;
            if (r < rel) {
                o = (kk[r] & 0x40000000) != 0;
                const float vr = fv[r], br = eb[r];
                for (int q = min(r, n_t) - 1; q >= 0 && !o; q--) {   // higher values (a pair needs one of the first n_t)
                    const float d = fv[q] - vr, sl = 2.4e-7f * (fv[q] + vr);
                    if (d > br + ebmax + sl) break;
                    const float sb = br + eb[q];
                    o = sb > 0.f && fabsf(d) <= sb + sl;
                }
                for (int q = r + 1; r < n_t && q < rel && !o; q++) {   // lower values
                    const float d = vr - fv[q], sl = 2.4e-7f * (fv[q] + vr);
                    if (d > br + ebmax + sl) break;
                    const float sb = br + eb[q];
                    o = sb > 0.f && fabsf(d) <= sb + sl;
                }
                if (o) kk[r] |= 0x20000000;        // only lane r touches kk[r] here
            }
            open += __popc(__ballot_sync(0xffffffffu, o));
        }
        __syncwarp();
        if (open == 0) break;
        for (int r = 0; r < rel; r++) {
            const int tag = kk[r];
            if (!(tag & 0x20000000)) continue;
            const int k = tag & 0x0fffffff;
            if (tag & 0x10000000) {                // exact already: nothing to recompute
                if (lane == 0) kk[r] = tag & ~0x20000000;
                __syncwarp();
                continue;
            }
            float bk = 0.f, bn = 0.f;
            const double sk = tier == 1 ? window_acc(pts, m, (uint64_t)k, lane, bk) : window_fp64(pts, m, (uint64_t)k, lane);
            int state = 1;                         // 1 a maximum, 0 not, 2 still uncertain
            if (tag & 0x40000000) {                // S(k) > S(k - 1) and S(k) >= S(k + 1) at this accuracy
                if (k > 0) {
                    const double sl = tier == 1 ? window_acc(pts, m, (uint64_t)(k - 1), lane, bn)
                                                : window_fp64(pts, m, (uint64_t)(k - 1), lane);
                    if (sk - sl > (double)(bk + bn)) state = 1;
                    else if (sl - sk >= (double)(bk + bn)) state = 0;
                    else state = 2;
                }
                if (state != 0 && k < K - 1) {
                    const double sr = tier == 1 ? window_acc(pts, m, (uint64_t)(k + 1), lane, bn)
                                                : window_fp64(pts, m, (uint64_t)(k + 1), lane);
                    if (sr - sk > (double)(bk + bn) || (tier == 2 && sr > sk)) state = 0;
                    else if (!(sk - sr > (double)(bk + bn) || tier == 2)) state = 2;
                }
            }
            if (lane == 0) {
                val[r] = sk;
                eb[r] = bk;
                fv[r] = (float)sk;
                kk[r] = state == 0 ? -1 : k | (state == 2 ? 0x40000000 : 0) | (tier == 2 ? 0x10000000 : 0);
            }
            __syncwarp();
        }
    }

    // the first n_t of the decided order are the trials
    int32_t* out = a.trials + (int64_t)job * n_t;
    for (int r = lane; r < n_t; r += 32) out[r] = r < rel ? (kk[r] & 0x0fffffff) : -1;
    // a full candidate list leaves out points whose FP32 value is below its last
    // entry: they cannot reach the trials when the n_t-th trial lies above it by
    // more than both error bounds; otherwise (peaks of nearly equal height, such
    // as the maxima 4 of a two-sample band) the band is scanned exactly
    int scan = 0;
    if (full)
        scan = rel < n_t || val[n_t - 1] - (double)eb[n_t - 1] <= (double)last32 + (double)win_err(last32, e);
    scan = __shfl_sync(0xffffffffu, scan, 0);
    if (!scan) return;
    if (lane == 0) atomicAdd(a.exact_scans, 1);

    // exact scan of the whole grid: lanes take k = k0 + lane, k0 advancing by 30 so that
    // lanes 1..30 have both neighbours; S(-1) = S(K) = -inf reproduce the end rules
    int cntl = 0;
    for (int k0 = -1; k0 + 1 < K; k0 += 30) {
        const int k = k0 + lane;
        const double v = (k >= 0 && k < K) ? window_fp64_lane(pts, m, (uint64_t)k) : -INFINITY;
        const double left = __shfl_up_sync(0xffffffffu, v, 1), right = __shfl_down_sync(0xffffffffu, v, 1);
        const bool ismax = lane >= 1 && lane <= 30 && k < K && v > left && v >= right && !(k >= a.ex_lo && k <= a.ex_hi);
        uint32_t bal = __ballot_sync(0xffffffffu, ismax);
        while (bal) {
            const int l = __ffs(bal) - 1;
            bal &= bal - 1;
            const double vv = __shfl_sync(0xffffffffu, v, l);
            if (lane == 0) list_insert(val, kk, cntl, n_t, vv, k0 + l);
        }
    }
    __syncwarp();
    if (lane == 0)
        for (int r = 0; r < n_t; r++) out[r] = r < cntl ? kk[r] : -1;
}

// ---------------------------------------------------------------------------
size_t bands_smem_bytes(int np2max) { return (size_t)np2max * (sizeof(unsigned long long) + 1); }

size_t window_smem_bytes(int max_band_points, int n_t) { return win_layout(max_band_points, n_t).total; }

size_t refine_smem_bytes(int max_band_points, int n_t)
{
    return (size_t)kRefineWarps * ((size_t)max_band_points * sizeof(ulonglong2) +
                                   (size_t)win_candidates(n_t) * (sizeof(double) + sizeof(int32_t) + 2 * sizeof(float)));
}

cudaError_t prepare_bands_kernels(int np2max, int max_band_points, int n_t)
{
    cudaError_t e = raise_dyn_smem((const void*)k_bands, bands_smem_bytes(np2max));
    if (e != cudaSuccess) return e;
    e = raise_dyn_smem((const void*)k_window_refine, refine_smem_bytes(max_band_points, n_t));
    if (e != cudaSuccess) return e;
    return raise_dyn_smem((const void*)k_window, window_smem_bytes(max_band_points, n_t));
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
    k_window<<<(unsigned)ctas, kWinThreads, window_smem_bytes(a.max_band_points, a.n_t), s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_window_refine<<<(unsigned)((ctas + kRefineWarps - 1) / kRefineWarps), 32 * kRefineWarps,
                      refine_smem_bytes(a.max_band_points, a.n_t), s>>>(a);
    return cudaGetLastError();
}

}  // namespace cpk
