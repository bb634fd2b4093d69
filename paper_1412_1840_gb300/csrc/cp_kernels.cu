// cp_kernels.cu -- sm_103a kernels of the correntropy kernelized periodogram.
//
// Hot path (arXiv:1412.1840, Section 3, Eq. (HP), (IP), (CKP)):
//   k_stats        per-curve scalars (sigma_y = med(e), pSNR, sigma_t, IP),
//                  scaled magnitudes y' and 64-bit fixed-point phase steps
//   k_build_w      period-independent magnitude-kernel tiles w_ij = g_ij - ip
//   k_pair_direct  persistent pair-sum kernel over (curve, frequency-chunk)
//                  work units: the N(N-1)/2 interactions of Section 8 per
//                  trial frequency, FP32 with packed f32x2 arithmetic
//   k_topk         coarse-grid local maxima for the coarse-then-fine search
//                  (the bands method of Section 3.1 is in cp_bands.cu)
//   k_finalize     best frequency, nCKP and Table tab:th discriminator
#include <cstdint>
#include <map>
#include <mutex>
#include <utility>
#include <cuda_runtime.h>

#include "cp_internal.cuh"

namespace cpk {

// Table "tab:th" of Section 4.1: pSNR bin lower edges and thresholds.
__constant__ double c_bin_lo[8] = {0.0, 1.5, 2.0, 2.5, 3.5, 5.0, 10.0, 20.0};
__constant__ float c_th[8] = {0.4584f, 0.4565f, 0.4537f, 0.4581f, 0.5875f, 1.1153f, 1.6464f, 2.4112f};

// ===========================================================================
// k_stats: one CTA per curve.
// ===========================================================================

constexpr int kStatsThreads = 256;

__device__ __forceinline__ double median_sorted(const float* s, int n) { return median_of_sorted(s, n); }

// Quantile by linear interpolation between order statistics at q*(n-1).
__device__ __forceinline__ double quantile_sorted(const float* s, int n, double q)
{
    const double pos = q * (double)(n - 1);
    const int lo = (int)floor(pos);
    const int hi = lo + 1 < n ? lo + 1 : n - 1;
    return (double)s[lo] + (pos - (double)lo) * ((double)s[hi] - (double)s[lo]);
}

__device__ __forceinline__ int snr_bin(double p)
{
    int b = 0;
#pragma unroll
    for (int k = 0; k < 8; k++)
        if (p >= c_bin_lo[k]) b = k;
    return b;
}

__global__ void __launch_bounds__(kStatsThreads) k_stats(const StatsArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    double* ts = reinterpret_cast<double*>(smem);
    float* ys = reinterpret_cast<float*>(ts + a.np2max);
    float* es = ys + a.np2max;
    float* ypl = es + a.np2max;
    __shared__ double s_red[kStatsThreads / 32];
    __shared__ double s_t0;
    __shared__ float s_yref, s_gamma, s_iph, s_ipl;
    __shared__ int s_bad;

    const int c = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    CurveParams* P = a.cp + c;
    const int64_t off = P->off;
    const int n = P->n;
    int np2 = 1;
    while (np2 < n) np2 <<= 1;
    if (tid == 0) s_bad = 0;
    __syncthreads();

    // 1. load, validate, min t
    double tmin = INFINITY;
    for (int i = tid; i < np2; i += kStatsThreads) {
        if (i < n) {
            const double t = a.times[off + i];
            const float y = a.mags[off + i];
            const float e = a.errs[off + i];
            if (!isfinite(t) || !isfinite(y) || !isfinite(e)) s_bad = 1;
            ts[i] = t;
            ys[i] = y;
            es[i] = e;
            tmin = fmin(tmin, t);
        } else {
            ys[i] = INFINITY;
            es[i] = INFINITY;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tmin = fmin(tmin, __shfl_xor_sync(0xffffffffu, tmin, o));
    if (lane == 0) s_red[warp] = tmin;
    __syncthreads();
    if (tid == 0) {
        double m = s_red[0];
        for (int w = 1; w < kStatsThreads / 32; w++) m = fmin(m, s_red[w]);
        s_t0 = m;
    }

    // 2. bitonic sort of magnitudes and error bars (ascending)
    for (int k = 2; k <= np2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            __syncthreads();
            for (int i = tid; i < np2; i += kStatsThreads) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const bool up = (i & k) == 0;
                    float u = ys[i], v = ys[ixj];
                    if ((u > v) == up) { ys[i] = v; ys[ixj] = u; }
                    u = es[i]; v = es[ixj];
                    if ((u > v) == up) { es[i] = v; es[ixj] = u; }
                }
            }
        }
    }
    __syncthreads();

    // 3. per-curve scalars (FP64, one thread)
    if (tid == 0) {
        const double sy = median_sorted(es, n);
        const double yref = median_sorted(ys, n);
        const double q1 = quantile_sorted(ys, n, 0.25), q3 = quantile_sorted(ys, n, 0.75);
        const double psnr = 0.7413 * (q3 - q1) / ((double)a.alpha * sy);
        double st;
        if (a.sigma_t_mode == 1) {
            st = (double)a.sigma_t_per_curve[c];
        } else if (a.sigma_t_mode == 2) {
            st = sigma_t_rule(ys, n);
        } else {
            st = (double)a.sigma_t;
        }
        if (!(sy > 0.0) || !isfinite(sy) || !(st > 0.0) || !isfinite(st)) s_bad = 1;
        const float stf = (float)st;
        // the planned harmonic count no longer covers this sigma_t: the host re-plans
        if (stf < P->st_floor) atomicOr(a.status, 4);
        P->sigma_y = (float)sy;
        P->sigma_t = stf;
        P->psnr = (float)psnr;
        P->th = c_th[snr_bin(psnr)];
        P->t0 = s_t0;
        const double gamma = sqrt(1.4426950408889634 / (2.0 * sy * sy));
        s_yref = (float)yref;
        s_gamma = (float)gamma;
        P->gamma = (float)gamma;
        // sqrt(beta), beta = sqrt(2 log2 e) / sigma_t
        P->tscale = (float)sqrt(sqrt(2.0 * 1.4426950408889634) / (double)stf);
    }
    __syncthreads();

    // 4. scaled magnitudes y' = (y - y_ref) * gamma (same values feed IP and W)
    const float yref = s_yref, gamma = s_gamma;
    for (int i = tid; i < n; i += kStatsThreads) {
        const float v = (a.mags[off + i] - yref) * gamma;
        ypl[i] = v;
        a.yp[off + i] = v;
    }
    __syncthreads();

    // 5. IP: ip = (N + 2 sum_{i<j} g_ij) / N^2.  Each row is summed in FP32 with
    //    Kahan compensation (error ~1 ulp of the row sum, independent of its
    //    length) and the rows are accumulated in FP64; an FP64 add per pair
    //    would cost more than the rest of the kernel (2.3 DFMA/clk/SM).
    double acc = 0.0;
    for (int i = tid; i < n; i += kStatsThreads) {
        const float yi = ypl[i];
        float sum = 0.f, comp = 0.f;
        for (int j = i + 1; j < n; j++) {
            const float y = gauss_g(yi, ypl[j]) - comp;
            const float t = sum + y;
            comp = (t - sum) - y;
            sum = t;
        }
        acc += (double)sum - (double)comp;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __syncthreads();
    if (lane == 0) s_red[warp] = acc;
    __syncthreads();
    if (tid == 0) {
        double s2 = 0.0;
        for (int w = 0; w < kStatsThreads / 32; w++) s2 += s_red[w];
        const double nn = (double)n;
        const double ip = (nn + 2.0 * s2) / (nn * nn);
        const float iph = (float)ip;
        P->ip = ip;
        P->ip_hi = iph;
        P->ip_lo = (float)(ip - (double)iph);
        s_iph = iph;
        s_ipl = P->ip_lo;
        P->norm = (float)(sqrt(nn) / (nn * nn * ip * sqrt(2.0 * CP_PI) * sqrt((double)P->sigma_t)));
        P->diag = (float)(nn * (1.0 - ip));
        if (s_bad) atomicOr(a.status, 1);
    }

    // 5b. tensor form: per sample i, the sum over j of the rounding error of the
    //     16-bit operand w_ij = (g_ij - ip_hi) - ip_lo (the same FP32 values the
    //     tile builder rounds), and its total.  With these the tensor epilogue
    //     removes the error's coherent part: for a Z column x with mean xm the
    //     operand error adds xm^2 sum(dW) + 2 xm drho^T (x - xm), which does not
    //     average out where x is nearly constant over the samples (low f T, or
    //     aliases of the sampling).  Full rows in a fixed order: deterministic.
    if (a.wrho) {
        __syncthreads();
        const float iph = s_iph, ipl = s_ipl;
        const bool bf = a.wrho_bf16 != 0;
        double tot = 0.0;
        for (int i = tid; i < n; i += kStatsThreads) {
            const float yi = ypl[i];
            float sum = 0.f;
            for (int j = 0; j < n; j++) sum += w16_err((gauss_g(yi, ypl[j]) - iph) - ipl, bf);
            a.wrho[off + i] = sum;
            tot += (double)sum;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
        __syncthreads();
        if (lane == 0) s_red[warp] = tot;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < kStatsThreads / 32; w++) t += s_red[w];
            P->dwsum = (float)t;
        }
    }

    // 6. fixed-point phase steps of t - t0 for each grid the search uses
    const double t0 = s_t0;
    for (int i = tid; i < n; i += kStatsThreads) {
        const double tp = ts[i] - t0;
        a.ph_base[off + i] = fixfrac(a.f_min, tp);
        a.ph_full[off + i] = fixfrac(a.df, tp);
        if (a.hierarchical) {
            a.ph_coarse[off + i] = fixfrac(a.coarse_df, tp);
            a.ph_fine[off + i] = fixfrac(a.fine_df, tp);
        }
    }
}

// ===========================================================================
// k_sigma_t_rule: sigma_t of the skewness rule per curve (one CTA per curve),
// the same sort and the same FP64 arithmetic as k_stats.
// ===========================================================================
__global__ void __launch_bounds__(kStatsThreads) k_sigma_t_rule(const float* mags, const int64_t* offsets,
                                                               int np2max, float* out)
{
    extern __shared__ __align__(16) unsigned char smem[];
    float* ys = reinterpret_cast<float*>(smem);
    const int c = blockIdx.x, tid = threadIdx.x;
    const int64_t off = offsets[c];
    const int n = (int)(offsets[c + 1] - off);
    int np2 = 1;
    while (np2 < n) np2 <<= 1;
    for (int i = tid; i < np2; i += kStatsThreads) ys[i] = i < n ? mags[off + i] : INFINITY;
    for (int k = 2; k <= np2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            __syncthreads();
            for (int i = tid; i < np2; i += kStatsThreads) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const bool up = (i & k) == 0;
                    const float u = ys[i], v = ys[ixj];
                    if ((u > v) == up) { ys[i] = v; ys[ixj] = u; }
                }
            }
        }
    }
    __syncthreads();
    if (tid == 0) out[c] = (float)sigma_t_rule(ys, n);
}

// Curves with sigma_t at or above this take the exponent in the cos form (see
// pair_item); below it the sin form keeps the exponent's rounding relative.
constexpr float kCosFormMinSigma = 0.3f;

// ===========================================================================
// k_build_w: one warp per 32x32 tile of the upper block triangle.
// Layout per tile: [k][lane][m] floats, k < 8 rows, m < 4 columns per lane.
// ===========================================================================

__device__ __forceinline__ void decode_tile(int t, int nb, int& bi, int& bj)
{
    int b = 0, rem = t;
    while (rem >= nb - b) { rem -= nb - b; ++b; }
    bi = b;
    bj = b + rem;
}

__global__ void __launch_bounds__(256) k_build_w(const BuildWArgs a)
{
    const int lane = threadIdx.x & 31;
    const int64_t T = a.tile_begin + (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (T >= a.tile_end) return;
    int lo = a.slot_begin, hi = a.slot_end - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.wtile_start[mid] <= T) lo = mid; else hi = mid - 1;
    }
    const int c = a.order[lo];
    const CurveParams P = a.cp[c];
    const int n = P.n;
    const int nb = (n + kTile - 1) / kTile;
    int bi, bj;
    decode_tile((int)(T - a.wtile_start[lo]), nb, bi, bj);
    const int la = lane >> 3, lb = lane & 7;
    // cos-form curves: w carries the exponent's constant term, w 2^(-beta/2), so
    // that the pair kernel's exponent is the bare product sum (see pair_item)
    const float tsc = P.tscale * P.tscale * 0.70710678f;
    const float wscale = P.sigma_t >= kCosFormMinSigma ? exp2f(-(tsc * tsc)) : 1.0f;
    float ypc[kColsPerLane];
    int jj[kColsPerLane];
#pragma unroll
    for (int m = 0; m < kColsPerLane; m++) {
        jj[m] = bj * kTile + lb + 8 * m;
        ypc[m] = jj[m] < n ? a.yp[P.off + jj[m]] : 0.f;
    }
    float* dst = a.W + (T - a.tile_begin) * kTileFloats;
#pragma unroll
    for (int k = 0; k < kRowsPerLane; k++) {
        const int i = bi * kTile + la + 4 * k;
        const float ypr = i < n ? a.yp[P.off + i] : 0.f;
        float w[kColsPerLane];
#pragma unroll
        for (int m = 0; m < kColsPerLane; m++) {
            const float g = gauss_g(ypr, ypc[m]);
            w[m] = (i < jj[m] && jj[m] < n) ? ((g - P.ip_hi) - P.ip_lo) * wscale : 0.f;
        }
        reinterpret_cast<float4*>(dst)[k * 32 + lane] = make_float4(w[0], w[1], w[2], w[3]);
    }
}

// ===========================================================================
// k_pair_direct: persistent CTAs pop (curve, frequency-chunk) units.
// ===========================================================================
constexpr int kPairThreads = 512;
// Rows per lane in one warp work item: 8 = a whole 32 x 32 tile (each lane 8
// rows x 4 columns), 4 = half a tile.  Every trig value a lane loads from
// shared memory serves (rows x columns) / (rows + columns) evaluations, so the
// whole-tile item needs a third fewer shared-memory loads per evaluation.
constexpr int kItemRows = 8;
constexpr int kItemsPerTile = kRowsPerLane / kItemRows;
constexpr bool kPrefetchW = kItemRows == 4;   // next item's W in registers (the half-tile item only)
// The unit's trig table is built by one thread per (point, half of the
// frequency pairs): each point's phase and step are loaded twice per unit
// instead of once per frequency pair, and the threads' shares stay even
// (one thread per point leaves a few threads with twice the work).
constexpr int kTableGroups = 2;

// One work item (4 kItemRows rows x 32 columns of a tile) at every frequency
// pair of the unit.  The exponent of the periodic kernel (Eq. (periodickernel)),
// -beta sin^2(pi dphi) with beta = 2 log2(e) / sigma_t^2, is taken in one of
// two forms from the trig table of the unit:
//   sin form  -(c_i s_j - s_i c_j)^2 with (s, c) = (sin, cos)(pi phi) sqrt(beta)
//             (three f32x2 operations per two frequencies);
//   cos form  C_i C_j + S_i S_j - beta/2 with (S, C) = (sin, cos)(2 pi phi)
//             sqrt(beta/2), from sin^2 x = (1 - cos 2x)/2; the constant
//             2^(-beta/2) is carried by the tile's w (k_build_w), so the
//             exponent is the bare sum, a multiply and an FMA (two operations,
//             one of them with two operands).
// The cos form's rounding is absolute, about beta 2^-24 in the exponent, so it
// is used only for sigma_t >= kCosFormMinSigma (beta <= 32: below 3e-6 per term;
// the exponent then lies in [-beta/2, beta/2], within FP32 range).
template <bool COSF>
__device__ __forceinline__ void pair_item(const ulonglong2* SC, const f2* NS, int npad, int nfp, int rbase,
                                          int cbase, const f2 (&w01)[kItemRows],
                                          const f2 (&w23)[kItemRows], f2 (&acc)[kFcMax / 2])
{
#pragma unroll
    for (int fp = 0; fp < kFcMax / 2; fp++) {
        if (fp < nfp) {
            const ulonglong2* SCf = SC + fp * npad;
            const f2* NSf = NS + fp * npad;
            ulonglong2 col[kColsPerLane];
#pragma unroll
            for (int m = 0; m < kColsPerLane; m++) col[m] = SCf[cbase + 8 * m];
            f2 tf0 = 0ull, tf1 = 0ull, tg0 = 0ull, tg1 = 0ull;
#pragma unroll
            for (int k = 0; k < kItemRows; k++) {
                const int i = rbase + 4 * k;
                float e[kColsPerLane][2];
                if (COSF) {
                    const ulonglong2 R = SCf[i];   // ((S_i(f), S_i(f')), (C_i(f), C_i(f')))
#pragma unroll
                    for (int m = 0; m < kColsPerLane; m++) {
                        const f2 a2 = fma2(R.y, col[m].y, mul2(R.x, col[m].x));
                        float a0, a1;
                        upk(a2, a0, a1);
                        e[m][0] = ex2_approx(a0);
                        e[m][1] = ex2_approx(a1);
                    }
                } else {
                    const f2 A = SCf[i].y;   // (c_i(f), c_i(f'))
                    const f2 B = NSf[i];     // (-s_i(f), -s_i(f'))
#pragma unroll
                    for (int m = 0; m < kColsPerLane; m++) {
                        const f2 t2 = mul2(B, col[m].y);
                        const f2 d2 = fma2(A, col[m].x, t2);
                        const f2 q2 = mul2(d2, d2);
                        float q0, q1;
                        upk(q2, q0, q1);
                        e[m][0] = ex2_approx(-q0);
                        e[m][1] = ex2_approx(-q1);
                    }
                }
                tf0 = fma2(w01[k], pk(e[0][0], e[1][0]), tf0);
                tf1 = fma2(w23[k], pk(e[2][0], e[3][0]), tf1);
                tg0 = fma2(w01[k], pk(e[0][1], e[1][1]), tg0);
                tg1 = fma2(w23[k], pk(e[2][1], e[3][1]), tg1);
            }
            float fx, fy, gx, gy;
            upk(add2(tf0, tf1), fx, fy);
            upk(add2(tg0, tg1), gx, gy);
            acc[fp] = add2(acc[fp], pk(fx + fy, gx + gy));
        }
    }
}

__global__ void __launch_bounds__(kPairThreads, 1) k_pair_direct(const PairArgs a)
{
    constexpr int NW = kPairThreads / 32;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_unit;
    __shared__ float s_red[NW][kFcMax];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int la = lane >> 3, lb = lane & 7;

    for (;;) {
        __syncthreads();
        if (tid == 0) s_unit = (long long)atomicAdd(a.queue, 1ull) + a.unit_begin;
        __syncthreads();
        const long long u = s_unit;
        if (u >= a.unit_end) break;

        int lo = a.slot_begin, hi = a.slot_end - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.unit_start[mid] <= u) lo = mid; else hi = mid - 1;
        }
        const int slot = lo;
        const int c = a.order[slot];
        const CurveParams& P = a.cp[c];
        const int n = P.n, fc = P.fc, nfp = fc >> 1;
        const int npad = (n + kTile - 1) & ~(kTile - 1);
        const long long chunk = u - a.unit_start[slot];
        const int64_t off = P.off;

        // frequencies of this unit: phase(i, kk) = base_i + mult0 * step_i + kk * step_i
        long long kfirst;      // full/coarse: first grid index; fine: first j
        int count;
        int peak = 0;
        uint64_t peak_mult = 0;  // fine: coarse peak index (phase offset kpeak * coarse_i)
        if (a.stage == kStageFine) {
            const int W = 2 * a.fine_half + 1;
            const int upp = (W + fc - 1) / fc;
            peak = (int)(chunk / upp);
            const int sub = (int)(chunk - (long long)peak * upp);
            if (peak >= a.n_peaks[c]) continue;
            peak_mult = (uint64_t)a.peaks[(int64_t)c * a.top_k + peak];
            kfirst = -a.fine_half + (long long)sub * fc;
            count = (int)min((long long)fc, (long long)a.fine_half - kfirst + 1);
        } else if (a.stage == kStageList) {
            kfirst = chunk * fc;     // first list position
            count = (int)min((long long)fc, (long long)a.n_trials - kfirst);
        } else {
            kfirst = chunk * fc;
            count = (int)min((long long)fc, a.n_freq - kfirst);
        }
        const int32_t* tl = a.trials + (int64_t)c * a.n_trials;   // list stage only

        // trig table: SC[fp][i] = {(s_f, s_f'), (c_f, c_f')} * sqrt(beta), NS[fp][i] = -(s_f, s_f')
        // (sin form), or the sines and cosines of the doubled angle * sqrt(beta / 2) (cos form)
        ulonglong2* SC = reinterpret_cast<ulonglong2*>(smem);
        f2* NS = reinterpret_cast<f2*>(SC + nfp * npad);
        const bool cosf = P.sigma_t >= kCosFormMinSigma;
        const float ts = cosf ? P.tscale * P.tscale * 0.70710678f : P.tscale;   // tscale^4 = beta
        // One thread per (point, group of frequency pairs): the point's phase and
        // step are loaded once for the whole group, and the phase advances by two
        // grid steps per pair (exact in the 2^-64 fixed point).
        const int gsz = (nfp + kTableGroups - 1) / kTableGroups;
        for (int it = tid; it < kTableGroups * npad; it += kPairThreads) {
            const int gi = it / npad, i = it - gi * npad;
            const int fp0 = gi * gsz, fp1 = min(nfp, fp0 + gsz);
            if (i < n) {
                const uint64_t st = a.ph_step[off + i];
                const uint64_t base = a.ph_base[off + i];
                uint64_t ph = base + (uint64_t)(kfirst + 2 * fp0) * st;
                if (a.stage == kStageFine) ph += peak_mult * a.ph_coarse[off + i];
                for (int fp = fp0; fp < fp1; fp++, ph += 2 * st) {
                    uint64_t p0 = ph, p1 = ph + st;
                    if (a.stage == kStageList) {
                        // grid indices of list positions kfirst + 2 fp (+1); a missing entry evaluates k = 0
                        const long long q0 = kfirst + 2 * fp;
                        const int k0 = q0 < a.n_trials ? max(tl[q0], 0) : 0;
                        const int k1 = q0 + 1 < a.n_trials ? max(tl[q0 + 1], 0) : 0;
                        p0 = base + (uint64_t)k0 * st;
                        p1 = base + (uint64_t)k1 * st;
                    }
                    float s0, c0, s1, c1;
                    if (cosf) {
                        sincos2pi_turns((uint32_t)(p0 >> 32), s0, c0);
                        sincos2pi_turns((uint32_t)(p1 >> 32), s1, c1);
                    } else {
                        sincospi_turns((uint32_t)(p0 >> 32), s0, c0);
                        sincospi_turns((uint32_t)(p1 >> 32), s1, c1);
                    }
                    s0 *= ts; c0 *= ts; s1 *= ts; c1 *= ts;
                    SC[fp * npad + i] = make_ulonglong2(pk(s0, s1), pk(c0, c1));
                    if (!cosf) NS[fp * npad + i] = pk(-s0, -s1);   // the cos form reads SC only
                }
            } else {
                for (int fp = fp0; fp < fp1; fp++) {
                    SC[fp * npad + i] = make_ulonglong2(0ull, 0ull);
                    if (!cosf) NS[fp * npad + i] = 0ull;
                }
            }
        }
        __syncthreads();

        const int nb = npad / kTile;
        const int ntiles = nb * (nb + 1) / 2;
        const int nitems = kItemsPerTile * ntiles;   // (tile, row part): 4 kItemRows x 32 pairs per warp item
        const float4* Wc = reinterpret_cast<const float4*>(a.W + (a.wtile_start[slot] - a.wtile_base) * kTileFloats);
        f2 acc[kFcMax / 2];                      // per f-pair: (sum at f, sum at f')
#pragma unroll
        for (int q = 0; q < kFcMax / 2; q++) acc[q] = 0ull;

        // W of an item: rows (item % kItemsPerTile) * kItemRows + k of the stored tile
        auto w_ptr = [&](int it, int k) {
            return Wc + (int64_t)(it / kItemsPerTile) * (kTileFloats / 4) + ((it % kItemsPerTile) * kItemRows + k) * 32 + lane;
        };
        float4 wn[kPrefetchW ? kItemRows : 1];
        int item = warp;
        if (kPrefetchW && item < nitems) {
#pragma unroll
            for (int k = 0; k < kItemRows; k++) wn[k] = __ldg(w_ptr(item, k));
        }
#pragma unroll 1
        for (; item < nitems; item += NW) {
            f2 w01[kItemRows], w23[kItemRows];
#pragma unroll
            for (int k = 0; k < kItemRows; k++) {
                const float4 wv = kPrefetchW ? wn[k] : __ldg(w_ptr(item, k));
                w01[k] = pk(wv.x, wv.y);
                w23[k] = pk(wv.z, wv.w);
            }
            const int nxt = item + NW;
            if (kPrefetchW && nxt < nitems) {
#pragma unroll
                for (int k = 0; k < kItemRows; k++) wn[k] = __ldg(w_ptr(nxt, k));
            }
            int bi, bj;
            decode_tile(item / kItemsPerTile, nb, bi, bj);
            const int rbase = bi * kTile + (item % kItemsPerTile) * (4 * kItemRows) + la;
            const int cbase = bj * kTile + lb;
            if (cosf) pair_item<true>(SC, NS, npad, nfp, rbase, cbase, w01, w23, acc);
            else pair_item<false>(SC, NS, npad, nfp, rbase, cbase, w01, w23, acc);
        }

        // warp reduction of the 2*nfp frequency sums, then a fixed-order CTA sum
#pragma unroll
        for (int fp = 0; fp < kFcMax / 2; fp++) {
            if (fp < nfp) {
                float vf, vg;
                upk(acc[fp], vf, vg);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    vf += __shfl_xor_sync(0xffffffffu, vf, o);
                    vg += __shfl_xor_sync(0xffffffffu, vg, o);
                }
                if (lane == 0) {
                    s_red[warp][2 * fp] = vf;
                    s_red[warp][2 * fp + 1] = vg;
                }
            }
        }
        __syncthreads();
        if (warp == 0) {
            unsigned long long key = 0ull;
            if (lane < count) {
                float S = 0.f;
#pragma unroll
                for (int w = 0; w < NW; w++) S += s_red[w][lane];
                const float v = (2.0f * S + P.diag) * P.norm;
                const long long kk = kfirst + lane;
                if (a.stage == kStageFull) {
                    if (a.out) a.out[(int64_t)c * a.out_ld + kk] = v;
                    if (!excluded_k(a.ex.full_k, a.ex.n, kk)) key = make_key(v, (uint32_t)kk);
                } else if (a.stage == kStageCoarse) {
                    a.coarse_out[(int64_t)c * a.n_freq + kk] = v;
                } else if (a.stage == kStageList) {
                    const bool valid = tl[kk] >= 0;
                    if (a.trial_stat) a.trial_stat[(int64_t)c * a.n_trials + kk] = valid ? v : __int_as_float(0x7fc00000);
                    if (valid && !excluded_k(a.ex.full_k, a.ex.n, tl[kk])) key = make_key(v, (uint32_t)kk);
                } else {
                    const double fpk = grid_freq(a.f_min, (double)peak_mult, a.coarse_df);
                    const double f = grid_freq(fpk, (double)kk, a.step);
                    if (f >= a.f_min && f <= a.f_max && !excluded_f(a.ex, f))
                        key = make_key(v, (uint32_t)(peak * (2 * a.fine_half + 1) + (kk + a.fine_half)));
                }
            }
            if (a.stage != kStageCoarse) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const unsigned long long other = __shfl_xor_sync(0xffffffffu, key, o);
                    key = other > key ? other : key;
                }
                if (lane == 0 && key) atomicMax(a.best_key + c, key);
            }
        }
    }
}

// ===========================================================================
// k_topk: one warp per curve, top_k local maxima of the coarse periodogram.
// Local maximum: v[k] > v[k-1] and v[k] >= v[k+1]; ends use one neighbour.
// Order: value descending, ties to the lower k (larger key).
// ===========================================================================

__global__ void __launch_bounds__(256) k_topk(const TopkArgs a)
{
    const int lane = threadIdx.x & 31;
    const int slot = a.slot_begin + blockIdx.x * 8 + (threadIdx.x >> 5);
    if (slot >= a.slot_end) return;
    const int c = a.order[slot];
    const float* v = a.coarse + (int64_t)c * a.n_freq;
    const int64_t K = a.n_freq;
    unsigned long long prev = ~0ull;
    int cnt = 0;
    for (int r = 0; r < a.top_k; r++) {
        unsigned long long best = 0ull;
        for (int64_t k = lane; k < K; k += 32) {
            const float x = v[k];
            const bool lok = (k == 0) || (x > v[k - 1]);
            const bool rok = (k == K - 1) || (x >= v[k + 1]);
            if (lok && rok && !excluded_k(a.ex.coarse_k, a.ex.n, k)) {
                const unsigned long long key = make_key(x, (uint32_t)k);
                if (key < prev && key > best) best = key;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long other = __shfl_xor_sync(0xffffffffu, best, o);
            best = other > best ? other : best;
        }
        if (best == 0ull) break;
        if (lane == 0) a.peaks[(int64_t)c * a.top_k + r] = (int32_t)(0xffffffffu - (uint32_t)(best & 0xffffffffu));
        prev = best;
        cnt++;
    }
    if (lane == 0) a.n_peaks[c] = cnt;
}

// ===========================================================================
// k_finalize: decode the best keys, apply the discriminator.
// ===========================================================================

__global__ void k_finalize(const FinalArgs a)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= a.n_curves) return;
    const unsigned long long key = a.best_key[c];
    if (key == 0ull) {   // no admissible candidate (cannot happen for valid grids)
        a.best_idx[c] = -1;
        a.best_freq[c] = __longlong_as_double(0x7ff8000000000000ll);
        a.best_stat[c] = __int_as_float(0x7fc00000);
        a.is_periodic[c] = 0;
        a.psnr[c] = a.cp[c].psnr;
        return;
    }
    const float v = from_orderable((uint32_t)(key >> 32));
    const uint32_t idx = 0xffffffffu - (uint32_t)(key & 0xffffffffu);
    double f;
    uint32_t kout = idx;
    if (a.hierarchical == CP_SEARCH_BANDS) {
        kout = (uint32_t)a.trials[(int64_t)c * a.n_trials + idx];   // list position -> grid index
        f = __dadd_rn(a.f_min, __dmul_rn((double)kout, a.df));
    } else if (a.hierarchical) {
        const int W = 2 * a.fine_half + 1;
        const int p = (int)(idx / (uint32_t)W);
        const int j = (int)(idx % (uint32_t)W) - a.fine_half;
        const double fpk = __dadd_rn(a.f_min, __dmul_rn((double)a.peaks[(int64_t)c * a.top_k + p], a.coarse_df));
        f = __dadd_rn(fpk, __dmul_rn((double)j, a.fine_df));
    } else {
        f = __dadd_rn(a.f_min, __dmul_rn((double)idx, a.df));
    }
    a.best_idx[c] = (int64_t)kout;
    a.best_freq[c] = f;
    a.best_stat[c] = v;
    a.is_periodic[c] = v > a.cp[c].th ? 1 : 0;
    a.psnr[c] = a.cp[c].psnr;
}

__global__ void k_zero_u64(unsigned long long* p, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = 0ull;
}

}  // namespace cpk

// ---------------------------------------------------------------------------
// Launchers used by the host API (C++ linkage, internal to the library).
// ---------------------------------------------------------------------------
namespace cpk {

cudaError_t launch_stats(const StatsArgs& a, int n_curves, cudaStream_t s)
{
    const size_t smem = stats_smem_bytes(a.np2max);
    k_stats<<<n_curves, kStatsThreads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_sigma_t_rule(const float* mags, const int64_t* offsets, int n_curves, int np2max, float* out,
                                cudaStream_t s)
{
    const size_t smem = (size_t)np2max * sizeof(float);
    cudaError_t e = raise_dyn_smem((const void*)k_sigma_t_rule, smem);
    if (e != cudaSuccess) return e;
    k_sigma_t_rule<<<n_curves, kStatsThreads, smem, s>>>(mags, offsets, np2max, out);
    return cudaGetLastError();
}

cudaError_t launch_build_w(const BuildWArgs& a, cudaStream_t s)
{
    const int64_t tiles = a.tile_end - a.tile_begin;
    if (tiles <= 0) return cudaSuccess;
    k_build_w<<<(unsigned)((tiles + 7) / 8), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_pair_direct(const PairArgs& a, int grid, size_t smem, cudaStream_t s)
{
    k_pair_direct<<<grid, kPairThreads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_topk(const TopkArgs& a, cudaStream_t s)
{
    const int n = a.slot_end - a.slot_begin;
    if (n <= 0) return cudaSuccess;
    k_topk<<<(n + 7) / 8, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const FinalArgs& a, cudaStream_t s)
{
    k_finalize<<<(a.n_curves + 255) / 256, 256, 0, s>>>(a);
    return cudaGetLastError();
}

int pair_direct_threads() { return kPairThreads; }

size_t stats_smem_bytes(int np2max) { return (size_t)np2max * (sizeof(double) + 3 * sizeof(float)); }

namespace {
std::mutex g_smem_mutex;
std::map<std::pair<const void*, int>, size_t> g_smem_limit;   // (kernel, device) -> limit set
}  // namespace

cudaError_t raise_dyn_smem(const void* func, size_t bytes)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_smem_mutex);
    size_t& cur = g_smem_limit[std::make_pair(func, dev)];
    if (bytes <= cur) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) cur = bytes;
    return e;
}

cudaError_t prepare_kernels(int np2max, size_t pair_smem)
{
    cudaError_t e = raise_dyn_smem((const void*)k_stats, stats_smem_bytes(np2max));
    if (e != cudaSuccess) return e;
    return raise_dyn_smem((const void*)k_pair_direct, pair_smem);
}

cudaError_t pair_direct_occupancy(int* blocks_per_sm, size_t smem)
{
    cudaError_t e = raise_dyn_smem((const void*)k_pair_direct, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_pair_direct, kPairThreads, smem);
}

cudaError_t launch_zero_u64(unsigned long long* p, int64_t n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_zero_u64<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, n);
    return cudaGetLastError();
}

}  // namespace cpk
