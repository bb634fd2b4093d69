// cp_prep.cu -- per-curve transforms around the periodogram search
// (arXiv:1412.1840):
//
//   cp_preprocess  Section 5.2: drop samples whose error bar is not below
//                  mean(e) + 3 std(e) (population std), discard curves with
//                  fewer than min_n samples left, fit x = a0 + a1 t by the
//                  weighted linear chi^2 of Eq. (chisquare) and subtract the
//                  fit when the Pearson correlation between the magnitudes and
//                  the fit exceeds 0.5.  The kept samples keep their order.
//   cp_whiten      Section 7.1 (multimodes): fold each curve at its P0
//                  (phase = frac(t / P0), equal phases by sample index),
//                  smooth the folded curve by a circular moving average of
//                  w = min(window, N) samples (folded positions k - w/2 ..
//                  k - w/2 + w - 1), subtract that template and return the
//                  samples in their original order.
//
// One CTA per curve; every sum is FP64 in a fixed order.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "cp.h"
#include "cp_internal.cuh"

namespace cpk {

constexpr int kPrepThreads = 256;

struct PrepStats {
    int64_t n_out;
    int32_t kept, detrended;
    double a0, a1, r;
};

// Fixed-order block sum of one double per thread (all threads call it).
__device__ double block_sum(double v, double* s_red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) s_red[warp] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < kPrepThreads / 32; w++) t += s_red[w];
    return t;
}

__global__ void __launch_bounds__(kPrepThreads) k_prep_stats(const double* times, const float* mags,
                                                             const float* errs, const int64_t* offsets,
                                                             int min_n, PrepStats* out)
{
    __shared__ double s_red[kPrepThreads / 32];
    const int c = blockIdx.x, tid = threadIdx.x;
    const int64_t off = offsets[c];
    const int n = (int)(offsets[c + 1] - off);

    // error-bar cut: e_i < mean + 3 std (population)
    double s = 0.0;
    for (int i = tid; i < n; i += kPrepThreads) s += (double)errs[off + i];
    const double mean = block_sum(s, s_red) / (double)n;
    s = 0.0;
    for (int i = tid; i < n; i += kPrepThreads) {
        const double d = (double)errs[off + i] - mean;
        s += d * d;
    }
    const double cut = mean + 3.0 * sqrt(block_sum(s, s_red) / (double)n);

    // weighted chi^2 sums over the kept samples (weights 1 / e^2)
    double cnt = 0, S = 0, St = 0, Sx = 0, Stt = 0, Stx = 0;
    for (int i = tid; i < n; i += kPrepThreads) {
        const double e = (double)errs[off + i];
        if (!(e < cut)) continue;
        const double t = times[off + i], x = (double)mags[off + i], w = 1.0 / (e * e);
        cnt += 1.0;
        S += w;
        St += w * t;
        Sx += w * x;
        Stt += w * t * t;
        Stx += w * t * x;
    }
    cnt = block_sum(cnt, s_red);
    S = block_sum(S, s_red);
    St = block_sum(St, s_red);
    Sx = block_sum(Sx, s_red);
    Stt = block_sum(Stt, s_red);
    Stx = block_sum(Stx, s_red);
    const int64_t k = (int64_t)cnt;
    double a0 = 0.0, a1 = 0.0, r = 0.0;
    if (k >= 2) {
        const double det = S * Stt - St * St;
        a1 = (S * Stx - St * Sx) / det;
        a0 = (Stt * Sx - St * Stx) / det;
        // Pearson correlation of the kept magnitudes with the fit
        double mx = 0, mf = 0;
        for (int i = tid; i < n; i += kPrepThreads) {
            if (!((double)errs[off + i] < cut)) continue;
            mx += (double)mags[off + i];
            mf += a0 + a1 * times[off + i];
        }
        mx = block_sum(mx, s_red) / (double)k;
        mf = block_sum(mf, s_red) / (double)k;
        double sxf = 0, sxx = 0, sff = 0;
        for (int i = tid; i < n; i += kPrepThreads) {
            if (!((double)errs[off + i] < cut)) continue;
            const double dx = (double)mags[off + i] - mx, df = (a0 + a1 * times[off + i]) - mf;
            sxf += dx * df;
            sxx += dx * dx;
            sff += df * df;
        }
        sxf = block_sum(sxf, s_red);
        sxx = block_sum(sxx, s_red);
        sff = block_sum(sff, s_red);
        r = (sxx == 0.0 || sff == 0.0) ? 0.0 : sxf / sqrt(sxx * sff);
    }
    if (tid == 0) {
        PrepStats p;
        p.n_out = k;
        p.kept = k >= min_n;
        p.detrended = r > 0.5;
        p.a0 = a0;
        p.a1 = a1;
        p.r = r;
        out[c] = p;
        // the cut itself is recomputed by the compaction kernel from the same sums
    }
}

// Order-preserving compaction of the kept samples, fit removed where flagged.
__global__ void __launch_bounds__(kPrepThreads) k_prep_compact(const double* times, const float* mags,
                                                               const float* errs, const int64_t* offsets,
                                                               const PrepStats* st, const int64_t* out_off,
                                                               double* out_t, float* out_x, float* out_e)
{
    __shared__ double s_red[kPrepThreads / 32];
    __shared__ int s_wsum[kPrepThreads / 32];
    const int c = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const PrepStats P = st[c];
    if (!P.kept) return;
    const int64_t off = offsets[c];
    const int n = (int)(offsets[c + 1] - off);
    // the same cut as k_prep_stats (same sums in the same order)
    double s = 0.0;
    for (int i = tid; i < n; i += kPrepThreads) s += (double)errs[off + i];
    const double mean = block_sum(s, s_red) / (double)n;
    s = 0.0;
    for (int i = tid; i < n; i += kPrepThreads) {
        const double d = (double)errs[off + i] - mean;
        s += d * d;
    }
    const double cut = mean + 3.0 * sqrt(block_sum(s, s_red) / (double)n);
    const int64_t o = out_off[c];
    int written = 0;
    for (int i0 = 0; i0 < n; i0 += kPrepThreads) {
        const int i = i0 + tid;
        const bool keep = i < n && (double)errs[off + i] < cut;
        const uint32_t bal = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) s_wsum[warp] = __popc(bal);
        __syncthreads();
        int before = written, chunk = 0;
        for (int w = 0; w < kPrepThreads / 32; w++) {
            if (w < warp) before += s_wsum[w];
            chunk += s_wsum[w];
        }
        if (keep) {
            const int64_t pos = o + before + __popc(bal & ((1u << lane) - 1u));
            const double t = times[off + i];
            double x = (double)mags[off + i];
            if (P.detrended) x -= P.a0 + P.a1 * t;
            out_t[pos] = t;
            out_x[pos] = (float)x;
            out_e[pos] = errs[off + i];
        }
        written += chunk;
        __syncthreads();
    }
}

// Whitening: bitonic sort of (phase, sample) pairs, circular moving average
// from FP64 prefix sums, subtraction, scatter back to the sample positions.
__global__ void __launch_bounds__(kPrepThreads) k_whiten(const double* times, const float* mags,
                                                         const int64_t* offsets, const double* p0, int window,
                                                         int np2max, float* out)
{
    extern __shared__ __align__(16) unsigned char smem[];
    double* ph = reinterpret_cast<double*>(smem);             // np2max
    double* pre = ph + np2max;                                // np2max + 1 prefix sums (folded order)
    int32_t* idx = reinterpret_cast<int32_t*>(pre + np2max + 1);
    const int c = blockIdx.x, tid = threadIdx.x;
    const int64_t off = offsets[c];
    const int n = (int)(offsets[c + 1] - off);
    const double P = p0[c];
    if (!(P > 0.0) || !isfinite(P)) {
        for (int i = tid; i < n; i += kPrepThreads) out[off + i] = mags[off + i];
        return;
    }
    int np2 = 1;
    while (np2 < n) np2 <<= 1;
    for (int i = tid; i < np2; i += kPrepThreads) {
        if (i < n) {
            const double q = times[off + i] / P;
            ph[i] = q - floor(q);
        } else {
            ph[i] = INFINITY;
        }
        idx[i] = i;
    }
    // ascending by (phase, sample index)
    for (int k = 2; k <= np2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            __syncthreads();
            for (int i = tid; i < np2; i += kPrepThreads) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const bool up = (i & k) == 0;
                    const double u = ph[i], v = ph[ixj];
                    const int iu = idx[i], iv = idx[ixj];
                    const bool greater = u > v || (u == v && iu > iv);
                    if (greater == up) {
                        ph[i] = v; ph[ixj] = u;
                        idx[i] = iv; idx[ixj] = iu;
                    }
                }
            }
        }
    }
    __syncthreads();
    // prefix sums of the folded magnitudes (one thread per 64-sample block, then block offsets)
    constexpr int kSeg = 64;
    const int nseg = (n + kSeg - 1) / kSeg;
    for (int sgi = tid; sgi < nseg; sgi += kPrepThreads) {
        double acc = 0.0;
        for (int k = sgi * kSeg; k < min(n, (sgi + 1) * kSeg); k++) {
            acc += (double)mags[off + idx[k]];
            pre[k + 1] = acc;
        }
    }
    __syncthreads();
    if (tid == 0) {
        pre[0] = 0.0;
        double carry = 0.0;
        for (int sgi = 0; sgi < nseg; sgi++) {
            const int end = min(n, (sgi + 1) * kSeg);
            const double seg_total = pre[end];
            for (int k = sgi * kSeg + 1; k <= end; k++) pre[k] += carry;
            carry += seg_total;
        }
    }
    __syncthreads();
    const int w = window < n ? window : n;
    const double total = pre[n];
    for (int k = tid; k < n; k += kPrepThreads) {
        // folded positions k - w/2 .. k - w/2 + w - 1, circular
        int a = k - w / 2, b = a + w;                          // [a, b)
        double sum;
        if (a >= 0 && b <= n) {
            sum = pre[b] - pre[a];
        } else if (a < 0) {
            sum = pre[b] + (total - pre[n + a]);
        } else {
            sum = (total - pre[a]) + pre[b - n];
        }
        const int i = idx[k];
        out[off + i] = (float)((double)mags[off + i] - sum / (double)w);
    }
}

size_t whiten_smem_bytes(int np2max) { return (size_t)np2max * 8 + (size_t)(np2max + 1) * 8 + (size_t)np2max * 4; }

}  // namespace cpk

using namespace cpk;

namespace {

cp_status pfail(cp_status s, const std::string& m) { return cpk::set_error(s, m.c_str()); }

#define PREP_CUDA(call)                                                                 \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            cudaGetLastError();                                                         \
            st = pfail(e_ == cudaErrorMemoryAllocation ? CP_ENOMEM : CP_ECUDA,          \
                       std::string(#call) + ": " + cudaGetErrorString(e_));             \
            goto done;                                                                  \
        }                                                                               \
    } while (0)

cp_status check_csr(const int64_t* offsets, int64_t n_curves, int min_size, const char* who)
{
    if (!offsets) return pfail(CP_EINVAL, std::string(who) + ": null offsets");
    if (n_curves < 1 || n_curves > ((int64_t)1 << 30)) return pfail(CP_EINVAL, std::string(who) + ": bad n_curves");
    if (offsets[0] != 0) return pfail(CP_EINVAL, std::string(who) + ": offsets[0] must be 0");
    for (int64_t c = 0; c < n_curves; c++) {
        const int64_t n = offsets[c + 1] - offsets[c];
        if (n < min_size) return pfail(CP_EINVAL, std::string(who) + ": curve " + std::to_string(c) + " is too short");
        if (n > kMaxN) return pfail(CP_EUNSUPPORTED, std::string(who) + ": curve " + std::to_string(c) + " exceeds cp_max_points()");
    }
    return CP_OK;
}

bool on_device(const void* p)
{
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" cp_status cp_preprocess(const double* times, const float* mags, const float* errs, const int64_t* offsets,
                                   int64_t n_curves, int32_t min_n, double* out_times, float* out_mags,
                                   float* out_errs, int64_t* out_offsets, uint8_t* flags, double* fit,
                                   void* cuda_stream)
{
    if (!times || !mags || !errs || !out_times || !out_mags || !out_errs || !out_offsets)
        return pfail(CP_EINVAL, "cp_preprocess: null argument");
    if (min_n < 1) return pfail(CP_EINVAL, "cp_preprocess: min_n must be >= 1");
    cp_status st = check_csr(offsets, n_curves, 1, "cp_preprocess");
    if (st != CP_OK) return st;
    for (const void* p : {(const void*)times, (const void*)mags, (const void*)errs, (const void*)out_times,
                          (const void*)out_mags, (const void*)out_errs})
        if (!on_device(p)) return pfail(CP_EINVAL, "cp_preprocess: inputs and outputs must be device memory");
    const cudaStream_t s = (cudaStream_t)cuda_stream;
    const int64_t nc = n_curves;
    int64_t* d_off = nullptr;
    int64_t* d_oout = nullptr;
    PrepStats* d_st = nullptr;
    std::vector<PrepStats> h_st((size_t)nc);
    PREP_CUDA(cudaMalloc(&d_off, (nc + 1) * sizeof(int64_t)));
    PREP_CUDA(cudaMalloc(&d_oout, (nc + 1) * sizeof(int64_t)));
    PREP_CUDA(cudaMalloc(&d_st, nc * sizeof(PrepStats)));
    PREP_CUDA(cudaMemcpyAsync(d_off, offsets, (nc + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    k_prep_stats<<<(unsigned)nc, kPrepThreads, 0, s>>>(times, mags, errs, d_off, min_n, d_st);
    PREP_CUDA(cudaGetLastError());
    PREP_CUDA(cudaMemcpyAsync(h_st.data(), d_st, nc * sizeof(PrepStats), cudaMemcpyDeviceToHost, s));
    PREP_CUDA(cudaStreamSynchronize(s));
    out_offsets[0] = 0;
    for (int64_t c = 0; c < nc; c++) {
        out_offsets[c + 1] = out_offsets[c] + (h_st[c].kept ? h_st[c].n_out : 0);
        if (flags) flags[c] = (uint8_t)((h_st[c].kept ? 1 : 0) | (h_st[c].kept && h_st[c].detrended ? 2 : 0));
        if (fit) {
            fit[3 * c] = h_st[c].a0;
            fit[3 * c + 1] = h_st[c].a1;
            fit[3 * c + 2] = h_st[c].r;
        }
    }
    PREP_CUDA(cudaMemcpyAsync(d_oout, out_offsets, (nc + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    k_prep_compact<<<(unsigned)nc, kPrepThreads, 0, s>>>(times, mags, errs, d_off, d_st, d_oout, out_times,
                                                         out_mags, out_errs);
    PREP_CUDA(cudaGetLastError());
    PREP_CUDA(cudaStreamSynchronize(s));
done:
    cudaFree(d_off);
    cudaFree(d_oout);
    cudaFree(d_st);
    return st;
}

extern "C" cp_status cp_whiten(const double* times, const float* mags, const int64_t* offsets, int64_t n_curves,
                               const double* p0, int32_t window, float* out_mags, void* cuda_stream)
{
    if (!times || !mags || !p0 || !out_mags) return pfail(CP_EINVAL, "cp_whiten: null argument");
    if (window < 1) return pfail(CP_EINVAL, "cp_whiten: window must be >= 1");
    cp_status st = check_csr(offsets, n_curves, 1, "cp_whiten");
    if (st != CP_OK) return st;
    for (const void* p : {(const void*)times, (const void*)mags, (const void*)out_mags})
        if (!on_device(p)) return pfail(CP_EINVAL, "cp_whiten: times, mags and out_mags must be device memory");
    const cudaStream_t s = (cudaStream_t)cuda_stream;
    const int64_t nc = n_curves;
    int max_n = 1;
    for (int64_t c = 0; c < nc; c++) max_n = std::max(max_n, (int)(offsets[c + 1] - offsets[c]));
    int np2 = 1;
    while (np2 < max_n) np2 <<= 1;
    const size_t smem = whiten_smem_bytes(np2);
    int64_t* d_off = nullptr;
    double* d_p0 = nullptr;
    PREP_CUDA(cudaMalloc(&d_off, (nc + 1) * sizeof(int64_t)));
    PREP_CUDA(cudaMalloc(&d_p0, nc * sizeof(double)));
    PREP_CUDA(cudaMemcpyAsync(d_off, offsets, (nc + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    PREP_CUDA(cudaMemcpyAsync(d_p0, p0, nc * sizeof(double), cudaMemcpyHostToDevice, s));
    PREP_CUDA(raise_dyn_smem((const void*)k_whiten, smem));
    k_whiten<<<(unsigned)nc, kPrepThreads, smem, s>>>(times, mags, d_off, d_p0, window, np2, out_mags);
    PREP_CUDA(cudaGetLastError());
    PREP_CUDA(cudaStreamSynchronize(s));
done:
    cudaFree(d_off);
    cudaFree(d_p0);
    return st;
}
