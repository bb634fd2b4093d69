// cp_peaks.cu -- instruction-rate probes of the pipes the pair kernels are
// bound by (measurement tool of the package, not part of the method).
//
// Each probe runs register-only dependency chains (eight independent chains
// per thread, 1,024 threads per SM, one CTA per SM) for a given number of
// iterations and reports the operations executed.  The caller times the
// launch; the kernel also reads clock64 and %globaltimer at its first and
// last instruction in every CTA, which gives the SM clock during the run.
//
//   kind 0  MUFU ex2.approx.f32, x <- ex2(x)               (1 op / instruction)
//   kind 1  MUFU ex2.approx.f32, x <- ex2(-x)              (1 op / instruction)
//   kind 2  FP32 FFMA, x <- x a + b                        (1 lane-op / instruction)
//   kind 3  packed f32x2 FFMA2                             (2 lane-ops / instruction)
//   kind 4  FP64 DFMA                                      (1 op / instruction)
//   kind 5  the direct form's sin-form pair term: per two evaluations one
//           f32x2 multiply, FMA, multiply, two MUFU ex2, one f32x2 FMA
//           (counts evaluations: ops = pair-frequency evaluations)
//   kind 6  the cos-form pair term: two f32x2 FMAs, two MUFU ex2, one f32x2 FMA
//   kind 7  MUFU ex2.approx.f16x2                          (2 ops / instruction)
//   kind 8  tcgen05.mma kind::f16, M = 128, N = 256, K = 16, FP16 operands
//           from shared memory, FP32 accumulation in TMEM, issued back to back
//           by one thread per CTA (ops = flops, 2 M N K per instruction)
//
// The MMA probe's only wait (for its last MMAs) is bounded: after the limit it
// reports a timeout instead of spinning on.
#include <cstdint>
#include <cuda_runtime.h>

#include "../cp_tc.cuh"

namespace {

using namespace cpk::tc;

constexpr int kThreads = 1024;
constexpr int kChains = 8;

__device__ __forceinline__ float ex2f(float x)
{
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ uint32_t ex2h2(uint32_t x)
{
    uint32_t y;
    asm volatile("ex2.approx.f16x2 %0, %1;" : "=r"(y) : "r"(x));
    return y;
}
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
    asm volatile("mul.rn.ftz.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c)
{
    f2 d;
    asm volatile("fma.rn.ftz.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

struct ProbeOut {
    unsigned long long clk0, clk1, ns0, ns1;
};

__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <int KIND>
__global__ void __launch_bounds__(kThreads, 1) k_probe(long long iters, float seed, float* sink, ProbeOut* out)
{
    unsigned long long c0 = 0, t0 = 0;
    if (threadIdx.x == 0) {
        t0 = globaltimer();
        c0 = clock64();
    }
    const float s = seed + 1e-3f * (float)(threadIdx.x & 31);
    float acc = 0.f;
    if (KIND == 0 || KIND == 1) {
        float x[kChains];
#pragma unroll
        for (int k = 0; k < kChains; k++) x[k] = s * (float)(k + 1);
        for (long long it = 0; it < iters; it++) {
#pragma unroll
            for (int u = 0; u < 16; u++)
#pragma unroll
                for (int k = 0; k < kChains; k++) x[k] = ex2f(KIND == 1 ? -x[k] : x[k]);
        }
#pragma unroll
        for (int k = 0; k < kChains; k++) acc += x[k];
    } else if (KIND == 2) {
        float x[kChains];
#pragma unroll
        for (int k = 0; k < kChains; k++) x[k] = s * (float)(k + 1);
        const float a = 0.999f, b = 1e-3f * s;
        for (long long it = 0; it < iters; it++) {
#pragma unroll
            for (int u = 0; u < 16; u++)
#pragma unroll
                for (int k = 0; k < kChains; k++) x[k] = fmaf(x[k], a, b);
        }
#pragma unroll
        for (int k = 0; k < kChains; k++) acc += x[k];
    } else if (KIND == 3) {
        f2 x[kChains];
#pragma unroll
        for (int k = 0; k < kChains; k++) x[k] = pk(s * (float)(k + 1), s * (float)(k + 2));
        const f2 a = pk(0.999f, 0.998f), b = pk(1e-3f * s, 2e-3f * s);
        for (long long it = 0; it < iters; it++) {
#pragma unroll
            for (int u = 0; u < 16; u++)
#pragma unroll
                for (int k = 0; k < kChains; k++) x[k] = fma2(x[k], a, b);
        }
#pragma unroll
        for (int k = 0; k < kChains; k++) {
            float lo, hi;
            upk(x[k], lo, hi);
            acc += lo + hi;
        }
    } else if (KIND == 4) {
        double x[kChains];
#pragma unroll
        for (int k = 0; k < kChains; k++) x[k] = (double)s * (k + 1);
        const double a = 0.999, b = 1e-3 * (double)s;
        for (long long it = 0; it < iters; it++) {
#pragma unroll
            for (int u = 0; u < 16; u++)
#pragma unroll
                for (int k = 0; k < kChains; k++) x[k] = fma(x[k], a, b);
        }
#pragma unroll
        for (int k = 0; k < kChains; k++) acc += (float)x[k];
    } else if (KIND == 5 || KIND == 6) {
        // chain k: (c, c') in f32x2; each step evaluates two pair terms and feeds
        // the exponentials back as the next step's column values
        f2 c[kChains], ac[kChains];
        const f2 A = pk(0.7f, 0.6f), B = pk(-0.5f, -0.4f), W = pk(0.01f, 0.02f), H = pk(-3.0f, -2.5f);
#pragma unroll
        for (int k = 0; k < kChains; k++) {
            c[k] = pk(s * 0.1f * (k + 1), s * 0.1f * (k + 2));
            ac[k] = 0ull;
        }
        for (long long it = 0; it < iters; it++) {
#pragma unroll
            for (int u = 0; u < 8; u++)
#pragma unroll
                for (int k = 0; k < kChains; k++) {
                    float e0, e1;
                    if (KIND == 5) {
                        const f2 t = mul2(B, c[k]);
                        const f2 d = fma2(A, c[k], t);
                        const f2 q = mul2(d, d);
                        float q0, q1;
                        upk(q, q0, q1);
                        e0 = ex2f(-q0);
                        e1 = ex2f(-q1);
                    } else {
                        const f2 a2 = fma2(A, c[k], fma2(B, c[k], H));
                        float a0, a1;
                        upk(a2, a0, a1);
                        e0 = ex2f(a0);
                        e1 = ex2f(a1);
                    }
                    const f2 e = pk(e0, e1);
                    ac[k] = fma2(W, e, ac[k]);
                    c[k] = e;
                }
        }
#pragma unroll
        for (int k = 0; k < kChains; k++) {
            float lo, hi;
            upk(ac[k], lo, hi);
            acc += lo + hi;
        }
    } else if (KIND == 7) {
        uint32_t x[kChains];
#pragma unroll
        for (int k = 0; k < kChains; k++) x[k] = 0x3c003c00u ^ (uint32_t)(k + threadIdx.x);
        for (long long it = 0; it < iters; it++) {
#pragma unroll
            for (int u = 0; u < 16; u++)
#pragma unroll
                for (int k = 0; k < kChains; k++) x[k] = ex2h2(x[k]);
        }
#pragma unroll
        for (int k = 0; k < kChains; k++) acc += (float)(x[k] & 0xffu);
    }
    if (acc == 1234.5f) sink[blockIdx.x * blockDim.x + threadIdx.x] = acc;   // keeps the chains live
    __syncthreads();
    if (threadIdx.x == 0) {
        out[blockIdx.x].clk1 = clock64();
        out[blockIdx.x].ns1 = globaltimer();
        out[blockIdx.x].clk0 = c0;
        out[blockIdx.x].ns0 = t0;
    }
}

// tcgen05 MMA issue rate: A (128 x 64) and B (256 x 64) FP16 tiles of zeros in
// shared memory, K-major 128-byte swizzle; iters x 4 MMAs of K = 16 into one of
// two TMEM accumulators (alternating per K = 64 step).
constexpr int kMmaA = 128 * 64 * 2, kMmaB = 256 * 64 * 2;

__global__ void __launch_bounds__(128, 1) k_probe_mma(long long iters, uint32_t wait_limit, int* status, ProbeOut* out)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t bar_done;
    __shared__ uint32_t s_taddr;
    __shared__ int s_abort;
    unsigned long long c0 = 0, t0 = 0;
    for (int i = threadIdx.x; i < (kMmaA + kMmaB) / 16; i += blockDim.x)
        reinterpret_cast<uint4*>(smem)[i] = make_uint4(0u, 0u, 0u, 0u);
    fence_proxy_async_smem();
    if (threadIdx.x == 0) {
        mbar_init(&bar_done, 1);
        s_abort = 0;
        fence_mbar_init();
    }
    if (threadIdx.x < 32) {
        tmem_alloc(&s_taddr, 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = s_taddr;
    if (threadIdx.x == 0) {
        t0 = globaltimer();
        c0 = clock64();
        constexpr uint32_t idesc = idesc_f16(128, 256, false);
        const uint32_t a0 = smem_u32(smem), b0 = a0 + kMmaA;
        for (long long it = 0; it < iters; it++) {
            const uint32_t d = taddr + (uint32_t)(it & 1) * 256u;
#pragma unroll
            for (int kk = 0; kk < 4; kk++)
                umma_f16(d, sw128_desc(a0 + kk * 32), sw128_desc(b0 + kk * 32), idesc, (it >= 2 || kk > 0) ? 1u : 0u);
        }
        umma_commit(&bar_done);
        if (!mbar_wait(&bar_done, 0, &s_abort, wait_limit)) atomicOr(status, 1);
        out[blockIdx.x].clk1 = clock64();
        out[blockIdx.x].ns1 = globaltimer();
        out[blockIdx.x].clk0 = c0;
        out[blockIdx.x].ns0 = t0;
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x < 32) {
        tc_fence_after();
        tmem_dealloc(taddr, 512);
    }
}

// Dynamic shared memory that no probe uses, so that at most one CTA fits on an
// SM and a grid of SM-count CTAs puts exactly one on every SM.
constexpr size_t kOneCtaSmem = 120 * 1024;

template <int K>
cudaError_t launch_kind(int grid, long long iters, float* sink, ProbeOut* out, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(k_probe<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kOneCtaSmem);
    if (e != cudaSuccess) return e;
    k_probe<K><<<grid, kThreads, kOneCtaSmem, s>>>(iters, 0.37f, sink, out);
    return cudaGetLastError();
}

}  // namespace

extern "C" {

/*
 * Runs probe `kind` (see the file header) once on every SM of the current
 * device: grid = SM count, 1,024 threads (128 for the MMA probe).
 *   iters        loop trips (each trip is 16 dependent steps of 8 chains; 8 for
 *                kinds 5 and 6; 4 MMAs for kind 8)
 *   ms           kernel time from CUDA events around the launch
 *   ops          operations executed in total (see the kinds)
 *   sm_mhz       SM clock during the run: mean over CTAs of
 *                delta clock64 / delta %globaltimer
 * Returns 0, or a CUDA error code (-1 for a bad kind, -2 for an MMA wait that
 * gave up).
 */
int cp_probe_rate(int kind, long long iters, double* ms, double* ops, double* sm_mhz)
{
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return (int)e;
    if (kind < 0 || kind > 8 || iters < 1) return -1;
    float* sink = nullptr;
    ProbeOut* out = nullptr;
    int* status = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = 0;
    const size_t mma_smem = kOneCtaSmem;   // operands use the first 49 KB
    if ((e = cudaMalloc(&sink, (size_t)nsm * kThreads * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&out, (size_t)nsm * sizeof(ProbeOut))) != cudaSuccess ||
        (e = cudaMalloc(&status, sizeof(int))) != cudaSuccess || (e = cudaMemset(status, 0, sizeof(int))) != cudaSuccess ||
        (e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess)
        rc = (int)e;
    if (rc == 0 && kind == 8)
        rc = (int)cudaFuncSetAttribute(k_probe_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mma_smem);
    if (rc == 0) {
        cudaEventRecord(e0, 0);
        switch (kind) {
        case 0: e = launch_kind<0>(nsm, iters, sink, out, 0); break;
        case 1: e = launch_kind<1>(nsm, iters, sink, out, 0); break;
        case 2: e = launch_kind<2>(nsm, iters, sink, out, 0); break;
        case 3: e = launch_kind<3>(nsm, iters, sink, out, 0); break;
        case 4: e = launch_kind<4>(nsm, iters, sink, out, 0); break;
        case 5: e = launch_kind<5>(nsm, iters, sink, out, 0); break;
        case 6: e = launch_kind<6>(nsm, iters, sink, out, 0); break;
        case 7: e = launch_kind<7>(nsm, iters, sink, out, 0); break;
        default:
            // bounded wait for the last MMAs: a generous multiple of their expected time
            k_probe_mma<<<nsm, 128, mma_smem, 0>>>(iters, (uint32_t)(iters * 64 > (1ll << 22) ? iters * 64 : (1ll << 22)),
                                                   status, out);
            e = cudaGetLastError();
        }
        cudaEventRecord(e1, 0);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        rc = (int)e;
    }
    if (rc == 0) {
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        *ms = t;
        const double per_thread_steps = (double)iters * (kind == 5 || kind == 6 ? 8 : 16) * kChains;
        const double threads = (double)nsm * kThreads;
        double per_step = 1.0;   // operations per dependent step
        if (kind == 3 || kind == 5 || kind == 6 || kind == 7) per_step = 2.0;
        *ops = kind == 8 ? (double)nsm * (double)iters * 4.0 * 2.0 * 128 * 256 * 16 : per_thread_steps * threads * per_step;
        ProbeOut* h = new ProbeOut[nsm];
        int st = 0;
        cudaMemcpy(h, out, (size_t)nsm * sizeof(ProbeOut), cudaMemcpyDeviceToHost);
        cudaMemcpy(&st, status, sizeof(int), cudaMemcpyDeviceToHost);
        double mhz = 0.0;
        for (int b = 0; b < nsm; b++)
            mhz += (double)(h[b].clk1 - h[b].clk0) / (double)(h[b].ns1 - h[b].ns0) * 1e3;
        *sm_mhz = mhz / nsm;
        delete[] h;
        if (st) rc = -2;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    cudaFree(out);
    cudaFree(status);
    return rc;
}

}  // extern "C"
