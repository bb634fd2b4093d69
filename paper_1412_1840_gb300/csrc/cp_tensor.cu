// cp_tensor.cu -- tensor-core form of the CKP pair sum (arXiv:1412.1840).
//
// Eq. (taylor) regrouped by harmonic gives
//   exp(-2 sin^2(pi f dt) / st^2) = b_0 + sum_{n>=1} a_n cos(2 pi n f dt),
//   a_n = 2 e^-k I_n(k), k = 1/st^2,
// and since sum_ij w_ij = 0 (Eq. (IP)) the pair sum of Eq. (HP) becomes
//   S(f) = sum_ij w_ij e_ij = sum_{n=1}^{n_max} a_n (c_n^T W c_n + s_n^T W s_n),
//   c_{n,i} = cos(2 pi n f t_i), s_{n,i} = sin(2 pi n f t_i).
// With W' = the upper block triangle of W in 128-row blocks (off-diagonal
// blocks doubled), S(f) = sum_I z_I^T (W' Z)_I, so each work unit (curve, tile of
// 256 columns = frequencies x harmonics x {cos, sin}) is a chain of GEMMs
// D_I = W'[I, J >= I] * Z[J, cols] on tcgen05 (M = 128, N = 256, K = 64 per
// stage, FP16 or BF16 operands, FP32 accumulation in TMEM), followed by the
// epilogue q = sum_i z[i, col] D_I[i, col].  Up to 16 harmonics the weights
// a_n are folded into the GEMM operand (column n of Z holds a_n z_n), so the
// epilogue multiplies by the unweighted z_n; with 32 harmonics the producers'
// registers are the tighter resource and the epilogue applies a_n.
//
// Warp roles: warp 0 bulk-copies pre-swizzled W' tiles, warp 1 issues the
// MMAs, the next 4 or 8 warps read TMEM (epilogue), the last 8 generate the Z
// tiles (cos/sin of every harmonic by the Chebyshev recurrence) straight into
// the swizzled shared-memory layout the MMA reads.  Every wait is bounded.
//
// The 16-bit rounding of W' leaves, per column, an error whose coherent part
// (xm^2 sum dW + 2 xm drho^T (x - xm), xm the samples' mean of the column's x)
// does not average out where x is nearly constant over the samples (f = 0,
// short f T, aliases of the sampling); two pseudo-rows at the top of W' give
// the products the epilogue needs to subtract it (see kTcPseudo).
//
// With folded weights both sides run the recurrence on x_n = sigma_n (cos n th,
// sin n th) with the sign pattern sigma = +, +, -, -, ... (period 4 in n,
// n = 0, 1, 2, ...).  Then x_{n+1} = K_n x_n + x_{n-1} with K_n = +2 cos th for
// even n and -2 cos th for odd n: one packed f32x2 FMA per step and no
// negation.  The signs cancel in the product z_n (W' z_n).
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "cp_internal.cuh"
#include "cp_tc.cuh"

namespace cpk {

using namespace tc;

constexpr int kTcA = 16384;            // 128 x 64 x 2 B
constexpr int kTcB = 32768;            // 256 x 64 x 2 B
// BF16 carries 8 significand bits, and the rounding of W' alone would exceed
// the tolerance of 1e-3 (Z's rounding stays below it).  With BF16 operands W'
// is therefore stored as two BF16 tiles, hi = bf16(w) and lo = bf16(w - hi),
// and every K slice issues two MMAs into the same accumulator: W' carries ~16
// significand bits.  FP16 (11 bits) needs no split.
// Split Z (ZS, BF16 only): Z's single BF16 rounding still leaves ~1.5e-3 on
// the harmonic-rich curves, so Z too is stored as hi + lo parts, the lo part
// in the upper half of the unit's 256 MMA columns: a unit holds half the
// frequencies, column c + 128 carries bf16(z - hi) of column c, and the
// epilogue reads D[c] + D[c + 128] = W' (Z_hi + Z_lo) less the lo x lo
// product (the W' lo MMA covers the first 128 columns only): three of the
// four hi/lo products.  Harmonic counts 4, 8, 16 and 32 (a half unit of
// exactly 128 columns).
__host__ __device__ constexpr int tc_wparts(bool bf) { return bf ? 2 : 1; }
// Stages of the operand ring: W' tiles (all parts) of two M-tiles + one Z tile.
__host__ __device__ constexpr int tc_stages(bool bf) { return bf ? 2 : 3; }
__host__ __device__ constexpr int tc_stage_bytes(bool bf) { return 2 * tc_wparts(bf) * kTcA + kTcB; }
constexpr int kTcMaxStages = 3;
constexpr int kTcCols = 256;           // columns per unit
// Epilogue warps: 8 for up to 16 harmonics (two warps per TMEM lane group,
// each taking half of the unit's frequencies), else 4; the drain of an
// accumulator is on the MMA's critical path (a warp's share must be an even
// number of frequencies: 12 harmonics keep 4 warps).  With 18 warps a quarter-SM
// holds up to 5 of them, which caps registers at 96 per thread: enough
// below 32 harmonics.
__host__ __device__ constexpr int tc_cols_h(bool zs) { return zs ? 128 : 256; }   // MMA columns of one Z part
__host__ __device__ constexpr int tc_ft(int nmax, bool zs) { return tc_cols_h(zs) / 2 / nmax; }   // frequencies per unit
__host__ __device__ constexpr int tc_ew(int nmax, bool zs) { return nmax <= 16 && (tc_ft(nmax, zs) / 2) % 2 == 0 ? 8 : 4; }
// Producer items split a frequency's harmonics into this many ranges for 32
// harmonics (4 frequencies per unit): 64 items per stage instead of 32, so
// three stages are produced by 192 threads instead of 96; 48 harmonics (2
// frequencies per unit, 192 columns): three ranges of 16.
// With split Z a unit has half the frequencies, so the harmonic ranges are
// halved too (8 and 16 harmonics: 2 ranges, 32: 4) to keep the items per stage.
__host__ __device__ constexpr int tc_hsplit(int nmax, bool zs)
{
    return zs ? (nmax == 4 ? 1 : nmax == 32 ? 4 : 2) : (nmax == 32 ? 2 : nmax == 48 ? 3 : 1);
}
// Items of one Z stage: (j-octet, frequency, harmonic range).  A stage group
// takes a whole number of warps: a warp split between two groups would run
// both groups' work one after the other.
__host__ __device__ constexpr int tc_items(int nmax, bool zs) { return 8 * tc_ft(nmax, zs) * tc_hsplit(nmax, zs); }
__host__ __device__ constexpr int tc_gstride(int nmax, bool zs) { return (tc_items(nmax, zs) + 31) / 32 * 32; }
// Producer threads: 8 warps; 9 for 12 harmonics, so that three 80-item groups
// (padded to 96 threads) produce three stages at once.
__host__ __device__ constexpr int tc_producers(int nmax) { return nmax == 12 ? 288 : 256; }
__host__ __device__ constexpr int tc_threads(int nmax, bool zs) { return 64 + 32 * tc_ew(nmax, zs) + tc_producers(nmax); }
constexpr int kTcTablePoints = 1024;   // per-unit phase table in shared memory (producers), by K row
// Table slot of K row j: one 16-byte pad after every 8 entries, so that the
// eight j-octets a warp reads at once (128 bytes apart unpadded) fall on
// different banks.
__device__ __forceinline__ int tc_tab(int j) { return j + (j >> 3); }
constexpr int kTcTableSlots = kTcTablePoints + kTcTablePoints / 8;

// Two pseudo-rows precede the samples in W' (rows 0 and 1 of its first
// M-tile, whose block row spans every K chunk): row 0 holds the row sums of
// the 16-bit rounding error of W, drho_j, row 1 ones.  Their products with a Z
// column are drho^T z and 1^T z, from which the epilogue removes the coherent
// part of the operand's rounding error (see k_stats).  Row / K index r is
// sample r - kTcPseudo; the pseudo-rows' own Z rows are zero.
constexpr int kTcPseudo = 2;
__host__ __device__ inline int tc_mtiles(int n) { return (n + 127) / 128; }
__host__ __device__ inline int tc_kchunks(int n) { return (n + 63) / 64; }
__host__ __device__ inline int tc_tiles_of(int n)
{
    const int nmt = tc_mtiles(n), nkc = tc_kchunks(n);
    int t = 0;
    for (int I = 0; I < nmt; I++) t += nkc - 2 * I > 0 ? nkc - 2 * I : 0;
    return t;
}
__host__ __device__ inline int tc_tile_index(int I, int J, int nkc)
{
    // tiles stored I-major: sum_{I' < I} (nkc - 2 I') + (J - 2 I)
    return I * nkc - I * (I - 1) + (J - 2 * I);
}

__device__ __forceinline__ uint16_t to16(float v, bool bf)
{
    return bf ? __bfloat16_as_ushort(__float2bfloat16_rn(v)) : __half_as_ushort(__float2half_rn(v));
}

// Two floats -> one packed 16-bit pair (low = lo), one conversion instruction.
template <bool BF>
__device__ __forceinline__ uint32_t pack16x2(float lo, float hi)
{
    uint32_t r;
    if (BF)
        asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    else
        asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

// The BF16 rounding residuals of a packed pair: (lo - bf16(lo), hi - bf16(hi))
// (exact in FP32), rounded to BF16 and packed the same way.
__device__ __forceinline__ uint32_t bf16x2_residual(float lo, float hi, uint32_t packed)
{
    return pack16x2<true>(lo - __uint_as_float(packed << 16), hi - __uint_as_float(packed & 0xffff0000u));
}

// ===========================================================================
// k_build_w16: pre-swizzled 128 x 64 tiles of W' (one CTA per tile).
// ===========================================================================
__global__ void __launch_bounds__(256) k_build_w16(const BuildW16Args a)
{
    const int64_t T = a.tile_begin + blockIdx.x;
    if (T >= a.tile_end) return;
    int lo = a.slot_begin, hi = a.slot_end - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.wtile_start[mid] <= T) lo = mid; else hi = mid - 1;
    }
    const int c = a.order[lo];
    const CurveParams P = a.cp[c];
    const int n = P.n, nkc = tc_kchunks(n + kTcPseudo);
    int t = (int)(T - a.wtile_start[lo]);
    int I = 0;
    while (t >= nkc - 2 * I) { t -= nkc - 2 * I; ++I; }
    const int J = 2 * I + t;
    const float scale = (J >= 2 * I + 2) ? 2.0f : 1.0f;
    const int r = threadIdx.x >> 1;                 // tile row
    const int kb = (threadIdx.x & 1) * 32;          // first of 32 columns
    const int i = I * 128 + r - kTcPseudo;          // sample of the row (-2, -1: pseudo-rows)
    const float ypi = i >= 0 && i < n ? a.yp[P.off + i] : 0.f;
    const bool bf = a.bf16 != 0;
    // tile T: its tc_wparts(bf) parts (hi, then lo for BF16) of kTcA bytes each
    unsigned char* dst = reinterpret_cast<unsigned char*>(a.W16) + (T - a.tile_begin) * (int64_t)(tc_wparts(bf) * kTcA);
#pragma unroll
    for (int ch = 0; ch < 4; ch++) {
        uint32_t packed[4], packed_lo[4];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
            float v2[2];
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int k = kb + ch * 8 + e + h;
                const int j = J * 64 + k - kTcPseudo;
                float w = 0.f;
                if (j >= 0 && j < n) {
                    if (i >= 0 && i < n) w = ((gauss_g(ypi, a.yp[P.off + j]) - P.ip_hi) - P.ip_lo) * scale;
                    else if (i == -kTcPseudo) w = a.wrho[P.off + j];
                    else if (i == 1 - kTcPseudo) w = 1.0f;
                }
                v2[h] = w;
            }
            const uint16_t h0 = to16(v2[0], bf), h1 = to16(v2[1], bf);
            packed[e >> 1] = (uint32_t)h0 | ((uint32_t)h1 << 16);
            if (bf) {
                // the remainder w - hi is exact in FP32; its BF16 rounding is the lo part
                const float l0 = v2[0] - __bfloat162float(__ushort_as_bfloat16(h0));
                const float l1 = v2[1] - __bfloat162float(__ushort_as_bfloat16(h1));
                packed_lo[e >> 1] = (uint32_t)to16(l0, true) | ((uint32_t)to16(l1, true) << 16);
            }
        }
        const uint32_t o = sw128_offset(r, kb + ch * 8);
        *reinterpret_cast<uint4*>(dst + o) = make_uint4(packed[0], packed[1], packed[2], packed[3]);
        if (bf)
            *reinterpret_cast<uint4*>(dst + kTcA + o) = make_uint4(packed_lo[0], packed_lo[1], packed_lo[2], packed_lo[3]);
    }
}

// ===========================================================================
// k_harmonic_coef: a_n = 2 e^-k I_n(k), n = 1..n_max, per curve (one warp),
// trapezoid rule on (1/pi) int_0^pi e^{k(cos t - 1)} cos(n t) dt.  The
// integrand is evaluated in FP32 (relative error ~1e-5 at most, from the
// exponent's rounding at k <= 100 and n^2 2^-24 from the Chebyshev recurrence
// for cos(n t), n <= 32; beyond 32, cos(n t) is evaluated directly on the
// exactly reduced angle (n k mod 2M) / M turns of pi; far below the tensor
// form's 1e-3), each lane sums its <= M/32 points in FP32, and the warp sum is
// FP64.  (FP64 transcendentals run at 1.68 operations/clk/SM here; this took
// 0.4 ms per 4096 curves in FP64.)  Written at coef[c * stride + n - 1].
// ===========================================================================
__global__ void __launch_bounds__(256) k_harmonic_coef(const CurveParams* cp, int n_curves, int n_max, int stride,
                                                       float* coef)
{
    const int c = blockIdx.x * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (c >= n_curves) return;
    const float st = cp[c].sigma_t;
    const float kap = 1.0f / (st * st);
    // quadrature points: enough for the integrand's width ~1/sqrt(k) and the
    // highest harmonic (k capped so that a tiny sigma_t cannot overflow M)
    const int M = 64 + 4 * (int)fminf(kap, (float)(1 << 20)) + 4 * n_max;
    float acc[kTcMaxHarmonics];
#pragma unroll
    for (int q = 0; q < kTcMaxHarmonics; q++) acc[q] = 0.f;
    for (int k = lane; k <= M; k += 32) {
        float sn, ct;
        sincospif((float)k / (float)M, &sn, &ct);
        const float wgt = (k == 0 || k == M) ? 0.5f : 1.0f;
        const float e = wgt * expf(kap * (ct - 1.0f));
        float cm2 = 1.0f, cm1 = ct;   // cos(0 t), cos(1 t)
#pragma unroll
        for (int q = 0; q < 32; q++) {
            if (q < n_max) acc[q] = fmaf(e, cm1, acc[q]);
            const float cn = fmaf(2.0f * ct, cm1, -cm2);
            cm2 = cm1;
            cm1 = cn;
        }
#pragma unroll
        for (int q = 32; q < kTcMaxHarmonics; q++)
            if (q < n_max)
                acc[q] = fmaf(e, cospif((float)(((int64_t)(q + 1) * k) % (2 * M)) / (float)M), acc[q]);
    }
#pragma unroll
    for (int q = 0; q < kTcMaxHarmonics; q++) {
        double v = (double)acc[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0 && q < n_max) coef[(int64_t)c * stride + q] = (float)(2.0 * v / (double)M);
    }
}

// Butterfly reduce-scatter over a warp: on return, lane l holds the warp-wide
// sum of x[(l >> (5 - log2 FT)) & (FT - 1)] (every value summed over 32 lanes).
template <int FT>
__device__ __forceinline__ float warp_reduce_scatter(float (&x)[FT], int lane)
{
    constexpr int L = FT == 1 ? 0 : FT == 2 ? 1 : FT == 4 ? 2 : FT == 8 ? 3 : FT == 16 ? 4 : 5;
#pragma unroll
    for (int step = 0; step < L; step++) {
        const int bit = 4 - step;
        const int half = FT >> (step + 1);
        const bool upper = (lane >> bit) & 1;
#pragma unroll
        for (int q = 0; q < half; q++) {
            const float send = upper ? x[q] : x[q + half];
            const float recv = __shfl_xor_sync(0xffffffffu, send, 1 << bit);
            x[q] = (upper ? x[q + half] : x[q]) + recv;
        }
    }
    float v = x[0];
#pragma unroll
    for (int b = 4 - L; b >= 0; b--) v += __shfl_xor_sync(0xffffffffu, v, 1 << b);
    return v;
}

template <bool SFU>
__device__ __forceinline__ void epi_sincos(uint32_t U, float& s, float& c)
{
    if (SFU) sincos2pi_turns_sfu(U, s, c);
    else sincos2pi_turns(U, s, c);
}

// ===========================================================================
// k_pair_tensor
// ===========================================================================
struct TcUnit {
    int c, n, nmt, nkc;
    int64_t kfirst;
    int count;
    int peak;
    uint64_t peak_mult;
    int64_t wbase;      // first W' tile of the curve (relative to the wave)
    bool empty;
};

__device__ __forceinline__ TcUnit tc_decode(const TensorArgs& a, int64_t u)
{
    TcUnit U;
    int lo = a.slot_begin, hi = a.slot_end - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.unit_start[mid] <= u) lo = mid; else hi = mid - 1;
    }
    const int slot = lo;
    U.c = a.order[slot];
    U.n = a.cp[U.c].n;
    U.nmt = tc_mtiles(U.n + kTcPseudo);
    U.nkc = tc_kchunks(U.n + kTcPseudo);
    U.wbase = a.wtile_start[slot] - a.wtile_base;
    const int64_t chunk = u - a.unit_start[slot];
    const int ft = a.ft;
    U.peak = 0;
    U.peak_mult = 0;
    U.empty = false;
    if (a.stage == kStageFine) {
        const int W = 2 * a.fine_half + 1;
        const int upp = (W + ft - 1) / ft;
        U.peak = (int)(chunk / upp);
        const int sub = (int)(chunk - (int64_t)U.peak * upp);
        U.empty = U.peak >= a.n_peaks[U.c];
        U.peak_mult = U.empty ? 0 : (uint64_t)a.peaks[(int64_t)U.c * a.top_k + U.peak];
        U.kfirst = -a.fine_half + (int64_t)sub * ft;
        U.count = (int)min((int64_t)ft, (int64_t)a.fine_half - U.kfirst + 1);
    } else if (a.stage == kStageList) {
        U.kfirst = chunk * ft;       // first list position
        U.count = (int)min((int64_t)ft, (int64_t)a.n_trials - U.kfirst);
    } else {
        U.kfirst = chunk * ft;
        U.count = (int)min((int64_t)ft, a.n_freq - U.kfirst);
    }
    return U;
}

// Frequency multiplier of the unit's f-th frequency relative to the phase
// table base: f for the uniform stages (base = ph_base + kfirst * step), the
// grid index of list position kfirst + f for the list stage (base = ph_base;
// a missing entry evaluates k = 0 and is never emitted).
template <bool LIST>
__device__ __forceinline__ uint64_t tc_mult(const TensorArgs& a, const TcUnit& U, int f)
{
    if (!LIST) return (uint64_t)f;
    const int64_t q = U.kfirst + f;
    return q < a.n_trials ? (uint64_t)max(a.trials[(int64_t)U.c * a.n_trials + q], 0) : 0ull;
}

template <bool LIST>
__device__ __forceinline__ uint64_t tc_base_mult(const TensorArgs& a, const TcUnit& U)
{
    return LIST ? 0ull : (uint64_t)U.kfirst;
}

template <bool LIST>
__device__ __forceinline__ uint32_t tc_phase_u32(const TensorArgs& a, const TcUnit& U, int64_t off, int i,
                                                 uint64_t mult)
{
    const uint64_t st = a.ph_step[off + i];
    uint64_t ph = a.ph_base[off + i] + (tc_base_mult<LIST>(a, U) + mult) * st;
    if (a.stage == kStageFine) ph += U.peak_mult * a.ph_coarse[off + i];
    return (uint32_t)(ph >> 32);
}

// Stages hold the W' tiles of two M-tiles and one Z tile: M-tiles 2P and
// 2P+1 share every Z stage of their common K range (two TMEM accumulators).
// LIST: the list stage (explicit grid indices per curve); a separate
// instantiation so that the uniform stages keep their rotation shortcut.
// ZS: Z split into hi + lo BF16 parts (see tc_cols_h).
template <int NMAX, bool BF, bool LIST, bool ZS>
__global__ void __launch_bounds__(tc_threads(NMAX, ZS), 1) k_pair_tensor(const TensorArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    constexpr int STG = tc_stages(BF);                // operand ring stages
    constexpr int SB = tc_stage_bytes(BF);            // bytes per stage
    constexpr int WP = tc_wparts(BF);                 // W' parts (BF16: hi and lo)
    constexpr int AB = WP * kTcA;                     // W' bytes of one M-tile in a stage
    // producers' phase table of the current unit: (phase at the unit's first frequency, step)
    ulonglong2* sPh = reinterpret_cast<ulonglong2*>(smem + STG * SB);
    __shared__ uint64_t bar_afull[kTcMaxStages], bar_bfull[kTcMaxStages], bar_empty[kTcMaxStages];
    __shared__ uint64_t bar_tfull, bar_tempty[2], bar_drain;
    __shared__ uint32_t s_taddr;
    __shared__ int s_abort;
    __shared__ float s_red[8][32];
    __shared__ float s_acc[32];                       // per-accumulator reduction: running sums
    __shared__ __align__(16) float s_pse[kTcPseudo][kTcCols];   // the pseudo-rows' accumulator values of the unit
    __shared__ float s_cc[kTcCols / 8];               // their correction, summed per 8 columns

    constexpr int FT = tc_ft(NMAX, ZS);               // frequencies per unit
    constexpr int CH = FT * 2 * NMAX;                 // columns of one Z part: 256 (240 for 12 harmonics), 128 split
    constexpr int COLS = ZS ? 2 * CH : CH;            // MMA columns of the unit
    constexpr int LW = ZS ? 16 : 32;                  // accumulator columns per TMEM load
    static_assert(!ZS || (BF && CH == 128), "split Z: BF16 operands and 4, 8, 16 or 32 harmonics");
    constexpr int EW = tc_ew(NMAX, ZS);               // epilogue warps
    constexpr int FH = FT / (EW / 4);                 // frequencies per epilogue warp
    constexpr int FHP = FH <= 2 ? 2 : FH <= 4 ? 4 : FH <= 8 ? 8 : FH <= 16 ? 16 : 32;   // padded to a power of 2
    constexpr int HS = tc_hsplit(NMAX, ZS);           // harmonic ranges per producer item
    constexpr int NH = NMAX / HS;                     // harmonics per producer item
    constexpr int items = tc_items(NMAX, ZS);         // (j-octet, frequency, harmonic range) per stage
    constexpr int PROD = tc_producers(NMAX);
    constexpr int GS = tc_gstride(NMAX, ZS);          // threads per stage group
    constexpr bool FOLD = NMAX <= 16;                 // a_n folded into Z (see the file header)
    // Row sums reduced across the warp once per unit (per-thread partial sums over
    // the M-tiles) or once per accumulator; the latter measured faster only for
    // 16 harmonics, where the former raises register spills.
    constexpr bool UNIT_RED = NMAX != 16;
    // Epilogue angles by the SFU approximations (absolute error ~1e-6, far below the
    // 16-bit rounding of Z), for every class.
    constexpr bool EPI_SFU = true;
    // a producer's harmonic range starts at n0 = hr NH + 1 with sigma_{n0-1} = sigma_{n0} = +
    static_assert(!FOLD || HS == 1 || NH % 4 == 0, "harmonic ranges must start on the sign pattern's period");
    static_assert(!FOLD || NH % 2 == 0, "the producers take the step's sign from the parity of nn");
    // Stages produced concurrently.  A group owns every use of its stages, so
    // it never waits more than one barrier phase ahead; hence groups <= stages.
    constexpr int groups = PROD / GS < STG ? PROD / GS : STG;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        for (int s = 0; s < STG; s++) {
            mbar_init(&bar_afull[s], 1);
            mbar_init(&bar_bfull[s], items);
            mbar_init(&bar_empty[s], 1);
        }
        mbar_init(&bar_tfull, 1);
        mbar_init(&bar_tempty[0], 32 * EW);
        mbar_init(&bar_tempty[1], 32 * EW);
        mbar_init(&bar_drain, 1);
        s_abort = 0;
        fence_mbar_init();
    }
    if (tid < 32) s_acc[tid] = 0.f;
    if (warp == 0) {
        tmem_alloc(&s_taddr, 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = s_taddr;

    if (warp == 0) {
        // ---------------- W' tile loader ----------------
        if (lane == 0) {
            uint32_t q = 0;
            bool ok = true;
            for (int64_t u = a.unit_begin + blockIdx.x / a.ctas_per_unit; ok && u < a.unit_end; u += gridDim.x) {
                const TcUnit U = tc_decode(a, u);
                if (U.empty) continue;
                for (int P = 0; ok && 2 * P < U.nmt; P++) {
                    const int I0 = 2 * P, I1 = 2 * P + 1;
                    for (int J = 2 * I0; J < U.nkc; J++, q++) {
                        const bool use1 = I1 < U.nmt && J >= 2 * I1;
                        const int s = q % STG;
                        if (!mbar_wait(&bar_empty[s], ((q / STG) & 1) ^ 1, &s_abort, a.wait_limit)) { ok = false; break; }
                        unsigned char* st = smem + s * SB;
                        const unsigned char* w16 = reinterpret_cast<const unsigned char*>(a.W16);
                        mbar_arrive_expect_tx(&bar_afull[s], use1 ? 2 * AB : AB);
                        bulk_g2s(st, w16 + (U.wbase + tc_tile_index(I0, J, U.nkc)) * (int64_t)AB, AB, &bar_afull[s]);
                        if (use1)
                            bulk_g2s(st + AB, w16 + (U.wbase + tc_tile_index(I1, J, U.nkc)) * (int64_t)AB, AB,
                                     &bar_afull[s]);
                    }
                }
            }
            if (!ok) {
                // let copies already issued land before the CTA exits
                for (uint32_t k = 0; k < STG && q > 0; k++) {
                    const uint32_t qq = q - 1 - k;
                    mbar_wait(&bar_afull[qq % STG], (qq / STG) & 1, &s_abort, 1u << 20);
                    if (qq == 0) break;
                }
                atomicOr(a.status, 2);
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_f16(128, COLS, BF);
            // W' lo against Z hi only: with split Z the lo x lo product (2^-18 of the
            // term) is left out, an N = 128 MMA over the first half of the columns
            constexpr uint32_t idesc_lo = idesc_f16(128, ZS ? CH : COLS, BF);
            uint32_t q = 0, m = 0;
            bool ok = true;
            for (int64_t u = a.unit_begin + blockIdx.x / a.ctas_per_unit; ok && u < a.unit_end; u += gridDim.x) {
                const TcUnit U = tc_decode(a, u);
                if (U.empty) continue;
                for (int P = 0; ok && 2 * P < U.nmt; P++, m++) {
                    const int I0 = 2 * P, I1 = 2 * P + 1;
                    const uint32_t epar = (m & 1) ^ 1;
                    if (!mbar_wait(&bar_tempty[0], epar, &s_abort, a.wait_limit)) { ok = false; break; }
                    tc_fence_after();
                    for (int J = 2 * I0; J < U.nkc; J++, q++) {
                        const bool use1 = I1 < U.nmt && J >= 2 * I1;
                        const int s = q % STG;
                        const uint32_t par = (q / STG) & 1;
                        if (J == 2 * I1 && use1) {
                            if (!mbar_wait(&bar_tempty[1], epar, &s_abort, a.wait_limit)) { ok = false; break; }
                        }
                        if (!mbar_wait(&bar_afull[s], par, &s_abort, a.wait_limit) ||
                            !mbar_wait(&bar_bfull[s], par, &s_abort, a.wait_limit)) { ok = false; break; }
                        tc_fence_after();
                        const uint32_t a0 = smem_u32(smem + s * SB);
                        const uint32_t a1 = a0 + AB, b0 = a0 + 2 * AB;
#pragma unroll
                        for (int kk = 0; kk < 4; kk++) {
                            const uint64_t bd = sw128_desc(b0 + kk * 32);
                            umma_f16(taddr, sw128_desc(a0 + kk * 32), bd, idesc, (J > 2 * I0 || kk > 0) ? 1u : 0u);
                            if (WP == 2) umma_f16(taddr, sw128_desc(a0 + kTcA + kk * 32), bd, idesc_lo, 1u);
                            if (use1) {
                                umma_f16(taddr + kTcCols, sw128_desc(a1 + kk * 32), bd, idesc,
                                         (J > 2 * I1 || kk > 0) ? 1u : 0u);
                                if (WP == 2) umma_f16(taddr + kTcCols, sw128_desc(a1 + kTcA + kk * 32), bd, idesc_lo, 1u);
                            }
                        }
                        umma_commit(&bar_empty[s]);
                    }
                    if (ok) umma_commit(&bar_tfull);
                }
            }
            // every MMA issued has completed before TMEM can be released
            umma_commit(&bar_drain);
            mbar_wait(&bar_drain, 0, &s_abort, 1u << 22);
            if (!ok) atomicOr(a.status, 2);
        }
    } else if (warp < 2 + EW) {
        // ---------------- epilogue: one TMEM lane (W' row) per thread ----------------
        const int lg = warp & 3;                      // TMEM lane group this warp may access
        const int row = lg * 32 + lane;
        const int ew = warp - 2;                      // epilogue warp index 0..EW-1
        const int fh = ew >> 2;                       // which FH frequencies of the unit
        const uint32_t hcol = (uint32_t)(fh * FH * 2 * NMAX);   // their first column (a multiple of 32)
        constexpr bool list = LIST;                   // explicit frequencies: no rotation shortcut
        constexpr int SH = FHP == 2 ? 4 : FHP == 4 ? 3 : FHP == 8 ? 2 : FHP == 16 ? 1 : 0;   // lanes per sum
        uint32_t m = 0;
        bool ok = true;
        for (int64_t u = a.unit_begin + blockIdx.x / a.ctas_per_unit; ok && u < a.unit_end; u += gridDim.x) {
            const TcUnit U = tc_decode(a, u);
            if (U.empty) continue;
            const CurveParams& P_ = a.cp[U.c];
            const int64_t off = P_.off;
            float an[FOLD ? 1 : NMAX];
            if constexpr (!FOLD) {
#pragma unroll
                for (int q = 0; q < NMAX; q++) an[q] = a.coef[(int64_t)U.c * a.coef_stride + q];
            }
            // this thread's rows summed over all M-tiles of the unit, per frequency of
            // the warp's share; reduced across the rows once per unit
            float accu[UNIT_RED ? FHP : 1];
#pragma unroll
            for (int fi = 0; fi < (UNIT_RED ? FHP : 1); fi++) accu[fi] = 0.f;
            for (int P = 0; 2 * P < U.nmt; P++, m++) {
                // the rows' phases for both M-tiles, loaded before the wait
                uint64_t ph0[2] = {0, 0}, pstep[2] = {0, 0};
                bool live[2];
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const int i = (2 * P + h) * 128 + row - kTcPseudo;   // sample of this row
                    live[h] = (unsigned)i < (unsigned)U.n;
                    if (live[h]) {
                        pstep[h] = a.ph_step[off + i];
                        ph0[h] = a.ph_base[off + i] + tc_base_mult<LIST>(a, U) * pstep[h];
                        if (a.stage == kStageFine) ph0[h] += U.peak_mult * a.ph_coarse[off + i];
                    }
                }
                mbar_wait(&bar_tfull, m & 1, &s_abort, a.wait_limit);
                // agree on the outcome: every epilogue thread sees the abort flag after the barrier
                asm volatile("bar.sync 1, %0;" ::"n"(32 * EW) : "memory");
                if (s_abort) { ok = false; break; }
                tc_fence_after();
#pragma unroll 1
                for (int h = 0; h < 2; h++) {
                    // scalars, not the arrays indexed by h: this loop is not unrolled, and
                    // indexing the arrays with h would place them in local memory
                    const bool live_h = h ? live[1] : live[0];
                    const uint64_t ph0_h = h ? ph0[1] : ph0[0];
                    const uint64_t pstep_h = h ? pstep[1] : pstep[0];
                    const bool has = 2 * P + h < U.nmt;
                    float accf[UNIT_RED ? 1 : FHP];             // per-accumulator reduction only
                    if constexpr (!UNIT_RED) {
#pragma unroll
                        for (int fi = FH; fi < FHP; fi++) accf[fi] = 0.f;
                    }
                    if (has) {
                        const uint32_t tbase = taddr + ((uint32_t)(lg * 32) << 16) + (uint32_t)(h * kTcCols) + hcol;
                        float v[LW];
                        // the angle of odd frequencies is the even one's rotated by one frequency step
                        float sr = 0.f, cr = 1.f, s1 = 0.f, c1 = 0.f;
                        if (live_h) epi_sincos<EPI_SFU>((uint32_t)(pstep_h >> 32), sr, cr);
#pragma unroll
                        for (int fi = 0; fi < FH; fi++) {
                            const int f = fh * FH + fi;       // FH is even: f and fi have the same parity
                            if (live_h) {
                                if ((fi & 1) == 0 || list) {
                                    epi_sincos<EPI_SFU>((uint32_t)((ph0_h + tc_mult<LIST>(a, U, f) * pstep_h) >> 32), s1, c1);
                                } else {
                                    const float cn = fmaf(c1, cr, -s1 * sr), sn = fmaf(s1, cr, c1 * sr);
                                    c1 = cn;
                                    s1 = sn;
                                }
                            }
                            if constexpr (FOLD) {
                                // x_{n-1}, x_n (signed as the producers sign them)
                                f2 xp = pk(1.f, 0.f), xc = pk(c1, s1), acc2 = 0ull;
                                const f2 kp = pk(2.f * c1, 2.f * c1), km = pk(-2.f * c1, -2.f * c1);
#pragma unroll
                                for (int n = 1; n <= NMAX; n++) {
                                    const int col = fi * 2 * NMAX + 2 * (n - 1);   // relative to hcol
                                    if (col % LW == 0) {
                                        if constexpr (ZS) tmem_ld16_sum(tbase + col, tbase + CH + col, v);
                                        else tmem_ld32(tbase + col, v);
                                    }
                                    acc2 = fma2(pk(v[col % LW], v[col % LW + 1]), xc, acc2);
                                    if (n < NMAX) {
                                        const f2 xn = fma2((n & 1) ? km : kp, xc, xp);
                                        xp = xc;
                                        xc = xn;
                                    }
                                }
                                float acc_c, acc_s;
                                upk(acc2, acc_c, acc_s);
                                if constexpr (UNIT_RED) {
                                    if (live_h) accu[fi] += acc_c + acc_s;
                                } else {
                                    accf[fi] = live_h ? acc_c + acc_s : 0.f;
                                }
                            } else {
                                float cp2 = 1.f, sp2 = 0.f, cp1 = c1, sp1 = s1;
                                float acc = 0.f;
#pragma unroll
                                for (int n = 1; n <= NMAX; n++) {
                                    const int col = fi * 2 * NMAX + 2 * (n - 1);   // relative to hcol
                                    if (col % LW == 0) {
                                        if constexpr (ZS) tmem_ld16_sum(tbase + col, tbase + CH + col, v);
                                        else tmem_ld32(tbase + col, v);
                                    }
                                    acc = fmaf(an[n - 1], fmaf(v[col % LW], cp1, v[col % LW + 1] * sp1), acc);
                                    const float cn = fmaf(2.f * c1, cp1, -cp2), sn = fmaf(2.f * c1, sp1, -sp2);
                                    cp2 = cp1; sp2 = sp1;
                                    cp1 = cn; sp1 = sn;
                                }
                                if constexpr (UNIT_RED) {
                                    if (live_h) accu[fi] += acc;
                                } else {
                                    accf[fi] = live_h ? acc : 0.f;
                                }
                            }
                        }
                    }
                    // the pseudo-rows (first M-tile: lanes 0 and 1 of lane group 0) keep their
                    // values for the unit's correction: one more read of this warp's columns
                    if (has && P == 0 && h == 0 && lg == 0) {
                        const uint32_t tb0 = taddr + (uint32_t)hcol;
#pragma unroll 1
                        for (int c0 = 0; c0 < FH * 2 * NMAX; c0 += LW) {
                            float v[LW];
                            if constexpr (ZS) tmem_ld16_sum(tb0 + c0, tb0 + CH + c0, v);
                            else tmem_ld32(tb0 + c0, v);
                            if (lane < kTcPseudo) {
                                float4* dst = reinterpret_cast<float4*>(&s_pse[lane][hcol + c0]);
#pragma unroll
                                for (int q = 0; q < LW / 4; q++)
                                    dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                            }
                        }
                    }
                    // release this accumulator (always, so the phases of both buffers advance per pair)
                    tc_fence_before();
                    mbar_arrive(&bar_tempty[h]);
                    if constexpr (!UNIT_RED) {
                        if (has) {
                            // sum over the 128 rows, fixed order
                            const float x = warp_reduce_scatter<FHP>(accf, lane);
                            if ((lane & ((1 << SH) - 1)) == 0) s_red[ew][lane >> SH] = x;
                            asm volatile("bar.sync 1, %0;" ::"n"(32 * EW) : "memory");
                            if (ew == 0 && lane < FT) {
                                const int w0 = (lane / FH) * 4, fi = lane % FH;
                                s_acc[lane] += ((s_red[w0][fi] + s_red[w0 + 1][fi]) + s_red[w0 + 2][fi]) + s_red[w0 + 3][fi];
                            }
                            asm volatile("bar.sync 1, %0;" ::"n"(32 * EW) : "memory");
                        }
                    }
                }
            }
            if (!ok) break;
            // The unit's correction for the coherent part of the operand's rounding error.
            // Per column, with the pseudo-rows' D0 = drho^T z and D1 = 1^T z (z = a_n x when
            // the weights are folded into Z, else x) and xm = 1^T x / N, that error adds
            // a_n (2 xm drho^T x - xm^2 sum dW).  Columns are spread over the epilogue
            // threads and summed in groups of eight (2 n_max is a multiple of 8).
            if (U.nmt <= 2) asm volatile("bar.sync 1, %0;" ::"n"(32 * EW) : "memory");   // stash of pair 0
            {
                const float inv_n = 1.0f / (float)U.n, dws = P_.dwsum;
                for (int c0 = ew * 32; c0 < CH; c0 += 32 * EW) {
                    const int col = c0 + lane;
                    float cc = 0.f;
                    if (col < CH) {
                        const float an = a.coef[(int64_t)U.c * a.coef_stride + ((col % (2 * NMAX)) >> 1)];
                        if (an > 0.f) {
                            const float d0 = s_pse[0][col], d1 = s_pse[1][col];
                            const float xm = FOLD ? __fdividef(d1 * inv_n, an) : d1 * inv_n;
                            cc = an * xm * (2.f * (FOLD ? __fdividef(d0, an) : d0) - xm * dws);
                        }
                    }
                    cc += __shfl_xor_sync(0xffffffffu, cc, 4);
                    cc += __shfl_xor_sync(0xffffffffu, cc, 2);
                    cc += __shfl_xor_sync(0xffffffffu, cc, 1);
                    if ((lane & 7) == 0 && col < CH) s_cc[col >> 3] = cc;
                }
            }
            if constexpr (!UNIT_RED) asm volatile("bar.sync 1, %0;" ::"n"(32 * EW) : "memory");
            if constexpr (UNIT_RED) {
                // unit complete: sum over the rows (lanes, then the four lane groups), fixed order
                const float x = warp_reduce_scatter<FHP>(accu, lane);
                if ((lane & ((1 << SH) - 1)) == 0) s_red[ew][lane >> SH] = x;
                asm volatile("bar.sync 1, %0;" ::"n"(32 * EW) : "memory");
            }
            // normalise and emit
            if (ew == 0) {
                float S = 0.f;
                if (UNIT_RED && lane < FT) {
                    const int w0 = (lane / FH) * 4, fi = lane % FH;
                    S = ((s_red[w0][fi] + s_red[w0 + 1][fi]) + s_red[w0 + 2][fi]) + s_red[w0 + 3][fi];
                }
                unsigned long long key = 0ull;
                if (lane < U.count) {
                    if constexpr (!UNIT_RED) S = s_acc[lane];
                    float corr = 0.f;
#pragma unroll
                    for (int q = 0; q < 2 * NMAX / 8; q++) corr += s_cc[lane * (2 * NMAX / 8) + q];
                    S -= corr;
                    const float v = S * P_.norm;
                    const long long kk = U.kfirst + lane;
                    if (a.stage == kStageFull) {
                        if (a.out) a.out[(int64_t)U.c * a.out_ld + kk] = v;
                        if (!excluded_k(a.ex.full_k, a.ex.n, kk)) key = make_key(v, (uint32_t)kk);
                    } else if (a.stage == kStageCoarse) {
                        a.coarse_out[(int64_t)U.c * a.n_freq + kk] = v;
                    } else if (list) {
                        const int32_t kg = a.trials[(int64_t)U.c * a.n_trials + kk];
                        const bool valid = kg >= 0;
                        if (a.trial_stat)
                            a.trial_stat[(int64_t)U.c * a.n_trials + kk] = valid ? v : __int_as_float(0x7fc00000);
                        if (valid && !excluded_k(a.ex.full_k, a.ex.n, kg)) key = make_key(v, (uint32_t)kk);
                    } else {
                        const double fpk = grid_freq(a.f_min, (double)U.peak_mult, a.coarse_df);
                        const double fr = grid_freq(fpk, (double)kk, a.step);
                        if (fr >= a.f_min && fr <= a.f_max && !excluded_f(a.ex, fr))
                            key = make_key(v, (uint32_t)(U.peak * (2 * a.fine_half + 1) + (kk + a.fine_half)));
                    }
                }
                if constexpr (!UNIT_RED) s_acc[lane] = 0.f;
                if (a.stage != kStageCoarse) {
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        const unsigned long long other = __shfl_xor_sync(0xffffffffu, key, o);
                        key = other > key ? other : key;
                    }
                    if (lane == 0 && key) atomicMax(a.best_key + U.c, key);
                }
            }
            asm volatile("bar.sync 1, %0;" ::"n"(32 * EW) : "memory");
        }
        if (!ok && ew == 0 && lane == 0) atomicOr(a.status, 2);
    } else {
        // ---------------- Z producers: PROD threads ----------------
        const int pt = tid - (2 + EW) * 32;           // 0..PROD-1
        const int grp = pt / GS;                      // stage group
        const int it = pt - grp * GS;
        const int g = it & 7;                         // j-octet of the K chunk (fastest: conflict-free stores)
        const int f = (it >> 3) % FT;                 // frequency within the unit
        const int hr = (it >> 3) / FT;                // harmonics hr*NH+1 .. (hr+1)*NH
        const bool active = grp < groups && (GS == items || it < items);
        uint32_t q = 0;
        bool ok = true;
        // After a timeout (ok == false) a producer keeps walking the units so that
        // every producer executes the same named barriers; it skips all work.
        for (int64_t u = a.unit_begin + blockIdx.x / a.ctas_per_unit; u < a.unit_end; u += gridDim.x) {
            const TcUnit U = tc_decode(a, u);
            if (U.empty) continue;
            const int64_t off = a.cp[U.c].off;
            const bool tab = U.n + kTcPseudo <= kTcTablePoints;   // table slot = K row (sample + kTcPseudo)
            const uint64_t mf = tc_mult<LIST>(a, U, f);   // this producer's frequency multiplier
            const float* anp = a.coef + (int64_t)U.c * a.coef_stride + hr * NH;   // a_n of this harmonic range
            if (tab) {
                // every producer is done with the previous unit's table
                asm volatile("bar.sync 2, %0;" ::"n"(PROD) : "memory");
                for (int j = pt; ok && j < U.n; j += PROD) {
                    const uint64_t stp = a.ph_step[off + j];
                    uint64_t ph0 = a.ph_base[off + j] + tc_base_mult<LIST>(a, U) * stp;
                    if (a.stage == kStageFine) ph0 += U.peak_mult * a.ph_coarse[off + j];
                    sPh[tc_tab(j + kTcPseudo)] = make_ulonglong2(ph0, stp);
                }
                asm volatile("bar.sync 2, %0;" ::"n"(PROD) : "memory");
            }
            for (int P = 0; ok && 2 * P < U.nmt; P++)
                for (int J = 4 * P; J < U.nkc; J++, q++) {
                    if (!active || (int)(q % (uint32_t)groups) != grp) continue;
                    const int s = q % STG;
                    const int j0 = J * 64 + g * 8;               // the octet's first K row (sample + kTcPseudo)
                    uint32_t pu[8];
#pragma unroll
                    for (int p = 0; p < 8; p++) {
                        uint32_t v = 0u;
                        if ((unsigned)(j0 + p - kTcPseudo) < (unsigned)U.n) {
                            if (tab) {
                                const ulonglong2 e = sPh[tc_tab(j0 + p)];
                                v = (uint32_t)((e.x + mf * e.y) >> 32);
                            } else {
                                v = tc_phase_u32<LIST>(a, U, off, j0 + p - kTcPseudo, mf);
                            }
                        }
                        pu[p] = v;
                    }
                    if (!mbar_wait(&bar_empty[s], ((q / STG) & 1) ^ 1, &s_abort, a.wait_limit)) { ok = false; break; }
                    if constexpr (FOLD) {
                        // x_{n0} and x_{n0-1} (n0 = hr*NH+1, both signed +) start the recurrence;
                        // f32x2 lanes are the points 2r and 2r+1
                        f2 cc[4], ss[4], cm[4], sm[4], kp[4], km[4];
#pragma unroll
                        for (int r = 0; r < 4; r++) {
                            float sv[2], cv[2], sb[2], cb[2], sa[2], ca[2];
#pragma unroll
                            for (int h = 0; h < 2; h++) {
                                const int p = 2 * r + h;
                                sv[h] = 0.f; cv[h] = 0.f; sb[h] = 0.f; cb[h] = 0.f; sa[h] = 0.f; ca[h] = 0.f;
                                if ((unsigned)(j0 + p - kTcPseudo) < (unsigned)U.n) {
                                    sincos2pi_turns_sfu(pu[p], sv[h], cv[h]);   // Z is rounded to 16 bits
                                    if (HS > 1 && hr > 0) {
                                        const uint32_t n0 = (uint32_t)(hr * NH + 1);
                                        sincos2pi_turns_sfu(pu[p] * n0, sb[h], cb[h]);
                                        sincos2pi_turns_sfu(pu[p] * (n0 - 1u), sa[h], ca[h]);
                                    } else {
                                        sb[h] = sv[h]; cb[h] = cv[h];
                                        sa[h] = 0.f; ca[h] = 1.f;
                                    }
                                }
                            }
                            kp[r] = pk(2.f * cv[0], 2.f * cv[1]);
                            km[r] = pk(-2.f * cv[0], -2.f * cv[1]);
                            cc[r] = pk(cb[0], cb[1]); ss[r] = pk(sb[0], sb[1]);     // n = n0
                            cm[r] = pk(ca[0], ca[1]); sm[r] = pk(sa[0], sa[1]);     // n = n0 - 1
                        }
                        unsigned char* Bs = smem + s * SB + 2 * AB;
                        // fully unrolled: measured fastest for every class (a partial unroll
                        // avoids the 16-harmonic spill but runs slower)
#pragma unroll
                        for (int nn = 0; nn < NH; nn++) {
                            const int n = hr * NH + 1 + nn;
                            const float an = __ldg(anp + nn);
                            const f2 a2 = pk(an, an);
                            uint32_t pc[4], ps[4], pcl[4], psl[4];
#pragma unroll
                            for (int r = 0; r < 4; r++) {
                                float lo, hi;
                                upk(mul2(a2, cc[r]), lo, hi);
                                pc[r] = pack16x2<BF>(lo, hi);
                                if constexpr (ZS) pcl[r] = bf16x2_residual(lo, hi, pc[r]);
                                upk(mul2(a2, ss[r]), lo, hi);
                                ps[r] = pack16x2<BF>(lo, hi);
                                if constexpr (ZS) psl[r] = bf16x2_residual(lo, hi, ps[r]);
                            }
                            const int col = f * 2 * NMAX + 2 * (n - 1);
                            *reinterpret_cast<uint4*>(Bs + sw128_offset(col, g * 8)) = make_uint4(pc[0], pc[1], pc[2], pc[3]);
                            *reinterpret_cast<uint4*>(Bs + sw128_offset(col + 1, g * 8)) = make_uint4(ps[0], ps[1], ps[2], ps[3]);
                            if constexpr (ZS) {
                                *reinterpret_cast<uint4*>(Bs + sw128_offset(CH + col, g * 8)) =
                                    make_uint4(pcl[0], pcl[1], pcl[2], pcl[3]);
                                *reinterpret_cast<uint4*>(Bs + sw128_offset(CH + col + 1, g * 8)) =
                                    make_uint4(psl[0], psl[1], psl[2], psl[3]);
                            }
                            if (nn + 1 < NH) {
#pragma unroll
                                for (int r = 0; r < 4; r++) {
                                    const f2 k = (nn & 1) ? kp[r] : km[r];   // n = hr NH + 1 + nn, hr NH even
                                    const f2 cn = fma2(k, cc[r], cm[r]);
                                    const f2 sn = fma2(k, ss[r], sm[r]);
                                    cm[r] = cc[r]; sm[r] = ss[r];
                                    cc[r] = cn; ss[r] = sn;
                                }
                            }
                        }
                    } else {
                        // cos/sin of harmonics n0 = hr*NH+1 and n0-1 start the Chebyshev recurrence
                        float cc[8], ss[8], c1[8], cm[8], sm[8];
#pragma unroll
                        for (int p = 0; p < 8; p++) {
                            float sv = 0.f, cv = 0.f, sb = 0.f, cb = 0.f, sa = 0.f, ca = 0.f;
                            if ((unsigned)(j0 + p - kTcPseudo) < (unsigned)U.n) {
                                sincos2pi_turns_sfu(pu[p], sv, cv);   // Z is rounded to 16 bits
                                if (HS > 1 && hr > 0) {
                                    const uint32_t n0 = (uint32_t)(hr * NH + 1);
                                    sincos2pi_turns_sfu(pu[p] * n0, sb, cb);
                                    sincos2pi_turns_sfu(pu[p] * (n0 - 1u), sa, ca);
                                } else {
                                    sb = sv; cb = cv;
                                    sa = 0.f; ca = 1.f;
                                }
                            }
                            c1[p] = cv;
                            cc[p] = cb; ss[p] = sb;           // n = n0
                            cm[p] = ca; sm[p] = sa;           // n = n0 - 1
                        }
                        unsigned char* Bs = smem + s * SB + 2 * AB;
#pragma unroll
                        for (int nn = 0; nn < NH; nn++) {
                            const int n = hr * NH + 1 + nn;
                            uint32_t pc[4], ps[4], pcl[4], psl[4];
#pragma unroll
                            for (int p = 0; p < 8; p += 2) {
                                pc[p >> 1] = pack16x2<BF>(cc[p], cc[p + 1]);
                                ps[p >> 1] = pack16x2<BF>(ss[p], ss[p + 1]);
                                if constexpr (ZS) {
                                    pcl[p >> 1] = bf16x2_residual(cc[p], cc[p + 1], pc[p >> 1]);
                                    psl[p >> 1] = bf16x2_residual(ss[p], ss[p + 1], ps[p >> 1]);
                                }
                            }
                            const int col = f * 2 * NMAX + 2 * (n - 1);
                            *reinterpret_cast<uint4*>(Bs + sw128_offset(col, g * 8)) = make_uint4(pc[0], pc[1], pc[2], pc[3]);
                            *reinterpret_cast<uint4*>(Bs + sw128_offset(col + 1, g * 8)) = make_uint4(ps[0], ps[1], ps[2], ps[3]);
                            if constexpr (ZS) {
                                *reinterpret_cast<uint4*>(Bs + sw128_offset(CH + col, g * 8)) =
                                    make_uint4(pcl[0], pcl[1], pcl[2], pcl[3]);
                                *reinterpret_cast<uint4*>(Bs + sw128_offset(CH + col + 1, g * 8)) =
                                    make_uint4(psl[0], psl[1], psl[2], psl[3]);
                            }
#pragma unroll
                            for (int p = 0; p < 8; p++) {
                                const float cn = fmaf(2.f * c1[p], cc[p], -cm[p]);
                                const float sn = fmaf(2.f * c1[p], ss[p], -sm[p]);
                                cm[p] = cc[p]; sm[p] = ss[p];
                                cc[p] = cn; ss[p] = sn;
                            }
                        }
                    }
                    fence_proxy_async_smem();
                    mbar_arrive(&bar_bfull[s]);
                }
        }
        if (!ok && it == 0) atomicOr(a.status, 2);
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(taddr, 512);
    }
}

// ---------------------------------------------------------------------------
size_t tensor_smem_bytes(bool bf16)
{
    return (size_t)tc_stages(bf16) * tc_stage_bytes(bf16) + kTcTableSlots * 16 + 1024;
}

size_t tensor_tile_bytes(bool bf16) { return (size_t)tc_wparts(bf16) * kTcA; }

int tensor_tiles_of(int n) { return tc_tiles_of(n + kTcPseudo); }

template <int NMAX, bool BF, bool ZS>
static cudaError_t set_tensor_smem()
{
    cudaError_t e = raise_dyn_smem((const void*)k_pair_tensor<NMAX, BF, false, ZS>, tensor_smem_bytes(BF));
    if (e != cudaSuccess) return e;
    return raise_dyn_smem((const void*)k_pair_tensor<NMAX, BF, true, ZS>, tensor_smem_bytes(BF));
}

cudaError_t prepare_tensor_kernel(int n_max)
{
    cudaError_t e = cudaErrorInvalidValue;
    switch (n_max) {
    case 4:
        e = set_tensor_smem<4, false, false>();
        if (e == cudaSuccess) e = set_tensor_smem<4, true, false>();
        if (e == cudaSuccess) e = set_tensor_smem<4, true, true>();
        break;
    case 8:
        e = set_tensor_smem<8, false, false>();
        if (e == cudaSuccess) e = set_tensor_smem<8, true, false>();
        if (e == cudaSuccess) e = set_tensor_smem<8, true, true>();
        break;
    case 12:
        e = set_tensor_smem<12, false, false>();
        if (e == cudaSuccess) e = set_tensor_smem<12, true, false>();
        break;
    case 16:
        e = set_tensor_smem<16, false, false>();
        if (e == cudaSuccess) e = set_tensor_smem<16, true, false>();
        if (e == cudaSuccess) e = set_tensor_smem<16, true, true>();
        break;
    case 32:
        e = set_tensor_smem<32, false, false>();
        if (e == cudaSuccess) e = set_tensor_smem<32, true, false>();
        if (e == cudaSuccess) e = set_tensor_smem<32, true, true>();
        break;
    case 48:
        e = set_tensor_smem<48, false, false>();
        if (e == cudaSuccess) e = set_tensor_smem<48, true, false>();
        break;
    }
    return e;
}

int tensor_freqs_per_unit(int n_max, bool zsplit) { return zsplit ? tc_ft(n_max, true) : tc_ft(n_max, false); }

cudaError_t launch_build_w16(const BuildW16Args& a, cudaStream_t s)
{
    const int64_t tiles = a.tile_end - a.tile_begin;
    if (tiles <= 0) return cudaSuccess;
    k_build_w16<<<(unsigned)tiles, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_harmonic_coef(const CurveParams* cp, int n_curves, int n_max, int stride, float* coef,
                                 cudaStream_t s)
{
    if (n_max < 1 || n_max > kTcMaxHarmonics || stride < n_max) return cudaErrorInvalidValue;
    k_harmonic_coef<<<(n_curves + 7) / 8, 256, 0, s>>>(cp, n_curves, n_max, stride, coef);
    return cudaGetLastError();
}

cudaError_t launch_pair_tensor(const TensorArgs& a, int grid, cudaStream_t s)
{
    const bool bf = a.bf16 != 0, list = a.stage == kStageList, zs = a.zsplit != 0;
    const size_t b = tensor_smem_bytes(bf);
    if (zs && (!bf || a.n_max == 12 || a.n_max == 48)) return cudaErrorInvalidValue;
#define CP_TC_GO(NM, BFV, LV, ZV) k_pair_tensor<NM, BFV, LV, ZV><<<grid, tc_threads(NM, ZV), b, s>>>(a)
#define CP_TC_LAUNCH(NM, ZOK)                                                                   \
    case NM:                                                                                    \
        if (zs) {                                                                               \
            if constexpr (ZOK) {                                                                \
                if (list) CP_TC_GO(NM, true, true, ZOK);                                        \
                else CP_TC_GO(NM, true, false, ZOK);                                            \
            }                                                                                   \
        } else if (list) {                                                                      \
            if (bf) CP_TC_GO(NM, true, true, false);                                            \
            else CP_TC_GO(NM, false, true, false);                                              \
        } else {                                                                                \
            if (bf) CP_TC_GO(NM, true, false, false);                                           \
            else CP_TC_GO(NM, false, false, false);                                             \
        }                                                                                       \
        break;
    switch (a.n_max) {
        CP_TC_LAUNCH(4, true)
        CP_TC_LAUNCH(8, true)
        CP_TC_LAUNCH(12, false)
        CP_TC_LAUNCH(16, true)
        CP_TC_LAUNCH(32, true)
        CP_TC_LAUNCH(48, false)
    default: return cudaErrorInvalidValue;
    }
#undef CP_TC_LAUNCH
#undef CP_TC_GO
    return cudaGetLastError();
}

}  // namespace cpk
