// Reduced-precision Gaussian sketch on the 5th-generation tensor cores
// (tcgen05, kind::f16 with bf16 operands, fp32 accumulation in TMEM).
//
// The sketch S X of Algorithm 6 (and S M of Algorithm 7) only has to
// be a subspace embedding (Section 3), so its product may run at reduced
// precision.  Y = S X with S generated on the fly: each CTA owns one tile of
// 128 sketch rows x NT columns of Y (M = 128, N = NT <= 256) and a contiguous
// chunk of rows of X (split-K).  For every 32 rows of X the 256 threads
//   * draw the 128 x 32 block of S (bf16 levels, defined below),
//   * load the 32 x NT block of X (binary64) and split each value into one
//     or three bf16 terms x1 = bf16(x), x2 = bf16(x - x1), x3 = bf16(x - x1 - x2),
//   * store both as K-major operand tiles (8 x 8 bf16 core matrices) in
//     shared memory,
// and one thread issues tcgen05.mma for the 16-row k-steps (one MMA per bf16
// term of X), committing to an mbarrier per stage.  Three stages let the
// tensor core consume stage k while the threads fill k+1 and k+2.  At the
// end the fp32 accumulator is read from TMEM (tcgen05.ld), scaled by
// 1/sqrt(s) in binary64 and written as this CTA's partial; partials are
// summed in a fixed order by the same reduction as the FP64 sketch.
//
// S at these tiers: since only an embedding is needed, its entries lie on
// the grid k / 32 of a discretised standard normal, T[j] = k_j / 32 with
// k_j = round(32 Phi^{-1}((j + 1/2) / 4096)) (half to even, |k_j| <= 117),
// drawn eight at a time: entry (r, i) = T[h >> 4] with h the 16-bit half
// (i mod 8) mod 2 of word (i mod 8) div 2 of Philox4x32-10 at counter
// (i div 8 mod 2^32, i div 2^35, r, 0x53424631), key = seed.  The operand
// holds the integer k (an exact bf16); the 1/32 joins 1/sqrt(s) in the
// epilogue.  One Philox block, eight table reads from shared memory and one
// 16-byte store give the eight K-consecutive entries of one operand row.
//
// The digit tier (k_sketch_digits) keeps the same S and writes X in six
// balanced base-256 digits per column (48 bits of each column's largest
// entry): every product k d is an integer below 2^14 and a level's fp32 sum
// over 1024 rows stays below 2^24, so the sums are exact; they are drained
// into int64 per window and into binary64 every 16 windows.  The sketch is
// then the exact sum over X's 48-bit rounding, rounded a few times in
// binary64: no fp32 accumulation error, so it suffices for kappa(X) far
// beyond the reach of the bf16 and three-term tiers.
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "emu.cuh"
#include "kernels.h"
#include "tcgen05.cuh"

namespace rq {
namespace {

constexpr int kTcThreads = 256;
constexpr int kTcBK = 32;      // rows of X per stage
constexpr int kTcStages = 3;
constexpr int kTcM = 128;      // sketch rows per CTA tile
constexpr int kLevels = 4096;  // levels of the discretised normal
constexpr uint32_t kLevelsDomain = 0x53424631u;

// bf16 bits of the integer k_j = round(32 Phi^{-1}((j + 1/2) / 4096)),
// written once per device by k_gauss_levels_init (ensure_sketch_levels()).
__device__ __align__(16) uint16_t g_gauss_levels[kLevels];

// ---- bf16 rounding (nearest, ties to even) ----------------------------------

// binary64 -> nearest bf16 (8 significant bits), as raw bits; normal range.
__device__ __forceinline__ uint16_t bf16_bits_from_f64(double x, double &rounded) {
    unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
    const unsigned long long mag = b & 0x7fffffffffffffffull;
    if (mag == 0) {
        rounded = x;
        return static_cast<uint16_t>((b >> 48) & 0x8000u);
    }
    const unsigned long long lsb = (b >> 45) & 1ull, rnd = (b >> 44) & 1ull;
    const unsigned long long sticky = (b & ((1ull << 44) - 1ull)) != 0ull;
    if (rnd && (sticky || lsb)) b += 1ull << 45;
    b &= ~((1ull << 45) - 1ull);
    rounded = __longlong_as_double(static_cast<long long>(b));
    // repack: sign | exponent rebased 1023 -> 127 | top 7 fraction bits
    const unsigned sign = static_cast<unsigned>(b >> 63);
    const int e = static_cast<int>((b >> 52) & 0x7ff) - 1023 + 127;
    const unsigned frac = static_cast<unsigned>((b >> 45) & 0x7f);
    if (e <= 0) return static_cast<uint16_t>(sign << 15);  // below bf16's normal range: zero
    return static_cast<uint16_t>((sign << 15) | (static_cast<unsigned>(e) << 7) | frac);
}

// Byte offset of element (row, k) inside a K-major operand tile of BK
// columns laid out as [row/8][k/8][row%8][k%8] (bf16).
__device__ __forceinline__ uint32_t kmajor_off(int row, int k) {
    return static_cast<uint32_t>(((row >> 3) * (kTcBK / 8) + (k >> 3)) * 128 + (row & 7) * 16 +
                                 (k & 7) * 2);
}

// k_j from CUDA's normcdfinv in binary64, rounded to the nearest integer
// (ties to even), stored as its bf16 bits.
__global__ void k_gauss_levels_init() {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= kLevels) return;
    const int k = __double2int_rn(32.0 * normcdfinv((double(j) + 0.5) / double(kLevels)));
    g_gauss_levels[j] = static_cast<uint16_t>(small_int_bf16(k));
}

// Eight entries (r, g0 .. g0 + 7) of the reduced tier's S as packed bf16;
// `lv` is the level table in shared memory.  g0 need not be a multiple of 8.
__device__ __forceinline__ uint4 sk_levels8(uint64_t seed, int r, int64_t g0, const uint16_t *lv) {
    const uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
    const uint64_t q = static_cast<uint64_t>(g0) >> 3;
    const int off = static_cast<int>(g0 & 7);
    const uint4 a = philox4x32_10(make_uint4(static_cast<uint32_t>(q), static_cast<uint32_t>(q >> 32),
                                             static_cast<uint32_t>(r), kLevelsDomain), k0, k1);
    uint32_t h[8];
    if (off == 0) {  // one block: word t / 2, half t % 2
        const uint32_t w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
        for (int t = 0; t < 8; ++t) h[t] = lv[((w[t >> 1] >> (16 * (t & 1))) & 0xffffu) >> 4];
    } else {  // entries off .. off + 7 of two consecutive blocks, selected without indexing
        const uint64_t q1 = q + 1;
        const uint4 b = philox4x32_10(make_uint4(static_cast<uint32_t>(q1), static_cast<uint32_t>(q1 >> 32),
                                                 static_cast<uint32_t>(r), kLevelsDomain), k0, k1);
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const int e = off + t, k = (e >> 1) & 3;
            const uint4 v = (e >> 3) ? b : a;
            const uint32_t w = k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
            h[t] = lv[((w >> (16 * (e & 1))) & 0xffffu) >> 4];
        }
    }
    return make_uint4(h[0] | (h[1] << 16), h[2] | (h[3] << 16), h[4] | (h[5] << 16),
                      h[6] | (h[7] << 16));
}

template <int NSL>
__global__ void __launch_bounds__(kTcThreads, 2)
    k_sketch_tc(const double *__restrict__ X, int64_t ldx, int64_t m, int n, int unit_lower,
                int64_t chunk, int n_st, int nt, uint64_t seed, double scale,
                double *__restrict__ part, int s_pad, int n_pad, DevStatus *st, int64_t row0) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar_mma[kTcStages];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    __shared__ __align__(16) uint16_t lv[kLevels];

    const int a_bytes = kTcM * kTcBK * 2;       // 8 KB
    const int b_bytes = nt * kTcBK * 2;         // per bf16 term of X
    const int stage_bytes = a_bytes + NSL * b_bytes;
    const int st_idx = blockIdx.x % n_st, ct_idx = blockIdx.x / n_st;
    const int rt0 = kTcM * st_idx;              // first sketch row of the tile
    const int c0 = 256 * ct_idx;                // first column of the tile
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint32_t ncols = 32;
    while (ncols < static_cast<uint32_t>(nt)) ncols <<= 1;

    if (warp == 0) tmem_alloc(&tmem_slot, ncols);
    if (tid == 0) {
        for (int s = 0; s < kTcStages; ++s) mbar_init(&bar_mma[s], 1);
        fence_mbar_init();
        abort_flag = 0;
    }
    for (int k = tid; k < kLevels / 8; k += kTcThreads)
        reinterpret_cast<uint4 *>(lv)[k] = reinterpret_cast<const uint4 *>(g_gauss_levels)[k];
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const uint32_t idesc = idesc_bf16_f32(kTcM, nt);
    const uint32_t smem_base = smem_u32(smem_raw);

    const int64_t rb = int64_t(blockIdx.y) * chunk;
    const int64_t re = std::min<int64_t>(m, rb + chunk);
    const int nsteps = static_cast<int>(ceil_div(re - rb, kTcBK));
    bool ok = true;
    for (int ks = 0; ks < nsteps; ++ks) {
        const int sidx = ks % kTcStages;
        unsigned char *stage = smem_raw + sidx * stage_bytes;
        const int64_t r0 = rb + int64_t(ks) * kTcBK;
        if (ks >= kTcStages) {
            // the MMAs issued kTcStages steps ago read this stage
            ok = mbar_wait_bounded(&bar_mma[sidx], static_cast<uint32_t>((ks / kTcStages - 1) & 1));
            if (!ok) abort_flag = 1;
        }
        __syncthreads();
        if (abort_flag) break;
        // (0) this stage's X block into registers first: its loads complete
        // while the threads generate S (the longest part of a stage)
        // tasks of 8 rows x 1 column: nt * 4 of them, at most 4 per thread
        const int ntasks = nt * (kTcBK / 8);
        double xv[4][8];
#pragma unroll
        for (int tt = 0; tt < 4; ++tt) {
            const int task = tid + kTcThreads * tt;
            if (task >= ntasks) break;
            const int kb = task % (kTcBK / 8), c = task / (kTcBK / 8);
            const int col = c0 + c;
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int64_t row = r0 + kb * 8 + t;
                double x = 0.0;
                if (row < re && col < n) {
                    x = __ldg(X + row + int64_t(col) * ldx);
                    if (unit_lower && row <= col) x = (row == col) ? 1.0 : 0.0;
                }
                xv[tt][t] = x;
            }
        }
        // (1) S block: entries (r, i) for 128 sketch rows x 32 rows of X, one
        // task per 8 K-consecutive entries of a row (X's rows past the end
        // are zero, so those entries need no masking)
#pragma unroll 2
        for (int task = tid; task < kTcM * (kTcBK / 8); task += kTcThreads) {
            const int kb = task % (kTcBK / 8), r = task / (kTcBK / 8);
            const uint4 v = sk_levels8(seed, rt0 + r, row0 + r0 + 8 * kb, lv);
            *reinterpret_cast<uint4 *>(stage + kmajor_off(r, 8 * kb)) = v;
        }
        // (2) X block split into NSL bf16 terms: 8 consecutive rows of one column per task
#pragma unroll
        for (int tt = 0; tt < 4; ++tt) {
            const int task = tid + kTcThreads * tt;
            if (task >= ntasks) break;
            const int kb = task % (kTcBK / 8), c = task / (kTcBK / 8);
            uint16_t hv[NSL][8];
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const double x = xv[tt][t];
                double rnd;
                hv[0][t] = bf16_bits_from_f64(x, rnd);
                if (NSL == 3) {
                    const double r1 = x - rnd;
                    double rnd2;
                    hv[NSL > 1 ? 1 : 0][t] = bf16_bits_from_f64(r1, rnd2);
                    double rnd3;
                    hv[NSL > 2 ? 2 : 0][t] = bf16_bits_from_f64(r1 - rnd2, rnd3);
                }
            }
#pragma unroll
            for (int p = 0; p < NSL; ++p) {
                uint4 v;
                v.x = uint32_t(hv[p][0]) | (uint32_t(hv[p][1]) << 16);
                v.y = uint32_t(hv[p][2]) | (uint32_t(hv[p][3]) << 16);
                v.z = uint32_t(hv[p][4]) | (uint32_t(hv[p][5]) << 16);
                v.w = uint32_t(hv[p][6]) | (uint32_t(hv[p][7]) << 16);
                *reinterpret_cast<uint4 *>(stage + a_bytes + p * b_bytes + kmajor_off(c, kb * 8)) = v;
            }
        }
        fence_proxy_async_smem();  // generic-proxy stores -> visible to the tensor core
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t a0 = smem_base + sidx * stage_bytes;
#pragma unroll
            for (int kk = 0; kk < kTcBK / 16; ++kk) {
                const uint64_t ad = smem_desc(a0 + kk * 256, 128, kTcBK * 16);
#pragma unroll
                for (int p = 0; p < NSL; ++p) {
                    const uint64_t bd = smem_desc(a0 + a_bytes + p * b_bytes + kk * 256, 128, kTcBK * 16);
                    mma_bf16(tmem, ad, bd, idesc, (ks > 0 || kk > 0 || p > 0) ? 1u : 0u);
                }
            }
            mma_commit(&bar_mma[sidx]);
        }
    }
    // all MMAs done: wait for the last commit (it covers every earlier MMA)
    if (!abort_flag && nsteps > 0) {
        const int last = nsteps - 1;
        const bool okw = mbar_wait_bounded(&bar_mma[last % kTcStages],
                                           static_cast<uint32_t>((last / kTcStages) & 1));
        if (!okw) abort_flag = 1;
    }
    __syncthreads();
    tc_fence_after();
    if (abort_flag) {
        if (tid == 0) report(st, kErrTimeout, 0, -1);
    } else {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 (sketch rows) and
        // half (w / 4) of the columns
        const int lane_base = 32 * (warp & 3);
        const int half = warp >> 2;
        const int nchunks = (nt + 31) / 32;  // 32-column loads (TMEM holds >= 32 columns)
        const int per_half = (nchunks + 1) / 2;
        const int r = rt0 + lane_base + lane;
        double *out = part + size_t(blockIdx.y) * s_pad * n_pad;
        for (int ch = half * per_half; ch < std::min(nchunks, (half + 1) * per_half); ++ch) {
            const int cb = 32 * ch;
            float v[32];
            tmem_ld32(tmem + (static_cast<uint32_t>(lane_base) << 16) + static_cast<uint32_t>(cb), v);
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int c = c0 + cb + j;
                if (cb + j < nt && c < n_pad && r < s_pad)
                    out[size_t(c) * s_pad + r] = double(v[j]) * scale;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, ncols);
}

// ---- digit tier --------------------------------------------------------------

constexpr int kDgDigits = 6;                         // 48 bits of each column of X
constexpr int kDgNC = 32;                            // columns of X per CTA (N of the MMA)
constexpr int kDgStages = 3;
constexpr int kDgWinSteps = 32;                      // 32 stages of 32 rows: 1024-row windows
constexpr int kDgFlushWindows = 16;                  // int64 drains between binary64 flushes
constexpr int kDgTileA = kTcM * kTcBK * 2;           // S: 128 x 32 bf16 (8 KB)
constexpr int kDgTileB = kDgNC * kTcBK * 2;          // one digit of X: 32 x 32 bf16 (2 KB)
constexpr int kDgStageBytes = kDgTileA + kDgDigits * kDgTileB;
constexpr int kDgTmemCols = 256;                     // 6 levels x 32 columns (192) rounded up

// Largest biased exponent field of each column (atomic max; colbits zeroed
// first); with unit_lower the column is read as a unit-lower factor (1 on
// the diagonal, nothing above it).
__global__ void k_dg_col_exponent(const double *__restrict__ A, int64_t lda, int64_t m,
                                  int unit_lower, int64_t chunk, int *__restrict__ colbits) {
    const int j = blockIdx.x;
    const int64_t rb = int64_t(blockIdx.y) * chunk;
    const int64_t re = std::min<int64_t>(m, rb + chunk);
    int e = 0;
    for (int64_t i = rb + threadIdx.x; i < re; i += blockDim.x) {
        double x = A[i + int64_t(j) * lda];
        if (unit_lower && i <= j) x = (i == j) ? 1.0 : 0.0;
        const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
        e = max(e, static_cast<int>((b >> 52) & 0x7ff));
    }
    for (int off = 16; off > 0; off >>= 1) e = max(e, __shfl_down_sync(0xffffffffu, e, off));
    if ((threadIdx.x & 31) == 0 && e > 0) atomicMax(colbits + j, e);
}

// Partial Y of one CTA: 128 sketch rows x 32 columns of X over a chunk of
// rows, in units of 2^(E_c - 44) (binary64), written to
// part[blockIdx.y][c * s_pad + r].  Per 32 rows of X the threads draw S
// (integers k), split X into six digit tiles, and thread 0 issues the six
// level products of each 16-row k-step (kind::f16, M = 128, N = 32): level t
// (digit t of X, weight 256^(5 - t)) in TMEM columns 32 t .. 32 t + 31.
__global__ void __launch_bounds__(kTcThreads, 2)
    k_sketch_digits(const double *__restrict__ X, int64_t ldx, int64_t m, int n, int unit_lower,
                    int64_t chunk, int n_st, uint64_t seed, const int *__restrict__ colbits,
                    double *__restrict__ part, int s_pad, int n_pad, DevStatus *st, int64_t row0) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar_mma[kDgStages];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    __shared__ __align__(16) uint16_t lv[kLevels];
    __shared__ int expB[kDgNC];
    // this thread's 16 int64 window sums (in shared memory: registers are
    // short), acc[q][tid]
    __shared__ long long acc[16][kTcThreads];

    const int st_idx = blockIdx.x % n_st, ct_idx = blockIdx.x / n_st;
    const int rt0 = kTcM * st_idx;  // first sketch row of the tile
    const int c0 = kDgNC * ct_idx;  // first column of X
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == 0) tmem_alloc(&tmem_slot, kDgTmemCols);
    if (tid == 0) {
        for (int q = 0; q < kDgStages; ++q) mbar_init(&bar_mma[q], 1);
        fence_mbar_init();
        abort_flag = 0;
    }
    for (int k = tid; k < kLevels / 8; k += kTcThreads)
        reinterpret_cast<uint4 *>(lv)[k] = reinterpret_cast<const uint4 *>(g_gauss_levels)[k];
    if (tid < kDgNC) expB[tid] = (c0 + tid < n) ? emu_exponent(colbits[c0 + tid]) : 0;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const uint32_t idesc = idesc_bf16_f32(kTcM, kDgNC);
    const uint32_t smem_base = smem_u32(smem_raw);

    // drain ownership: TMEM lanes 32 (warp % 4) .. +31 (sketch rows), columns
    // 16 (warp / 4) .. +15
    const int lane_base = 32 * (warp & 3);
    const int half = warp >> 2;
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q][tid] = 0;
    double *mine = part + size_t(blockIdx.y) * s_pad * n_pad + size_t(c0 + 16 * half) * s_pad +
                   rt0 + lane_base + lane;
    int windows = 0;
    bool flushed = false;
    auto flush = [&]() {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const double v = static_cast<double>(acc[q][tid]);
            mine[size_t(q) * s_pad] = flushed ? mine[size_t(q) * s_pad] + v : v;
            acc[q][tid] = 0;
        }
        flushed = true;
    };

    const int64_t rb = int64_t(blockIdx.y) * chunk;
    const int64_t re = std::min<int64_t>(m, rb + chunk);
    const int nsteps = re > rb ? static_cast<int>(ceil_div(re - rb, kTcBK)) : 0;
    // this thread's X task: column c0 + (tid % 32), rows 4 (tid / 32) .. +3 of a stage
    const int xc = tid % kDgNC, xq = tid / kDgNC;
    const int xcol = c0 + xc;
    for (int ks = 0; ks < nsteps; ++ks) {
        const int sidx = ks % kDgStages;
        unsigned char *stage = smem_raw + sidx * kDgStageBytes;
        const int64_t r0 = rb + int64_t(ks) * kTcBK;
        // (0) the thread's four values of X (in flight during the wait and S)
        double xv[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int64_t row = r0 + 4 * xq + t;
            double x = 0.0;
            if (row < re && xcol < n) {
                x = __ldg(X + row + int64_t(xcol) * ldx);
                if (unit_lower && row <= xcol) x = (row == xcol) ? 1.0 : 0.0;
            }
            xv[t] = x;
        }
        if (ks >= kDgStages &&
            !mbar_wait_bounded(&bar_mma[sidx], static_cast<uint32_t>((ks / kDgStages - 1) & 1)))
            abort_flag = 1;
        __syncthreads();
        if (abort_flag) break;
        // (1) S block: 128 sketch rows x 32 rows of X, eight K-consecutive
        // entries per task (X's rows past the end are zero)
#pragma unroll 1
        for (int task = tid; task < kTcM * (kTcBK / 8); task += kTcThreads) {
            const int kb = task % (kTcBK / 8), r = task / (kTcBK / 8);
            *reinterpret_cast<uint4 *>(stage + kmajor_off(r, 8 * kb)) =
                sk_levels8(seed, rt0 + r, row0 + r0 + 8 * kb, lv);
        }
        // (2) six digits of the thread's four values: one 8-byte piece per digit tile
        {
            const int E = expB[xc];
            uint32_t w[kDgDigits][2];
#pragma unroll
            for (int t = 0; t < 4; t += 2) {
                uint32_t wp[kDgDigits];
                emu_digits2_packed<kDgDigits>(xv[t], xv[t + 1], E, wp);
#pragma unroll
                for (int q = 0; q < kDgDigits; ++q) w[q][t >> 1] = wp[q];
            }
            const uint32_t off = static_cast<uint32_t>(((xc >> 3) * (kTcBK / 8) + (xq >> 1)) * 128 +
                                                       (xc & 7) * 16 + (xq & 1) * 8);
#pragma unroll
            for (int q = 0; q < kDgDigits; ++q)
                *reinterpret_cast<uint2 *>(stage + kDgTileA + q * kDgTileB + off) = make_uint2(w[q][0], w[q][1]);
        }
        fence_proxy_async_smem();  // generic-proxy stores -> visible to the tensor core
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t a0 = smem_base + sidx * kDgStageBytes;
            const bool fresh = (ks % kDgWinSteps) == 0;
#pragma unroll
            for (int kk = 0; kk < kTcBK / 16; ++kk) {
                const uint64_t ad = smem_desc(a0 + kk * 256, 128, kTcBK * 16);
#pragma unroll
                for (int t = 0; t < kDgDigits; ++t) {
                    const uint64_t bd = smem_desc(a0 + kDgTileA + t * kDgTileB + kk * 256, 128, kTcBK * 16);
                    mma_bf16(tmem + static_cast<uint32_t>(t * kDgNC), ad, bd, idesc,
                             (fresh && kk == 0) ? 0u : 1u);
                }
            }
            mma_commit(&bar_mma[sidx]);
        }
        // (3) end of a window: drain the six level accumulators into int64,
        // in units of 2^8 (level 5 rounded to that unit)
        if ((ks % kDgWinSteps) == kDgWinSteps - 1 || ks == nsteps - 1) {
            if (!mbar_wait_bounded(&bar_mma[sidx], static_cast<uint32_t>((ks / kDgStages) & 1)))
                abort_flag = 1;
            tc_fence_after();
            const uint32_t tl = tmem + (static_cast<uint32_t>(lane_base) << 16) +
                                static_cast<uint32_t>(16 * half);
            float v[16];
#pragma unroll
            for (int t = 0; t < kDgDigits; ++t) {
                tmem_ld16(tl + static_cast<uint32_t>(t * kDgNC), v);
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    long long a;
                    switch (t) {  // compile-time after unrolling
                        case 0: a = emu_level<32>(v[q]); break;
                        case 1: a = emu_level<24>(v[q]); break;
                        case 2: a = emu_level<16>(v[q]); break;
                        case 3: a = emu_level<8>(v[q]); break;
                        case 4: a = emu_level<0>(v[q]); break;
                        default: a = emu_level<-8>(v[q]); break;
                    }
                    acc[q][tid] += a;
                }
            }
            if (++windows == kDgFlushWindows) {
                flush();
                windows = 0;
            }
            tc_fence_before();  // the next iteration's barrier orders these reads before its MMAs
        }
    }
    __syncthreads();
    if (abort_flag) {
        if (tid == 0) report(st, kErrTimeout, 0, -1);
    } else {
        flush();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kDgTmemCols);
}

// Y[r][c] = 2^(E_c - 44) / sqrt(s) times the sum over the CTAs (in order) of
// their partials; NaN where column c holds a non-finite value.
__global__ void k_reduce_sketch_digits(const double *__restrict__ part, int nparts, int s, int n,
                                       int s_pad, int n_pad, const int *__restrict__ colbits,
                                       double scale, double *__restrict__ Y, int64_t ldy) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= int64_t(s) * n) return;
    const int r = static_cast<int>(e % s), c = static_cast<int>(e / s);
    const double v = ordered_sum(part + size_t(c) * s_pad + r, size_t(s_pad) * n_pad, nparts);
    const int bits = __ldg(colbits + c);
    Y[r + int64_t(c) * ldy] = bits == 0x7ff ? __longlong_as_double(0x7ff8000000000000ll)
                                            : ldexp(v, emu_exponent(bits) - 44) * scale;
}

}  // namespace

// Writes the level table of the reduced tier's S on the current device,
// once per device, on a private stream, and waits for it.  Called when a
// handle is created, so that no launch that reads the table (or a graph
// captured later) can run before it is written.
cudaError_t ensure_sketch_levels() {
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> g(mu);
    if (done[dev]) return cudaSuccess;
    cudaStream_t s = nullptr;
    if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) return e;
    RQ_LAUNCH(KID_SKETCH_TC, s, k_gauss_levels_init<<<kLevels / 256, 256, 0, s>>>());
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    if (e == cudaSuccess) done[dev] = true;
    return e;
}

size_t tc_sketch_smem_bytes(int n, int nterms) {
    const int nt = std::min(pad16(n), 256);
    return size_t(kTcStages) * (size_t(kTcM) * kTcBK * 2 + size_t(nterms) * nt * kTcBK * 2);
}

cudaError_t launch_sketch_tc(const double *X, int64_t ldx, int64_t m, int n, int unit_lower,
                             int64_t s, uint64_t seed, int nterms, double *Y, int64_t ldy,
                             double *part, DevStatus *st, cudaStream_t stream, int64_t row0) {
    if (n > 256 || (nterms != 1 && nterms != 3)) return cudaErrorInvalidValue;
    const int nt = std::min(pad16(n), 256);
    const int s_pad = static_cast<int>(round_up(s, kTcM));
    const int n_pad = static_cast<int>(round_up(n, 32));
    const int n_st = s_pad / kTcM;
    const int tiles = n_st;  // n <= 256: one column tile
    // CTAs per SM: two when their TMEM columns (<= 256 each) and shared
    // memory both fit, so that one CTA's generation of S covers the other's
    // load latency; each CTA's stages stay below half the SM's shared memory
    const size_t smem = tc_sketch_smem_bytes(n, nterms);
    const int per_sm = smem <= 100 * 1024 ? 2 : 1;  // plus 8 KB of levels each
    int p = std::max(1, per_sm * grid_sms() / tiles);
    int64_t chunk = round_up(ceil_div(m, p), kTcBK);
    p = static_cast<int>(ceil_div(m, chunk));
    const dim3 grid(tiles, p);
    const double scale = 1.0 / (32.0 * sqrt(double(s)));  // the grid's 1/32 and 1/sqrt(s)
    if (nterms == 1) {
        cudaFuncSetAttribute(k_sketch_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        RQ_LAUNCH(KID_SKETCH_TC, stream,
                  k_sketch_tc<1><<<grid, kTcThreads, smem, stream>>>(X, ldx, m, n, unit_lower, chunk,
                                                                   n_st, nt, seed, scale, part,
                                                                   s_pad, n_pad, st, row0));
    } else {
        cudaFuncSetAttribute(k_sketch_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        RQ_LAUNCH(KID_SKETCH_TC, stream,
                  k_sketch_tc<3><<<grid, kTcThreads, smem, stream>>>(X, ldx, m, n, unit_lower, chunk,
                                                                   n_st, nt, seed, scale, part,
                                                                   s_pad, n_pad, st, row0));
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_reduce_sketch(part, p, static_cast<int>(s), n, s_pad, n_pad, Y, ldy, stream);
}

size_t sketch_digits_partials_doubles(int64_t s, int n) {
    const size_t tiles = size_t(round_up(s, kTcM) / kTcM) * size_t(ceil_div(n, kDgNC));
    const size_t p = std::max<size_t>(1, size_t(2) * num_sms() / tiles) + 1;
    return p * size_t(round_up(s, kTcM)) * size_t(round_up(n, kDgNC)) + size_t(n) + 64;
}

cudaError_t launch_sketch_digits(const double *X, int64_t ldx, int64_t m, int n, int unit_lower,
                                 int64_t s, uint64_t seed, double *Y, int64_t ldy, double *part,
                                 DevStatus *st, cudaStream_t stream, int64_t row0) {
    if (n > 256 || s > 4096) return cudaErrorInvalidValue;
    const int s_pad = static_cast<int>(round_up(s, kTcM));
    const int n_pad = static_cast<int>(round_up(n, kDgNC));
    const int n_st = s_pad / kTcM, n_ct = n_pad / kDgNC;
    const int tiles = n_st * n_ct;
    int p = std::max(1, 2 * grid_sms() / tiles);
    const int64_t chunk = round_up(ceil_div(m, p), kTcBK);
    p = static_cast<int>(ceil_div(m, chunk));
    int *colbits = reinterpret_cast<int *>(part + size_t(p) * s_pad * n_pad);
    cudaError_t e = cudaMemsetAsync(colbits, 0, sizeof(int) * size_t(n), stream);
    if (e != cudaSuccess) return e;
    const int64_t cchunk = std::max<int64_t>(4096, ceil_div(m, 64));
    RQ_LAUNCH(KID_EMU_AUX, stream,
              k_dg_col_exponent<<<dim3(n, static_cast<unsigned>(ceil_div(m, cchunk))), 256, 0, stream>>>(
                  X, ldx, m, unit_lower, cchunk, colbits));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const size_t smem = size_t(kDgStages) * kDgStageBytes;
    cudaFuncSetAttribute(k_sketch_digits, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    RQ_LAUNCH(KID_SKETCH_TC, stream,
              k_sketch_digits<<<dim3(tiles, p), kTcThreads, smem, stream>>>(
                  X, ldx, m, n, unit_lower, chunk, n_st, seed, colbits, part, s_pad, n_pad, st, row0));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int64_t ne = s * int64_t(n);
    RQ_LAUNCH(KID_REDUCE, stream,
              k_reduce_sketch_digits<<<static_cast<unsigned>(ceil_div(ne, 256)), 256, 0, stream>>>(
                  part, p, static_cast<int>(s), n, s_pad, n_pad, colbits, 1.0 / sqrt(double(s)), Y, ldy));
    return cudaGetLastError();
}

}  // namespace rq
