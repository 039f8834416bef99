// Triangular solve Q = A R^{-1} for a well-conditioned upper-triangular R as
// one binary64-emulating product Q = A W with W = R^{-1} (the precision form
// of the second and final solves of CholeskyQR2, C3 and C7, whose factors R2
// and R4 have the condition number of Q1 and of Q2: a few units after a
// sketch that embeds).
//
// W is formed once in binary64 by forward substitution along its rows
// (k_tri_inverse, one warp per row), and Skeel's condition number
// cond(R) = || |R^{-1}| |R| ||_inf, which bounds the product's residual
// (|Q R - A| <= c u |A| |W| |R|), is taken on the way.  Both this product and
// the substitution kernel of emu_trsm.cu are launched; each reads cond(R) and
// only one of them runs: the product when cond(R) <= max(kWprodMaxCond, n)
// (its residual bound then stays within the substitution's own, gamma_n
// |Q| |R| ~ n u), the substitution otherwise.  No host round trip, so the
// pair can be captured in a graph.
//
// The product: digits of A's rows (one exponent per row over all n columns of
// A, known before anything is written) and of W's columns (one exponent per
// column), levels s + t <= 7 summed exactly in fp32 over at most 128
// K-columns, drained into int64 (units 2^-40 of level 0), scaled into
// binary64.  One CTA per SM owns 128-row tiles; passes of 64 output columns
// (all 512 TMEM columns: eight levels) run from the last to the first, so
// that a pass reads only columns of A below the ones it writes and Q may
// alias A.  Warp-specialised (k_wprod_emu): 16 producer warps split each
// 32-column K-chunk of their rows into eight K-major digit tiles while the
// control warp bulk-copies W's precomputed digit tiles and issues the level
// products as 24 wide MMAs (kind::f16, M = 128, N = 64 .. 256, K = 16: one
// digit of A times up to four side-by-side digits of W).  No binary64
// arithmetic remains on the rows.
#include <algorithm>
#include <cstring>

#include "common.cuh"
#include "emu.cuh"
#include "kernels.h"
#include "tcgen05.cuh"

namespace rq {
namespace {

constexpr int kWpProducers = 512;    // 16 producer warps
constexpr int kWpThreads = kWpProducers + 32;  // plus the control warp
constexpr int kWpM = 128;            // rows per tile
constexpr int kWpK = 32;             // K-columns per chunk (two k-steps of the MMA)
constexpr int kWpN = 64;             // output columns per pass
constexpr int kWpWinChunks = 4;      // K-chunks per exact window (128 K-columns)
constexpr int kWpStages = 2;
constexpr int kWpTileA = kWpM * kWpK * 2;   // one digit tile of A: 8 KB
constexpr int kWpTileB = kWpN * kWpK * 2;   // one digit tile of W: 4 KB
constexpr int kWpStageA = kEmuDigits * kWpTileA;
constexpr int kWpStageB = kEmuDigits * kWpTileB;
constexpr int kWpStageBytes = kWpStageA + kWpStageB;
constexpr int kWpTmemCols = 512;     // eight 64-column level accumulators
constexpr int kWpUnit = 16;          // drain units: 2^-(24 + 16) of level 0

// Byte offset of element (row, k) of a K-major tile of 32 K-columns laid
// out as [row/8][k/8][row%8][k%8] (bf16).
__host__ __device__ __forceinline__ uint32_t wp_off(int row, int k) {
    return static_cast<uint32_t>(((row >> 3) * (kWpK / 8) + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// Index of W's digit tiles for (pass g, K-chunk kc), kc <= 2g + 1.
__host__ __device__ __forceinline__ size_t wp_tile(int g, int kc) {
    return size_t(g) * (g + 1) + kc;
}

// Scratch layout (bytes from its start): the two norm maxima (as ordered
// bits), then W's column exponents, then W (n_pad x n_pad binary64), then the
// digit tiles.
struct WpLayout {
    size_t norms, cbits, w, tiles, total;
};

__host__ __device__ __forceinline__ WpLayout wp_layout(int n) {
    const int n_pad = pad16(n);
    const int npn = (n + kWpN - 1) / kWpN * kWpN;
    const int passes = npn / kWpN;
    WpLayout l;
    l.norms = 0;
    l.cbits = 256;
    l.w = l.cbits + ((size_t(npn) * sizeof(int) + 255) / 256) * 256;
    l.tiles = l.w + ((size_t(n_pad) * n_pad * 8 + 1023) / 1024) * 1024;
    l.total = l.tiles + wp_tile(passes, 0) * kWpStageB + 256;
    return l;
}

// W = R^{-1} (binary64, column-major n_pad x n_pad, zeros below the diagonal
// and in the padding) by rows, one warp per row i: w_ii = 1 / r_ii,
// w_ij = -(sum_{k = i..j-1} w_ik r_kj) / r_jj for j > i (the reciprocal
// multiplied, as in the binary64 substitution), the sum split over the lanes
// and combined by shuffles.  Each row is a forward substitution with R, so
// the left residual is small, |W R - I| <= c_n u |W| |R|, and the product
// Q = A W then has the residual |Q R - A| <= c u |A| |W| |R|.  Its bound,
// Skeel's condition number cond(R) = || |W| |R| ||_inf = max_i sum_k |w_ik|
// rho_k (rho_k = sum_j |r_kj|), is folded into norms[0]; block 0 stores the
// selection limit max(kWprodMaxCond, n) in norms[1].
__global__ void k_tri_inverse(const double *__restrict__ RP, const double *__restrict__ rinv, int n,
                              int n_pad, double *__restrict__ W, unsigned long long *norms) {
    extern __shared__ double ti_smem[];  // rho (n_pad), then one row of W per warp
    const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double *rho = ti_smem;
    double *wr = ti_smem + n_pad + size_t(warp) * n_pad;
    const double *RT = RP + size_t(n_pad) * n_pad;  // row-major copy: RT[k * n_pad + j] = r_kj
    for (int k = warp; k < n_pad; k += nw) {
        double a = 0.0;
        for (int j = lane; j < n_pad; j += 32) a += fabs(RT[size_t(k) * n_pad + j]);
        for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
        if (lane == 0) rho[k] = a;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const double lim = n > kWprodMaxCond ? double(n) : kWprodMaxCond;
        norms[1] = static_cast<unsigned long long>(__double_as_longlong(lim));
    }
    __syncthreads();
    const int i = blockIdx.x * nw + warp;
    if (i >= n_pad) return;
    for (int j = lane; j < n_pad; j += 32) wr[j] = 0.0;
    __syncwarp();
    if (i < n) {
        if (lane == 0) wr[i] = rinv[i];
        __syncwarp();
        for (int j = i + 1; j < n; ++j) {
            double acc = 0.0;
            for (int k = i + lane; k < j; k += 32) acc = fma(wr[k], RP[size_t(j) * n_pad + k], acc);
            for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
            if (lane == 0) wr[j] = -acc * rinv[j];
            __syncwarp();
        }
    }
    double t = 0.0;
    for (int j = lane; j < n_pad; j += 32) {
        W[size_t(j) * n_pad + i] = wr[j];
        t = fma(fabs(wr[j]), rho[j], t);
    }
    for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
    // non-negative doubles order like their bits; a NaN sum maps to the
    // largest bits and rejects the product
    if (lane == 0) atomicMax(norms, static_cast<unsigned long long>(__double_as_longlong(t == t ? t : INFINITY)));
}

// Column exponents of W (over all its rows) and its digit tiles for every
// (pass g, K-chunk kc <= 2g + 1): one CTA per pass.
__global__ void k_wprod_prep(const double *__restrict__ W, int n, int n_pad,
                             const unsigned long long *norms, int *__restrict__ cbits,
                             unsigned char *__restrict__ tiles) {
    if (!wprod_selected(norms)) return;
    const int g = blockIdx.x;
    const int c0 = kWpN * g;
    __shared__ int cb[kWpN];
    if (threadIdx.x < kWpN) {
        const int c = c0 + threadIdx.x;
        int e = 0;
        if (c < n)
            for (int k = 0; k <= c; ++k) {
                const unsigned long long b =
                    static_cast<unsigned long long>(__double_as_longlong(W[size_t(c) * n_pad + k]));
                e = max(e, static_cast<int>((b >> 52) & 0x7ff));
            }
        cb[threadIdx.x] = e;
        cbits[c] = e;
    }
    __syncthreads();
    const int nk = std::min(2 * g + 2, (n + kWpK - 1) / kWpK);
    for (int idx = threadIdx.x; idx < nk * kWpK * kWpN; idx += blockDim.x) {
        const int k = idx % (nk * kWpK), c = idx / (nk * kWpK);
        const int col = c0 + c;
        const double w = (col < n && k < n_pad) ? W[size_t(col) * n_pad + k] : 0.0;
        int d[kEmuDigits];
        emu_digits(w, emu_exponent(cb[c]), d);
        unsigned char *tile = tiles + wp_tile(g, k / kWpK) * kWpStageB;
#pragma unroll
        for (int s = 0; s < kEmuDigits; ++s)
            *reinterpret_cast<uint16_t *>(tile + s * kWpTileB + wp_off(c, k % kWpK)) =
                static_cast<uint16_t>(small_int_bf16(d[s]));
    }
}

// Pipeline state of k_wprod_emu: per stage, the producers' digit tiles of A
// are written (full, one arrival per producer warp), W's digit tiles have
// landed (wfull) and the MMAs that read the stage are done (empty); per
// window, the MMAs are complete (win_done) and the accumulators are drained
// (tmem_empty).  Every thread that waits on a barrier waits on each of its
// completions in order.
struct WpPipe {
    uint64_t full[kWpStages], wfull[kWpStages], empty[kWpStages];
    uint64_t win_done, tmem_empty;
    uint64_t rowx;  // a tile's row-exponent parts are written
    uint32_t tmem_slot;
    int abort_flag;
};

__device__ __forceinline__ bool wp_aborted(WpPipe &pp) {
    return *reinterpret_cast<volatile int *>(&pp.abort_flag) != 0;
}

__device__ __forceinline__ bool wp_wait(WpPipe &pp, uint64_t *bar, uint32_t parity) {
    if (wp_aborted(pp)) return false;
    if (mbar_wait_bounded(bar, parity)) return true;
    *reinterpret_cast<volatile int *>(&pp.abort_flag) = 1;
    return false;
}

// Warp-specialised: per 128-row tile and 64-column pass (last first, so
// that a pass reads only columns of A below the ones it writes and Q may
// alias A), per 32-column K-chunk the 16 producer warps split their rows'
// values into eight digit tiles of A (four threads per row, eight K-columns
// each), while lane 0 of the control warp bulk-copies W's precomputed digit
// tiles into the same stage and issues the chunk's level products as 24 wide
// MMAs (kind::f16, M = 128, N = 64 .. 256, K = 16).  After each window (at most four
// chunks: 128 K-columns) the producers drain the eight levels into int64;
// at a pass's end they write Q.
__global__ void __launch_bounds__(kWpThreads, 1)
    k_wprod_emu(const double *A, int64_t lda, int64_t m, int n, int64_t chunk,
                const unsigned long long *norms, const int *__restrict__ cbits,
                const unsigned char *__restrict__ tiles, double *Q, int64_t ldq, DevStatus *st) {
    if (!wprod_selected(norms)) return;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ WpPipe pp;
    __shared__ int rowbits_part[kWpProducers / kWpM][kWpM];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool control = warp == kWpProducers / 32;
    if (control) tmem_alloc(&pp.tmem_slot, kWpTmemCols);
    if (tid == 0) {
        for (int q = 0; q < kWpStages; ++q) {
            mbar_init(&pp.full[q], kWpProducers / 32);
            mbar_init(&pp.wfull[q], 1);
            mbar_init(&pp.empty[q], 1);
        }
        mbar_init(&pp.win_done, 1);
        mbar_init(&pp.tmem_empty, kWpProducers / 32);
        mbar_init(&pp.rowx, kWpProducers / 32);
        fence_mbar_init();
        pp.abort_flag = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = pp.tmem_slot;
    const int nkc = (n + kWpK - 1) / kWpK;
    const int passes = (n + kWpN - 1) / kWpN;
    const int64_t rb = int64_t(blockIdx.x) * chunk;
    const int64_t re = std::min<int64_t>(m, rb + chunk);
    const int ntiles = re > rb ? static_cast<int>(ceil_div(re - rb, kWpM)) : 0;
    int committed = -1, wcopies = 0;  // the control thread's last commit, W copies issued

    if (control) {
        // W's tiles of chunk `it` (pass g, K-chunk kc) into its stage, once
        // the MMAs that last read the stage are done (lane 0)
        auto copy_w = [&](int it, int g, int kc) -> bool {
            const int s = it % kWpStages;
            if (it >= kWpStages &&
                !wp_wait(pp, &pp.empty[s], static_cast<uint32_t>((it / kWpStages - 1) & 1)))
                return false;
            mbar_arrive_expect_tx(&pp.wfull[s], kWpStageB);
            bulk_load(smem_raw + s * kWpStageBytes + kWpStageA, tiles + wp_tile(g, kc) * kWpStageB,
                      kWpStageB, &pp.wfull[s]);
            wcopies = it + 1;
            return true;
        };
        int it = 0, win = 0;
        bool ok = true;
        // the chunk after (it, g, kc) in the schedule, for the copy one ahead
        int ng = passes - 1, nkn = 0, ntile = 0;
        auto advance = [&]() {
            if (++nkn == std::min(2 * ng + 2, nkc)) {
                nkn = 0;
                if (--ng < 0) {
                    ng = passes - 1;
                    ++ntile;
                }
            }
        };
        if (ntiles > 0 && lane == 0) ok = copy_w(0, ng, nkn);
        advance();
        for (int t = 0; t < ntiles && ok; ++t)
            for (int g = passes - 1; g >= 0 && ok; --g) {
                const int nk = std::min(2 * g + 2, nkc);
                for (int kc = 0; kc < nk; ++kc, ++it) {
                    const int s = it % kWpStages;
                    const bool fresh = (kc % kWpWinChunks) == 0;
                    const bool wend = (kc % kWpWinChunks) == kWpWinChunks - 1 || kc == nk - 1;
                    int okw = 1;
                    if (lane == 0)
                        okw = (!fresh || win == 0 ||
                               wp_wait(pp, &pp.tmem_empty, static_cast<uint32_t>((win - 1) & 1))) &&
                              wp_wait(pp, &pp.full[s], static_cast<uint32_t>((it / kWpStages) & 1)) &&
                              wp_wait(pp, &pp.wfull[s], static_cast<uint32_t>((it / kWpStages) & 1));
                    if (!__shfl_sync(0xffffffffu, okw, 0)) {
                        ok = false;
                        break;
                    }
                    const uint32_t sa = smem_u32(smem_raw + s * kWpStageBytes);
                    const uint64_t adA = smem_desc(sa, 128, (kWpK / 8) * 128);
                    const uint64_t adB = smem_desc(sa + kWpStageA, 128, (kWpK / 8) * 128);
                    if (lane == 0) {
                        tc_fence_after();
                        // W's eight digit tiles lie side by side (64 rows of the
                        // K-major operand each): digit sd of A times up to four
                        // adjacent digits t0 .. t0 + w - 1 of W is one MMA of
                        // N = 64 w into levels sd + t0 .. (TMEM columns
                        // 64 (sd + t0) ..); twelve MMAs per k-step for the 36
                        // pairs, the two with sd = 0 first (they write every
                        // level, so only they start a window afresh)
#pragma unroll
                        for (int kk = 0; kk < kWpK / 16; ++kk) {
                            const uint32_t a0 = (fresh && kk == 0) ? 0u : 1u;
                            const uint64_t ak = adA + static_cast<uint64_t>(kk * 16);
                            const uint64_t bk = adB + static_cast<uint64_t>(kk * 16);
                            const uint64_t bk4 = bk + static_cast<uint64_t>(4 * (kWpTileB >> 4));
                            mma_bf16(tmem, ak, bk, idesc_bf16_f32(kWpM, 4 * kWpN), a0);
                            mma_bf16(tmem + 4 * kWpN, ak, bk4, idesc_bf16_f32(kWpM, 4 * kWpN), a0);
#pragma unroll
                            for (int sd = 1; sd < kEmuDigits; ++sd) {
                                const uint64_t as = ak + static_cast<uint64_t>(sd * (kWpTileA >> 4));
                                const int w0 = (kEmuDigits - sd) < 4 ? (kEmuDigits - sd) : 4;
                                mma_bf16(tmem + static_cast<uint32_t>(sd * kWpN), as, bk,
                                         idesc_bf16_f32(kWpM, w0 * kWpN), 1u);
                                if (sd < 4)
                                    mma_bf16(tmem + static_cast<uint32_t>((sd + 4) * kWpN), as, bk4,
                                             idesc_bf16_f32(kWpM, (4 - sd) * kWpN), 1u);
                            }
                        }
                        mma_commit(&pp.empty[s]);
                        if (wend) mma_commit(&pp.win_done);
                        committed = it;
                        // the next chunk's W while these products run
                        if (ntile < ntiles) ok = copy_w(it + 1, ng, nkn);
                    }
                    ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
                    if (!ok) break;
                    advance();
                    if (wend) ++win;
                }
            }
    } else {
        const int r = 32 * (warp & 3) + lane;                   // this thread's row of the tile
        const int kb = warp >> 2;                              // its eight K-columns of a chunk
        const int cgrp = warp >> 2;                            // its 16 drain columns of a pass
        long long acc[16];
        int it = 0, win = 0;
        bool ok = true;
        for (int t = 0; t < ntiles && ok; ++t) {
            const int64_t row = rb + int64_t(t) * kWpM + r;
            const bool live = row < re;
            // the row's exponent over all n columns of A (its four threads
            // scan a quarter each)
            int eb = 0;
            if (live)
                for (int c = kb; c < n; c += 4) {
                    const unsigned long long b = static_cast<unsigned long long>(
                        __double_as_longlong(__ldcg(A + row + int64_t(c) * lda)));
                    eb = max(eb, static_cast<int>((b >> 52) & 0x7ff));
                }
            rowbits_part[kb][r] = eb;
            __syncwarp();
            if (lane == 0) mbar_arrive(&pp.rowx);
            if (!wp_wait(pp, &pp.rowx, static_cast<uint32_t>(t & 1))) {
                ok = false;
                break;
            }
            const int rowbits = max(max(rowbits_part[0][r], rowbits_part[1][r]),
                                    max(rowbits_part[2][r], rowbits_part[3][r]));
            const int E = emu_exponent(rowbits);
            for (int g = passes - 1; g >= 0 && ok; --g) {
                const int nk = std::min(2 * g + 2, nkc);
#pragma unroll
                for (int q = 0; q < 16; ++q) acc[q] = 0;
                for (int kc = 0; kc < nk; ++kc, ++it) {
                    const int s = it % kWpStages;
                    unsigned char *stage = smem_raw + s * kWpStageBytes;
                    // this thread's eight values of the chunk (in flight during the wait)
                    double xv[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int col = kWpK * kc + 8 * kb + u;
                        xv[u] = (live && col < n) ? __ldcg(A + row + int64_t(col) * lda) : 0.0;
                    }
                    if (it >= kWpStages &&
                        !wp_wait(pp, &pp.empty[s], static_cast<uint32_t>((it / kWpStages - 1) & 1))) {
                        ok = false;
                        break;
                    }
                    // digits, two K-neighbours per 32-bit word; the eight of a digit
                    // are one 16-byte row of a core matrix, stored at once
                    {
                        uint32_t w[kEmuDigits][4];
#pragma unroll
                        for (int u = 0; u < 8; u += 2) {
                            uint32_t wp[kEmuDigits];
                            emu_digits2_packed<kEmuDigits>(xv[u], xv[u + 1], E, wp);
#pragma unroll
                            for (int d = 0; d < kEmuDigits; ++d) w[d][u >> 1] = wp[d];
                        }
#pragma unroll
                        for (int d = 0; d < kEmuDigits; ++d)
                            *reinterpret_cast<uint4 *>(stage + d * kWpTileA + wp_off(r, 8 * kb)) =
                                make_uint4(w[d][0], w[d][1], w[d][2], w[d][3]);
                    }
                    fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&pp.full[s]);
                    if ((kc % kWpWinChunks) == kWpWinChunks - 1 || kc == nk - 1) {
                        // window end: drain the eight levels of this thread's 16 columns
                        if (!wp_wait(pp, &pp.win_done, static_cast<uint32_t>(win & 1))) {
                            ok = false;
                            break;
                        }
                        ++win;
                        tc_fence_after();
                        const uint32_t tl = tmem + (static_cast<uint32_t>(32 * (warp & 3)) << 16) +
                                            static_cast<uint32_t>(16 * cgrp);
                        float v[16];
#pragma unroll
                        for (int L = 0; L < kEmuDigits; ++L) {
                            tmem_ld16(tl + static_cast<uint32_t>(L * kWpN), v);
#pragma unroll
                            for (int q = 0; q < 16; ++q) {
                                switch (L) {  // compile-time after unrolling
                                    case 0: acc[q] += emu_level<24 + kWpUnit>(v[q]); break;
                                    case 1: acc[q] += emu_level<16 + kWpUnit>(v[q]); break;
                                    case 2: acc[q] += emu_level<8 + kWpUnit>(v[q]); break;
                                    case 3: acc[q] += emu_level<0 + kWpUnit>(v[q]); break;
                                    case 4: acc[q] += emu_level<-8 + kWpUnit>(v[q]); break;
                                    case 5: acc[q] += emu_level<-16 + kWpUnit>(v[q]); break;
                                    case 6: acc[q] += emu_level<-24 + kWpUnit>(v[q]); break;
                                    default: acc[q] += emu_level<-32 + kWpUnit>(v[q]); break;
                                }
                            }
                        }
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&pp.tmem_empty);
                        if (kc == nk - 1 && live) {
                            // Q[row, 64 g + 16 cgrp + q] = 2^(E + E'_c - 54) acc[q]
#pragma unroll
                            for (int q = 0; q < 16; ++q) {
                                const int col = kWpN * g + 16 * cgrp + q;
                                if (col < n) {
                                    const int cb = __ldg(cbits + col);
                                    Q[row + int64_t(col) * ldq] =
                                        (rowbits == 0x7ff || cb == 0x7ff)
                                            ? __longlong_as_double(0x7ff8000000000000ll)
                                            : emu_i64_scaled(acc[q], E + emu_exponent(cb) - 14 - 24 - kWpUnit);
                                }
                            }
                        }
                    }
                }
            }
        }
    }
    __syncthreads();
    if (wp_aborted(pp)) {
        if (tid == 0) report(st, kErrTimeout, 0, -1);
        if (control && lane == 0) {
            // the copies and products in flight land before the shared
            // memory and TMEM are released (bounded waits)
            for (int q = 0; q < kWpStages && q < wcopies; ++q) {
                const int c = q + ((wcopies - 1 - q) / kWpStages) * kWpStages;
                (void)mbar_wait_bounded(&pp.wfull[q], static_cast<uint32_t>((c / kWpStages) & 1));
            }
            if (committed >= 0)
                (void)mbar_wait_bounded(&pp.empty[committed % kWpStages],
                                        static_cast<uint32_t>((committed / kWpStages) & 1));
        }
    }
    tc_fence_before();
    __syncthreads();
    if (control) tmem_dealloc(tmem, kWpTmemCols);
}

}  // namespace

size_t wprod_scratch_bytes(int n) { return wp_layout(n).total; }

// After a launch_trsm_emu_wellcond on `stream` with this scratch: 1 if the
// product form ran, 0 if the substitution did, -1 on a CUDA error
// (synchronizes the stream).
int wellcond_used_product(const void *scratch, int n, cudaStream_t stream) {
    const unsigned char *wp = static_cast<const unsigned char *>(scratch) +
                              round_up(int64_t(trsm_emu_scratch_bytes(n)), 1024);
    unsigned long long h[2] = {0, 0};
    if (cudaMemcpyAsync(h, wp + wp_layout(n).norms, sizeof h, cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
        return -1;
    double cond, lim;
    memcpy(&cond, &h[0], sizeof cond);
    memcpy(&lim, &h[1], sizeof lim);
    return cond <= lim ? 1 : 0;
}

cudaError_t launch_trsm_emu_wellcond(const double *A, int64_t lda, int64_t m, int n, const double *RP,
                                     const double *rinv, double *Q, int64_t ldq, void *scratch,
                                     DevStatus *st, cudaStream_t stream) {
    if (n < 1 || n > 256 || m < 1) return cudaErrorInvalidValue;
    const int n_pad = pad16(n);
    unsigned char *base = static_cast<unsigned char *>(scratch);
    unsigned char *wp = base + round_up(int64_t(trsm_emu_scratch_bytes(n)), 1024);
    const WpLayout l = wp_layout(n);
    unsigned long long *norms = reinterpret_cast<unsigned long long *>(wp + l.norms);
    int *cbits = reinterpret_cast<int *>(wp + l.cbits);
    double *W = reinterpret_cast<double *>(wp + l.w);
    unsigned char *tiles = wp + l.tiles;
    cudaError_t e = cudaMemsetAsync(norms, 0, 2 * sizeof(unsigned long long), stream);
    if (e != cudaSuccess) return e;
    constexpr int kWarps = 8;
    const size_t ism = size_t(kWarps + 1) * n_pad * sizeof(double);
    RQ_LAUNCH(KID_EMU_AUX, stream,
              k_tri_inverse<<<static_cast<unsigned>(ceil_div(n_pad, kWarps)), 32 * kWarps, ism, stream>>>(
                  RP, rinv, n, n_pad, W, norms));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int passes = (n + kWpN - 1) / kWpN;
    RQ_LAUNCH(KID_EMU_AUX, stream,
              k_wprod_prep<<<passes, 256, 0, stream>>>(W, n, n_pad, norms, cbits, tiles));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int64_t ntiles = ceil_div(m, kWpM);
    const int64_t grid = std::min<int64_t>(ntiles, int64_t(grid_sms()));  // one CTA per SM
    const int64_t chunk = ceil_div(ntiles, grid) * kWpM;
    const int g = static_cast<int>(ceil_div(m, chunk));
    const size_t smem = size_t(kWpStages) * kWpStageBytes;
    if ((e = cudaFuncSetAttribute(k_wprod_emu, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem))) !=
        cudaSuccess)
        return e;
    RQ_LAUNCH(KID_TRSM_EMU, stream,
              k_wprod_emu<<<g, kWpThreads, smem, stream>>>(A, lda, m, n, chunk, norms, cbits, tiles, Q,
                                                           ldq, st));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // the substitution form, which runs only when the estimate rejected the product
    return launch_trsm_emu(A, lda, m, n, RP, rinv, Q, ldq, scratch, st, stream, norms);
}

}  // namespace rq
