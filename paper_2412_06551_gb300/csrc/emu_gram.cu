// Gram product G = A^T A emulating binary64 on the tensor cores (the
// precision form of the CholeskyQR pass: Gram as split-bf16 products with
// fp32 accumulation; Algorithm 1, C1).
//
// Splitting (emu.cuh): per column j of A, with 2^E_j above every |a_ij|,
// a_ij = 2^(E_j - 7) sum_{s=0..7} d_s 2^(-8s) up to 2^(E_j - 64), |d_s| <= 128.
// Level L = s + t collects the products d_s(i, j) d_t(i, k); levels 0..7 are
// kept (36 digit pairs).
//
// Exactness: over a window of 128 rows a level's sum has at most 8 x 128
// products of magnitude <= 2^14, so it stays within 2^24 and the tensor
// core's fp32 accumulation of these integers is exact.  After each window
// the eight fp32 accumulators are drained into one int64 per element in
// units of 2^-36 of level 0 (levels 0..4 exactly, 5..7 rounded: at most 1.5
// units, 2^-50 of a window's scale).  Every 16 windows, and at the end, the
// int64 (|sum| < 2^62) is added to the CTA's binary64 partial in global
// memory.  The partials are reduced in a fixed order and scaled by
// 2^(E_j + E_k - 50).
//
// Tiles: a CTA owns 128 rows (columns j of A) x 64 columns (k of A) of G and
// a contiguous chunk of rows of A (split-K).  Its eight 128 x 64 fp32
// accumulators take the 512 TMEM columns.  Per 32 rows of A the 16 producer
// warps split the block into digits (K-major 8 x 8 bf16 core matrices in
// shared memory; the k columns' eight digit tiles side by side) while the
// control warp issues the previous blocks' 36 digit-pair products as 12 x 2
// wide MMAs (kind::f16, M=128, N=64 .. 256, K=16): one digit of the j columns
// times up to four adjacent digits of the k columns lands in as many adjacent
// levels; mbarriers hand the stages back and forth (see k_gram_emu).
#include <algorithm>
#include <climits>

#include "common.cuh"
#include "kernels.h"
#include "emu.cuh"
#include "tcgen05.cuh"

namespace rq {
namespace {

constexpr int kEmuProducers = 512;                 // 16 producer warps
constexpr int kEmuThreads = kEmuProducers + 32;   // plus the control warp
constexpr int kEmuWinSteps = 4; // stages per exact window (128 rows)
constexpr int kEmuM = 128;      // rows of G per tile (columns j of A)
constexpr int kEmuN = 64;       // columns of G per tile (columns k of A)
constexpr int kEmuMaxStages = 2;  // one stage per producer group
constexpr int kTileA = kEmuM * kEmuBK * 2;  // bytes of one digit tile of the j columns
constexpr int kTileB = kEmuN * kEmuBK * 2;  // ... of the k columns
constexpr int kEmuStageBytes = kEmuDigits * (kTileA + kTileB);
constexpr int kEmuTmemCols = 512;
constexpr int kEmuSlot = kEmuM * kEmuN;  // elements of one per-CTA partial
constexpr int kEmuFlushWindows = 16;     // int64 drains between binary64 flushes
constexpr int kEmuUnit = 12;             // drain units: 2^-(24 + 12) of level 0
constexpr int kEmuGroups = 2;            // producer groups taking alternate blocks
constexpr int kEmuGroupWarps = kEmuProducers / 32 / kEmuGroups;

// Tile t of the upper triangle of G: rows [128 jb, +128), columns [64 kb, +64),
// kb >= 2 jb, enumerated jb-major.
__host__ __device__ __forceinline__ void emu_tile(int t, int n, int &j0, int &k0) {
    const int nJ = (n + kEmuM - 1) / kEmuM, nK = (n + kEmuN - 1) / kEmuN;
    int jb = 0;
    for (; jb < nJ; ++jb) {
        const int cnt = nK - 2 * jb;
        if (t < cnt) break;
        t -= cnt;
    }
    j0 = kEmuM * jb;
    k0 = kEmuN * (2 * jb + t);
}

int emu_tiles(int n) {
    const int nJ = (n + kEmuM - 1) / kEmuM, nK = (n + kEmuN - 1) / kEmuN;
    int c = 0;
    for (int jb = 0; jb < nJ; ++jb) c += nK - 2 * jb;
    return c;
}

// Largest biased binary64 exponent of each column (atomic max; colbits zeroed first).
__global__ void k_col_exponent(const double *__restrict__ A, int64_t lda, int64_t m, int64_t chunk,
                               int *__restrict__ colbits) {
    const int j = blockIdx.x;
    const int64_t rb = int64_t(blockIdx.y) * chunk;
    const int64_t re = std::min<int64_t>(m, rb + chunk);
    int e = 0;
    for (int64_t i = rb + threadIdx.x; i < re; i += blockDim.x) {
        const unsigned long long b =
            static_cast<unsigned long long>(__double_as_longlong(A[i + int64_t(j) * lda]));
        e = max(e, static_cast<int>((b >> 52) & 0x7ff));
    }
    for (int off = 16; off > 0; off >>= 1) e = max(e, __shfl_down_sync(0xffffffffu, e, off));
    if ((threadIdx.x & 31) == 0 && e > 0) atomicMax(colbits + j, e);
}

// Warp-specialised: two groups of 8 producer warps take alternate 32-row
// blocks of A, split each into digit tiles in the block's stage and arrive on
// the stage's full barrier (one arrival per warp); the control warp's lane 0
// waits for it,
// issues the block's 24 MMAs and commits them to the stage's empty barrier.
// A window's eight accumulators are drained by the producers after they
// have filled the next block (so that its split overlaps the window's last
// MMAs); the control lane starts a window only when the previous one is
// drained (tmem_empty).  No block-wide barrier inside the loop.
struct GePipe {
    uint64_t full[kEmuMaxStages], empty[kEmuMaxStages];
    uint64_t win_done;    // a window's MMAs are complete
    uint64_t tmem_empty;  // its accumulators are drained
    uint32_t tmem_slot;
    int abort_flag;
};

__device__ __forceinline__ bool ge_wait(GePipe &pp, uint64_t *bar, uint32_t parity) {
    if (*reinterpret_cast<volatile int *>(&pp.abort_flag)) return false;
    if (mbar_wait_bounded(bar, parity)) return true;
    *reinterpret_cast<volatile int *>(&pp.abort_flag) = 1;
    return false;
}

__global__ void __launch_bounds__(kEmuThreads, 1)
    k_gram_emu(const double *__restrict__ A, int64_t lda, int64_t m, int n,
               const int *__restrict__ colbits, int64_t chunk, double *__restrict__ part,
               DevStatus *st) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ GePipe pp;
    __shared__ int expA[kEmuM], expB[kEmuN];

    int j0, k0;
    emu_tile(blockIdx.x, n, j0, k0);
    const bool b_in_a = (k0 >= j0) && (k0 + kEmuN <= j0 + kEmuM);
    // one stage per producer group (block ks in stage ks % 2, so that each
    // stage's empty barrier is waited on by one group, phase after phase);
    // the k columns inside the j columns need no digits of their own
    constexpr int nst = kEmuGroups;
    // the k columns' digit tiles sit side by side after the j columns' (when
    // the k columns lie inside the j columns, their digits are stored twice)
    const int stage_bytes = kEmuStageBytes;
    const int kin = b_in_a ? k0 - j0 : -kEmuN;  // first k column inside the j columns
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool control = warp == kEmuProducers / 32;

    if (control) tmem_alloc(&pp.tmem_slot, kEmuTmemCols);
    if (tid == 0) {
        for (int s = 0; s < nst; ++s) {
            mbar_init(&pp.full[s], kEmuGroupWarps);
            mbar_init(&pp.empty[s], 1);
        }
        mbar_init(&pp.win_done, 1);
        mbar_init(&pp.tmem_empty, kEmuProducers / 32);
        fence_mbar_init();
        pp.abort_flag = 0;
    }
    for (int c = tid; c < kEmuM; c += kEmuThreads)
        expA[c] = (j0 + c < n) ? emu_exponent(colbits[j0 + c]) : 0;
    for (int c = tid; c < kEmuN; c += kEmuThreads)
        expB[c] = (k0 + c < n) ? emu_exponent(colbits[k0 + c]) : 0;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = pp.tmem_slot;

    const int64_t rb = int64_t(blockIdx.y) * chunk;
    const int64_t re = std::min<int64_t>(m, rb + chunk);
    const int nsteps = re > rb ? static_cast<int>(ceil_div(re - rb, kEmuBK)) : 0;
    int committed = -1;  // the control thread's last commit

    if (control) {
        // the whole warp runs the loop, so that the stage addresses and
        // descriptors are warp-uniform values; lane 0 waits and issues
        // the level products as wide MMAs: the k columns' digit tiles t0 ..
        // t0 + w - 1 side by side form one operand of N = 64 w, whose product
        // with digit s of the j columns lands in levels s + t0 .. s + t0 + w - 1
        // (TMEM columns 64 (s + t0) ..); twelve MMAs per k-step cover the 36
        // pairs s + t <= 7.  The two with s = 0 come first: they write every
        // level, so only they start a window afresh.
        const uint32_t idn[5] = {0u, idesc_bf16_f32(kEmuM, kEmuN), idesc_bf16_f32(kEmuM, 2 * kEmuN),
                                 idesc_bf16_f32(kEmuM, 3 * kEmuN), idesc_bf16_f32(kEmuM, 4 * kEmuN)};
        for (int ks = 0; ks < nsteps; ++ks) {
            const int s = ks % nst;
            const bool fresh = (ks % kEmuWinSteps) == 0;
            int okw = 1;
            if (lane == 0)
                okw = (!fresh || ks == 0 ||
                       ge_wait(pp, &pp.tmem_empty, static_cast<uint32_t>((ks / kEmuWinSteps - 1) & 1))) &&
                      ge_wait(pp, &pp.full[s], static_cast<uint32_t>((ks / nst) & 1));
            if (!__shfl_sync(0xffffffffu, okw, 0)) break;
            const uint32_t sa = smem_u32(smem_raw + s * stage_bytes);
            // descriptors of digit 0, k-step 0; digit d, k-step kk add their
            // byte offsets / 16 to the start-address field (no carry: shared
            // addresses stay below 2^18)
            const uint64_t adA = smem_desc(sa, 128, (kEmuBK / 8) * 128);
            const uint64_t adB = smem_desc(sa + kEmuDigits * kTileA, 128, (kEmuBK / 8) * 128);
            if (lane == 0) {
                tc_fence_after();
#pragma unroll
                for (int kk = 0; kk < kEmuBK / 16; ++kk) {
                    const uint32_t a0 = fresh && kk == 0 ? 0u : 1u;
                    const uint64_t ak = adA + static_cast<uint64_t>(kk * 16);
                    const uint64_t bk = adB + static_cast<uint64_t>(kk * 16);
                    // s = 0: k tiles 0-3 -> levels 0-3, k tiles 4-7 -> levels 4-7
                    mma_bf16(tmem, ak, bk, idn[4], a0);
                    mma_bf16(tmem + 4 * kEmuN, ak, bk + static_cast<uint64_t>(4 * (kTileB >> 4)), idn[4], a0);
#pragma unroll
                    for (int sd = 1; sd < kEmuDigits; ++sd) {
                        const uint64_t as = ak + static_cast<uint64_t>(sd * (kTileA >> 4));
                        // k tiles 0 .. min(3, 7 - sd)
                        mma_bf16(tmem + static_cast<uint32_t>(sd * kEmuN), as, bk,
                                 idn[(8 - sd) < 4 ? (8 - sd) : 4], 1u);
                        // k tiles 4 .. 7 - sd
                        if (sd <= 3)
                            mma_bf16(tmem + static_cast<uint32_t>((sd + 4) * kEmuN), as,
                                     bk + static_cast<uint64_t>(4 * (kTileB >> 4)), idn[4 - sd], 1u);
                    }
                }
                mma_commit(&pp.empty[s]);
                if ((ks % kEmuWinSteps) == kEmuWinSteps - 1 || ks == nsteps - 1) mma_commit(&pp.win_done);
                committed = ks;
            }
            __syncwarp();
        }
    } else {
        // drain ownership: TMEM lanes 32 (warp % 4) .. +31 (rows j of the
        // tile), columns 16 (warp / 4) .. +15
        const int lane_base = 32 * (warp & 3);
        const int cgrp = warp >> 2;
        long long acc[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) acc[q] = 0;
        // this thread's elements of the CTA's binary64 partial, [col][row]
        double *mine = part + (size_t(blockIdx.x) * gridDim.y + blockIdx.y) * kEmuSlot +
                       size_t(16 * cgrp) * kEmuM + lane_base + lane;
        int windows = 0;
        bool flushed = false;
        auto flush = [&]() {
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const double v = static_cast<double>(acc[q]);
                mine[q * kEmuM] = flushed ? mine[q * kEmuM] + v : v;
                acc[q] = 0;
            }
            flushed = true;
        };
        // window w: its MMAs are done; add the eight levels into int64 and
        // release TMEM (every producer warp drains every window, in order)
        auto drain = [&](int w) -> bool {
            if (!ge_wait(pp, &pp.win_done, static_cast<uint32_t>(w & 1))) return false;
            tc_fence_after();
            const uint32_t tl = tmem + (static_cast<uint32_t>(lane_base) << 16) +
                                static_cast<uint32_t>(16 * cgrp);
            float v[16];
#pragma unroll
            for (int L = 0; L < kEmuDigits; ++L) {
                tmem_ld16(tl + static_cast<uint32_t>(L * kEmuN), v);
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    switch (L) {  // compile-time after unrolling
                        case 0: acc[q] += emu_level<24 + kEmuUnit>(v[q]); break;
                        case 1: acc[q] += emu_level<16 + kEmuUnit>(v[q]); break;
                        case 2: acc[q] += emu_level<8 + kEmuUnit>(v[q]); break;
                        case 3: acc[q] += emu_level<0 + kEmuUnit>(v[q]); break;
                        case 4: acc[q] += emu_level<-8 + kEmuUnit>(v[q]); break;
                        case 5: acc[q] += emu_level<-16 + kEmuUnit>(v[q]); break;
                        case 6: acc[q] += emu_level<-24 + kEmuUnit>(v[q]); break;
                        default: acc[q] += emu_level<-32 + kEmuUnit>(v[q]); break;
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&pp.tmem_empty);
            if (++windows == kEmuFlushWindows) {
                flush();
                windows = 0;
            }
            return true;
        };
        const int ncolsB = b_in_a ? 0 : kEmuN;
        const int ntasks = (kEmuM + ncolsB) * (kEmuBK / 8);
        // the two groups of eight producer warps take alternate blocks, so that
        // one group's loads are in flight while the other splits
        const int grp = warp / kEmuGroupWarps;
        const int gtid = tid % (kEmuGroupWarps * 32);
        constexpr int kG = kEmuGroupWarps * 32;
        // split this thread's task (8 rows x 1 column) held in x into the stage
        auto split = [&](unsigned char *stage, int task, const double (&x)[8]) {
            const int kb = task % (kEmuBK / 8), c = task / (kEmuBK / 8);
            const bool isA = c < kEmuM;
            const int cc = isA ? c : c - kEmuM;
            const int E = isA ? expA[cc] : expB[cc];
            unsigned char *base = stage + (isA ? 0 : kEmuDigits * kTileA);
            const int tbytes = isA ? kTileA : kTileB;
            // a j column that is also a k column: its digits again in the k tiles
            const int kc = isA ? c - kin : -1;
            const bool dup = kc >= 0 && kc < kEmuN;
            unsigned char *bdup = stage + kEmuDigits * kTileA;
            // two rows at a time: one 32-bit word (two bf16) per digit
#pragma unroll
            for (int t = 0; t < 8; t += 2) {
                uint32_t w[kEmuDigits];
                emu_digits2_packed<kEmuDigits>(x[t], x[t + 1], E, w);
#pragma unroll
                for (int sd = 0; sd < kEmuDigits; ++sd) {
                    *reinterpret_cast<uint32_t *>(base + sd * tbytes + emu_off(cc, kb * 8 + t)) = w[sd];
                    if (dup) *reinterpret_cast<uint32_t *>(bdup + sd * kTileB + emu_off(kc, kb * 8 + t)) = w[sd];
                }
            }
        };
        auto load = [&](int64_t r0, int task, double (&x)[8]) {
            const int kb = task % (kEmuBK / 8), c = task / (kEmuBK / 8);
            const int col = c < kEmuM ? j0 + c : k0 + (c - kEmuM);
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int64_t row = r0 + kb * 8 + t;
                x[t] = (task < ntasks && row < re && col < n) ? A[row + int64_t(col) * lda] : 0.0;
            }
        };
        bool ok = true;
        int next_w = 0;  // the next window this warp drains
        for (int ks = grp; ks < nsteps && ok; ks += kEmuGroups) {
            const int s = ks % nst;
            unsigned char *stage = smem_raw + s * stage_bytes;
            const int64_t r0 = rb + int64_t(ks) * kEmuBK;
            // (1) this thread's first two blocks of 8 rows x 1 column (in
            // flight during the wait); a third, for the k columns outside the
            // j columns, after them
            double x0[8], x1[8];
            load(r0, gtid, x0);
            load(r0, gtid + kG, x1);
            // the MMAs that last read this stage are done
            if (ks >= nst && !ge_wait(pp, &pp.empty[s], static_cast<uint32_t>((ks / nst - 1) & 1))) break;
            // (2) digits, stored as K-major operand tiles
            split(stage, gtid, x0);
            if (gtid + kG < ntasks) split(stage, gtid + kG, x1);
            if (gtid + 2 * kG < ntasks) {
                load(r0, gtid + 2 * kG, x0);
                split(stage, gtid + 2 * kG, x0);
            }
            fence_proxy_async_smem();  // generic-proxy stores -> visible to the tensor core
            __syncwarp();
            if (lane == 0) mbar_arrive(&pp.full[s]);
            // (3) the window that ended before this block
            if (kEmuWinSteps * next_w + kEmuWinSteps - 1 < ks) {
                ok = drain(next_w);
                ++next_w;
            }
        }
        // the windows left (the last one may be short)
        const int nwin = static_cast<int>(ceil_div(nsteps, kEmuWinSteps));
        for (; ok && next_w < nwin; ++next_w) ok = drain(next_w);
        if (ok && nsteps > 0) flush();
    }
    __syncthreads();
    if (*reinterpret_cast<volatile int *>(&pp.abort_flag)) {
        if (tid == 0) report(st, kErrTimeout, 0, -1);
        if (control && lane == 0 && committed >= 0)
            (void)mbar_wait_bounded(&pp.empty[committed % nst], static_cast<uint32_t>((committed / nst) & 1));
    }
    tc_fence_before();
    __syncthreads();
    if (control) tmem_dealloc(tmem, kEmuTmemCols);
}

// G[j][k] = G[k][j] = 2^(E_j + E_k - 50) times the sum over the tile's CTAs
// (in order) of their binary64 partials; NaN where a column holds a
// non-finite value.
__global__ void k_reduce_gram_emu(const double *__restrict__ part, int nsplit, int n,
                                  const int *__restrict__ colbits, double *__restrict__ G,
                                  int64_t ldg) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= int64_t(n) * n) return;
    const int j = static_cast<int>(e % n), k = static_cast<int>(e / n);
    if (j > k) return;
    const int jb = j / kEmuM, kb = k / kEmuN;
    const int nK = (n + kEmuN - 1) / kEmuN;
    int t = 0;
    for (int q = 0; q < jb; ++q) t += nK - 2 * q;
    t += kb - 2 * jb;
    const size_t off = size_t(k - kEmuN * kb) * kEmuM + (j - kEmuM * jb);
    const double s = ordered_sum(part + size_t(t) * nsplit * kEmuSlot + off, kEmuSlot, nsplit);
    const int bj = __ldg(colbits + j), bk = __ldg(colbits + k);
    double g;
    if (bj == 0x7ff || bk == 0x7ff)
        g = __longlong_as_double(0x7ff8000000000000ll);
    else
        g = ldexp(s, emu_exponent(bj) + emu_exponent(bk) - 14 - 24 - kEmuUnit);
    G[j + int64_t(k) * ldg] = g;
    G[k + int64_t(j) * ldg] = g;
}

int emu_split(int n, int64_t m) {
    const int tiles = emu_tiles(n);
    int p = std::max(1, grid_sms() / tiles);
    const int64_t windows = ceil_div(m, int64_t(kEmuBK) * kEmuWinSteps);
    return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(p, windows)));
}

}  // namespace

size_t gram_emu_partials_doubles(int n) {
    const size_t slots = size_t(num_sms()) + 8;
    (void)n;
    // one binary64 partial per CTA slot, plus the column exponents
    return slots * kEmuSlot + 64;
}

cudaError_t launch_gram_emu(const double *A, int64_t lda, int64_t m, int n, double *G, int64_t ldg,
                            double *part, DevStatus *st, cudaStream_t stream) {
    if (n < 1 || n > 256 || m < 1) return cudaErrorInvalidValue;
    const int tiles = emu_tiles(n);
    const int p = emu_split(n, m);
    // chunks of whole windows, so that every window but the last is full
    const int64_t win = int64_t(kEmuBK) * kEmuWinSteps;
    int64_t chunk = round_up(ceil_div(m, p), win);
    const int nsplit = static_cast<int>(ceil_div(m, chunk));
    int *colbits = reinterpret_cast<int *>(part + size_t(tiles) * nsplit * kEmuSlot);
    cudaError_t e = cudaMemsetAsync(colbits, 0, sizeof(int) * size_t(n), stream);
    if (e != cudaSuccess) return e;
    const int64_t cchunk = std::max<int64_t>(4096, ceil_div(m, 64));
    const dim3 gx(n, static_cast<unsigned>(ceil_div(m, cchunk)));
    RQ_LAUNCH(KID_EMU_AUX, stream, k_col_exponent<<<gx, 256, 0, stream>>>(A, lda, m, cchunk, colbits));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const size_t smem = size_t(kEmuMaxStages) * kEmuStageBytes;
    cudaFuncSetAttribute(k_gram_emu, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    RQ_LAUNCH(KID_GRAM_EMU, stream,
              k_gram_emu<<<dim3(tiles, nsplit), kEmuThreads, smem, stream>>>(
                  A, lda, m, n, colbits, chunk, part, st));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int64_t ne = int64_t(n) * n;
    RQ_LAUNCH(KID_EMU_AUX, stream,
              k_reduce_gram_emu<<<static_cast<unsigned>(ceil_div(ne, 256)), 256, 0, stream>>>(
                  part, nsplit, n, colbits, G, ldg));
    return cudaGetLastError();
}

}  // namespace rq
