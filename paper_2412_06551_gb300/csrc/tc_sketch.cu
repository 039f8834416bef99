// Reduced-precision Gaussian sketch on the 5th-generation tensor cores
// (tcgen05, kind::f16 with bf16 operands, fp32 accumulation in TMEM).
//
// The sketch S X of Algorithm 6 (and S M of Algorithm 7) only has to
// be a subspace embedding (Section 3), so its product may run at reduced
// precision.  Y = S X with S generated on the fly: each CTA owns ts = 1 or 2
// tiles of 128 sketch rows x all NT <= 256 columns of Y and every p-th
// 32-row step of X (split-K over p CTAs, interleaved: see the X ring).  X streams through a ring of 16-row boxes
// that thread 0 keeps in flight by TMA (the X ring below), so its loads
// overlap the generation of S.  For every 32 rows of X the 256 threads
//   * draw the ts 128 x 32 blocks of S (bf16 levels, defined below),
//   * split the 32 x NT block of X (binary64) into one or three bf16 terms
//     x1 = bf16(x), x2 = bf16(x - x1), x3 = bf16(x - x1 - x2), once for all
//     ts tiles,
//   * store both as K-major operand tiles (8 x 8 bf16 core matrices) in
//     shared memory,
// and one thread issues tcgen05.mma for the 16-row k-steps (one MMA per tile
// and bf16 term of X), committing to an mbarrier per stage; two operand
// stages let the tensor core consume step k while the threads fill k + 1.
// At the end the fp32 accumulators are read from TMEM (tcgen05.ld), scaled
// by 1/sqrt(s) in binary64 and written as this CTA's partial; partials are
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
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "emu.cuh"
#include "kernels.h"
#include "tcgen05.cuh"

namespace rq {
namespace {

constexpr int kSkProducers = 512;              // producer threads of the sketch kernels
constexpr int kSkWarps = kSkProducers / 32;     // producer warps (one barrier arrival each)
constexpr int kTcThreads = kSkProducers + 32;   // plus one control warp
constexpr int kSkMaxStages = 4;
constexpr int kTcBK = 32;      // rows of X per step (two 16-row k-steps of the MMA)
constexpr int kTcM = 128;      // sketch rows per tile (M of the MMA)
constexpr int kLevels = 4096;  // levels of the discretised normal
constexpr uint32_t kLevelsDomain = 0x53424631u;
constexpr int kXBoxRows = 16;  // rows of X per ring box: one 128-byte swizzle line per column
constexpr int kXRingMax = 8;   // ring slots at most

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
    if (e >= 255) return static_cast<uint16_t>((sign << 15) | 0x7f80u);  // beyond it: infinity
    return static_cast<uint16_t>((sign << 15) | (static_cast<unsigned>(e) << 7) | frac);
}

// The same rounding on 32-bit words (the one-term split needs no rounded
// binary64 value): the top word holds sign, exponent and the kept 7 bits,
// the round bit (bit 12) and part of the sticky bits.
__device__ __forceinline__ uint32_t bf16_bits_from_f64_fast(double x) {
    uint32_t hi = static_cast<uint32_t>(__double2hiint(x));
    const uint32_t lo = static_cast<uint32_t>(__double2loint(x));
    const uint32_t sticky = (hi & 0xfffu) | lo;
    if (((hi >> 12) & 1u) && (sticky != 0u || ((hi >> 13) & 1u))) hi += 0x2000u;
    const uint32_t sign = (hi >> 16) & 0x8000u;
    const int e = static_cast<int>((hi >> 20) & 0x7ffu) - 1023 + 127;
    if (e <= 0) return sign;
    if (e >= 255) return sign | 0x7f80u;
    return sign | (static_cast<uint32_t>(e) << 7) | ((hi >> 13) & 0x7fu);
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

// Eight entries (r, 8q .. 8q + 7) of the reduced tier's S as packed bf16:
// one Philox block; `lv` is the level table in shared memory.
__device__ __forceinline__ uint4 sk_levels8_aligned(uint32_t k0, uint32_t k1, int r, uint64_t q,
                                                    const uint16_t *lv) {
    const uint4 a = philox4x32_10(make_uint4(static_cast<uint32_t>(q), static_cast<uint32_t>(q >> 32),
                                             static_cast<uint32_t>(r), kLevelsDomain), k0, k1);
    // entry 2 w + 0 is the low half of word w, 2 w + 1 the high half; level index = half >> 4
    const uint32_t h0 = lv[(a.x >> 4) & 0xfffu], h1 = lv[a.x >> 20];
    const uint32_t h2 = lv[(a.y >> 4) & 0xfffu], h3 = lv[a.y >> 20];
    const uint32_t h4 = lv[(a.z >> 4) & 0xfffu], h5 = lv[a.z >> 20];
    const uint32_t h6 = lv[(a.w >> 4) & 0xfffu], h7 = lv[a.w >> 20];
    return make_uint4(h0 | (h1 << 16), h2 | (h3 << 16), h4 | (h5 << 16), h6 | (h7 << 16));
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

// ---- X ring ------------------------------------------------------------------
//
// The CTAs of a grid column take the steps of 32 rows of X in turn (CTA y
// of p takes rows 32 (t p + y) .. + 31 at its step t), so that the CTAs
// running at the same time read neighbouring pieces of every column and
// the DRAM pages they open serve several of them.  A CTA walks its steps in
// boxes of 16 rows x ncx columns (binary64): box g holds rows
// xbox_row(g) .. + 15 of columns c0 .. c0 + ncx - 1,
// column c's 16 values in the 128-byte line c of the box, its 16-byte chunk j
// (rows 2 j, 2 j + 1) at chunk j ^ (c % 8) (the TMA's 128-byte swizzle; the
// ring starts on a 1024-byte boundary and every box spans a multiple of 1024
// bytes).  Box g sits in slot g % kx and completes on that slot's mbarrier
// (phase g / kx).  Thread 0 keeps up to kx boxes in flight ahead of the
// threads.  Rows past the end of X and columns past n arrive as zeros.  When
// X does not meet TMA's alignment rules the threads fill the same layout
// with plain loads just before the step that reads it.

__device__ __forceinline__ uint32_t xbox_off(int c, int j) {
    return static_cast<uint32_t>(c * 128 + ((j ^ (c & 7)) << 4));
}

// First row of X of the CTA's step t (32 rows), of its box g (16 rows).
__device__ __forceinline__ int64_t xstep_row(int t) {
    return (int64_t(t) * gridDim.y + blockIdx.y) * kTcBK;
}
__device__ __forceinline__ int64_t xbox_row(int g) {
    return xstep_row(g >> 1) + kXBoxRows * (g & 1);
}

// Steps of the CTA: the 32-row steps y, y + p, y + 2p, ... of X's rows.
__device__ __forceinline__ int xsteps(int64_t m) {
    const int64_t total = ceil_div(m, kTcBK);
    return blockIdx.y < total ? static_cast<int>((total - 1 - blockIdx.y) / gridDim.y + 1) : 0;
}

// Thread 0, TMA path: box g into slot g % kx.
__device__ __forceinline__ void xring_issue(unsigned char *ring, uint64_t *bar, const CUtensorMap *map,
                                            int g, int kx, uint32_t box_bytes, int c0) {
    const int q = g % kx;
    mbar_arrive_expect_tx(&bar[q], box_bytes);
    tma_load_2d(ring + size_t(q) * box_bytes, map, &bar[q], static_cast<int32_t>(xbox_row(g)), c0);
}

// Threads t0, t0 + nthr, ... of the producers, plain-load path: their part
// of box g into slot g % kx.
__device__ __forceinline__ void xring_fill(unsigned char *ring, int g, int kx, uint32_t box_bytes,
                                           const double *__restrict__ X, int64_t ldx, int64_t m,
                                           int n, int c0, int ncx, int t0, int nthr) {
    unsigned char *box = ring + size_t(g % kx) * box_bytes;
    const int64_t r = xbox_row(g);
    for (int idx = t0; idx < ncx * 8; idx += nthr) {
        const int c = idx >> 3, j = idx & 7;
        const int64_t row = r + 2 * j;
        const int col = c0 + c;
        double2 v = make_double2(0.0, 0.0);
        if (col < n) {
            const double *xc = X + int64_t(col) * ldx;
            if (row < m) v.x = xc[row];
            if (row + 1 < m) v.y = xc[row + 1];
        }
        *reinterpret_cast<double2 *>(box + xbox_off(c, j)) = v;
    }
}

// Eight K-consecutive values (rows 8 kb .. 8 kb + 7 of the step) of column c
// from the two boxes of a step; rows at or past re read as zero, and with
// unit_lower the column is read as a unit-lower factor.
__device__ __forceinline__ void xring_read8(const unsigned char *box0, const unsigned char *box1, int c,
                                            int kb, int64_t row8, int64_t re, int col, int unit_lower,
                                            double (&v)[8]) {
    const unsigned char *box = (kb >> 1) ? box1 : box0;
#pragma unroll
    for (int tt = 0; tt < 4; ++tt) {
        const double2 d = *reinterpret_cast<const double2 *>(box + xbox_off(c, (kb & 1) * 4 + tt));
        v[2 * tt] = d.x;
        v[2 * tt + 1] = d.y;
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const int64_t row = row8 + t;
        if (row >= re) v[t] = 0.0;
        else if (unit_lower && row <= col) v[t] = (row == col) ? 1.0 : 0.0;
    }
}

// Pipeline state shared by the sketch kernels' warps: operand stages
// (full: every producer warp has written it; empty: the MMAs that read it
// are done), ring slots (xfull: the TMA box has landed; xempty: every
// producer warp has read it) and the abort flag.  A producer warp's lanes
// fence their stores for the async proxy, meet at __syncwarp, and lane 0
// arrives for the warp.
struct SkPipe {
    uint64_t full[kSkMaxStages], empty[kSkMaxStages];
    uint64_t xfull[kXRingMax], xempty[kXRingMax];
    uint64_t tmem_empty;  // the digit tier: a window's accumulators are drained
    uint32_t tmem_slot;
    int abort_flag;
};

__device__ __forceinline__ bool sk_aborted(SkPipe &pp) {
    return *reinterpret_cast<volatile int *>(&pp.abort_flag) != 0;
}

// Named barrier over `count` threads (barrier 0 is __syncthreads).
__device__ __forceinline__ void named_bar_sync(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Named barrier that also returns, in every participating thread, whether
// any of them passed p = true.
__device__ __forceinline__ bool named_bar_or(int id, int count, bool p) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred pi, po;\n\t"
        "setp.ne.u32 pi, %1, 0;\n\t"
        "bar.red.or.pred po, %2, %3, pi;\n\t"
        "selp.u32 %0, 1, 0, po;\n\t}"
        : "=r"(r)
        : "r"(static_cast<uint32_t>(p)), "r"(id), "r"(count)
        : "memory");
    return r != 0;
}

// A bounded wait that gives up at once when another thread already has.
__device__ __forceinline__ bool sk_wait(SkPipe &pp, uint64_t *bar, uint32_t parity) {
    if (sk_aborted(pp)) return false;
    if (mbar_wait_bounded(bar, parity)) return true;
    *reinterpret_cast<volatile int *>(&pp.abort_flag) = 1;
    return false;
}

// After an abort: the control thread lets the copies and products in flight
// land (each slot's latest box, the latest commit; every wait bounded)
// before the CTA's shared memory and TMEM are released.
__device__ __forceinline__ void sk_drain(SkPipe &pp, int issued, int kx, int committed, int nst) {
    for (int q = 0; q < kx && q < issued; ++q) {
        const int g = q + ((issued - 1 - q) / kx) * kx;  // the latest box issued into slot q
        (void)mbar_wait_bounded(&pp.xfull[q], static_cast<uint32_t>((g / kx) & 1));
    }
    if (committed >= 0)
        (void)mbar_wait_bounded(&pp.empty[committed % nst], static_cast<uint32_t>((committed / nst) & 1));
}

// One CTA: ts sketch tiles (128 rows each, ts = 1 or 2) x all nt columns of
// X over the CTA's steps (split-K).  Warp-specialised: the 16 producer warps
// draw the ts S blocks of a step, wait for its two ring boxes, split X into
// NSL bf16 terms (once for all ts tiles) and arrive on the stage's full
// barrier; one lane of the control warp waits for it, issues the ts x NSL
// MMAs of each 16-row k-step (tile t accumulates in TMEM columns t tcols ..),
// commits them to the stage's empty barrier and refills the ring slots the
// producers have released.  No block-wide barrier inside the loop.
template <int NSL, bool kAlignedS>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_sketch_tc(const __grid_constant__ CUtensorMap xmap, int use_tma, const double *__restrict__ X,
                int64_t ldx, int64_t m, int n, int unit_lower, int ts, int nt, int nst, int kx,
                uint64_t seed, double scale, double *__restrict__ part, int s_pad, int n_pad,
                DevStatus *st, int64_t row0) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ SkPipe pp;
    __shared__ __align__(16) uint16_t lv[kLevels];

    const int a_bytes = kTcM * kTcBK * 2;  // 8 KB per sketch tile
    const int b_bytes = nt * kTcBK * 2;    // per bf16 term of X
    const int stage_bytes = ts * a_bytes + NSL * b_bytes;  // a multiple of 1024
    const uint32_t box_bytes = static_cast<uint32_t>(nt) * 128u;
    unsigned char *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    unsigned char *ring = smem + nst * stage_bytes;
    const int rt0 = kTcM * ts * static_cast<int>(blockIdx.x);  // first sketch row of the CTA
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool control = warp == kSkProducers / 32;
    uint32_t tcols = 32;  // TMEM columns per sketch tile
    while (tcols < static_cast<uint32_t>(nt)) tcols <<= 1;
    const uint32_t ncols = tcols * static_cast<uint32_t>(ts);
    const int64_t re = m;
    const int nsteps = xsteps(m);
    const int nboxes = 2 * nsteps;

    if (control) tmem_alloc(&pp.tmem_slot, ncols);
    if (tid == 0) {
        for (int q = 0; q < nst; ++q) {
            mbar_init(&pp.full[q], kSkWarps);
            mbar_init(&pp.empty[q], 1);
        }
        for (int q = 0; q < kx; ++q) {
            mbar_init(&pp.xfull[q], 1);
            mbar_init(&pp.xempty[q], kSkWarps);
        }
        fence_mbar_init();
        pp.abort_flag = 0;
    }
    for (int k = tid; k < kLevels / 8; k += kTcThreads)
        reinterpret_cast<uint4 *>(lv)[k] = reinterpret_cast<const uint4 *>(g_gauss_levels)[k];
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = pp.tmem_slot;
    int issued = 0, committed = -1;  // the control thread's ring and MMA bookkeeping

    if (control) {
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16_f32(kTcM, nt);
            if (use_tma) {
                prefetch_tensormap(&xmap);
                for (; issued < std::min(kx, nboxes); ++issued)
                    xring_issue(ring, pp.xfull, &xmap, issued, kx, box_bytes, 0);
            }
            for (int ks = 0; ks < nsteps; ++ks) {
                const int s = ks % nst;
                if (!sk_wait(pp, &pp.full[s], static_cast<uint32_t>((ks / nst) & 1))) break;
                tc_fence_after();
                const uint32_t a0 = smem_u32(smem + s * stage_bytes);
#pragma unroll
                for (int kk = 0; kk < kTcBK / 16; ++kk) {
                    for (int t = 0; t < ts; ++t) {
                        const uint64_t ad = smem_desc(a0 + t * a_bytes + kk * 256, 128, kTcBK * 16);
#pragma unroll
                        for (int p = 0; p < NSL; ++p) {
                            const uint64_t bd =
                                smem_desc(a0 + ts * a_bytes + p * b_bytes + kk * 256, 128, kTcBK * 16);
                            mma_bf16(tmem + static_cast<uint32_t>(t) * tcols, ad, bd, idesc,
                                     (ks > 0 || kk > 0 || p > 0) ? 1u : 0u);
                        }
                    }
                }
                mma_commit(&pp.empty[s]);
                committed = ks;
                // refill the step's two slots once every producer has read them
                // (they arrive there before arriving on full, so no wait is long)
                if (use_tma)
                    for (int g = 2 * ks; g < 2 * ks + 2 && g + kx < nboxes; ++g) {
                        if (!sk_wait(pp, &pp.xempty[g % kx], static_cast<uint32_t>((g / kx) & 1))) break;
                        xring_issue(ring, pp.xfull, &xmap, g + kx, kx, box_bytes, 0);
                        issued = g + kx + 1;
                    }
            }
        }
    } else {
        for (int ks = 0; ks < nsteps; ++ks) {
            const int s = ks % nst;
            unsigned char *stage = smem + s * stage_bytes;
            const int64_t r0 = xstep_row(ks);
            const int g0 = 2 * ks;
            // the MMAs of step ks - nst read this stage
            if (use_tma) {
                if (ks >= nst && !sk_wait(pp, &pp.empty[s], static_cast<uint32_t>(((ks / nst) - 1) & 1)))
                    break;
            } else {
                const bool w = ks < nst || sk_wait(pp, &pp.empty[s], static_cast<uint32_t>(((ks / nst) - 1) & 1));
                // one verdict for all producers before their shared fills (the
                // previous step's reads of the ring are complete)
                if (named_bar_or(1, kSkProducers, !w || sk_aborted(pp))) break;
                xring_fill(ring, g0, kx, box_bytes, X, ldx, m, n, 0, nt, tid, kSkProducers);
                xring_fill(ring, g0 + 1, kx, box_bytes, X, ldx, m, n, 0, nt, tid, kSkProducers);
            }
            // (1) the ts S blocks: entries (r, i) for ts x 128 sketch rows x 32
            // rows of X, one task per 8 K-consecutive entries of a row; eight
            // neighbouring threads take eight rows (one 128-byte line of the
            // operand tile); X's rows past the end are zero, so those entries
            // need no masking
            for (int task = tid; task < ts * kTcM * (kTcBK / 8); task += kSkProducers) {
                const int kb = (task >> 3) & 3;
                const int r = ((task >> 5) << 3) | (task & 7);
                const uint4 v = kAlignedS ? sk_levels8_aligned(static_cast<uint32_t>(seed),
                                                               static_cast<uint32_t>(seed >> 32), rt0 + r,
                                                               static_cast<uint64_t>(row0 + r0) / 8 + kb, lv)
                                          : sk_levels8(seed, rt0 + r, row0 + r0 + 8 * kb, lv);
                *reinterpret_cast<uint4 *>(stage + (r >> 7) * a_bytes + kmajor_off(r & 127, 8 * kb)) = v;
            }
            // (2) the step's X boxes, split into NSL bf16 terms: task (column
            // c, rows 8 kb .. 8 kb + 7), eight neighbouring threads on eight
            // columns
            if (use_tma) {
                if (!sk_wait(pp, &pp.xfull[g0 % kx], static_cast<uint32_t>((g0 / kx) & 1))) break;
                if (!sk_wait(pp, &pp.xfull[(g0 + 1) % kx], static_cast<uint32_t>(((g0 + 1) / kx) & 1))) break;
            } else {
                named_bar_sync(1, kSkProducers);  // the fills are complete
            }
            const unsigned char *box0 = ring + size_t(g0 % kx) * box_bytes;
            const unsigned char *box1 = ring + size_t((g0 + 1) % kx) * box_bytes;
            for (int task = tid; task < nt * (kTcBK / 8); task += kSkProducers) {
                const int c = ((task >> 5) << 3) | (task & 7), kb = (task >> 3) & 3;
                double v[8];
                xring_read8(box0, box1, c, kb, r0 + 8 * kb, re, c, unit_lower, v);
                const uint32_t off = static_cast<uint32_t>(ts * a_bytes) + kmajor_off(c, 8 * kb);
                if (NSL == 1) {
                    uint32_t h[8];
#pragma unroll
                    for (int t = 0; t < 8; ++t) h[t] = bf16_bits_from_f64_fast(v[t]);
                    *reinterpret_cast<uint4 *>(stage + off) =
                        make_uint4(h[0] | (h[1] << 16), h[2] | (h[3] << 16), h[4] | (h[5] << 16),
                                   h[6] | (h[7] << 16));
                } else {
                    uint32_t h[3][8];
#pragma unroll
                    for (int t = 0; t < 8; ++t) {
                        double rnd, rnd2, rnd3;
                        h[0][t] = bf16_bits_from_f64(v[t], rnd);
                        const double r1 = v[t] - rnd;
                        h[1][t] = bf16_bits_from_f64(r1, rnd2);
                        h[2][t] = bf16_bits_from_f64(r1 - rnd2, rnd3);
                    }
#pragma unroll
                    for (int p = 0; p < 3; ++p)
                        *reinterpret_cast<uint4 *>(stage + off + p * b_bytes) =
                            make_uint4(h[p][0] | (h[p][1] << 16), h[p][2] | (h[p][3] << 16),
                                       h[p][4] | (h[p][5] << 16), h[p][6] | (h[p][7] << 16));
                }
            }
            fence_proxy_async_smem();  // generic-proxy stores -> visible to the tensor core
            __syncwarp();
            if (lane == 0) {  // one arrival per warp
                if (use_tma) {
                    mbar_arrive(&pp.xempty[g0 % kx]);
                    mbar_arrive(&pp.xempty[(g0 + 1) % kx]);
                }
                mbar_arrive(&pp.full[s]);
            }
        }
        // the last commit covers every MMA
        if (nsteps > 0) {
            const int last = nsteps - 1;
            (void)sk_wait(pp, &pp.empty[last % nst], static_cast<uint32_t>((last / nst) & 1));
        }
    }
    __syncthreads();
    tc_fence_after();
    if (pp.abort_flag) {
        if (tid == 0) report(st, kErrTimeout, 0, -1);
        if (control && lane == 0) sk_drain(pp, issued, kx, committed, nst);
    } else if (!control) {
        // epilogue: producer warp w reads TMEM lanes 32 (w % 4) .. +31 (sketch
        // rows of each tile) and the 32-column chunks ch with ch % 4 = w / 4
        const int lane_base = 32 * (warp & 3);
        const int cgrp = warp >> 2;
        const int nchunks = (nt + 31) / 32;
        double *out = part + size_t(blockIdx.y) * s_pad * n_pad;
        for (int t = 0; t < ts; ++t) {
            const int r = rt0 + kTcM * t + lane_base + lane;
            for (int ch = cgrp; ch < nchunks; ch += kSkProducers / 128) {
                const int cb = 32 * ch;
                if (nsteps > 0) {
                    float v[32];
                    tmem_ld32(tmem + (static_cast<uint32_t>(lane_base) << 16) +
                                  static_cast<uint32_t>(t) * tcols + static_cast<uint32_t>(cb),
                              v);
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int c = cb + j;
                        if (c < nt && c < n_pad && r < s_pad) out[size_t(c) * s_pad + r] = double(v[j]) * scale;
                    }
                } else {  // a CTA without rows contributes zeros
                    for (int j = 0; j < 32; ++j) {
                        const int c = cb + j;
                        if (c < nt && c < n_pad && r < s_pad) out[size_t(c) * s_pad + r] = 0.0;
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (control) tmem_dealloc(tmem, ncols);
}

// ---- digit tier --------------------------------------------------------------

constexpr int kDgDigits = 6;                         // 48 bits of each column of X
constexpr int kDgNC = 64;                            // columns of X per CTA (N of the MMA)
constexpr int kDgThreads = kSkProducers + 32;      // 16 producer warps + the control warp
constexpr int kDgStages = 3;
constexpr int kDgWinSteps = 32;                      // 32 steps of 32 rows: 1024-row windows
constexpr int kDgFlushWindows = 16;                  // int64 drains between binary64 flushes
constexpr int kDgTileA = kTcM * kTcBK * 2;           // S: 128 x 32 bf16 (8 KB)
constexpr int kDgTileB = kDgNC * kTcBK * 2;          // one digit of X: 64 x 32 bf16 (4 KB)
constexpr int kDgStageBytes = kDgTileA + kDgDigits * kDgTileB;
constexpr int kDgTmemCols = 512;                     // 6 levels x 64 columns (384) rounded up
constexpr int kDgAccPerThread = kTcM * kDgNC / kSkProducers;  // 16 int64 window sums
constexpr uint32_t kDgBoxBytes = kDgNC * 128;        // one ring box: 16 rows x 64 columns
constexpr int kDgRing = 6;
constexpr size_t kDgSmemBytes = size_t(kDgStages) * kDgStageBytes + size_t(kDgRing) * kDgBoxBytes +
                                size_t(kDgAccPerThread) * kSkProducers * 8 + 1024;

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

// Partial Y of one CTA: 128 sketch rows x 64 columns of X over the CTA's
// steps of rows, in units of 2^(E_c - 44) (binary64), written to
// part[blockIdx.y][c * s_pad + r].  Warp-specialised like k_sketch_tc: per
// 32 rows of X the 16 producer warps draw S (integers k) and split X (from
// the ring) into six digit tiles; the control lane issues the six level
// products of each 16-row k-step as two MMAs over the side-by-side digit
// tiles (kind::f16, M = 128, N = 256 and 128): level t (digit t of X,
// weight 256^(5 - t)) in TMEM columns 64 t .. 64 t + 63.
// After the last step of each 1024-row window the producers drain the
// levels into int64 window sums (exact) and release TMEM (tmem_empty) before
// the control lane starts the next window; every 16 windows the sums go
// into the binary64 partial.
template <bool kAlignedS>
__global__ void __launch_bounds__(kDgThreads, 1)
    k_sketch_digits(const __grid_constant__ CUtensorMap xmap, int use_tma, const double *__restrict__ X,
                    int64_t ldx, int64_t m, int n, int unit_lower, int n_st,
                    uint64_t seed, const int *__restrict__ colbits, double *__restrict__ part,
                    int s_pad, int n_pad, DevStatus *st, int64_t row0) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ SkPipe pp;
    __shared__ __align__(16) uint16_t lv[kLevels];
    __shared__ int expB[kDgNC];

    unsigned char *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    unsigned char *ring = smem + kDgStages * kDgStageBytes;
    // the producers' window sums acc[q * kSkProducers + tid] (registers are short)
    long long *acc = reinterpret_cast<long long *>(ring + size_t(kDgRing) * kDgBoxBytes);

    const int st_idx = blockIdx.x % n_st, ct_idx = blockIdx.x / n_st;
    const int rt0 = kTcM * st_idx;  // first sketch row of the tile
    const int c0 = kDgNC * ct_idx;  // first column of X
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool control = warp == kSkProducers / 32;
    const int64_t re = m;
    const int nsteps = xsteps(m);
    const int nboxes = 2 * nsteps;

    if (control) tmem_alloc(&pp.tmem_slot, kDgTmemCols);
    if (tid == 0) {
        for (int q = 0; q < kDgStages; ++q) {
            mbar_init(&pp.full[q], kSkWarps);
            mbar_init(&pp.empty[q], 1);
        }
        for (int q = 0; q < kDgRing; ++q) {
            mbar_init(&pp.xfull[q], 1);
            mbar_init(&pp.xempty[q], kSkWarps);
        }
        mbar_init(&pp.tmem_empty, kSkWarps);
        fence_mbar_init();
        pp.abort_flag = 0;
    }
    for (int k = tid; k < kLevels / 8; k += kDgThreads)
        reinterpret_cast<uint4 *>(lv)[k] = reinterpret_cast<const uint4 *>(g_gauss_levels)[k];
    if (tid < kDgNC) expB[tid] = (c0 + tid < n) ? emu_exponent(colbits[c0 + tid]) : 0;
    if (!control)
#pragma unroll
        for (int q = 0; q < kDgAccPerThread; ++q) acc[q * kSkProducers + tid] = 0;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = pp.tmem_slot;
    int issued = 0, committed = -1;  // the control thread's ring and MMA bookkeeping

    if (control) {
        if (lane == 0) {
            const uint32_t idesc4 = idesc_bf16_f32(kTcM, 4 * kDgNC);
            const uint32_t idesc2 = idesc_bf16_f32(kTcM, 2 * kDgNC);
            if (use_tma) {
                prefetch_tensormap(&xmap);
                for (; issued < (nboxes < kDgRing ? nboxes : kDgRing); ++issued)
                    xring_issue(ring, pp.xfull, &xmap, issued, kDgRing, kDgBoxBytes, c0);
            }
            for (int ks = 0; ks < nsteps; ++ks) {
                const int s = ks % kDgStages;
                const bool fresh = (ks % kDgWinSteps) == 0;
                // a new window overwrites the levels: the previous one is drained
                if (fresh && ks > 0 &&
                    !sk_wait(pp, &pp.tmem_empty, static_cast<uint32_t>((ks / kDgWinSteps - 1) & 1)))
                    break;
                if (!sk_wait(pp, &pp.full[s], static_cast<uint32_t>((ks / kDgStages) & 1))) break;
                tc_fence_after();
                const uint32_t a0 = smem_u32(smem + s * kDgStageBytes);
                // the digit tiles lie side by side (K-major, 64 rows each), so
                // digits 0-3 form one N = 256 operand whose product lands in
                // levels 0-3 (TMEM columns 0-255) and digits 4-5 one N = 128
                // operand (columns 256-383): two MMAs per k-step instead of six
#pragma unroll
                for (int kk = 0; kk < kTcBK / 16; ++kk) {
                    const uint64_t ad = smem_desc(a0 + kk * 256, 128, kTcBK * 16);
                    const uint64_t bd = smem_desc(a0 + kDgTileA + kk * 256, 128, kTcBK * 16);
                    mma_bf16(tmem, ad, bd, idesc4, (fresh && kk == 0) ? 0u : 1u);
                    mma_bf16(tmem + static_cast<uint32_t>(4 * kDgNC), ad,
                             bd + static_cast<uint64_t>((4 * kDgTileB) >> 4), idesc2, (fresh && kk == 0) ? 0u : 1u);
                }
                mma_commit(&pp.empty[s]);
                committed = ks;
                if (use_tma)
                    for (int g = 2 * ks; g < 2 * ks + 2 && g + kDgRing < nboxes; ++g) {
                        if (!sk_wait(pp, &pp.xempty[g % kDgRing], static_cast<uint32_t>((g / kDgRing) & 1)))
                            break;
                        xring_issue(ring, pp.xfull, &xmap, g + kDgRing, kDgRing, kDgBoxBytes, c0);
                        issued = g + kDgRing + 1;
                    }
            }
        }
    } else {
        // drain ownership: TMEM lanes 32 (warp % 4) .. +31 (sketch rows),
        // columns 16 (warp / 4) .. +15
        const int lane_base = 32 * (warp & 3);
        const int cgrp = warp >> 2;
        double *mine = part + size_t(blockIdx.y) * s_pad * n_pad + size_t(c0 + 16 * cgrp) * s_pad +
                       rt0 + lane_base + lane;
        int windows = 0;
        bool flushed = false;
        auto flush = [&]() {
#pragma unroll
            for (int q = 0; q < kDgAccPerThread; ++q) {
                const double v = static_cast<double>(acc[q * kSkProducers + tid]);
                mine[size_t(q) * s_pad] = flushed ? mine[size_t(q) * s_pad] + v : v;
                acc[q * kSkProducers + tid] = 0;
            }
            flushed = true;
        };
        // this thread's X task: column xc, rows 4 xq .. 4 xq + 3 of a step
        // (eight neighbouring threads on eight columns); its S task: row sr,
        // entries 8 skb .. 8 skb + 7
        const int xc = ((warp & 7) << 3) | (lane & 7), xq = (lane >> 3) + 4 * (warp >> 3);
        const int sr = (warp << 3) | (lane & 7), skb = (lane >> 3) & 3;
        const uint32_t xoff = static_cast<uint32_t>(((xc >> 3) * (kTcBK / 8) + (xq >> 1)) * 128 +
                                                    (xc & 7) * 16 + (xq & 1) * 8);
        bool ok = true;
        for (int ks = 0; ks < nsteps; ++ks) {
            const int s = ks % kDgStages;
            unsigned char *stage = smem + s * kDgStageBytes;
            const int64_t r0 = xstep_row(ks);
            const int g0 = 2 * ks;
            if (use_tma) {
                if (ks >= kDgStages &&
                    !sk_wait(pp, &pp.empty[s], static_cast<uint32_t>(((ks / kDgStages) - 1) & 1))) {
                    ok = false;
                    break;
                }
            } else {
                const bool w = ks < kDgStages ||
                               sk_wait(pp, &pp.empty[s], static_cast<uint32_t>(((ks / kDgStages) - 1) & 1));
                // one verdict for all producers before their shared fills
                if (named_bar_or(1, kSkProducers, !w || sk_aborted(pp))) {
                    ok = false;
                    break;
                }
                xring_fill(ring, g0, kDgRing, kDgBoxBytes, X, ldx, m, n, c0, kDgNC, tid, kSkProducers);
                xring_fill(ring, g0 + 1, kDgRing, kDgBoxBytes, X, ldx, m, n, c0, kDgNC, tid, kSkProducers);
            }
            // (1) S block: 128 sketch rows x 32 rows of X (X's rows past the end are zero)
            *reinterpret_cast<uint4 *>(stage + kmajor_off(sr, 8 * skb)) =
                kAlignedS ? sk_levels8_aligned(static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32),
                                               rt0 + sr, static_cast<uint64_t>(row0 + r0) / 8 + skb, lv)
                          : sk_levels8(seed, rt0 + sr, row0 + r0 + 8 * skb, lv);
            // (2) six digits of the thread's four values: one 8-byte piece per digit tile
            if (use_tma) {
                if (!sk_wait(pp, &pp.xfull[g0 % kDgRing], static_cast<uint32_t>((g0 / kDgRing) & 1)) ||
                    !sk_wait(pp, &pp.xfull[(g0 + 1) % kDgRing], static_cast<uint32_t>(((g0 + 1) / kDgRing) & 1))) {
                    ok = false;
                    break;
                }
            } else {
                named_bar_sync(1, kSkProducers);  // the fills are complete
            }
            {
                const unsigned char *box = ring + size_t((g0 + (xq >> 2)) % kDgRing) * kDgBoxBytes;
                const int j0 = (4 * xq & 15) >> 1;  // chunks j0, j0 + 1: rows 4 xq .. 4 xq + 3
                const double2 d0 = *reinterpret_cast<const double2 *>(box + xbox_off(xc, j0));
                const double2 d1 = *reinterpret_cast<const double2 *>(box + xbox_off(xc, j0 + 1));
                double xv[4] = {d0.x, d0.y, d1.x, d1.y};
                const int col = c0 + xc;
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int64_t row = r0 + 4 * xq + t;
                    if (row >= re) xv[t] = 0.0;
                    else if (unit_lower && row <= col) xv[t] = (row == col) ? 1.0 : 0.0;
                }
                const int E = expB[xc];
                uint32_t w0[kDgDigits], w1[kDgDigits];
                emu_digits2_packed<kDgDigits>(xv[0], xv[1], E, w0);
                emu_digits2_packed<kDgDigits>(xv[2], xv[3], E, w1);
#pragma unroll
                for (int q = 0; q < kDgDigits; ++q)
                    *reinterpret_cast<uint2 *>(stage + kDgTileA + q * kDgTileB + xoff) = make_uint2(w0[q], w1[q]);
            }
            fence_proxy_async_smem();  // generic-proxy stores -> visible to the tensor core
            __syncwarp();
            if (lane == 0) {  // one arrival per warp
                if (use_tma) {
                    mbar_arrive(&pp.xempty[g0 % kDgRing]);
                    mbar_arrive(&pp.xempty[(g0 + 1) % kDgRing]);
                }
                mbar_arrive(&pp.full[s]);
            }
            // (3) end of a window: drain the six level accumulators into int64,
            // in units of 2^8 (level 5 rounded to that unit), and release TMEM
            if ((ks % kDgWinSteps) == kDgWinSteps - 1 || ks == nsteps - 1) {
                if (!sk_wait(pp, &pp.empty[s], static_cast<uint32_t>((ks / kDgStages) & 1))) {
                    ok = false;
                    if (use_tma) break;
                    continue;  // the plain-load path leaves at the next step's common verdict
                }
                tc_fence_after();
                const uint32_t tl = tmem + (static_cast<uint32_t>(lane_base) << 16) +
                                    static_cast<uint32_t>(16 * cgrp);
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
                        acc[q * kSkProducers + tid] += a;
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&pp.tmem_empty);
                if (++windows == kDgFlushWindows) {
                    flush();
                    windows = 0;
                }
            }
        }
        if (ok && !sk_aborted(pp)) flush();
    }
    __syncthreads();
    if (pp.abort_flag) {
        if (tid == 0) report(st, kErrTimeout, 0, -1);
        if (control && lane == 0) sk_drain(pp, issued, kDgRing, committed, kDgStages);
    }
    tc_fence_before();
    __syncthreads();
    if (control) tmem_dealloc(tmem, kDgTmemCols);
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

namespace {

// Launch shape of the tensor-core sketch (one CTA of 16 producer warps and a
// control warp per SM): sketch tiles per CTA (ts), operand stages (nst),
// ring slots (kx) and dynamic shared memory.  Among the shapes that fit,
// the one with the most ring slots up to four (two steps of look-ahead),
// then the most tiles per CTA (X split once for both), then the most stages.
struct TcShape {
    int nt, ts, nst, kx;
    size_t smem;
};

constexpr size_t kTcStaticBytes = kLevels * 2 + 1024;  // level table, barriers (1024-aligned)

TcShape tc_shape(int n, int64_t s, int nterms) {
    TcShape best = {std::min(pad16(n), 256), 1, 2, 0, 0};
    int tcols = 32;
    while (tcols < best.nt) tcols <<= 1;
    const int n_st = static_cast<int>(round_up(s, kTcM) / kTcM);
    const size_t box = size_t(best.nt) * 128;
    const size_t dyn = 227 * 1024 - kTcStaticBytes;
    int best_key = -1;
    for (int ts = 1; ts <= ((n_st % 2 == 0 && 2 * tcols <= 512) ? 2 : 1); ++ts)
        for (int nst = 2; nst <= 3; ++nst) {
            const size_t fixed =
                size_t(nst) * (size_t(ts) * kTcM * kTcBK * 2 + size_t(nterms) * best.nt * kTcBK * 2) + 1024;
            if (fixed + 2 * box > dyn) continue;
            const int kx = static_cast<int>(std::min<size_t>(kXRingMax, (dyn - fixed) / box));
            const int key = std::min(kx, 4) * 100 + ts * 10 + nst;
            if (key > best_key) {
                best_key = key;
                best.ts = ts;
                best.nst = nst;
                best.kx = kx;
                best.smem = fixed + size_t(kx) * box;
            }
        }
    return best;
}

}  // namespace

size_t tc_sketch_smem_bytes(int n, int nterms) {
    return tc_shape(n, 256, nterms).smem;
}

cudaError_t launch_sketch_tc(const double *X, int64_t ldx, int64_t m, int n, int unit_lower,
                             int64_t s, uint64_t seed, int nterms, double *Y, int64_t ldy,
                             double *part, DevStatus *st, cudaStream_t stream, int64_t row0) {
    if (n > 256 || (nterms != 1 && nterms != 3)) return cudaErrorInvalidValue;
    const TcShape sh = tc_shape(n, s, nterms);
    if (sh.kx < 2) return cudaErrorInvalidValue;
    const int s_pad = static_cast<int>(round_up(s, kTcM));
    const int n_pad = static_cast<int>(round_up(n, 32));
    const int tiles = s_pad / kTcM / sh.ts;  // n <= 256: one column tile
    // one CTA per SM over the tiles, no more partials than the workspace holds
    const int64_t pmax = std::max<int64_t>(
        1, int64_t(sketch_partials_doubles(m, n, s, 0) / (size_t(s_pad) * size_t(n_pad))));
    int64_t p = std::min<int64_t>(pmax, std::max(1, grid_sms() / tiles));
    p = std::max<int64_t>(1, std::min<int64_t>(p, ceil_div(m, kTcBK)));
    CUtensorMap map;
    const bool tma = m < (int64_t(1) << 31) - 2 * kTcBK &&  // TMA row coordinates are int32
                     make_tma_map(&map, X, m, n, ldx, kXBoxRows, sh.nt, true);
    if (!tma) memset(&map, 0, sizeof map);
    const dim3 grid(tiles, static_cast<unsigned>(p));
    const double scale = 1.0 / (32.0 * sqrt(double(s)));  // the grid's 1/32 and 1/sqrt(s)
    // rows of S start on Philox block boundaries unless the rows of X are
    // offset by a non-multiple of 8 (a row block of a sharded matrix)
    const bool aligned = (row0 % 8) == 0;
    auto run = [&](auto kern) -> cudaError_t {
        cudaError_t e2 = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sh.smem));
        if (e2 != cudaSuccess) return e2;
        RQ_LAUNCH(KID_SKETCH_TC, stream,
                  kern<<<grid, kTcThreads, sh.smem, stream>>>(map, tma ? 1 : 0, X, ldx, m, n, unit_lower,
                                                              sh.ts, sh.nt, sh.nst, sh.kx, seed, scale, part,
                                                              s_pad, n_pad, st, row0));
        return cudaSuccess;
    };
    cudaError_t e;
    if (nterms == 1)
        e = aligned ? run(k_sketch_tc<1, true>) : run(k_sketch_tc<1, false>);
    else
        e = aligned ? run(k_sketch_tc<3, true>) : run(k_sketch_tc<3, false>);
    if (e != cudaSuccess) return e;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_reduce_sketch(part, static_cast<int>(p), static_cast<int>(s), n, s_pad, n_pad, Y,
                                ldy, stream);
}

size_t sketch_digits_partials_doubles(int64_t s, int n) {
    const size_t tiles = size_t(round_up(s, kTcM) / kTcM) * size_t(ceil_div(n, kDgNC));
    const size_t p = std::max<size_t>(1, size_t(num_sms()) / tiles) + 1;
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
    // one CTA per SM (its TMEM holds 384 of the SM's 512 columns)
    int p = std::max(1, grid_sms() / tiles);
    p = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(p, ceil_div(m, kTcBK))));
    int *colbits = reinterpret_cast<int *>(part + size_t(p) * s_pad * n_pad);
    cudaError_t e = cudaMemsetAsync(colbits, 0, sizeof(int) * size_t(n), stream);
    if (e != cudaSuccess) return e;
    const int64_t cchunk = std::max<int64_t>(4096, ceil_div(m, 64));
    RQ_LAUNCH(KID_EMU_AUX, stream,
              k_dg_col_exponent<<<dim3(n, static_cast<unsigned>(ceil_div(m, cchunk))), 256, 0, stream>>>(
                  X, ldx, m, unit_lower, cchunk, colbits));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    CUtensorMap map;
    const bool tma = m < (int64_t(1) << 31) - 2 * kTcBK &&  // TMA row coordinates are int32
                     make_tma_map(&map, X, m, n, ldx, kXBoxRows, kDgNC, true);
    if (!tma) memset(&map, 0, sizeof map);
    auto kern = (row0 % 8) == 0 ? k_sketch_digits<true> : k_sketch_digits<false>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kDgSmemBytes));
    if (e != cudaSuccess) return e;
    RQ_LAUNCH(KID_SKETCH_TC, stream,
              kern<<<dim3(tiles, p), kDgThreads, kDgSmemBytes, stream>>>(
                  map, tma ? 1 : 0, X, ldx, m, n, unit_lower, n_st, seed, colbits, part, s_pad,
                  n_pad, st, row0));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int64_t ne = s * int64_t(n);
    RQ_LAUNCH(KID_REDUCE, stream,
              k_reduce_sketch_digits<<<static_cast<unsigned>(ceil_div(ne, 256)), 256, 0, stream>>>(
                  part, p, static_cast<int>(s), n, s_pad, n_pad, colbits, 1.0 / sqrt(double(s)), Y, ldy));
    return cudaGetLastError();
}

}  // namespace rq
