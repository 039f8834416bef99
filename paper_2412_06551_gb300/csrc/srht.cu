// Subsampled randomized Hadamard sketch Y = S A, S = R H D / sqrt(s): the
// third common sketch Section 3 names next to the Gaussian sketch and
// CountSketch.  H is the Sylvester-Hadamard matrix of order m' = 2^b >= m
// (A padded with zero rows), H(p, i) = (-1)^popcount(p AND i); D holds random
// signs; R keeps the s rows p_r = pi(r) of a keyed Feistel permutation pi.
//
// The kernel never forms S.  Row index i = 256 g + i_lo splits H into a sign
// per 256-row block g and a Hadamard matrix of order 256 inside the block:
//   (S A)(r, j) = 1/sqrt(s) sum_g (-1)^popcount(p_hi AND g) (H256 D_g A_g)(p_lo, j)
// with p_r = 256 p_hi + p_lo.  So each block of each column is transformed
// once (eight butterfly levels) and the s sampled entries are gathered from
// it: 8 + s/256 operations per element of A instead of 2s for a dense S.
//
// The butterflies run on integers, exactly: the block's entries are scaled by
// one power of two (the block's largest exponent) and rounded to 53-bit
// integers, whose transform needs at most 61 bits.  This puts the transform on
// the integer pipes (the FP64 pipe is the scarcest one) and makes it exact;
// the one rounding is that of entries more than 2^53 times smaller than the
// block's largest.  The sampled values enter binary64 accumulators with one
// fused multiply-add each.
#include "common.cuh"
#include "kernels.h"

namespace rq {
namespace {

constexpr int kSrhtBlock = 256;  // rows per Hadamard block (order 2^8)
constexpr int kSrhtThreads = 256;

// pi(x) on b bits: four Feistel rounds (L, R) -> (R, L ^ F_k(R)) with widths
// (ceil(b/2), floor(b/2)) swapping after each round; F_k(R) is the first
// Philox word for counter (R, k, b, 0x53524850), reduced to the left width.
__device__ uint32_t srht_perm(int b, uint32_t k0, uint32_t k1, uint32_t x) {
    int wl = (b + 1) >> 1, wr = b >> 1;
    uint32_t L = x >> wr, R = x & ((1u << wr) - 1u);
#pragma unroll 1
    for (uint32_t k = 0; k < 4; ++k) {
        const uint4 w = philox4x32_10(make_uint4(R, k, static_cast<uint32_t>(b), 0x53524850u), k0, k1);
        const uint32_t nl = R, nr = L ^ (w.x & ((1u << wl) - 1u));
        const int t = wl;
        wl = wr;
        wr = t;
        L = nl;
        R = nr;
    }
    return (L << wr) | R;
}

// Bank-conflict-free position of row i of a 256-entry int64 column: the low
// four bits are XORed with the next four, so both the row-block and the
// transposed access of a half-warp touch sixteen distinct 8-byte slots.
__device__ __forceinline__ int srht_swz(int i) { return i ^ ((i >> 4) & 15); }

// Unnormalised Walsh-Hadamard transform of 16 values in natural order.
__device__ __forceinline__ void fwht16(long long (&v)[16]) {
#pragma unroll
    for (int h = 1; h < 16; h <<= 1)
#pragma unroll
        for (int k = 0; k < 16; ++k)
            if (!(k & h)) {
                const long long a = v[k], c = v[k | h];
                v[k] = a + c;
                v[k | h] = a - c;
            }
}

// One CTA: NC columns (tile blockIdx.y) over a range of 256-row blocks
// (blockIdx.x), NR sampled rows per thread (s <= 256 NR).  Phase A: each
// half-warp owns one column, holds 16 entries per lane, transforms over the
// register index, transposes through shared memory and transforms over the
// other four bits.  Phase B: thread t gathers rows p_r (r = t + 256 q) of
// every column's transformed block and accumulates them.
template <int NC, int NR>
__global__ void __launch_bounds__(kSrhtThreads, 2)
k_sketch_srht(const double *__restrict__ A, int64_t lda, int64_t m, int n, int unit_lower,
              int64_t row0, int s, uint64_t seed, int b, int64_t gb0, int64_t nblk, int64_t chunk,
              double inv_sqrt_s, double *__restrict__ part, int s_pad, int n_pad) {
    extern __shared__ __align__(16) unsigned char smem[];
    long long *T = reinterpret_cast<long long *>(smem);          // NC x 256, swizzled
    double *scale = reinterpret_cast<double *>(T + NC * kSrhtBlock);  // NC: 2^(E - 1075) or NaN
    uint32_t *sw = reinterpret_cast<uint32_t *>(scale + NC);     // 8 words of sign bits
    int *pidx = reinterpret_cast<int *>(sw + 8);                 // s sampled rows of H
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int half = lane >> 4, l16 = lane & 15;
    const uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
    for (int r = tid; r < s; r += kSrhtThreads)
        pidx[r] = static_cast<int>(srht_perm(b, k0, k1, static_cast<uint32_t>(r)));

    const int j0 = blockIdx.y * NC;
    const int64_t g_begin = gb0 + int64_t(blockIdx.x) * chunk;
    const int64_t g_end = min(gb0 + nblk, g_begin + chunk);
    const int c = 2 * warp + half;  // phase-A column of this half-warp
    const bool a_active = c < NC;   // warp-uniform (NC even)
    const int j = j0 + c;
    const bool col_ok = a_active && j < n;
    const double *Aj = A + int64_t(col_ok ? j : 0) * lda;

    double y[NR][NC];
#pragma unroll
    for (int q = 0; q < NR; ++q)
#pragma unroll
        for (int cc = 0; cc < NC; ++cc) y[q][cc] = 0.0;

#pragma unroll 1
    for (int64_t gb = g_begin; gb < g_end; ++gb) {
        if (tid < 2) {  // sign bits of rows 256 gb .. 256 gb + 255
            const uint64_t q = uint64_t(gb) * 2 + tid;
            const uint4 w = philox4x32_10(
                make_uint4(static_cast<uint32_t>(q), static_cast<uint32_t>(q >> 32), 0u, 0x53524844u), k0,
                k1);
            sw[4 * tid + 0] = w.x;
            sw[4 * tid + 1] = w.y;
            sw[4 * tid + 2] = w.z;
            sw[4 * tid + 3] = w.w;
        }
        __syncthreads();  // sign bits visible; the previous block's gathers are done
        if (a_active) {
            long long v[16];
            int emax = 1;
            const int64_t base = gb * kSrhtBlock - row0;  // local row of the block's first row
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const int64_t li = base + l16 + 16 * k;
                double x = 0.0;
                if (col_ok && li >= 0 && li < m) {
                    if (!unit_lower || li > j)
                        x = __ldg(Aj + li);
                    else
                        x = li == j ? 1.0 : 0.0;
                }
                v[k] = __double_as_longlong(x);
                emax = max(emax, static_cast<int>((v[k] >> 52) & 0x7FF));
            }
#pragma unroll
            for (int o = 8; o >= 1; o >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
            // x 2^(1075 - emax) rounded to an integer (|.| < 2^53), sign of x times d_i
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const long long bits = v[k];
                const int e = static_cast<int>((bits >> 52) & 0x7FF);
                const unsigned long long mant =
                    (static_cast<unsigned long long>(bits) & 0xFFFFFFFFFFFFFull) | (e ? (1ull << 52) : 0ull);
                const int sh = min(emax - max(e, 1), 63);
                const unsigned long long mag =
                    sh == 0 ? mant : (sh >= 54 ? 0ull : (mant + (1ull << (sh - 1))) >> sh);
                const uint32_t dw = sw[(k >> 3) * 4 + ((k & 7) >> 1)];
                const uint32_t neg = ((dw >> (l16 + 16 * (k & 1))) & 1u) ^
                                     static_cast<uint32_t>(static_cast<unsigned long long>(bits) >> 63);
                v[k] = neg ? -static_cast<long long>(mag) : static_cast<long long>(mag);
            }
            fwht16(v);  // row bits 4..7 (register index k of row l16 + 16 k)
            long long *Tc = T + c * kSrhtBlock;
#pragma unroll
            for (int k = 0; k < 16; ++k) Tc[srht_swz(l16 + 16 * k)] = v[k];
            __syncwarp();
#pragma unroll
            for (int k = 0; k < 16; ++k) v[k] = Tc[srht_swz(16 * l16 + k)];
            fwht16(v);  // row bits 0..3; each lane rewrites exactly the slots it read
#pragma unroll
            for (int k = 0; k < 16; ++k) Tc[srht_swz(16 * l16 + k)] = v[k];
            if (l16 == 0) {
                double f;
                if (emax == 2047)
                    f = __longlong_as_double(0x7FF8000000000000ll);  // non-finite entry in the block
                else if (emax >= 53)
                    f = __longlong_as_double(static_cast<long long>(emax - 52) << 52);
                else
                    f = __longlong_as_double(1ll << (emax - 1));  // subnormal 2^(emax - 1075)
                scale[c] = f;
            }
        }
        __syncthreads();  // transformed blocks ready
#pragma unroll
        for (int q = 0; q < NR; ++q) {
            const int r = tid + kSrhtThreads * q;
            if (r < s) {
                const int pr = pidx[r];
                const int ps = srht_swz(pr & 255);
                const bool neg = __popc(static_cast<uint32_t>(pr >> 8) & static_cast<uint32_t>(gb)) & 1;
#pragma unroll
                for (int cc = 0; cc < NC; ++cc) {
                    const long long t = T[cc * kSrhtBlock + ps];
                    y[q][cc] = fma(static_cast<double>(neg ? -t : t), scale[cc], y[q][cc]);
                }
            }
        }
    }
    double *P = part + size_t(blockIdx.x) * s_pad * n_pad;
#pragma unroll
    for (int q = 0; q < NR; ++q) {
        const int r = tid + kSrhtThreads * q;
        if (r >= s) continue;
#pragma unroll
        for (int cc = 0; cc < NC; ++cc)
            if (j0 + cc < n) P[size_t(j0 + cc) * s_pad + r] = y[q][cc] * inv_sqrt_s;
    }
}

template <int NC, int NR>
cudaError_t launch_srht_t(const double *A, int64_t lda, int64_t m, int n, int unit_lower, int64_t row0,
                          int s, uint64_t seed, int b, double *part, int s_pad, int n_pad, int *nparts,
                          cudaStream_t stream) {
    const int64_t gb0 = row0 / kSrhtBlock;
    const int64_t nblk = (row0 + m - 1) / kSrhtBlock - gb0 + 1;
    const int tiles = static_cast<int>(ceil_div(n, NC));
    const int64_t want = std::max<int64_t>(1, int64_t(2) * grid_sms() / tiles);
    const int64_t chunk = ceil_div(nblk, std::min(want, nblk));
    const int grid_x = static_cast<int>(ceil_div(nblk, chunk));
    const size_t smem = size_t(NC) * kSrhtBlock * 8 + size_t(NC) * 8 + 8 * 4 + size_t(s) * 4;
    auto k = k_sketch_srht<NC, NR>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    RQ_LAUNCH(KID_SKETCH_SRHT, stream,
              k<<<dim3(grid_x, tiles), kSrhtThreads, smem, stream>>>(
                  A, lda, m, n, unit_lower, row0, s, seed, b, gb0, nblk, chunk, 1.0 / sqrt(double(s)),
                  part, s_pad, n_pad));
    *nparts = grid_x;
    return cudaGetLastError();
}

}  // namespace

int srht_order_log2(int64_t rows) {
    int b = 0;
    while ((int64_t(1) << b) < rows) ++b;
    return b;
}

cudaError_t launch_sketch_srht(const double *A, int64_t lda, int64_t m, int n, int unit_lower, int64_t s,
                               uint64_t seed, int b, double *Y, int64_t ldy, double *part,
                               cudaStream_t stream, int64_t row0) {
    const int s_pad = static_cast<int>(round_up(s, 64));
    const int n_pad = static_cast<int>(round_up(n, 32));
    const int si = static_cast<int>(s);
    int nparts = 0;
    cudaError_t e;
    if (s <= 256)
        e = launch_srht_t<16, 1>(A, lda, m, n, unit_lower, row0, si, seed, b, part, s_pad, n_pad, &nparts,
                                 stream);
    else if (s <= 512)
        e = launch_srht_t<16, 2>(A, lda, m, n, unit_lower, row0, si, seed, b, part, s_pad, n_pad, &nparts,
                                 stream);
    else if (s <= 1024)
        e = launch_srht_t<8, 4>(A, lda, m, n, unit_lower, row0, si, seed, b, part, s_pad, n_pad, &nparts,
                                stream);
    else if (s <= 2048)
        e = launch_srht_t<4, 8>(A, lda, m, n, unit_lower, row0, si, seed, b, part, s_pad, n_pad, &nparts,
                                stream);
    else
        e = launch_srht_t<2, 16>(A, lda, m, n, unit_lower, row0, si, seed, b, part, s_pad, n_pad, &nparts,
                                 stream);
    if (e != cudaSuccess) return e;
    return launch_reduce_sketch(part, nparts, si, n, s_pad, n_pad, Y, ldy, stream);
}

}  // namespace rq
