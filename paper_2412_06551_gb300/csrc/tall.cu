// Tall m x n passes over X (FP64): the sketch S X (Algorithm 6; S M in
// Algorithm 7), the Gram product A^T A (Algorithm 1, C1/C5), and the
// triangular solve A R^{-1} fused with the Gram of its result (Algorithm 1,
// C1; C3 + C5; C7).
//
// Design (GB300, FP64 pipe bound): each CTA owns a contiguous chunk of rows
// and walks it in row tiles of BM x ncols staged in shared memory by a 2-D
// TMA box (cp.async.bulk.tensor, mbarrier completion; plain loads when the
// matrix misses TMA's alignment rules).  Per-CTA partial sums go to a
// workspace and are reduced in a fixed order, so results are bitwise
// reproducible for a given launch shape.  Work inside a CTA is assigned per
// warp (16 x 16 warp tiles of the output) so that all four SM sub-partitions
// get equal FP64 work.  Two CTAs per SM cover each other's load and
// synchronization bubbles.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace rq {

constexpr int kThreads = 256;

// ------------------------------------------------------------ plumbing ---

LaunchPolicy &launch_policy() {
    static thread_local LaunchPolicy p;
    return p;
}

int grid_sms() { return std::max(1, num_sms() / std::max(1, launch_policy().grid_div)); }

int num_sms() {
    static int cached = 0;
    if (cached == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&cached, cudaDevAttrMultiProcessorCount, dev);
        // no visible device (a host-only size query): the GB300's 152 SMs,
        // the only GPU this build targets
        if (cached <= 0) cached = 152;
    }
    return cached;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

bool make_tma_map(CUtensorMap *map, const double *A, int64_t rows, int64_t cols, int64_t ld,
                  int box_rows, int box_cols, bool swizzle128) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    if (reinterpret_cast<uintptr_t>(A) % 16 != 0) return false;
    if ((ld * 8) % 16 != 0 || ld * 8 >= (int64_t(1) << 40)) return false;
    if ((box_rows * 8) % 16 != 0 || box_rows > 256 || box_cols > 256 || box_rows < 1 || box_cols < 1)
        return false;
    if (swizzle128 && box_rows * 8 != 128) return false;  // one 128-byte swizzle span per column
    if (rows >= (int64_t(1) << 32) || cols >= (int64_t(1) << 32)) return false;
    cuuint64_t gdim[2] = {static_cast<cuuint64_t>(rows), static_cast<cuuint64_t>(cols)};
    cuuint64_t gstride[1] = {static_cast<cuuint64_t>(ld * 8)};
    cuuint32_t box[2] = {static_cast<cuuint32_t>(box_rows), static_cast<cuuint32_t>(box_cols)};
    cuuint32_t es[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<double *>(A), gdim, gstride, box,
              es, CU_TENSOR_MAP_INTERLEAVE_NONE,
              swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

TallPlan plan_rows(int64_t m, int bm, int ctas_per_sm, int ytiles) {
    TallPlan p;
    p.bm = bm;
    p.ncb = 0;
    const int64_t tiles = ceil_div(m, bm);
    int64_t want = std::max<int64_t>(1, int64_t(grid_sms()) * ctas_per_sm / std::max(1, ytiles));
    want = std::min<int64_t>(want, tiles);
    const int64_t tiles_per = ceil_div(tiles, want);
    p.chunk = tiles_per * bm;
    p.grid_x = static_cast<int>(ceil_div(m, p.chunk));
    if (p.grid_x < 1) p.grid_x = 1;
    return p;
}

// ------------------------------------------------------------- tiles ---

// Stage rows [r0, r0+BM) x columns [c0, c0+ncb) of A into T[c*BM + i]
// (zero outside the matrix).  TMA path: thread 0 issues one box; everyone
// waits on the mbarrier.  Returns false on a wait timeout.
template <int BM>
__device__ __forceinline__ bool stage_tile(double *T, const CUtensorMap *map, bool use_tma,
                                           uint64_t *bar, uint32_t &phase, const double *A,
                                           int64_t lda, int64_t m, int ncols, int64_t r0, int c0,
                                           int ncb) {
    if (use_tma) {
        if (threadIdx.x == 0) {
            mbar_arrive_expect_tx(bar, static_cast<uint32_t>(BM * ncb * 8));
            tma_load_2d(T, map, bar, static_cast<int32_t>(r0), c0);
        }
        const bool ok = mbar_wait_bounded(bar, phase);
        phase ^= 1u;
        return ok;
    }
    for (int idx = threadIdx.x; idx < BM * ncb; idx += blockDim.x) {
        const int i = idx % BM, c = idx / BM;
        const int64_t r = r0 + i;
        const int cc = c0 + c;
        T[idx] = (r < m && cc < ncols) ? A[r + int64_t(cc) * lda] : 0.0;
    }
    __syncthreads();
    return true;
}

// Replace the staged entries of a unit-lower trapezoidal factor M: ones on
// the diagonal, zeros above it (rows < ncols only).  Ends with a barrier.
template <int BM>
__device__ __forceinline__ void mask_unit_lower(double *T, int64_t r0, int c0, int ncb, int ncols) {
    if (r0 < ncols) {
        for (int idx = threadIdx.x; idx < BM * ncb; idx += blockDim.x) {
            const int i = idx % BM, c = idx / BM;
            const int64_t r = r0 + i;
            const int cc = c0 + c;
            if (cc < ncols && r <= cc) T[idx] = (r == cc) ? 1.0 : 0.0;
        }
    }
    __syncthreads();
}

// Before the next TMA overwrites a tile that threads wrote or read through
// the generic proxy: order those accesses before the async-proxy write.
__device__ __forceinline__ void tile_release() {
    fence_proxy_async_smem();
    __syncthreads();
}

// Shared abort flag: a thread whose bounded wait timed out sets it; all
// threads test it after the next barrier and leave together.
__device__ __forceinline__ bool check_abort(int *abort_flag, bool ok, DevStatus *st, int step) {
    if (!ok) {
        *abort_flag = 1;
        report(st, kErrTimeout, step, -1);
    }
    __syncthreads();
    return *abort_flag != 0;
}

// --------------------------------------------------- Gram accumulation ---

// Warp tiles of a 16-aligned output block (rows jn = 16*ntj, cols 16*ntk).
// Lane (a, b) = (lane / 4, lane % 4) of a full tile owns rows 2a, 2a+1 and
// cols 4b..4b+3.  In a diagonal block (diag) warp w < ntj owns the diagonal
// tile (w, w) and the tiles (a, b) with a < b go round-robin to warps
// (t + ntj) mod 8; otherwise all ntj x ntk tiles go to warps t mod 8.
// Coordinates (a, b) of the t-th of those tiles in row-major order (strict
// upper triangle when diag).  False if t is past the last tile.
__device__ __forceinline__ bool warp_tile_coords(int t, int ntj, int ntk, bool diag, int &a,
                                                 int &b) {
    a = 0;
    b = 0;
    int cnt = 0;
    for (int aa = 0; aa < ntj; ++aa) {
        const int len = diag ? (ntk - aa - 1) : ntk;
        if (len > 0 && t < cnt + len) {
            a = aa;
            b = (diag ? aa + 1 : 0) + (t - cnt);
            return true;
        }
        cnt += max(len, 0);
    }
    return false;
}

// A diagonal warp tile needs only its upper triangle: its 136 entries
// (r <= c, row-major) go to lane e % 32, slot e / 32, i.e. five FMAs per row
// instead of the eight of a full tile (lanes 8..31 idle in slot 4).  Each
// entry still sums its rows in order, so the values are those of a full tile.
constexpr int kDiagSlots = 5;

// NOFF full (off-diagonal) tiles per warp; DIAG: the block is a diagonal
// block and warps w < ntj also own the diagonal tile (w, w).
template <int NOFF, bool DIAG>
struct GramAcc {
    double acc[NOFF][8];
    double dacc[DIAG ? kDiagSlots : 1];
    int tj[NOFF], tk[NOFF];
    int drc[DIAG ? kDiagSlots : 1];  // this lane's diagonal-tile entry per slot: (r << 4) | c, or -1
    int nw;
    int dtile;  // the warp's diagonal tile, or -1

    __device__ __forceinline__ void init(int ntj, int ntk) {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const int shift = DIAG ? ntj : 0;
        nw = 0;
#pragma unroll
        for (int w = 0; w < NOFF; ++w) {
            int a, b;
            // tiles t with (t + shift) mod 8 == warp
            const int t = ((warp - shift) % 8 + 8) % 8 + 8 * w;
            if (warp_tile_coords(t, ntj, ntk, DIAG, a, b)) nw = w + 1;
            tj[w] = a;
            tk[w] = b;
        }
        dtile = (DIAG && warp < ntj) ? warp : -1;
#pragma unroll
        for (int q = 0; q < (DIAG ? kDiagSlots : 1); ++q) {
            int e = lane + 32 * q, r = 0;
            drc[q] = -1;
            if (DIAG && e < 136) {
                while (e >= 16 - r) {
                    e -= 16 - r;
                    ++r;
                }
                drc[q] = (r << 4) | (r + e);
            }
            dacc[q] = 0.0;
        }
#pragma unroll
        for (int w = 0; w < NOFF; ++w)
#pragma unroll
            for (int e = 0; e < 8; ++e) acc[w][e] = 0.0;
    }

    // Accumulate rows [0, rows) of the staged tiles TJ (column block of j)
    // and TK (column block of k), both laid out [col][BM].
    template <int BM>
    __device__ __forceinline__ void accumulate(const double *TJ, const double *TK, int rows) {
        const int lane = threadIdx.x & 31;
        const int a = lane >> 2, b = lane & 3;
        for (int i = 0; i < rows; ++i) {
            if (DIAG && dtile >= 0) {
#pragma unroll
                for (int q = 0; q < (DIAG ? kDiagSlots : 1); ++q) {
                    if (drc[q] >= 0) {
                        const double x = TJ[(dtile * 16 + (drc[q] >> 4)) * BM + i];
                        const double y = TK[(dtile * 16 + (drc[q] & 15)) * BM + i];
                        dacc[q] = fma(x, y, dacc[q]);
                    }
                }
            }
#pragma unroll
            for (int w = 0; w < NOFF; ++w) {
                if (w < nw) {
                    const double *pj = TJ + (tj[w] * 16 + 2 * a) * BM + i;
                    const double *pk = TK + (tk[w] * 16 + 4 * b) * BM + i;
                    const double x0 = pj[0], x1 = pj[BM];
                    const double y0 = pk[0], y1 = pk[BM], y2 = pk[2 * BM], y3 = pk[3 * BM];
                    acc[w][0] = fma(x0, y0, acc[w][0]);
                    acc[w][1] = fma(x0, y1, acc[w][1]);
                    acc[w][2] = fma(x0, y2, acc[w][2]);
                    acc[w][3] = fma(x0, y3, acc[w][3]);
                    acc[w][4] = fma(x1, y0, acc[w][4]);
                    acc[w][5] = fma(x1, y1, acc[w][5]);
                    acc[w][6] = fma(x1, y2, acc[w][6]);
                    acc[w][7] = fma(x1, y3, acc[w][7]);
                }
            }
        }
    }

    // Store the block partial (128 x 128 column-major slot) to part; a
    // diagonal tile stores its upper triangle (the reduction reads j <= k).
    __device__ __forceinline__ void store(double *part) const {
        const int lane = threadIdx.x & 31;
        const int a = lane >> 2, b = lane & 3;
        if (DIAG && dtile >= 0) {
#pragma unroll
            for (int q = 0; q < (DIAG ? kDiagSlots : 1); ++q) {
                if (drc[q] >= 0) {
                    const int j = dtile * 16 + (drc[q] >> 4);
                    const int k = dtile * 16 + (drc[q] & 15);
                    part[k * 128 + j] = dacc[q];
                }
            }
        }
#pragma unroll
        for (int w = 0; w < NOFF; ++w) {
            if (w < nw) {
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int j = tj[w] * 16 + 2 * a + (e >> 2);
                    const int k = tk[w] * 16 + 4 * b + (e & 3);
                    part[k * 128 + j] = acc[w][e];
                }
            }
        }
    }
};

// Gram partials.  blockIdx.y selects the output block: with diag != 0 the
// diagonal block (y, y); otherwise the off-diagonal block (0, 1) (n <= 256).
template <int BM, int MAXW>
__global__ void __launch_bounds__(kThreads, (MAXW > 5 ? 1 : 2))
    k_gram(const __grid_constant__ CUtensorMap map, int use_tma, const double *__restrict__ A,
           int64_t lda, int64_t m, int n, int unit_lower, int64_t chunk, int ncb, int diag,
           double *__restrict__ part, int nslots, DevStatus *st) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    double *T0 = reinterpret_cast<double *>(smem_raw);
    __shared__ __align__(8) uint64_t bar;
    __shared__ int abort_flag;
    const int bj = diag ? blockIdx.y : 0;
    const int bk = diag ? blockIdx.y : 1;
    double *T1 = diag ? T0 : T0 + BM * ncb;
    const int nj = std::min(ncb, pad16(n - bj * 128));
    const int nk = std::min(ncb, pad16(n - bk * 128));
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        abort_flag = 0;
        if (use_tma) prefetch_tensormap(&map);
    }
    __syncthreads();
    // MAXW warp tiles per warp: <BM, 5> serves diagonal blocks (one diagonal
    // tile and up to four full tiles per warp), <32, 8> the off-diagonal
    // block (eight full tiles per warp)
    constexpr bool kDiagBlock = MAXW <= 5;
    GramAcc<kDiagBlock ? MAXW - 1 : MAXW, kDiagBlock> g;
    g.init(nj / 16, nk / 16);
    uint32_t phase = 0;
    const int64_t rb = int64_t(blockIdx.x) * chunk;
    const int64_t re = std::min<int64_t>(m, rb + chunk);
    for (int64_t r0 = rb; r0 < re; r0 += BM) {
        bool ok;
        if (diag) {
            ok = stage_tile<BM>(T0, &map, use_tma, &bar, phase, A, lda, m, n, r0, bj * 128, ncb);
        } else {
            // two column slices waited on one barrier phase
            if (use_tma) {
                if (threadIdx.x == 0) {
                    mbar_arrive_expect_tx(&bar, static_cast<uint32_t>(2 * BM * ncb * 8));
                    tma_load_2d(T0, &map, &bar, static_cast<int32_t>(r0), 0);
                    tma_load_2d(T1, &map, &bar, static_cast<int32_t>(r0), 128);
                }
                ok = mbar_wait_bounded(&bar, phase);
                phase ^= 1u;
            } else {
                stage_tile<BM>(T0, &map, false, &bar, phase, A, lda, m, n, r0, 0, ncb);
                ok = stage_tile<BM>(T1, &map, false, &bar, phase, A, lda, m, n, r0, 128, ncb);
            }
        }
        if (check_abort(&abort_flag, ok, st, 0)) return;
        if (unit_lower) {
            mask_unit_lower<BM>(T0, r0, bj * 128, ncb, n);
            if (!diag) mask_unit_lower<BM>(T1, r0, 128, ncb, n);
        }
        const int rows = static_cast<int>(std::min<int64_t>(BM, re - r0));
        g.template accumulate<BM>(T0, T1, rows);
        tile_release();
    }
    g.store(part + (size_t(blockIdx.x) * nslots + blockIdx.y) * 16384);
}

// G[j][k] = G[k][j] = sum over CTAs (in CTA order) of the slot partials.
__global__ void k_reduce_gram(const double *__restrict__ part_diag, int nslots_diag,
                              int nparts_diag, const double *__restrict__ part_off,
                              int nparts_off, int n, double *__restrict__ G, int64_t ldg) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= int64_t(n) * n) return;
    const int j = static_cast<int>(e % n), k = static_cast<int>(e / n);
    if (j > k) return;
    const int bj = j / 128, bk = k / 128;
    const double *base;
    size_t stride;
    int nparts;
    if (bj == bk) {
        base = part_diag + size_t(bj) * 16384;
        stride = size_t(nslots_diag) * 16384;
        nparts = nparts_diag;
    } else {
        base = part_off;
        stride = 16384;
        nparts = nparts_off;
    }
    const int off = (k % 128) * 128 + (j % 128);
    const double s = ordered_sum(base + off, stride, nparts);
    G[j + int64_t(k) * ldg] = s;
    G[k + int64_t(j) * ldg] = s;
}

size_t gram_partials_doubles(int64_t m, int n) {
    // upper bound: grid_x <= 2 * SMs for the widest launch, 2 diagonal slots
    // plus one off-diagonal slot of 128 x 128
    const size_t p = size_t(2) * num_sms() + 8;
    return p * 3 * 16384;
}

static int gram_bm(int n) {
    if (launch_policy().fine_tiles) return n <= 64 ? 64 : 32;
    return n <= 64 ? 128 : (n <= 128 ? 64 : 32);
}

cudaError_t launch_gram(const double *A, int64_t lda, int64_t m, int n, int unit_lower, double *G,
                        int64_t ldg, double *part, DevStatus *st, cudaStream_t stream) {
    const int ncb = n <= 128 ? pad16(n) : 128;
    const int nd = n <= 128 ? 1 : 2;
    CUtensorMap map;
    int bm = gram_bm(std::min(n, 128));
    if (n > 128) bm = 32;  // off-diagonal launches stage two 128-column slices
    const bool tma = make_tma_map(&map, A, m, n, lda, bm, ncb);
    if (!tma) memset(&map, 0, sizeof map);
    // diagonal blocks: two CTAs per SM over nd slots; the off-diagonal block
    // (n > 128, 8 warp tiles per warp) runs alone per SM: each launch gets its
    // own row partition so that both fill every SM
    const TallPlan pl = plan_rows(m, bm, 2, nd);
    const TallPlan po = plan_rows(m, bm, 1, 1);
    double *part_diag = part;
    double *part_off = part + size_t(pl.grid_x) * nd * 16384;
    const size_t smem1 = size_t(bm) * ncb * 8;
    cudaError_t e;
    dim3 grid(pl.grid_x, nd);
    if (bm == 128) {
        auto k = k_gram<128, 5>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem1));
        RQ_LAUNCH(KID_GRAM, stream, k<<<grid, kThreads, smem1, stream>>>(map, tma, A, lda, m, n, unit_lower, pl.chunk, ncb, 1,
                                              part_diag, nd, st));
    } else if (bm == 64) {
        auto k = k_gram<64, 5>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem1));
        RQ_LAUNCH(KID_GRAM, stream, k<<<grid, kThreads, smem1, stream>>>(map, tma, A, lda, m, n, unit_lower, pl.chunk, ncb, 1,
                                              part_diag, nd, st));
    } else {
        auto k = k_gram<32, 5>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem1));
        RQ_LAUNCH(KID_GRAM, stream, k<<<grid, kThreads, smem1, stream>>>(map, tma, A, lda, m, n, unit_lower, pl.chunk, ncb, 1,
                                              part_diag, nd, st));
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (n > 128) {
        auto k = k_gram<32, 8>;
        const size_t smem2 = size_t(2) * 32 * 128 * 8;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem2));
        RQ_LAUNCH(KID_GRAM, stream, k<<<dim3(po.grid_x, 1), kThreads, smem2, stream>>>(map, tma, A, lda, m, n, unit_lower,
                                                            po.chunk, 128, 0, part_off, 1, st));
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const int64_t ne = int64_t(n) * n;
    RQ_LAUNCH(KID_REDUCE, stream, k_reduce_gram<<<static_cast<unsigned>(ceil_div(ne, 256)), 256, 0, stream>>>(
        part_diag, nd, pl.grid_x, part_off, po.grid_x, n, G, ldg));
    return cudaGetLastError();
}

// G = A^T A for n <= 128 with at most max_parts CTAs, so that the partial
// sums fit a caller-supplied buffer of max_parts x 16384 doubles.  Same
// kernels as launch_gram; only the row partition differs.
cudaError_t launch_gram_bounded(const double *A, int64_t lda, int64_t m, int n, double *G,
                                int64_t ldg, double *part, int max_parts, DevStatus *st,
                                cudaStream_t stream) {
    if (n > 128 || max_parts < 1) return cudaErrorInvalidValue;
    const int ncb = pad16(n);
    // the default row tiles of launch_gram, chosen here without the per-thread
    // launch policy: only the two instantiations below exist for this helper
    const int bm = n <= 64 ? 128 : 64;
    CUtensorMap map;
    const bool tma = make_tma_map(&map, A, m, n, lda, bm, ncb);
    if (!tma) memset(&map, 0, sizeof map);
    TallPlan pl = plan_rows(m, bm, 2, 1);
    if (pl.grid_x > max_parts) {
        pl.chunk = round_up(ceil_div(m, max_parts), bm);
        pl.grid_x = static_cast<int>(ceil_div(m, pl.chunk));
    }
    const size_t smem = size_t(bm) * ncb * 8;
    const dim3 grid(pl.grid_x, 1);
    if (bm == 128) {
        auto k = k_gram<128, 5>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        RQ_LAUNCH(KID_GRAM, stream, k<<<grid, kThreads, smem, stream>>>(map, tma, A, lda, m, n, 0,
                                                                       pl.chunk, ncb, 1, part, 1, st));
    } else {
        auto k = k_gram<64, 5>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        RQ_LAUNCH(KID_GRAM, stream, k<<<grid, kThreads, smem, stream>>>(map, tma, A, lda, m, n, 0,
                                                                       pl.chunk, ncb, 1, part, 1, st));
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t ne = int64_t(n) * n;
    RQ_LAUNCH(KID_REDUCE, stream,
              k_reduce_gram<<<static_cast<unsigned>(ceil_div(ne, 256)), 256, 0, stream>>>(
                  part, 1, pl.grid_x, part, pl.grid_x, n, G, ldg));
    return cudaGetLastError();
}

// ------------------------------------------------------- TRSM (+ Gram) ---

// Q = A R^{-1} tile by tile: blocked substitution with 16-column blocks.
// Each row of the tile belongs to P = 256 / BM adjacent lanes of one warp;
// lane p holds columns j0 + p + cP (c < CPT = 16 / P) of the current block
// in registers.  Update: a_ij -= sum_{k < j0} q_ik r_kj in increasing k (q_ik
// from shared memory, row k of R from its row-major copy).  Diagonal block,
// column t = 0..15 in turn: its owner scales it by 1 / r_jj, a shuffle
// broadcasts it and the row's later columns subtract q_ij r_jc.  Every
// column thus sees the same subtractions in the same order as the column
// formula q_ij = (a_ij - sum_{k<j} q_ik r_kj) / r_jj, and no barrier is
// needed inside the tile: a row's values only move within its warp.
// Interleaved columns retire early from the diagonal steps, so few of the
// predicated updates issue for nothing.  Optional fused Gram of the solved
// tile (n_pad <= 128).
template <int BM, bool kGram>
__global__ void __launch_bounds__(kThreads, 2)
    k_trsm(const __grid_constant__ CUtensorMap map, int use_tma, const double *__restrict__ A,
           int64_t lda, int64_t m, int n, int n_pad, int64_t chunk, const double *__restrict__ RT,
           const double *__restrict__ rinv, double *Q, int64_t ldq, double *__restrict__ part,
           DevStatus *st) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    double *T = reinterpret_cast<double *>(smem_raw);
    __shared__ __align__(8) uint64_t bar;
    __shared__ int abort_flag;
    constexpr int P = kThreads / BM;  // lanes per row
    constexpr int CPT = 16 / P;       // block columns per lane
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        abort_flag = 0;
        if (use_tma) prefetch_tensormap(&map);
    }
    __syncthreads();
    GramAcc<kGram ? (BM == 128 ? 1 : 4) : 1, kGram> g;
    if (kGram) g.init(n_pad / 16, n_pad / 16);
    uint32_t phase = 0;
    const int tid = threadIdx.x;
    const int p = tid % P, ti = tid / P;
    const int src0 = (tid & 31) - p;  // lane of this row's p = 0
    const int64_t rb = int64_t(blockIdx.x) * chunk;
    const int64_t re = std::min<int64_t>(m, rb + chunk);
    const int nblk = n_pad / 16;
    for (int64_t r0 = rb; r0 < re; r0 += BM) {
        const bool ok = stage_tile<BM>(T, &map, use_tma, &bar, phase, A, lda, m, n, r0, 0, n_pad);
        if (check_abort(&abort_flag, ok, st, 0)) return;
        for (int J = 0; J < nblk; ++J) {
            const int cb = 16 * J + p;  // column of c = 0
            double acc[CPT];
#pragma unroll
            for (int c = 0; c < CPT; ++c) acc[c] = T[(cb + c * P) * BM + ti];
            const double *rrow = RT + cb;
            for (int k = 0; k < 16 * J; ++k) {
                const double q = T[k * BM + ti];
                const double *rk = rrow + int64_t(k) * n_pad;
#pragma unroll
                for (int c = 0; c < CPT; ++c) acc[c] = fma(-q, __ldg(rk + c * P), acc[c]);
            }
#pragma unroll
            for (int t = 0; t < 16; ++t) {
                const int owner = t % P, lc = t / P;
                if (p == owner) acc[lc] *= __ldg(rinv + 16 * J + t);
                const double q = __shfl_sync(0xffffffffu, acc[lc], src0 + owner);
                const double *rk = RT + int64_t(16 * J + t) * n_pad + cb;
#pragma unroll
                for (int c = 0; c < CPT; ++c) {
                    if ((P - 1) + c * P <= t) continue;  // no lane has a column past t
                    if (p + c * P > t) acc[c] = fma(-q, __ldg(rk + c * P), acc[c]);
                }
            }
#pragma unroll
            for (int c = 0; c < CPT; ++c) T[(cb + c * P) * BM + ti] = acc[c];
            __syncwarp();
        }
        __syncthreads();
        const int rows = static_cast<int>(std::min<int64_t>(BM, re - r0));
        for (int idx = tid; idx < BM * n; idx += kThreads) {
            const int i = idx % BM, c = idx / BM;
            if (i < rows) Q[(r0 + i) + int64_t(c) * ldq] = T[c * BM + i];
        }
        if (kGram) g.template accumulate<BM>(T, T, rows);
        tile_release();
    }
    if (kGram) g.store(part + size_t(blockIdx.x) * 16384);
}

// (fine tiles: 64 rows for n <= 64; the fused Gram needs 64 or 128 rows, so
// wider matrices keep their tile)
static int trsm_bm(int n_pad) {
    if (launch_policy().fine_tiles && n_pad <= 64) return 64;
    return n_pad <= 64 ? 128 : (n_pad <= 128 ? 64 : 32);
}

cudaError_t launch_trsm_gram(const double *A, int64_t lda, int64_t m, int n, const double *RP,
                             const double *rinv, double *Q, int64_t ldq, double *G, int64_t ldg,
                             double *part, DevStatus *st, cudaStream_t stream) {
    const int n_pad = pad16(n);
    const int bm = trsm_bm(n_pad);
    const bool fuse = (G != nullptr) && n_pad <= 128;
    const double *RT = RP + size_t(n_pad) * n_pad;
    CUtensorMap map;
    const bool tma = make_tma_map(&map, A, m, n, lda, bm, n_pad);
    if (!tma) memset(&map, 0, sizeof map);
    const TallPlan pl = plan_rows(m, bm, 2, 1);
    const size_t smem = size_t(bm) * n_pad * 8;
    cudaError_t e;
#define RQ_TRSM_LAUNCH(BMV, GV)                                                                  \
    do {                                                                                         \
        auto k = k_trsm<BMV, GV>;                                                                \
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));         \
        RQ_LAUNCH(GV ? KID_TRSM_GRAM : KID_TRSM, stream,                                         \
                  k<<<pl.grid_x, kThreads, smem, stream>>>(map, tma, A, lda, m, n, n_pad,        \
                                                            pl.chunk, RT, rinv, Q, ldq, part, st)); \
    } while (0)
    if (bm == 128) {
        if (fuse) RQ_TRSM_LAUNCH(128, true); else RQ_TRSM_LAUNCH(128, false);
    } else if (bm == 64) {
        if (fuse) RQ_TRSM_LAUNCH(64, true); else RQ_TRSM_LAUNCH(64, false);
    } else {
        RQ_TRSM_LAUNCH(32, false);
    }
#undef RQ_TRSM_LAUNCH
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (G == nullptr) return cudaSuccess;
    if (fuse) {
        const int64_t ne = int64_t(n) * n;
        RQ_LAUNCH(KID_REDUCE, stream, k_reduce_gram<<<static_cast<unsigned>(ceil_div(ne, 256)), 256, 0, stream>>>(
            part, 1, pl.grid_x, part, pl.grid_x, n, G, ldg));
        return cudaGetLastError();
    }
    // n > 128: Gram of the solved Q in a separate pass
    return launch_gram(Q, ldq, m, n, 0, G, ldg, part, st, stream);
}

// --------------------------------------------------------------- sketch ---

// Y partials for an output tile of 64 sketch rows x NT columns.  S entries
// for the tile's rows are generated on the fly (Gaussian, scaled 1/sqrt(s))
// or read from an explicit S.  Per row of X the tile's 64 x NT outer
// product is accumulated in warp tiles (lane (a, b): sketch rows 2a, 2a+1,
// columns 4b..4b+3).
template <int BM>
__global__ void __launch_bounds__(kThreads, 2)
    k_sketch_gauss(const __grid_constant__ CUtensorMap map, int use_tma,
                   const double *__restrict__ A, int64_t lda, int64_t m, int n, int unit_lower,
                   int64_t chunk, int ncb, int n_st, int64_t s, uint64_t seed, double scale,
                   const double *__restrict__ S, int64_t lds, double *__restrict__ part, int s_pad,
                   int n_pad, DevStatus *st, int64_t row0) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    double *T = reinterpret_cast<double *>(smem_raw);
    double *Sg = T + BM * ncb;  // [i][64]
    __shared__ __align__(8) uint64_t bar;
    __shared__ int abort_flag;
    const int st_idx = blockIdx.y % n_st, ct_idx = blockIdx.y / n_st;
    const int rt0 = 64 * st_idx, c0 = 128 * ct_idx;
    const int nt = std::min(ncb, pad16(n - c0));
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        abort_flag = 0;
        if (use_tma) prefetch_tensormap(&map);
    }
    __syncthreads();
    // warp tiles of the 64 x nt output: 4 x (nt/16), warp w takes w, w+8, ...
    double acc[4][8];
    int wr[4], wc[4];
    int nw = 0;
    {
        const int warp = threadIdx.x >> 5;
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            int a, b;
            if (warp_tile_coords(warp + 8 * w, 4, nt / 16, false, a, b)) nw = w + 1;
            wr[w] = a;
            wc[w] = b;
        }
#pragma unroll
        for (int w = 0; w < 4; ++w)
#pragma unroll
            for (int e = 0; e < 8; ++e) acc[w][e] = 0.0;
    }
    const int lane = threadIdx.x & 31, la = lane >> 2, lb = lane & 3;
    uint32_t phase = 0;
    const int64_t rb = int64_t(blockIdx.x) * chunk;
    const int64_t re = std::min<int64_t>(m, rb + chunk);
    for (int64_t r0 = rb; r0 < re; r0 += BM) {
        if (use_tma && threadIdx.x == 0) {
            mbar_arrive_expect_tx(&bar, static_cast<uint32_t>(BM * ncb * 8));
            tma_load_2d(T, &map, &bar, static_cast<int32_t>(r0), c0);
        }
        // sketch entries for rows r0 .. r0+BM-1 (overlaps the TMA)
        if (S == nullptr) {
            for (int idx = threadIdx.x; idx < BM * 16; idx += kThreads) {
                const int i = idx >> 4, q = idx & 15;
                const int64_t row = r0 + i;
                double *dst = Sg + i * 64 + 4 * q;
                if (row < m) {
                    const float4 z = sk_gauss4(seed, row0 + row, (rt0 >> 2) + q);
                    dst[0] = double(z.x) * scale;
                    dst[1] = double(z.y) * scale;
                    dst[2] = double(z.z) * scale;
                    dst[3] = double(z.w) * scale;
                } else {
                    dst[0] = dst[1] = dst[2] = dst[3] = 0.0;
                }
            }
        } else {
            for (int idx = threadIdx.x; idx < BM * 64; idx += kThreads) {
                const int r = idx & 63, i = idx >> 6;
                const int64_t row = r0 + i;
                const int64_t rg = rt0 + r;
                Sg[i * 64 + r] = (row < m && rg < s) ? S[rg + row * lds] : 0.0;
            }
        }
        bool ok = true;
        if (use_tma) {
            ok = mbar_wait_bounded(&bar, phase);
            phase ^= 1u;
        } else {
            stage_tile<BM>(T, &map, false, &bar, phase, A, lda, m, n, r0, c0, ncb);
        }
        if (check_abort(&abort_flag, ok, st, 0)) return;
        if (unit_lower) mask_unit_lower<BM>(T, r0, c0, ncb, n);
        const int rows = static_cast<int>(std::min<int64_t>(BM, re - r0));
        for (int i = 0; i < rows; ++i) {
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                if (w < nw) {
                    const double *ps = Sg + i * 64 + wr[w] * 16 + 2 * la;
                    const double *px = T + (wc[w] * 16 + 4 * lb) * BM + i;
                    const double s0 = ps[0], s1 = ps[1];
                    const double x0 = px[0], x1 = px[BM], x2 = px[2 * BM], x3 = px[3 * BM];
                    acc[w][0] = fma(s0, x0, acc[w][0]);
                    acc[w][1] = fma(s0, x1, acc[w][1]);
                    acc[w][2] = fma(s0, x2, acc[w][2]);
                    acc[w][3] = fma(s0, x3, acc[w][3]);
                    acc[w][4] = fma(s1, x0, acc[w][4]);
                    acc[w][5] = fma(s1, x1, acc[w][5]);
                    acc[w][6] = fma(s1, x2, acc[w][6]);
                    acc[w][7] = fma(s1, x3, acc[w][7]);
                }
            }
        }
        tile_release();
    }
    double *out = part + size_t(blockIdx.x) * s_pad * n_pad;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        if (w < nw) {
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int r = rt0 + wr[w] * 16 + 2 * la + (e >> 2);
                const int c = c0 + wc[w] * 16 + 4 * lb + (e & 3);
                if (r < s_pad && c < n_pad) out[size_t(c) * s_pad + r] = acc[w][e];
            }
        }
    }
}

// Sparse-sign sketch partials.  Each CTA keeps the s_pad x 32 block of Y for
// its column slice in shared memory; warp w owns the Y rows r with
// r mod 8 == w (lane = column), so each entry has one writer and sums in
// increasing row order of X (deterministic, no atomics).  The +-1 entries
// are added exactly; the 1/sqrt(zeta) scale is applied once at the end.
constexpr int kSparseBM = 64;
constexpr int kSparseNT = 32;

__global__ void __launch_bounds__(kThreads, 2)
    k_sketch_sparse(const double *__restrict__ A, int64_t lda, int64_t m, int n, int unit_lower,
                    int64_t chunk, int s, int zeta, uint64_t seed, double scale,
                    double *__restrict__ part, int s_pad, int n_pad, int64_t row0) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    double *acc = reinterpret_cast<double *>(smem_raw);                    // [s_pad][32]
    double *T2 = acc + size_t(s_pad) * kSparseNT;                          // [BM][33]
    int *tgt = reinterpret_cast<int *>(T2 + kSparseBM * (kSparseNT + 1));  // [BM][zeta]
    const int c0 = blockIdx.y * kSparseNT;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int idx = threadIdx.x; idx < s_pad * kSparseNT; idx += kThreads) acc[idx] = 0.0;
    const int64_t rb = int64_t(blockIdx.x) * chunk;
    const int64_t re = std::min<int64_t>(m, rb + chunk);
    for (int64_t r0 = rb; r0 < re; r0 += kSparseBM) {
        for (int idx = threadIdx.x; idx < kSparseBM * kSparseNT; idx += kThreads) {
            const int i = idx % kSparseBM, c = idx / kSparseBM;
            const int64_t r = r0 + i;
            const int cc = c0 + c;
            double v = (r < m && cc < n) ? A[r + int64_t(cc) * lda] : 0.0;
            if (unit_lower && cc < n && r <= cc) v = (r == cc) ? 1.0 : 0.0;
            T2[i * (kSparseNT + 1) + c] = v;
        }
        if (threadIdx.x < kSparseBM) {
            const int64_t row = r0 + threadIdx.x;
            int rows_[16], sg[16];
            if (row < m) {
                sk_sparse_column(seed, row0 + row, s, zeta, rows_, sg);
                // target row (bits 0..15), this block row (bits 16..23), sign (bit 31)
                for (int t = 0; t < zeta; ++t)
                    tgt[threadIdx.x * zeta + t] =
                        rows_[t] | (threadIdx.x << 16) | (sg[t] < 0 ? int(0x80000000u) : 0);
            } else {
                for (int t = 0; t < zeta; ++t) tgt[threadIdx.x * zeta + t] = -1;
            }
        }
        __syncthreads();
        // warp w owns the accumulator rows r = w (mod 8).  The warp scans the
        // block's (row, t) entries 32 at a time, a ballot picks its own, and
        // they are added in increasing (row, t) order: the order of a plain
        // loop over rows and nonzeros, so every sum is reproducible.
        const int rows = static_cast<int>(std::min<int64_t>(kSparseBM, re - r0));
        const int total = rows * zeta;
        for (int base = 0; base < total; base += 32) {
            const int e = base + lane < total ? tgt[base + lane] : 0;
            unsigned mine = __ballot_sync(0xffffffffu, base + lane < total && (e & 7) == warp);
            while (mine) {
                const int src = __ffs(mine) - 1;
                mine &= mine - 1;
                const int ee = __shfl_sync(0xffffffffu, e, src);
                const double x = T2[((ee >> 16) & 0xff) * (kSparseNT + 1) + lane];
                // +-x by the sign bit, one binary64 add
                const unsigned long long sbit =
                    static_cast<unsigned long long>(static_cast<uint32_t>(ee) & 0x80000000u) << 32;
                const double xs = __longlong_as_double(static_cast<long long>(
                    static_cast<unsigned long long>(__double_as_longlong(x)) ^ sbit));
                double *p = acc + (ee & 0xffff) * kSparseNT + lane;
                *p += xs;
            }
        }
        __syncthreads();
    }
    double *out = part + size_t(blockIdx.x) * s_pad * n_pad;
    for (int idx = threadIdx.x; idx < s_pad * kSparseNT; idx += kThreads) {
        const int r = idx / kSparseNT, c = idx % kSparseNT;
        if (c0 + c < n_pad) out[size_t(c0 + c) * s_pad + r] = acc[idx] * scale;
    }
}

// Y[r][c] = sum over CTAs (in CTA order) of the partials.
__global__ void k_reduce_sketch(const double *__restrict__ part, int nparts, int s, int n,
                                int s_pad, int n_pad, double *__restrict__ Y, int64_t ldy) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= int64_t(s) * n) return;
    const int r = static_cast<int>(e % s), c = static_cast<int>(e / s);
    const size_t off = size_t(c) * s_pad + r;
    const size_t stride = size_t(s_pad) * n_pad;
    Y[r + int64_t(c) * ldy] = ordered_sum(part + off, stride, nparts);
}

cudaError_t launch_reduce_sketch(const double *part, int nparts, int s, int n, int s_pad, int n_pad,
                                 double *Y, int64_t ldy, cudaStream_t stream) {
    const int64_t ne = int64_t(s) * n;
    RQ_LAUNCH(KID_REDUCE, stream,
              k_reduce_sketch<<<static_cast<unsigned>(ceil_div(ne, 256)), 256, 0, stream>>>(
                  part, nparts, s, n, s_pad, n_pad, Y, ldy));
    return cudaGetLastError();
}

size_t sketch_partials_doubles(int64_t m, int n, int64_t s, int kind) {
    const size_t s_pad = size_t(round_up(s, 64)), n_pad = size_t(round_up(n, 32));
    const size_t p = size_t(2) * num_sms() + 8;
    (void)m;
    (void)kind;
    return p * s_pad * n_pad;
}

cudaError_t launch_sketch(const double *A, int64_t lda, int64_t m, int n, int unit_lower, int kind,
                          int64_t s, int zeta, uint64_t seed, const double *S, int64_t lds,
                          double *Y, int64_t ldy, double *part, DevStatus *st,
                          cudaStream_t stream, int64_t row0, int srht_b) {
    if (kind == 2 && S == nullptr)
        return launch_sketch_srht(A, lda, m, n, unit_lower, s, seed,
                                  srht_b > 0 ? srht_b : srht_order_log2(row0 + m), Y, ldy, part, stream,
                                  row0);
    const int s_pad = static_cast<int>(round_up(s, 64));
    const int n_pad = static_cast<int>(round_up(n, 32));
    cudaError_t e;
    int nparts;
    if (kind == 1 && S == nullptr) {
        const int ny = static_cast<int>(ceil_div(n, kSparseNT));
        const TallPlan pl = plan_rows(m, kSparseBM, 2, ny);
        const size_t smem = size_t(s_pad) * kSparseNT * 8 + size_t(kSparseBM) * (kSparseNT + 1) * 8 +
                            size_t(kSparseBM) * zeta * 4;
        cudaFuncSetAttribute(k_sketch_sparse, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        RQ_LAUNCH(KID_SKETCH_SPARSE, stream, k_sketch_sparse<<<dim3(pl.grid_x, ny), kThreads, smem, stream>>>(
            A, lda, m, n, unit_lower, pl.chunk, static_cast<int>(s), zeta, seed,
            1.0 / sqrt(double(zeta)), part, s_pad, n_pad, row0));
        nparts = pl.grid_x;
    } else {
        const int ncb = std::min(pad16(n), 128);
        const int bm = 64;
        const int n_st = s_pad / 64;
        const int n_ct = static_cast<int>(ceil_div(n, 128));
        CUtensorMap map;
        const bool tma = make_tma_map(&map, A, m, n, lda, bm, ncb);
        if (!tma) memset(&map, 0, sizeof map);
        const TallPlan pl = plan_rows(m, bm, 2, n_st * n_ct);
        const size_t smem = size_t(bm) * ncb * 8 + size_t(bm) * 64 * 8;
        auto k = k_sketch_gauss<64>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        RQ_LAUNCH(KID_SKETCH_GAUSS, stream, k<<<dim3(pl.grid_x, n_st * n_ct), kThreads, smem, stream>>>(
            map, tma, A, lda, m, n, unit_lower, pl.chunk, ncb, n_st, s, seed,
            1.0 / sqrt(double(s)), S, lds, part, s_pad, n_pad, st, row0));
        nparts = pl.grid_x;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int64_t ne = s * int64_t(n);
    RQ_LAUNCH(KID_REDUCE, stream, k_reduce_sketch<<<static_cast<unsigned>(ceil_div(ne, 256)), 256, 0, stream>>>(
        part, nparts, static_cast<int>(s), n, s_pad, n_pad, Y, ldy));
    return cudaGetLastError();
}

// RP = triu(R) zero-padded to n_pad x n_pad (ld n_pad), followed by its
// row-major copy; rinv = 1/diag (0 in padding).
__global__ void k_pad_upper(const double *__restrict__ R, int64_t ldr, int n, int n_pad,
                            double *__restrict__ RP, double *__restrict__ rinv) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= int64_t(n_pad) * n_pad) return;
    const int i = static_cast<int>(e % n_pad), j = static_cast<int>(e / n_pad);
    const double v = (i <= j && j < n) ? R[i + int64_t(j) * ldr] : 0.0;
    RP[e] = v;
    RP[int64_t(n_pad) * n_pad + int64_t(i) * n_pad + j] = v;
    if (i == j) rinv[i] = (i < n) ? 1.0 / v : 0.0;
}

cudaError_t launch_pad_upper(const double *R, int64_t ldr, int n, double *RP, double *rinv,
                             cudaStream_t stream) {
    const int n_pad = pad16(n);
    const int64_t ne = int64_t(n_pad) * n_pad;
    RQ_LAUNCH(KID_PAD, stream, k_pad_upper<<<static_cast<unsigned>(ceil_div(ne, 256)), 256, 0, stream>>>(R, ldr, n, n_pad, RP,
                                                                             rinv));
    return cudaGetLastError();
}

}  // namespace rq
