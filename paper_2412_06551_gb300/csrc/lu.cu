// Tall LU with partial pivoting of an m x n FP64 matrix, in place
// ([M, N, P] = LU(X) of Algorithms 4 and 7): PX = MN with the pivot of
// column k the first row of largest magnitude among rows >= k.
//
// Blocked right-looking schedule with panels of NB columns:
//   * column step k (one launch): l_ik = a_ik / u_kk for rows i > k, rank-1
//     update of the remaining panel columns, and the block-partial pivot
//     search of column k+1 on the freshly updated values;
//   * panel end: U12 = L11^{-1} A12 (one CTA), then the trailing update
//     A22 -= L21 U12 (all CTAs) fused with the pivot search of the next
//     panel's first column.
// The global pivot of each column is chosen by the last CTA to finish
// (atomic ticket, no waiting): it combines the per-CTA candidates, records
// ipiv, and swaps the two rows across all n columns before the next launch.
// Updates subtract in increasing elimination index, the order of the
// unblocked algorithm.  Selection is exact, so pivots are deterministic.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace rq {

constexpr int kLuThreads = 256;
constexpr int kLuNB = 8;

struct ArgCand {
    double v;     // |a|, -1 for "none"
    long long i;  // row index
};

__device__ __forceinline__ bool cand_better(double v1, long long i1, double v2, long long i2) {
    return v1 > v2 || (v1 == v2 && i1 < i2);
}

// Block-wide argmax of (v, i); result valid in thread 0.
__device__ __forceinline__ ArgCand block_argmax(double v, long long i) {
    __shared__ double sv[32];
    __shared__ long long si[32];
    for (int off = 16; off > 0; off >>= 1) {
        const double v2 = __shfl_down_sync(0xffffffffu, v, off);
        const long long i2 = __shfl_down_sync(0xffffffffu, i, off);
        if (cand_better(v2, i2, v, i)) {
            v = v2;
            i = i2;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        sv[warp] = v;
        si[warp] = i;
    }
    __syncthreads();
    ArgCand r{-1.0, 0x7fffffffffffffffll};
    if (threadIdx.x == 0) {
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
            if (cand_better(sv[w], si[w], r.v, r.i)) {
                r.v = sv[w];
                r.i = si[w];
            }
    }
    return r;
}

// Publish this CTA's candidate; the last CTA to arrive picks the pivot of
// column `col` (when col < n), records it, and swaps rows col <-> pivot.
__device__ __forceinline__ void finish_pivot(ArgCand mine, ArgCand *cands, unsigned *ticket,
                                             double *A, int64_t lda, int n, int col,
                                             int32_t *ipiv, DevStatus *st, int step) {
    __shared__ bool last;
    __shared__ long long piv_row;
    if (threadIdx.x == 0) {
        cands[blockIdx.x] = mine;
        __threadfence();
        const unsigned t = atomicAdd(ticket, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // all threads of the last CTA combine the candidates (L2 reads: other
    // CTAs wrote them in this launch)
    double cv = -1.0;
    long long ci = 0x7fffffffffffffffll;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
        const double v = __ldcg(&cands[b].v);
        const long long i = __ldcg(&cands[b].i);
        if (cand_better(v, i, cv, ci)) {
            cv = v;
            ci = i;
        }
    }
    const ArgCand best = block_argmax(cv, ci);
    if (threadIdx.x == 0) {
        long long p = best.i;
        if (!(best.v > 0.0)) {  // zero (or non-finite) column: rank < n
            report(st, best.v == 0.0 ? kErrLuZeroPivot : kErrNonfinite, step, col);
            p = col;
        }
        ipiv[col] = static_cast<int32_t>(p);
        piv_row = p;
        *ticket = 0u;
    }
    __syncthreads();
    const long long p = piv_row;
    if (p != col) {
        // L2 reads: the panel entries of both rows were written by other
        // CTAs in this launch
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            const double t = __ldcg(A + col + int64_t(j) * lda);
            A[col + int64_t(j) * lda] = __ldcg(A + p + int64_t(j) * lda);
            A[p + int64_t(j) * lda] = t;
        }
    }
}

// Column step k of the panel [.., pe): scale column k below the diagonal,
// update panel columns k+1 .. pe-1, and search the pivot of column k+1.
// Each thread takes kColRows rows at a time and loads all their panel
// entries before its first store, so that the loads of a row are in flight
// together instead of one memory round trip per column.
constexpr int kColRows = 4;

__global__ void __launch_bounds__(kLuThreads, 2)
    k_lu_col(double *A, int64_t lda, int64_t m, int n, int k, int pe, int64_t chunk,
             ArgCand *cands, unsigned *ticket, int32_t *ipiv, DevStatus *st, int step) {
    constexpr int NC = kLuNB - 1;
    __shared__ double urow[kLuNB];
    const int ncol = pe - k - 1;  // panel columns right of k
    if (threadIdx.x < ncol) urow[threadIdx.x] = A[k + int64_t(k + 1 + threadIdx.x) * lda];
    __syncthreads();
    const double rcp = 1.0 / A[k + int64_t(k) * lda];
    double u[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) u[c] = (c < ncol) ? urow[c] : 0.0;
    const bool search = (k + 1 < pe);
    double bv = -1.0;
    long long bi = 0x7fffffffffffffffll;
    const int64_t rb = k + 1 + int64_t(blockIdx.x) * chunk;
    const int64_t re = std::min<int64_t>(m, rb + chunk);
    double *colk = A + int64_t(k) * lda;
    double *col1 = A + int64_t(k + 1) * lda;
    for (int64_t i0 = rb + threadIdx.x; i0 < re; i0 += int64_t(kLuThreads) * kColRows) {
        double l[kColRows], a[kColRows][NC];
#pragma unroll
        for (int r = 0; r < kColRows; ++r) {
            const int64_t i = i0 + int64_t(r) * kLuThreads;
            const bool in = i < re;
            l[r] = in ? colk[i] : 0.0;
#pragma unroll
            for (int c = 0; c < NC; ++c) a[r][c] = (in && c < ncol) ? col1[i + int64_t(c) * lda] : 0.0;
        }
#pragma unroll
        for (int r = 0; r < kColRows; ++r) {
            const int64_t i = i0 + int64_t(r) * kLuThreads;
            if (i >= re) break;
            const double li = l[r] * rcp;
            colk[i] = li;
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                if (c >= ncol) break;
                const double v = fma(-li, u[c], a[r][c]);
                col1[i + int64_t(c) * lda] = v;
                if (c == 0 && cand_better(fabs(v), i, bv, bi)) {
                    bv = fabs(v);
                    bi = i;
                }
            }
        }
    }
    if (!search) return;
    __threadfence();  // this thread's updates before the CTA's ticket
    // the pivot of column k+1 may also be row k+1 itself: it is among rows >= k+1
    const ArgCand mine = block_argmax(bv, bi);
    finish_pivot(mine, cands, ticket, A, lda, n, k + 1, ipiv, st, step);
}

// U12 = L11^{-1} A12: rows k0 .. pe-1, columns pe .. n-1 (one CTA).
__global__ void __launch_bounds__(kLuThreads)
    k_lu_u12(double *A, int64_t lda, int n, int k0, int pe) {
    const int nb = pe - k0;
    for (int c = pe + threadIdx.x; c < n; c += blockDim.x) {
        double u[kLuNB];
        for (int t = 0; t < nb; ++t) {
            double a = A[k0 + t + int64_t(c) * lda];
            for (int q = 0; q < t; ++q) a = fma(-A[k0 + t + int64_t(k0 + q) * lda], u[q], a);
            u[t] = a;
            A[k0 + t + int64_t(c) * lda] = a;
        }
    }
}

// Trailing update A22 -= L21 U12 for rows >= pe, columns >= pe (in
// increasing elimination index), then the pivot search of column pe.
// With k0 == pe it only searches (the first column of the matrix).
__global__ void __launch_bounds__(kLuThreads)
    k_lu_trailing(double *A, int64_t lda, int64_t m, int n, int k0, int pe, int64_t chunk,
                  ArgCand *cands, unsigned *ticket, int32_t *ipiv, DevStatus *st, int step) {
    extern __shared__ double U[];  // [nb][n - pe]
    const int nb = pe - k0, nt = n - pe;
    for (int idx = threadIdx.x; idx < nb * nt; idx += blockDim.x) {
        const int t = idx % nb, c = idx / nb;
        U[t * nt + c] = A[k0 + t + int64_t(pe + c) * lda];
    }
    __syncthreads();
    double bv = -1.0;
    long long bi = 0x7fffffffffffffffll;
    const int64_t rb = pe + int64_t(blockIdx.x) * chunk;
    const int64_t re = std::min<int64_t>(m, rb + chunk);
    for (int64_t i = rb + threadIdx.x; i < re; i += kLuThreads) {
        double l[kLuNB];
        for (int t = 0; t < nb; ++t) l[t] = A[i + int64_t(k0 + t) * lda];
        for (int c = 0; c < nt; ++c) {
            double *p = A + i + int64_t(pe + c) * lda;
            double a = *p;
            for (int t = 0; t < nb; ++t) a = fma(-l[t], U[t * nt + c], a);
            *p = a;
            if (c == 0) {
                const double v = fabs(a);
                if (cand_better(v, i, bv, bi)) {
                    bv = v;
                    bi = i;
                }
            }
        }
    }
    __threadfence();  // this thread's updates before the CTA's ticket
    const ArgCand mine = block_argmax(bv, bi);
    finish_pivot(mine, cands, ticket, A, lda, n, pe, ipiv, st, step);
}

// CTAs per SM: the column step holds kColRows x kLuNB values per thread
// (two CTAs fit); the trailing update is latency-bound on its
// load-update-store chain per column and takes as many CTAs as fit.
constexpr int kColCtasPerSm = 2;
constexpr int kTrailCtasPerSm = 6;
constexpr int kMaxCtasPerSm = 6;

static size_t cand_slots() { return size_t(kMaxCtasPerSm) * num_sms() + 8; }

size_t lu_scratch_bytes(int64_t m, int n) {
    (void)m;
    (void)n;
    return cand_slots() * sizeof(ArgCand) + 256;
}

static int lu_grid(int64_t rows, int64_t &chunk, int per_sm) {
    const int64_t maxg = int64_t(per_sm) * grid_sms();
    int64_t g = std::max<int64_t>(1, std::min<int64_t>(maxg, ceil_div(rows, 2 * kLuThreads)));
    chunk = std::max<int64_t>(1, ceil_div(rows, g));
    g = std::max<int64_t>(1, ceil_div(rows, chunk));
    return static_cast<int>(g);
}

cudaError_t launch_tall_lupp(double *A, int64_t lda, int64_t m, int n, int32_t *ipiv,
                             void *scratch, DevStatus *st, int step_id, cudaStream_t stream) {
    ArgCand *cands = reinterpret_cast<ArgCand *>(scratch);
    unsigned *ticket =
        reinterpret_cast<unsigned *>(static_cast<char *>(scratch) + cand_slots() * sizeof(ArgCand));
    cudaError_t e = cudaMemsetAsync(ticket, 0, sizeof(unsigned), stream);
    if (e != cudaSuccess) return e;
    const size_t smax = size_t(kLuNB) * n * sizeof(double);
    cudaFuncSetAttribute(k_lu_trailing, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smax));
    int64_t chunk;
    int g = lu_grid(m, chunk, kTrailCtasPerSm);
    RQ_LAUNCH(KID_LU_TRAILING, stream, k_lu_trailing<<<g, kLuThreads, 0, stream>>>(A, lda, m, n, 0, 0, chunk, cands, ticket, ipiv, st,
                                                step_id));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    for (int k0 = 0; k0 < n; k0 += kLuNB) {
        const int pe = std::min(n, k0 + kLuNB);
        for (int k = k0; k < pe; ++k) {
            const int64_t rows = m - k - 1;
            if (rows <= 0) break;
            g = lu_grid(rows, chunk, kColCtasPerSm);
            RQ_LAUNCH(KID_LU_COL, stream, k_lu_col<<<g, kLuThreads, 0, stream>>>(A, lda, m, n, k, pe, chunk, cands, ticket, ipiv,
                                                   st, step_id));
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        if (pe < n) {
            RQ_LAUNCH(KID_LU_U12, stream, k_lu_u12<<<1, kLuThreads, 0, stream>>>(A, lda, n, k0, pe));
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            const int64_t rows = m - pe;
            g = lu_grid(rows, chunk, kTrailCtasPerSm);
            const size_t sm = size_t(pe - k0) * (n - pe) * sizeof(double);
            RQ_LAUNCH(KID_LU_TRAILING, stream, k_lu_trailing<<<g, kLuThreads, sm, stream>>>(A, lda, m, n, k0, pe, chunk, cands, ticket,
                                                         ipiv, st, step_id));
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

}  // namespace rq
