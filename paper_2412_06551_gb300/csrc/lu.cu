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
// ipiv, and swaps the two rows across all n columns.
// Updates subtract in increasing elimination index, the order of the
// unblocked algorithm.  Selection is exact, so pivots are deterministic.
//
// A panel's column steps run in one cooperative launch (k_lu_panel): after
// each pivot selection every CTA waits at a grid-wide barrier, so that the
// swapped rows are in place before the next column; the barrier's wait is
// bounded (the kernel reports a timeout and returns) and it reads rows that
// other CTAs may have swapped through L2.  Where a cooperative launch is not
// possible (stream capture, or the launch is refused) each column step is a
// launch of its own (k_lu_col) and the launch boundary is the barrier.
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

// Grid-wide barrier of a cooperative launch with a bounded wait.  Thread 0
// of each CTA reads the generation, arrives on `count`, and waits until the
// generation moves on; the last of `expected` arrivals resets `count` and
// advances the generation.  Every wait gives up after limit_ns of
// %globaltimer time; the return value (the same in all threads of the CTA)
// says whether the barrier completed.  With expected > gridDim.x the barrier
// cannot complete (fault injection for tests).
__device__ bool grid_barrier_bounded(unsigned *count, unsigned *gen, unsigned expected,
                                     uint64_t limit_ns) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        const unsigned g = atomicAdd(gen, 0u);
        __threadfence();  // this CTA's writes before its arrival
        if (atomicAdd(count, 1u) == expected - 1u) {
            atomicExch(count, 0u);
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            const uint64_t t0 = globaltimer_ns();
            for (uint32_t it = 1; atomicAdd(gen, 0u) == g; ++it) {
                __nanosleep(64);
                if ((it & 63u) == 0 && globaltimer_ns() - t0 > limit_ns) {
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// All column steps k0 .. pe-1 of one panel in a cooperative launch.  Column
// k's pivot row is in place on entry (for k0: the previous trailing update
// chose it; later columns: the previous iteration).  Per column every CTA
// scales column k below the diagonal in its rows, updates the panel's
// remaining columns and proposes its candidate for column k+1; the last CTA
// to take a ticket picks the pivot, records it and swaps the two rows across
// all n columns; then the grid waits at the bounded barrier.  Loads of A go
// through L2 (__ldcg): a swap by another CTA in this launch is not in this
// SM's L1.  `stall` makes the first barrier expect one arrival too many.
__global__ void __launch_bounds__(kLuThreads, 2)
    k_lu_panel(double *A, int64_t lda, int64_t m, int n, int k0, int pe, int64_t chunk,
               ArgCand *cands, unsigned *ticket, unsigned *bar_count, unsigned *bar_gen,
               int32_t *ipiv, DevStatus *st, int step, uint64_t limit_ns, int stall) {
    constexpr int NC = kLuNB - 1;
    __shared__ double urow[kLuNB];
    // after a failure earlier in this factorization (a timed-out barrier
    // leaves the barrier's counters behind) the remaining panels do nothing
    if (*reinterpret_cast<volatile int *>(&st->code) != 0) return;
    const int64_t rb = k0 + 1 + int64_t(blockIdx.x) * chunk;
    const int64_t re = std::min<int64_t>(m, rb + chunk);
    for (int k = k0; k < pe; ++k) {
        const int ncol = pe - k - 1;  // panel columns right of k
        if (threadIdx.x < ncol) urow[threadIdx.x] = __ldcg(A + k + int64_t(k + 1 + threadIdx.x) * lda);
        __syncthreads();
        const double rcp = 1.0 / __ldcg(A + k + int64_t(k) * lda);
        double u[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) u[c] = (c < ncol) ? urow[c] : 0.0;
        double bv = -1.0;
        long long bi = 0x7fffffffffffffffll;
        double *colk = A + int64_t(k) * lda;
        double *col1 = A + int64_t(k + 1) * lda;
        const int64_t r0 = std::max<int64_t>(rb, k + 1);
        for (int64_t i0 = r0 + threadIdx.x; i0 < re; i0 += int64_t(kLuThreads) * kColRows) {
            double l[kColRows], a[kColRows][NC];
#pragma unroll
            for (int r = 0; r < kColRows; ++r) {
                const int64_t i = i0 + int64_t(r) * kLuThreads;
                const bool in = i < re;
                l[r] = in ? __ldcg(colk + i) : 0.0;
#pragma unroll
                for (int c = 0; c < NC; ++c)
                    a[r][c] = (in && c < ncol) ? __ldcg(col1 + i + int64_t(c) * lda) : 0.0;
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
        if (k + 1 >= pe) break;  // the next panel's first pivot: the trailing update
        __threadfence();  // this thread's updates before the CTA's ticket
        const ArgCand mine = block_argmax(bv, bi);
        finish_pivot(mine, cands, ticket, A, lda, n, k + 1, ipiv, st, step);
        const unsigned expected = gridDim.x + ((stall && k == k0) ? 1u : 0u);
        if (!grid_barrier_bounded(bar_count, bar_gen, expected, limit_ns)) {
            if (threadIdx.x == 0) report(st, kErrTimeout, step, k + 1);
            return;
        }
    }
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

// Scratch: the candidates, then three counters (ticket, barrier arrivals,
// barrier generation), zeroed at the start of every factorization.
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

// CTAs of a panel launch: co-resident (cooperative), at most two per SM, and
// about two row blocks of the column-step size per CTA.
static int panel_grid(int64_t rows, int64_t &chunk) {
    static int per_sm[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (per_sm[dev] == 0) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_lu_panel, kLuThreads, 0) != cudaSuccess)
            nb = 1;
        per_sm[dev] = std::max(1, std::min(nb, kColCtasPerSm));
    }
    return lu_grid(rows, chunk, per_sm[dev]);
}

static bool stream_capturing(cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
}

cudaError_t launch_tall_lupp(double *A, int64_t lda, int64_t m, int n, int32_t *ipiv,
                             void *scratch, DevStatus *st, int step_id, cudaStream_t stream,
                             const LuWaitOptions *wopt) {
    ArgCand *cands = reinterpret_cast<ArgCand *>(scratch);
    unsigned *ticket =
        reinterpret_cast<unsigned *>(static_cast<char *>(scratch) + cand_slots() * sizeof(ArgCand));
    unsigned *bar_count = ticket + 1, *bar_gen = ticket + 2;
    cudaError_t e = cudaMemsetAsync(ticket, 0, 3 * sizeof(unsigned), stream);
    if (e != cudaSuccess) return e;
    const uint64_t limit_ns = wopt && wopt->limit_ns ? wopt->limit_ns : kWaitLimitNs;
    int stall = wopt ? wopt->stall : 0;
    bool coop = !stream_capturing(stream);
    const size_t smax = size_t(kLuNB) * n * sizeof(double);
    cudaFuncSetAttribute(k_lu_trailing, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smax));
    int64_t chunk;
    int g = lu_grid(m, chunk, kTrailCtasPerSm);
    RQ_LAUNCH(KID_LU_TRAILING, stream, k_lu_trailing<<<g, kLuThreads, 0, stream>>>(A, lda, m, n, 0, 0, chunk, cands, ticket, ipiv, st,
                                                step_id));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    for (int k0 = 0; k0 < n; k0 += kLuNB) {
        const int pe = std::min(n, k0 + kLuNB);
        bool done = false;
        if (coop && m - k0 - 1 > 0) {
            int64_t pchunk;
            const int pg = panel_grid(m - k0 - 1, pchunk);
            int k0v = k0, pev = pe, stallv = stall;
            int64_t mv = m, ldav = lda;
            int nv = n, stepv = step_id;
            uint64_t limv = limit_ns;
            void *args[] = {&A, &ldav, &mv, &nv, &k0v, &pev, &pchunk, &cands, &ticket, &bar_count,
                            &bar_gen, &ipiv, &st, &stepv, &limv, &stallv};
            RQ_LAUNCH(KID_LU_COL, stream,
                      e = cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(k_lu_panel), pg,
                                                      kLuThreads, args, 0, stream));
            if (e == cudaSuccess) {
                done = true;
                stall = 0;
            } else {
                cudaGetLastError();  // refused (e.g. too large): column launches from here on
                coop = false;
            }
        }
        for (int k = k0; k < pe && !done; ++k) {
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
