// Small dense FP64 factorizations held in the shared memory of one thread
// block cluster: the s x n matrix is split by rows over C = 1, 2, 4 or 8
// CTAs, each keeping its slab of h = ceil(s / C) rows (column-major, ld h)
// in shared memory for the whole factorization.  Pivot candidates, partial
// sums and the pivot row move between the CTAs through distributed shared
// memory; two cluster barriers per column order them.
//
//   k_precond_cluster, mode 0 (RCLUPP, Algorithm 6): LU with
//     partial pivoting of Y (eq. (elu); first largest magnitude, smallest row
//     on ties), R0 = R-factor of the Householder QR of M (eq. (eh), LAPACK
//     larfg convention), R1 = R0 N (eq. (ey)) with rows of negative diagonal
//     negated.
//   mode 1 (RCLUPPr, Algorithm 7; RCholeskyQR, Algorithm 5): the
//     Householder R of Y, R1 = R0 N with N the upper triangle of an external
//     factor, or N = I.
//   mode | kGivensMode: R0 by Givens rotations instead of Householder (the
//     alternative of Section 1 and of the remark after Algorithm 5): per
//     column a binary tree of rotations over each CTA's rows, then over the
//     CTAs' head rows; r = hypot(a, b) >= 0, c = a / r, s = b / r.
//   k_cholesky_cluster: upper Cholesky of an n x n Gram matrix (C2, C6),
//     right-looking, with the same breakdown status as the one-CTA kernel.
//
// The arithmetic of every column step is that of the one-CTA kernels
// (small.cu): same divisions, same Householder scalars; only the order of
// the partial sums across CTAs differs.
#include <cooperative_groups.h>

#include <algorithm>
#include <climits>

#include "common.cuh"
#include "kernels.h"

namespace cg = cooperative_groups;

namespace rq {
namespace {

constexpr int kClThreads = 512;
constexpr int kClMaxCtas = 8;
constexpr size_t kClSmemBudget = 200 * 1024;
constexpr int kClRowLanes = 128;                     // update loops: rows by tid % 128,
constexpr int kClColLanes = kClThreads / kClRowLanes;  // columns by tid / 128
constexpr int kGivensMode = 2;                          // mode bit: R0 by Givens rotations

// Deterministic block sum (shuffle tree, then warps in order), in every thread.
__device__ __forceinline__ double cl_block_sum(double v, double *red) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        red[32] = s;
    }
    __syncthreads();
    return red[32];
}

__device__ __forceinline__ bool cl_better(double v1, int g1, double v2, int g2) {
    return v1 > v2 || (v1 == v2 && g1 < g2);
}

// Block argmax of (v, g); result in thread 0's (rv, rg).
__device__ __forceinline__ void cl_block_argmax(double v, int g, double *redv, int *redg,
                                                double &rv, int &rg) {
    for (int off = 16; off > 0; off >>= 1) {
        const double v2 = __shfl_down_sync(0xffffffffu, v, off);
        const int g2 = __shfl_down_sync(0xffffffffu, g, off);
        if (cl_better(v2, g2, v, g)) {
            v = v2;
            g = g2;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) {
        redv[warp] = v;
        redg[warp] = g;
    }
    __syncthreads();
    rv = -1.0;
    rg = INT_MAX;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
            if (cl_better(redv[w], redg[w], rv, rg)) {
                rv = redv[w];
                rg = redg[w];
            }
}

struct ClShared {
    double redv[33];
    int redg[33];
    double cand_v;  // this CTA's pivot candidate / partial sum
    int cand_g;
    double alpha;   // Householder alpha (owner of row k)
    double piv_v;   // combined values, same in every CTA
    int piv_g;
    double sigma;
    double beta, tau, scal;  // reflector scalars of the current column
    double gc, gs;           // rotation of the current cross-CTA pair
};

// Cluster-wide barrier and remote shared-memory pointers; a single CTA
// (kCl == false, launched without a cluster) uses the block barrier and its
// own shared memory directly.
template <bool kCl>
struct ClOps {
    __device__ __forceinline__ static int size() {
        if constexpr (kCl) return static_cast<int>(cg::this_cluster().num_blocks());
        return 1;
    }
    __device__ __forceinline__ static int rank() {
        if constexpr (kCl) return static_cast<int>(cg::this_cluster().block_rank());
        return 0;
    }
    __device__ __forceinline__ static void sync() {
        if constexpr (kCl)
            cg::this_cluster().sync();
        else
            __syncthreads();
    }
    template <class Tp>
    __device__ __forceinline__ static Tp *at(Tp *p, int r) {
        if constexpr (kCl) return cg::this_cluster().map_shared_rank(p, r);
        (void)r;
        return p;
    }
};

template <bool kCl>
__global__ void __launch_bounds__(kClThreads)
    k_precond_cluster(const double *__restrict__ Y, int64_t ldy, int s, int n, int h, int mode,
                      const double *__restrict__ Nsrc, int64_t ldn, double *Nbuf, double *RP,
                      double *rinv, double *R1, int64_t ldr, DevStatus *st, int step) {
    using Cl = ClOps<kCl>;
    const int C = Cl::size();
    const int rank = Cl::rank();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *A = reinterpret_cast<double *>(smem_raw);  // slab, h x n, ld h
    double *urow = A + size_t(h) * n;                  // pivot row / w vector
    double *tmprow = urow + n;
    double *pw = tmprow + n;                           // partial w (this CTA)
    __shared__ ClShared sh;
    const int tid = threadIdx.x, T = blockDim.x;
    const int r0 = rank * h;
    const int rows = max(0, min(h, s - r0));
    const bool givens = (mode & kGivensMode) != 0;
    mode &= ~kGivensMode;

    for (int idx = tid; idx < h * n; idx += T) {
        const int i = idx % h, j = idx / h;
        A[idx] = i < rows ? Y[(r0 + i) + int64_t(j) * ldy] : 0.0;
    }
    __syncthreads();

    if (mode == 0) {
        // ---- LU with partial pivoting (eq. (elu))
        for (int k = 0; k < n; ++k) {
            double bv = -1.0;
            int bg = INT_MAX;
            for (int i = tid; i < rows; i += T) {
                const int g = r0 + i;
                if (g >= k) {
                    const double v = fabs(A[i + size_t(k) * h]);
                    if (cl_better(v, g, bv, bg)) {
                        bv = v;
                        bg = g;
                    }
                }
            }
            double rv;
            int rg;
            cl_block_argmax(bv, bg, sh.redv, sh.redg, rv, rg);
            if (tid == 0) {
                sh.cand_v = rv;
                sh.cand_g = rg;
            }
            Cl::sync();
            if (tid == 0) {
                double v = -1.0;
                int g = INT_MAX;
                for (int q = 0; q < C; ++q) {
                    const ClShared *o = Cl::at(&sh, q);
                    if (cl_better(o->cand_v, o->cand_g, v, g)) {
                        v = o->cand_v;
                        g = o->cand_g;
                    }
                }
                sh.piv_v = v;
                sh.piv_g = g;
            }
            __syncthreads();
            const double best = sh.piv_v;
            const int p = sh.piv_g;
            if (!(best > 0.0)) {  // the same verdict in every CTA
                if (rank == 0 && tid == 0)
                    report(st, best == 0.0 ? kErrLuZeroPivot : kErrNonfinite, step, k);
                Cl::sync();  // no CTA leaves while another may read its shared memory
                return;
            }
            const int rk = k / h, rp = p / h;
            {
                const double *rowp = Cl::at(A, rp) + (p - rp * h);
                for (int j = tid; j < n; j += T) urow[j] = rowp[size_t(j) * h];
                if (rank == rp && p != k) {
                    const double *rowk = Cl::at(A, rk) + (k - rk * h);
                    for (int j = tid; j < n; j += T) tmprow[j] = rowk[size_t(j) * h];
                }
            }
            Cl::sync();  // every CTA has both rows before either is overwritten
            if (rank == rk)
                for (int j = tid; j < n; j += T) A[(k - rk * h) + size_t(j) * h] = urow[j];
            if (rank == rp && p != k)
                for (int j = tid; j < n; j += T) A[(p - rp * h) + size_t(j) * h] = tmprow[j];
            __syncthreads();
            const double piv = urow[k];
            for (int i = tid; i < rows; i += T)
                if (r0 + i > k) A[i + size_t(k) * h] = A[i + size_t(k) * h] / piv;
            __syncthreads();
            // rows by tid % 128, columns by tid / 128 (no division in the loop)
            for (int i = tid % kClRowLanes; i < rows; i += kClRowLanes) {
                if (r0 + i <= k) continue;
                const double l = A[i + size_t(k) * h];
                for (int j = k + 1 + tid / kClRowLanes; j < n; j += kClColLanes)
                    A[i + size_t(j) * h] = fma(-l, urow[j], A[i + size_t(j) * h]);
            }
            __syncthreads();
        }
        // N (rows < n, upper part) to global scratch; the slab becomes M
        for (int idx = tid; idx < rows * n; idx += T) {
            const int i = idx % rows, j = idx / rows, g = r0 + i;
            const double a = A[i + size_t(j) * h];
            if (g < n) Nbuf[g + size_t(j) * n] = g <= j ? a : 0.0;
            A[i + size_t(j) * h] = g > j ? a : (g == j ? 1.0 : 0.0);
        }
        __threadfence();
        __syncthreads();
    }

    if (givens) {
        // ---- R0 by Givens rotations.  Column k: a tree over this slab's rows
        // g >= k (round d rotates rows lo + 2dq and lo + 2dq + d, zeroing the
        // second's entry), then a tree over the CTAs' head rows.
        double *gc = pw + n;                 // cosines of the current round
        double *gsn = gc + (h + 2) / 2;      // sines
        for (int k = 0; k < n; ++k) {
            const int lo = max(0, k - r0);
            const int cnt = rows - lo;       // the same in every thread of this CTA
            for (int d = 1; d < cnt; d <<= 1) {
                const int np = (cnt - d + 2 * d - 1) / (2 * d);
                for (int p = tid; p < np; p += T) {
                    const int top = lo + 2 * d * p, bot = top + d;
                    const double a = A[top + size_t(k) * h], b = A[bot + size_t(k) * h];
                    double c = 1.0, sn = 0.0;
                    if (b != 0.0) {
                        const double r = hypot(a, b);
                        c = a / r;
                        sn = b / r;
                        A[top + size_t(k) * h] = r;
                        A[bot + size_t(k) * h] = 0.0;
                    }
                    gc[p] = c;
                    gsn[p] = sn;
                }
                __syncthreads();
                // pairs by the low bits of tid, columns by the high bits
                int pl = 1;
                while (pl < np && pl < T) pl <<= 1;
                const int psh = __ffs(pl) - 1;
                for (int p = tid & (pl - 1); p < np; p += pl) {
                    const double c = gc[p], sn = gsn[p];
                    if (sn == 0.0) continue;
                    const int top = lo + 2 * d * p, bot = top + d;
                    for (int j = k + 1 + (tid >> psh); j < n; j += T >> psh) {
                        const double x = A[top + size_t(j) * h], y = A[bot + size_t(j) * h];
                        A[top + size_t(j) * h] = c * x + sn * y;
                        A[bot + size_t(j) * h] = c * y - sn * x;
                    }
                }
                __syncthreads();
            }
            if (C > 1) {
                Cl::sync();  // every CTA's tree is done
                const int rk = k / h, last = (s - 1) / h;
                for (int d = 1; rk + d <= last; d <<= 1) {
                    if (rank >= rk && (rank - rk) % (2 * d) == 0 && rank + d <= last) {
                        // the head of CTA rank + d is its local row 0 (its rows are all > k)
                        double *B = Cl::at(A, rank + d);
                        if (tid == 0) {
                            const double a = A[lo + size_t(k) * h], b = B[size_t(k) * h];
                            double c = 1.0, sn = 0.0;
                            if (b != 0.0) {
                                const double r = hypot(a, b);
                                c = a / r;
                                sn = b / r;
                                A[lo + size_t(k) * h] = r;
                                B[size_t(k) * h] = 0.0;
                            }
                            sh.gc = c;
                            sh.gs = sn;
                        }
                        __syncthreads();
                        const double c = sh.gc, sn = sh.gs;
                        if (sn != 0.0)
                            for (int j = k + 1 + tid; j < n; j += T) {
                                const double x = A[lo + size_t(j) * h], y = B[size_t(j) * h];
                                A[lo + size_t(j) * h] = c * x + sn * y;
                                B[size_t(j) * h] = c * y - sn * x;
                            }
                    }
                    Cl::sync();  // the pair's rows are final before the next round reads them
                }
            }
        }
    } else {
    // ---- Householder R of the slab matrix (eq. (eh), larfg convention)
    for (int k = 0; k < n; ++k) {
        const int rk = k / h;
        double part = 0.0;
        for (int i = tid; i < rows; i += T)
            if (r0 + i > k) {
                const double v = A[i + size_t(k) * h];
                part = fma(v, v, part);
            }
        part = cl_block_sum(part, sh.redv);
        if (tid == 0) {
            sh.cand_v = part;
            if (rank == rk) sh.alpha = A[(k - rk * h) + size_t(k) * h];
        }
        Cl::sync();
        // one thread forms the reflector's scalars (the FP64 pipe is too slow
        // for every thread to repeat a square root and two divisions)
        if (tid == 0) {
            double sg = 0.0;
            for (int q = 0; q < C; ++q) sg += Cl::at(&sh, q)->cand_v;
            sh.sigma = sg;
            if (sg != 0.0) {
                const double alpha = Cl::at(&sh, rk)->alpha;
                const double norm = sqrt(alpha * alpha + sg);
                const double beta = alpha >= 0.0 ? -norm : norm;
                sh.beta = beta;
                sh.tau = (beta - alpha) / beta;
                sh.scal = 1.0 / (alpha - beta);
            }
        }
        __syncthreads();
        if (sh.sigma == 0.0) {  // the same in every CTA: no reflection
            Cl::sync();  // partials read everywhere before the next column's are written
            continue;
        }
        const double beta = sh.beta, tau = sh.tau, scal = sh.scal;
        for (int i = tid; i < rows; i += T)
            if (r0 + i > k) A[i + size_t(k) * h] *= scal;
        __syncthreads();
        // partial w_j = sum over this slab's rows g >= k of v_g a_gj (v_k = 1)
        {
            const int lane = tid & 31, warp = tid >> 5, nw = T >> 5;
            for (int j = k + 1 + warp; j < n; j += nw) {
                double acc = 0.0;
                for (int i = lane; i < rows; i += 32) {
                    const int g = r0 + i;
                    if (g >= k) {
                        const double v = g == k ? 1.0 : A[i + size_t(k) * h];
                        acc = fma(v, A[i + size_t(j) * h], acc);
                    }
                }
                for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
                if (lane == 0) pw[j] = acc;
            }
        }
        Cl::sync();
        for (int j = k + 1 + tid; j < n; j += T) {
            double sw = 0.0;
            for (int q = 0; q < C; ++q) sw += Cl::at(pw, q)[j];
            urow[j] = sw * tau;
        }
        __syncthreads();
        for (int i = tid % kClRowLanes; i < rows; i += kClRowLanes) {
            const int g = r0 + i;
            if (g < k) continue;
            const double v = g == k ? 1.0 : A[i + size_t(k) * h];
            for (int j = k + 1 + tid / kClRowLanes; j < n; j += kClColLanes)
                A[i + size_t(j) * h] = fma(-v, urow[j], A[i + size_t(j) * h]);
        }
        __syncthreads();
        if (rank == rk && tid == 0) A[(k - rk * h) + size_t(k) * h] = beta;
        __syncthreads();
    }
    }
    Cl::sync();  // Nbuf written by every CTA before any reads it

    // ---- R1 = R0 N (rows of this slab below n), diagonal signs, padded outputs
    const int n_pad = pad16(n);
    double *RT = RP + size_t(n_pad) * n_pad;
    const double *N = mode == 0 ? Nbuf : Nsrc;
    const int64_t ldN = mode == 0 ? n : ldn;
    const int own = max(0, min(rows, n - r0));  // rows g < n held here
    for (int idx = tid; idx < own * n_pad; idx += T) {
        const int i = idx % own, j = idx / own, g = r0 + i;
        double acc = 0.0;
        if (j < n && g <= j) {
            if (N == nullptr)
                acc = A[i + size_t(j) * h];
            else
                for (int t = g; t <= j; ++t) acc = fma(A[i + size_t(t) * h], N[t + int64_t(j) * ldN], acc);
        }
        const double dgg = N == nullptr ? A[i + size_t(g) * h] : A[i + size_t(g) * h] * N[g + int64_t(g) * ldN];
        if (dgg < 0.0 && j < n && g <= j) acc = -acc;
        RP[g + size_t(j) * n_pad] = acc;
        RT[size_t(g) * n_pad + j] = acc;
        if (R1 != nullptr && j < n) R1[g + int64_t(j) * ldr] = acc;
        if (j == g) rinv[g] = 1.0 / acc;
    }
    if (rank == 0) {  // padding rows n .. n_pad - 1
        for (int idx = tid; idx < (n_pad - n) * n_pad; idx += T) {
            const int g = n + idx % (n_pad - n), j = idx / (n_pad - n);
            RP[g + size_t(j) * n_pad] = 0.0;
            RT[size_t(g) * n_pad + j] = 0.0;
        }
        for (int g = n + tid; g < n_pad; g += T) rinv[g] = 0.0;
    }
}

// ---- preconditioner with one exchange per column step ----------------------
// The factorizations of k_precond_cluster's modes 0 and 1 (Householder R0),
// arranged so that each column step needs one cluster barrier and no remote
// read: before the barrier every CTA stores what the others need into their
// shared memory (distributed shared-memory stores); after it, every CTA reads
// only its own.
//   LU column k: each CTA pushes its pivot candidate (largest |a_gk| over its
//   rows g >= k, smallest g on ties, NaN never a candidate) with that row in
//   full, and the owner of row k pushes row k.  After the barrier every
//   thread picks the same pivot p from the C candidates; the owner of row k
//   takes the pushed pivot row, the owner of row p takes row k, and the
//   trailing update reads the pivot row from the exchange buffer.
//   Householder column k: each CTA pushes P_j = sum over its rows g > k of
//   a_gk a_gj (j >= k; P_k is its share of sigma) and the owner of row k
//   pushes row k.  After the barrier every CTA forms sigma = sum_q P_k^q, the
//   reflector's scalars (eq. (eh), larfg convention) and
//   u_j = tau (a_kj + scal sum_q P_j^q) = tau (v^T A)_j, v_g = scal a_gk,
//   v_k = 1, on its own.
// Two exchange buffers, used alternately: a CTA stores into buffer b only
// after the barrier that every CTA reaches once it has read buffer b.
// The slab's leading dimension is odd, so that a warp reading one row of 32
// columns hits distinct banks.
constexpr int kPxThreads = 256;
constexpr int kPxMaxCtas = 8;
constexpr int kPxWarps = kPxThreads / 32;

// |v| as an order-preserving integer, plus one; 0 for NaN (not a candidate).
__device__ __forceinline__ unsigned long long px_key(double v) {
    const unsigned long long b =
        static_cast<unsigned long long>(__double_as_longlong(v)) & 0x7fffffffffffffffull;
    return b <= 0x7ff0000000000000ull ? b + 1ull : 0ull;
}

__device__ __forceinline__ bool px_better(unsigned long long k1, int g1, unsigned long long k2, int g2) {
    return k1 > k2 || (k1 == k2 && g1 < g2);
}

template <bool kCl>
__global__ void __launch_bounds__(kPxThreads)
    k_precond_push(const double *__restrict__ Y, int64_t ldy, int s, int n, int h, int ld, int mode,
                   const double *__restrict__ Nsrc, int64_t ldn, double *Nbuf, double *RP,
                   double *rinv, double *R1, int64_t ldr, DevStatus *st, int step) {
    using Cl = ClOps<kCl>;
    const int C = Cl::size();
    const int rank = Cl::rank();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *A = reinterpret_cast<double *>(smem_raw);  // slab, h x n, leading dimension ld
    const size_t xs = size_t(C + 1) * n;               // one exchange buffer: C rows, then row k
    double *X = A + size_t(ld) * n;
    double *Ssum = X + 2 * xs;                         // combined partial sums
    double *U = Ssum + n;                              // u_j of the current reflector
    __shared__ unsigned long long ckey[2][kPxMaxCtas];
    __shared__ int cidx[2][kPxMaxCtas];
    __shared__ double csc[4];                          // sigma, beta, tau, scal
    const int tid = threadIdx.x, T = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const int r0 = rank * h;
    const int rows = max(0, min(h, s - r0));

    for (int idx = tid; idx < h * n; idx += T) {
        const int i = idx % h, j = idx / h;
        A[i + size_t(j) * ld] = i < rows ? Y[(r0 + i) + int64_t(j) * ldy] : 0.0;
    }
    __syncthreads();
    int xc = 0;  // exchanges so far (buffer parity)

    if (mode == 0) {
        // ---- LU with partial pivoting (eq. (elu))
        for (int k = 0; k < n; ++k) {
            const int b = (xc++) & 1;
            double *xb = X + size_t(b) * xs;
            const int rk = k / h;
            // (1) this CTA's candidate, in every warp
            unsigned long long bk = 0;
            int bg = INT_MAX;
            for (int i = lane; i < rows; i += 32) {
                const int g = r0 + i;
                if (g >= k) {
                    const unsigned long long kk = px_key(A[i + size_t(k) * ld]);
                    if (px_better(kk, g, bk, bg)) {
                        bk = kk;
                        bg = g;
                    }
                }
            }
            for (int off = 16; off > 0; off >>= 1) {
                const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, bk, off);
                const int g2 = __shfl_xor_sync(0xffffffffu, bg, off);
                if (px_better(k2, g2, bk, bg)) {
                    bk = k2;
                    bg = g2;
                }
            }
            // (2) push the candidate row, row k (its owner) and the candidate
            {
                const int li = bg - r0;
                for (int idx = tid; idx < C * n; idx += T) {
                    const int q = idx / n, j = idx - q * n;
                    double *dst = Cl::at(xb, q);
                    if (bg != INT_MAX) dst[size_t(rank) * n + j] = A[li + size_t(j) * ld];
                    if (rank == rk) dst[size_t(C) * n + j] = A[(k - r0) + size_t(j) * ld];
                }
                if (tid < C) {
                    Cl::at(&ckey[b][0], tid)[rank] = bk;
                    Cl::at(&cidx[b][0], tid)[rank] = bg;
                }
            }
            Cl::sync();
            // (3) the pivot: the same in every thread of every CTA
            unsigned long long pk = 0;
            int p = INT_MAX, rp = 0;
            for (int q = 0; q < C; ++q)
                if (px_better(ckey[b][q], cidx[b][q], pk, p)) {
                    pk = ckey[b][q];
                    p = cidx[b][q];
                    rp = q;
                }
            if (pk <= 1ull) {  // key 1: the largest magnitude is 0; key 0: only NaN
                if (rank == 0 && tid == 0) report(st, pk == 1ull ? kErrLuZeroPivot : kErrNonfinite, step, k);
                Cl::sync();
                return;
            }
            const double *prow = xb + size_t(rp) * n;  // row p, pushed by its owner
            const double *krow = xb + size_t(C) * n;   // row k before the swap
            const double piv = prow[k];
            // (4) swap; multipliers l_g = a_gk / piv of the rows below k
            if (rank == rk)
                for (int j = tid; j < n; j += T) A[(k - r0) + size_t(j) * ld] = prow[j];
            if (rank == rp && p != k)
                for (int j = tid; j < n; j += T)
                    if (j != k) A[(p - r0) + size_t(j) * ld] = krow[j];
            for (int i = tid; i < rows; i += T) {
                const int g = r0 + i;
                if (g > k) A[i + size_t(k) * ld] = (g == p ? krow[k] : A[i + size_t(k) * ld]) / piv;
            }
            __syncthreads();
            // (5) trailing update with the pivot row: rows by lane, columns by warp
            for (int i = lane; i < rows; i += 32) {
                if (r0 + i <= k) continue;
                const double l = A[i + size_t(k) * ld];
                for (int j = k + 1 + warp; j < n; j += kPxWarps)
                    A[i + size_t(j) * ld] = fma(-l, prow[j], A[i + size_t(j) * ld]);
            }
            __syncthreads();
        }
        // N (rows < n, upper part) to global scratch; the slab becomes M
        for (int idx = tid; idx < rows * n; idx += T) {
            const int i = idx % rows, j = idx / rows, g = r0 + i;
            const double a = A[i + size_t(j) * ld];
            if (g < n) Nbuf[g + size_t(j) * n] = g <= j ? a : 0.0;
            A[i + size_t(j) * ld] = g > j ? a : (g == j ? 1.0 : 0.0);
        }
        __threadfence();
        __syncthreads();
    }

    // ---- Householder R of the slab matrix (eq. (eh), larfg convention)
    for (int k = 0; k < n; ++k) {
        const int b = (xc++) & 1;
        double *xb = X + size_t(b) * xs;
        const int rk = k / h;
        // (1) partial sums over this CTA's rows g > k; row k from its owner.
        // tpc adjacent lanes share a column, each summing every tpc-th row
        // (the FP64 work spread over all warps when few columns are left),
        // combined by shuffles.
        {
            const int i0 = max(0, k + 1 - r0);
            const int ncol = n - k;
            int tpc = 1;
            while (tpc < 8 && tpc * 2 * ncol <= T) tpc *= 2;
            for (int base = 0; base < ncol * tpc; base += T) {  // the same trip count in every thread
                const int idx = base + tid;
                const int jl = idx / tpc, part = idx - jl * tpc;
                const int j = k + jl;
                double acc = 0.0;
                if (jl < ncol)
                    for (int i = i0 + part; i < rows; i += tpc)
                        acc = fma(A[i + size_t(k) * ld], A[i + size_t(j) * ld], acc);
                for (int off = tpc >> 1; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
                if (part == 0 && jl < ncol) {
                    const double akj = rank == rk ? A[(k - r0) + size_t(j) * ld] : 0.0;
                    for (int q = 0; q < C; ++q) {
                        double *dst = Cl::at(xb, q);
                        dst[size_t(rank) * n + j] = acc;
                        if (rank == rk) dst[size_t(C) * n + j] = akj;
                    }
                }
            }
        }
        Cl::sync();
        // (2) the sums over the CTAs (in rank order) and the reflector's
        // scalars (one thread: the FP64 pipe is too slow for every thread to
        // repeat a square root and two divisions)
        for (int j = k + tid; j < n; j += T) {
            double sj = 0.0;
            for (int q = 0; q < C; ++q) sj += xb[size_t(q) * n + j];
            Ssum[j] = sj;
            if (j == k) {
                csc[0] = sj;
                if (sj != 0.0) {
                    const double alpha = xb[size_t(C) * n + k];
                    const double norm = sqrt(alpha * alpha + sj);
                    const double beta = alpha >= 0.0 ? -norm : norm;
                    csc[1] = beta;
                    csc[2] = (beta - alpha) / beta;
                    csc[3] = 1.0 / (alpha - beta);
                }
            }
        }
        __syncthreads();
        if (csc[0] == 0.0) continue;  // the same in every CTA: no reflection
        const double beta = csc[1], tau = csc[2], scal = csc[3];
        // (3) u_j, the reflector's vector v_g = scal a_gk in column k, r_kk
        {
            const double *krow = xb + size_t(C) * n;
            for (int j = k + 1 + tid; j < n; j += T) U[j] = tau * fma(scal, Ssum[j], krow[j]);
            for (int i = tid; i < rows; i += T)
                if (r0 + i > k) A[i + size_t(k) * ld] *= scal;
            if (rank == rk && tid == 0) A[(k - r0) + size_t(k) * ld] = beta;
        }
        __syncthreads();
        // (4) a_gj -= v_g u_j, rows g >= k by lane, columns by warp
        for (int i = lane; i < rows; i += 32) {
            const int g = r0 + i;
            if (g < k) continue;
            const double v = g == k ? 1.0 : A[i + size_t(k) * ld];
            for (int j = k + 1 + warp; j < n; j += kPxWarps)
                A[i + size_t(j) * ld] = fma(-v, U[j], A[i + size_t(j) * ld]);
        }
        __syncthreads();
    }
    Cl::sync();  // Nbuf written by every CTA before any reads it

    // ---- R1 = R0 N (rows of this slab below n), diagonal signs, padded outputs
    const int n_pad = pad16(n);
    double *RT = RP + size_t(n_pad) * n_pad;
    const double *N = mode == 0 ? Nbuf : Nsrc;
    const int64_t ldN = mode == 0 ? n : ldn;
    const int own = max(0, min(rows, n - r0));  // rows g < n held here
    for (int idx = tid; idx < own * n_pad; idx += T) {
        const int i = idx % own, j = idx / own, g = r0 + i;
        double acc = 0.0;
        if (j < n && g <= j) {
            if (N == nullptr)
                acc = A[i + size_t(j) * ld];
            else
                for (int t = g; t <= j; ++t) acc = fma(A[i + size_t(t) * ld], N[t + int64_t(j) * ldN], acc);
        }
        const double dgg =
            N == nullptr ? A[i + size_t(g) * ld] : A[i + size_t(g) * ld] * N[g + int64_t(g) * ldN];
        if (dgg < 0.0 && j < n && g <= j) acc = -acc;
        RP[g + size_t(j) * n_pad] = acc;
        RT[size_t(g) * n_pad + j] = acc;
        if (R1 != nullptr && j < n) R1[g + int64_t(j) * ldr] = acc;
        if (j == g) rinv[g] = 1.0 / acc;
    }
    if (rank == 0) {  // padding rows n .. n_pad - 1
        for (int idx = tid; idx < (n_pad - n) * n_pad; idx += T) {
            const int g = n + idx % (n_pad - n), j = idx / (n_pad - n);
            RP[g + size_t(j) * n_pad] = 0.0;
            RT[size_t(g) * n_pad + j] = 0.0;
        }
        for (int g = n + tid; g < n_pad; g += T) rinv[g] = 0.0;
    }
}

// Upper Cholesky of G (n x n) by rows over the cluster: step k takes
// r_kk = sqrt(w_kk) (breakdown if w_kk is not > 0), r_kj = w_kj / r_kk (the
// owner of row k), then every CTA subtracts r_ki r_kj from its rows i > k,
// j >= i -- the subtractions and order of the one-CTA kernel.
template <bool kCl>
__global__ void __launch_bounds__(kClThreads)
    k_cholesky_cluster(const double *__restrict__ G, int64_t ldg, int n, int h, double *RP,
                       double *rinv, double *R, int64_t ldr, DevStatus *st, int step) {
    using Cl = ClOps<kCl>;
    const int rank = Cl::rank();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *A = reinterpret_cast<double *>(smem_raw);  // rows [r0, r0 + rows), ld h
    double *urow = A + size_t(h) * n;
    __shared__ int fail_at;
    __shared__ int fail_all;
    __shared__ double rkk_sh;
    const int tid = threadIdx.x, T = blockDim.x;
    const int r0 = rank * h;
    const int rows = max(0, min(h, n - r0));
    if (tid == 0) fail_at = -1;
    for (int idx = tid; idx < h * n; idx += T) {
        const int i = idx % h, j = idx / h, g = r0 + i;
        A[idx] = (i < rows && g <= j) ? G[g + int64_t(j) * ldg] : 0.0;
    }
    __syncthreads();
    int failed = -1;
    for (int k = 0; k < n; ++k) {
        const int rk = k / h;
        if (rank == rk) {
            const int lk = k - rk * h;
            const double d = A[lk + size_t(k) * h];
            if (!(d > 0.0)) {
                if (tid == 0) fail_at = k;
            } else {
                if (tid == 0) rkk_sh = sqrt(d);  // one square root, shared
                __syncthreads();
                const double rkk = rkk_sh;
                for (int j = k + 1 + tid; j < n; j += T) A[lk + size_t(j) * h] = A[lk + size_t(j) * h] / rkk;
                __syncthreads();
                if (tid == 0) A[lk + size_t(k) * h] = rkk;
            }
        }
        Cl::sync();
        if (tid == 0) fail_all = Cl::at(&fail_at, rk)[0];
        __syncthreads();
        if (fail_all >= 0) {  // the same verdict in every CTA
            failed = fail_all;
            Cl::sync();  // no CTA leaves while another may read its shared memory
            break;
        }
        const double *rowk = Cl::at(A, rk) + (k - rk * h);
        for (int j = k + 1 + tid; j < n; j += T) urow[j] = rowk[size_t(j) * h];
        __syncthreads();
        for (int i = tid % kClRowLanes; i < rows; i += kClRowLanes) {
            const int g = r0 + i;
            if (g <= k) continue;
            const double rg = urow[g];
            for (int j = g + tid / kClRowLanes; j < n; j += kClColLanes)
                A[i + size_t(j) * h] = fma(-rg, urow[j], A[i + size_t(j) * h]);
        }
        Cl::sync();  // row k read by every CTA before its owner moves on
    }
    if (failed >= 0 && rank == 0 && tid == 0) report(st, kErrCholBreakdown, step, failed);
    const int n_pad = pad16(n);
    double *RT = RP + size_t(n_pad) * n_pad;
    for (int idx = tid; idx < rows * n_pad; idx += T) {
        const int i = idx % rows, j = idx / rows, g = r0 + i;
        const double v = (g <= j && j < n) ? A[i + size_t(j) * h] : 0.0;
        RP[g + size_t(j) * n_pad] = v;
        RT[size_t(g) * n_pad + j] = v;
        if (R != nullptr && j < n) R[g + int64_t(j) * ldr] = v;
        if (j == g) rinv[g] = (failed < 0) ? 1.0 / v : 0.0;
    }
    if (rank == 0) {
        for (int idx = tid; idx < (n_pad - n) * n_pad; idx += T) {
            const int g = n + idx % (n_pad - n), j = idx / (n_pad - n);
            RP[g + size_t(j) * n_pad] = 0.0;
            RT[size_t(g) * n_pad + j] = 0.0;
        }
        for (int g = n + tid; g < n_pad; g += T) rinv[g] = 0.0;
    }
}

// Upper Cholesky of G with one exchange per step, the arithmetic of
// k_cholesky_cluster: the owner of row k takes r_kk = sqrt(w_kk) (or records
// the breakdown) and r_kj = w_kj / r_kk, and pushes row k and the verdict into
// every CTA's shared memory; after the cluster barrier each CTA reads only
// its own copy and subtracts r_kg r_kj from its rows g > k, j >= g.  Two
// exchange buffers, used alternately, as in k_precond_push.
template <bool kCl>
__global__ void __launch_bounds__(kPxThreads)
    k_cholesky_push(const double *__restrict__ G, int64_t ldg, int n, int h, int ld, double *RP,
                    double *rinv, double *R, int64_t ldr, DevStatus *st, int step) {
    using Cl = ClOps<kCl>;
    const int C = Cl::size();
    const int rank = Cl::rank();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *A = reinterpret_cast<double *>(smem_raw);  // rows [r0, r0 + rows), leading dimension ld
    double *X = A + size_t(ld) * n;                    // two copies of the current row of R
    __shared__ int cfail[2];
    __shared__ double rkk_sh;
    const int tid = threadIdx.x, T = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const int r0 = rank * h;
    const int rows = max(0, min(h, n - r0));
    for (int idx = tid; idx < h * n; idx += T) {
        const int i = idx % h, j = idx / h, g = r0 + i;
        A[i + size_t(j) * ld] = (i < rows && g <= j) ? G[g + int64_t(j) * ldg] : 0.0;
    }
    __syncthreads();
    int failed = -1;
    for (int k = 0; k < n; ++k) {
        const int b = k & 1;
        const int rk = k / h;
        if (rank == rk) {  // the owner of row k (uniform in the CTA)
            const int lk = k - r0;
            const double d = A[lk + size_t(k) * ld];
            const bool ok = d > 0.0;
            if (tid == 0 && ok) rkk_sh = sqrt(d);  // one square root, shared
            __syncthreads();
            if (ok) {
                const double rkk = rkk_sh;
                for (int j = k + 1 + tid; j < n; j += T) {
                    const double r = A[lk + size_t(j) * ld] / rkk;
                    A[lk + size_t(j) * ld] = r;
                    for (int q = 0; q < C; ++q) Cl::at(X, q)[size_t(b) * n + j] = r;
                }
                if (tid == 0) A[lk + size_t(k) * ld] = rkk;
            }
            if (tid < C) Cl::at(&cfail[0], tid)[b] = ok ? -1 : k;
        }
        Cl::sync();
        if (cfail[b] >= 0) {  // the same verdict in every CTA
            failed = cfail[b];
            break;
        }
        const double *rowk = X + size_t(b) * n;
        // rows g > k by lane, columns j >= g by warp (all lanes on one column)
        for (int i = lane; i < rows; i += 32) {
            const int g = r0 + i;
            if (g <= k) continue;
            const double rg = rowk[g];
            for (int j = k + 1 + warp; j < n; j += kPxWarps)
                if (j >= g) A[i + size_t(j) * ld] = fma(-rg, rowk[j], A[i + size_t(j) * ld]);
        }
        __syncthreads();
    }
    if (failed >= 0 && rank == 0 && tid == 0) report(st, kErrCholBreakdown, step, failed);
    const int n_pad = pad16(n);
    double *RT = RP + size_t(n_pad) * n_pad;
    for (int idx = tid; idx < rows * n_pad; idx += T) {
        const int i = idx % rows, j = idx / rows, g = r0 + i;
        const double v = (g <= j && j < n) ? A[i + size_t(j) * ld] : 0.0;
        RP[g + size_t(j) * n_pad] = v;
        RT[size_t(g) * n_pad + j] = v;
        if (R != nullptr && j < n) R[g + int64_t(j) * ldr] = v;
        if (j == g) rinv[g] = (failed < 0) ? 1.0 / v : 0.0;
    }
    if (rank == 0) {
        for (int idx = tid; idx < (n_pad - n) * n_pad; idx += T) {
            const int g = n + idx % (n_pad - n), j = idx / (n_pad - n);
            RP[g + size_t(j) * n_pad] = 0.0;
            RT[size_t(g) * n_pad + j] = 0.0;
        }
        for (int g = n + tid; g < n_pad; g += T) rinv[g] = 0.0;
    }
}

// Smallest power-of-two cluster whose slabs fit the shared-memory budget,
// and at least four CTAs from 256 rows on: the column steps' FP64 updates
// then spread over four SMs (256 x 128: 2.76 -> 2.30 ms on GB300; eight
// CTAs gain nothing more, their cluster barriers cost what the FP64 work
// saves).
bool cl_shape(int rows, int n, int extra_vectors, int &C, int &h, size_t &smem, bool per_row = false) {
    for (C = rows >= 256 ? 4 : 1; C <= kClMaxCtas; C *= 2) {
        h = (rows + C - 1) / C;
        smem = (size_t(h) * n + size_t(extra_vectors) * n + (per_row ? size_t(h) + 2 : 0)) * sizeof(double);
        if (smem <= kClSmemBudget) return true;
    }
    return false;
}

// One CTA: the kCl == false instance, a plain launch.  Otherwise a cluster
// of C CTAs (the kCl == true instance).
template <class K1, class KC, class... Args>
cudaError_t cl_launch_t(K1 k1, KC kc, int C, int threads, size_t smem, cudaStream_t stream,
                        Args... args) {
    if (C == 1) {
        cudaError_t e = cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return e;
        k1<<<1, threads, smem, stream>>>(args...);
        return cudaGetLastError();
    }
    cudaError_t e = cudaFuncSetAttribute(kc, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C, 1, 1);
    cfg.blockDim = dim3(threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kc, args...);
}

template <class K1, class KC, class... Args>
cudaError_t cl_launch(K1 k1, KC kc, int C, size_t smem, cudaStream_t stream, Args... args) {
    return cl_launch_t(k1, kc, C, kClThreads, smem, stream, args...);
}

// Shape of k_precond_push: eight CTAs from 128 rows on (four from 32, else
// one), each slab with an odd leading dimension, two exchange buffers and two
// vectors, within the shared-memory budget of the other cluster kernels.
bool px_shape(int s, int n, int &C, int &h, int &ld, size_t &smem) {
    C = s >= 128 ? kPxMaxCtas : (s >= 32 ? 4 : 1);
    h = (s + C - 1) / C;
    ld = h | 1;
    smem = (size_t(ld) * n + 2 * size_t(C + 1) * n + 2 * size_t(n)) * sizeof(double);
    return smem <= kClSmemBudget;
}

}  // namespace

bool precond_cluster_fits(int s, int n, bool givens) {
    int C, h;
    size_t smem;
    return cl_shape(s, n, 3, C, h, smem, givens);
}

cudaError_t launch_precond_cluster(const double *Y, int64_t ldy, int s, int n, int mode,
                                   const double *Nsrc, int64_t ldn, double *Nbuf, double *RP,
                                   double *rinv, double *R1, int64_t ldr, DevStatus *st, int step,
                                   cudaStream_t stream) {
    int C, h, ld;
    size_t smem;
    cudaError_t e;
    if ((mode & kGivensMode) == 0 && px_shape(s, n, C, h, ld, smem)) {
        RQ_LAUNCH(KID_SMALL_PRECOND, stream,
                  e = cl_launch_t(k_precond_push<false>, k_precond_push<true>, C, kPxThreads, smem, stream,
                                  Y, ldy, s, n, h, ld, mode, Nsrc, ldn, Nbuf, RP, rinv, R1, ldr, st, step));
        if (e != cudaSuccess) return e;
        return cudaGetLastError();
    }
    if (!cl_shape(s, n, 3, C, h, smem, (mode & kGivensMode) != 0)) return cudaErrorInvalidValue;
    RQ_LAUNCH(KID_SMALL_PRECOND, stream,
              e = cl_launch(k_precond_cluster<false>, k_precond_cluster<true>, C, smem, stream, Y, ldy,
                            s, n, h, mode, Nsrc, ldn, Nbuf, RP, rinv, R1, ldr, st, step));
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

bool cholesky_cluster_fits(int n) {
    int C, h;
    size_t smem;
    return cl_shape(n, n, 1, C, h, smem);
}

cudaError_t launch_cholesky_cluster(const double *G, int64_t ldg, int n, double *RP, double *rinv,
                                    double *R, int64_t ldr, DevStatus *st, int step,
                                    cudaStream_t stream) {
    int C, h;
    size_t smem;
    cudaError_t e;
    {
        // one exchange per step: eight CTAs from n = 128 on (four from 32)
        const int Cx = n >= 128 ? kPxMaxCtas : (n >= 32 ? 4 : 1);
        const int hx = (n + Cx - 1) / Cx, ldx = hx | 1;
        const size_t sx = (size_t(ldx) * n + 2 * size_t(n)) * sizeof(double);
        if (sx <= kClSmemBudget) {
            RQ_LAUNCH(KID_CHOLESKY, stream,
                      e = cl_launch_t(k_cholesky_push<false>, k_cholesky_push<true>, Cx, kPxThreads, sx,
                                      stream, G, ldg, n, hx, ldx, RP, rinv, R, ldr, st, step));
            if (e != cudaSuccess) return e;
            return cudaGetLastError();
        }
    }
    if (!cl_shape(n, n, 1, C, h, smem)) return cudaErrorInvalidValue;
    RQ_LAUNCH(KID_CHOLESKY, stream,
              e = cl_launch(k_cholesky_cluster<false>, k_cholesky_cluster<true>, C, smem, stream, G,
                            ldg, n, h, RP, rinv, R, ldr, st, step));
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace rq
