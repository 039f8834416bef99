// Small dense FP64 factorizations that stay on the device (s x n and n x n,
// n <= 256): the LU with partial pivoting of the sketch (Algorithm 6,
// eq. (elu)), the R-factor of a thin Householder QR (eq. (eh)), the
// triangular products R1 = R0 N, R3 = R2 R1, R = R4 R3 (eq. (ey), C4, C8),
// and the Cholesky factorizations of the Gram matrices (C2, C6) with a
// breakdown status instead of NaNs.  This file holds the general one-CTA
// form with the working arrays in the (L2-resident) workspace; when the
// matrix fits the shared memory of a thread block cluster the launchers use
// the cluster form of small_cluster.cu instead.  These steps are O(s n^2)
// against the O(m n^2) tall passes.  Triangular factors are handed to the
// tall kernels in padded form: n_pad x n_pad (n_pad = 16-multiple), ld
// n_pad, zeros outside the upper triangle, followed by the row-major copy,
// plus the reciprocals of the diagonal.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace rq {

constexpr int kSmallThreads = 1024;

// Deterministic block sum (fixed shuffle tree, then warps in order).
__device__ __forceinline__ double block_sum(double v, double *red) {
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

// In-place LU with partial pivoting of W (rows x n, ld = rows), first
// largest magnitude wins.  Returns false (after reporting) on a zero pivot.
__device__ bool small_gepp(double *W, int rows, int n, DevStatus *st, int step, double *redv,
                           long long *redi) {
    for (int k = 0; k < n; ++k) {
        // pivot search
        double bv = -1.0;
        long long bi = 0x7fffffffffffffffll;
        for (int i = k + threadIdx.x; i < rows; i += blockDim.x) {
            const double v = fabs(W[i + int64_t(k) * rows]);
            if (v > bv || (v == bv && i < bi)) {
                bv = v;
                bi = i;
            }
        }
        for (int off = 16; off > 0; off >>= 1) {
            const double v2 = __shfl_down_sync(0xffffffffu, bv, off);
            const long long i2 = __shfl_down_sync(0xffffffffu, bi, off);
            if (v2 > bv || (v2 == bv && i2 < bi)) {
                bv = v2;
                bi = i2;
            }
        }
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        __syncthreads();
        if (lane == 0) {
            redv[warp] = bv;
            redi[warp] = bi;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double v = -1.0;
            long long ii = 0x7fffffffffffffffll;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
                if (redv[w] > v || (redv[w] == v && redi[w] < ii)) {
                    v = redv[w];
                    ii = redi[w];
                }
            redv[32] = v;
            redi[32] = ii;
        }
        __syncthreads();
        const double best = redv[32];
        const int p = static_cast<int>(redi[32]);
        if (!(best > 0.0)) {
            if (threadIdx.x == 0) report(st, best == 0.0 ? kErrLuZeroPivot : kErrNonfinite, step, k);
            return false;
        }
        if (p != k)
            for (int j = threadIdx.x; j < n; j += blockDim.x) {
                const double t = W[k + int64_t(j) * rows];
                W[k + int64_t(j) * rows] = W[p + int64_t(j) * rows];
                W[p + int64_t(j) * rows] = t;
            }
        __syncthreads();
        const double piv = W[k + int64_t(k) * rows];
        for (int i = k + 1 + threadIdx.x; i < rows; i += blockDim.x)
            W[i + int64_t(k) * rows] = W[i + int64_t(k) * rows] / piv;
        __syncthreads();
        const int nr = rows - k - 1, nc = n - k - 1;
        for (int idx = threadIdx.x; idx < nr * nc; idx += blockDim.x) {
            const int i = k + 1 + idx % nr, j = k + 1 + idx / nr;
            W[i + int64_t(j) * rows] =
                fma(-W[i + int64_t(k) * rows], W[k + int64_t(j) * rows], W[i + int64_t(j) * rows]);
        }
        __syncthreads();
    }
    return true;
}

// Householder reduction of H (rows x n, ld rows) in place; afterwards its top
// n x n upper triangle is R (LAPACK larfg convention: beta = -sign(alpha)||x||,
// sign(0) = +1, no reflection when the subcolumn is zero).  wv: n doubles.
__device__ void small_householder(double *H, int rows, int n, double *wv, double *red) {
    for (int k = 0; k < n; ++k) {
        double part = 0.0;
        for (int i = k + 1 + threadIdx.x; i < rows; i += blockDim.x) {
            const double v = H[i + int64_t(k) * rows];
            part = fma(v, v, part);
        }
        const double sigma = block_sum(part, red);
        if (sigma == 0.0) continue;  // uniform: every thread read the same sum
        // one thread forms the scalars (a square root and two divisions per
        // thread would load the slow FP64 pipe 1024-fold)
        if (threadIdx.x == 0) {
            const double alpha = H[k + int64_t(k) * rows];
            const double norm = sqrt(alpha * alpha + sigma);
            const double beta = alpha >= 0.0 ? -norm : norm;
            red[33] = beta;
            red[34] = (beta - alpha) / beta;
            red[35] = 1.0 / (alpha - beta);
        }
        __syncthreads();
        const double beta = red[33], tau = red[34], scal = red[35];
        for (int i = k + 1 + threadIdx.x; i < rows; i += blockDim.x)
            H[i + int64_t(k) * rows] *= scal;
        __syncthreads();
        // w_j = v^T H[k:, j] for j > k (v_k = 1): one warp per column
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int j = k + 1 + warp; j < n; j += nw) {
            double acc = 0.0;
            for (int i = k + 1 + lane; i < rows; i += 32)
                acc = fma(H[i + int64_t(k) * rows], H[i + int64_t(j) * rows], acc);
            for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
            if (lane == 0) wv[j] = (acc + H[k + int64_t(j) * rows]) * tau;
        }
        __syncthreads();
        const int nr = rows - k, nc = n - k - 1;
        for (int idx = threadIdx.x; idx < nr * nc; idx += blockDim.x) {
            const int i = k + idx % nr, j = k + 1 + idx / nr;
            const double vi = (i == k) ? 1.0 : H[i + int64_t(k) * rows];
            H[i + int64_t(j) * rows] = fma(-vi, wv[j], H[i + int64_t(j) * rows]);
        }
        __syncthreads();
        if (threadIdx.x == 0) H[k + int64_t(k) * rows] = beta;
        __syncthreads();
    }
}

// RP = A_up * B_up (upper triangular, padded output ld n_pad), where A_up is
// the upper triangle of A (lda) and B_up of B (ldb); then row signs
// normalised so that diag > 0 (when sign_fix), and rinv = 1/diag.
__device__ void small_trmm_to_padded(const double *A, int64_t lda, const double *B, int64_t ldb,
                                     int n, int n_pad, double *RP, double *rinv, bool sign_fix,
                                     int *sgn) {
    for (int idx = threadIdx.x; idx < n_pad * n_pad; idx += blockDim.x) {
        const int i = idx % n_pad, j = idx / n_pad;
        double acc = 0.0;
        if (i <= j && j < n) {
            if (B == nullptr)  // B = I
                acc = A[i + int64_t(j) * lda];
            else
                for (int t = i; t <= j; ++t)
                    acc = fma(A[i + int64_t(t) * lda], B[t + int64_t(j) * ldb], acc);
        }
        RP[idx] = acc;
    }
    __syncthreads();
    if (sign_fix) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) sgn[i] = RP[i + int64_t(i) * n_pad] < 0.0;
        __syncthreads();
        for (int idx = threadIdx.x; idx < n_pad * n_pad; idx += blockDim.x) {
            const int i = idx % n_pad;
            if (i < n && sgn[i]) RP[idx] = -RP[idx];
        }
        __syncthreads();
    }
    store_r_rows(RP, n_pad);
    for (int i = threadIdx.x; i < n_pad; i += blockDim.x)
        rinv[i] = (i < n) ? 1.0 / RP[i + int64_t(i) * n_pad] : 0.0;
    __syncthreads();
}

__device__ void copy_out_upper(const double *RP, int n, int n_pad, double *R, int64_t ldr) {
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int i = idx % n, j = idx / n;
        R[i + int64_t(j) * ldr] = (i <= j) ? RP[i + int64_t(j) * n_pad] : 0.0;
    }
}

// mode 0 (RCLUPP, Algorithm 6): LU of Y, Householder R of M,
//   R1 = R0 N.   mode 1 (RCLUPPr, Algorithm 7): Y is already M_s;
//   Householder R of Y, R1 = R0 N with N the top of an in-place tall LU (ldn).
__global__ void __launch_bounds__(kSmallThreads)
    k_small_precond(const double *__restrict__ Y, int64_t ldy, int s, int n, int mode,
                    const double *__restrict__ Nsrc, int64_t ldn, double *W, double *RP,
                    double *rinv, double *R1, int64_t ldr, DevStatus *st, int step) {
    __shared__ double red[36];
    __shared__ long long redi[33];
    __shared__ double wv[256];
    __shared__ int sgn[256];
    const int n_pad = pad16(n);
    double *W1 = W;                          // LU of Y (mode 0)
    double *W2 = W + int64_t(s) * n;         // Householder work
    for (int idx = threadIdx.x; idx < s * n; idx += blockDim.x) {
        const int i = idx % s, j = idx / s;
        W1[idx] = Y[i + int64_t(j) * ldy];
    }
    __syncthreads();
    const double *N = Nsrc;
    int64_t ldN = ldn;
    if (mode == 0) {
        if (!small_gepp(W1, s, n, st, step, red, redi)) return;
        // M: unit lower trapezoidal factor
        for (int idx = threadIdx.x; idx < s * n; idx += blockDim.x) {
            const int i = idx % s, j = idx / s;
            W2[idx] = i > j ? W1[idx] : (i == j ? 1.0 : 0.0);
        }
        N = W1;
        ldN = s;
    } else {
        for (int idx = threadIdx.x; idx < s * n; idx += blockDim.x) W2[idx] = W1[idx];
    }
    __syncthreads();
    small_householder(W2, s, n, wv, red);
    small_trmm_to_padded(W2, s, N, ldN, n, n_pad, RP, rinv, true, sgn);
    if (R1 != nullptr) copy_out_upper(RP, n, n_pad, R1, ldr);
}

cudaError_t launch_sketch_precond(const double *Y, int64_t ldy, int s, int n, double *W,
                                  double *RP, double *rinv, double *R1, int64_t ldr,
                                  DevStatus *st, int step_id, cudaStream_t stream, int r0_method) {
    if (r0_method == 1) {
        if (!precond_cluster_fits(s, n, true)) return cudaErrorNotSupported;
        return launch_precond_cluster(Y, ldy, s, n, kPrecondGivens, nullptr, 0, W, RP, rinv, R1, ldr, st,
                                      step_id, stream);
    }
    if (precond_cluster_fits(s, n))  // the matrix fits a cluster's shared memory
        return launch_precond_cluster(Y, ldy, s, n, 0, nullptr, 0, W, RP, rinv, R1, ldr, st, step_id,
                                      stream);
    RQ_LAUNCH(KID_SMALL_PRECOND, stream, k_small_precond<<<1, kSmallThreads, 0, stream>>>(Y, ldy, s, n, 0, nullptr, 0, W, RP, rinv, R1,
                                                     ldr, st, step_id));
    return cudaGetLastError();
}

cudaError_t launch_rcholqr_r1(const double *K, int64_t ldk, int s, int n, double *W, double *RP,
                              double *rinv, cudaStream_t stream, int r0_method) {
    if (r0_method == 1) {
        if (!precond_cluster_fits(s, n, true)) return cudaErrorNotSupported;
        return launch_precond_cluster(K, ldk, s, n, 1 | kPrecondGivens, nullptr, 0, W, RP, rinv, nullptr,
                                      0, nullptr, 0, stream);
    }
    // mode 1 with N = I: R1 = R-factor of HouseholderQR(K), signs normalised
    if (precond_cluster_fits(s, n))
        return launch_precond_cluster(K, ldk, s, n, 1, nullptr, 0, W, RP, rinv, nullptr, 0, nullptr, 0,
                                      stream);
    RQ_LAUNCH(KID_SMALL_PRECOND, stream,
              k_small_precond<<<1, kSmallThreads, 0, stream>>>(K, ldk, s, n, 1, nullptr, 0, W, RP,
                                                               rinv, nullptr, 0, nullptr, 0));
    return cudaGetLastError();
}

// G + s I with the SCholeskyQR3 shift s = 11 (m n u + n (n+1) u) max_j G_jj
// (||X||_g^2 = max_j ||X_j||^2 = max_j G_jj), written to Gs (ld n).
__global__ void __launch_bounds__(256)
    k_shifted_gram(const double *__restrict__ G, int64_t ldg, int n, int64_t m, double *Gs) {
    __shared__ double red[33];
    double g = 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) g = fmax(g, G[j + int64_t(j) * ldg]);
    for (int off = 16; off > 0; off >>= 1) g = fmax(g, __shfl_down_sync(0xffffffffu, g, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = g;
    __syncthreads();
    if (threadIdx.x == 0) {
        double mx = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, red[w]);
        const double u = 0x1p-53;
        red[32] = 11.0 * (double(m) * double(n) * u + double(n) * double(n + 1) * u) * mx;
    }
    __syncthreads();
    const double shift = red[32];
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int i = idx % n, j = idx / n;
        Gs[idx] = G[i + int64_t(j) * ldg] + (i == j ? shift : 0.0);
    }
}

cudaError_t launch_shifted_gram(const double *G, int64_t ldg, int n, int64_t m, double *Gs,
                                cudaStream_t stream) {
    RQ_LAUNCH(KID_CHOLESKY, stream, k_shifted_gram<<<1, 256, 0, stream>>>(G, ldg, n, m, Gs));
    return cudaGetLastError();
}

cudaError_t launch_rcluppr_r1(const double *Ms, int64_t ldm, int s, int n, const double *LU,
                              int64_t lda, double *W, double *RP, double *rinv,
                              cudaStream_t stream, int r0_method) {
    if (r0_method == 1) {
        if (!precond_cluster_fits(s, n, true)) return cudaErrorNotSupported;
        return launch_precond_cluster(Ms, ldm, s, n, 1 | kPrecondGivens, LU, lda, W, RP, rinv, nullptr, 0,
                                      nullptr, 0, stream);
    }
    if (precond_cluster_fits(s, n))
        return launch_precond_cluster(Ms, ldm, s, n, 1, LU, lda, W, RP, rinv, nullptr, 0, nullptr, 0,
                                      stream);
    RQ_LAUNCH(KID_SMALL_PRECOND, stream, k_small_precond<<<1, kSmallThreads, 0, stream>>>(Ms, ldm, s, n, 1, LU, lda, W, RP, rinv,
                                                     nullptr, 0, nullptr, 0));
    return cudaGetLastError();
}

__global__ void __launch_bounds__(kSmallThreads)
    k_householder_r(const double *__restrict__ A, int64_t lda, int s, int n, double *W, double *R,
                    int64_t ldr) {
    __shared__ double red[36];
    __shared__ double wv[256];
    for (int idx = threadIdx.x; idx < s * n; idx += blockDim.x) {
        const int i = idx % s, j = idx / s;
        W[idx] = A[i + int64_t(j) * lda];
    }
    __syncthreads();
    small_householder(W, s, n, wv, red);
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int i = idx % n, j = idx / n;
        R[i + int64_t(j) * ldr] = (i <= j) ? W[i + int64_t(j) * s] : 0.0;
    }
}

cudaError_t launch_givens_r(const double *A, int64_t lda, int s, int n, double *W, double *RP,
                            double *rinv, double *R, int64_t ldr, cudaStream_t stream) {
    if (!precond_cluster_fits(s, n, true)) return cudaErrorNotSupported;
    return launch_precond_cluster(A, lda, s, n, 1 | kPrecondGivens, nullptr, 0, W, RP, rinv, R, ldr, nullptr,
                                  0, stream);
}

cudaError_t launch_householder_r(const double *A, int64_t lda, int s, int n, double *W, double *R,
                                 int64_t ldr, cudaStream_t stream) {
    RQ_LAUNCH(KID_SMALL_PRECOND, stream, k_householder_r<<<1, kSmallThreads, 0, stream>>>(A, lda, s, n, W, R, ldr));
    return cudaGetLastError();
}

// Upper Cholesky, right-looking: step k takes r_kk = sqrt(w_kk) (breakdown
// if w_kk is not > 0), r_kj = w_kj / r_kk, then w_ij -= r_ki r_kj for
// k < i <= j -- the same subtractions, in the same order, as the column
// formula r_ij = (g_ij - sum_{k<i} r_ki r_kj) / r_ii.
__global__ void __launch_bounds__(kSmallThreads)
    k_cholesky(const double *__restrict__ G, int64_t ldg, int n, double *W, double *RP,
               double *rinv, double *R, int64_t ldr, DevStatus *st, int step) {
    __shared__ int fail;
    __shared__ double rkk_sh;
    const int n_pad = pad16(n);
    if (threadIdx.x == 0) fail = 0;
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int i = idx % n, j = idx / n;
        W[idx] = (i <= j) ? G[i + int64_t(j) * ldg] : 0.0;
    }
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        const double d = W[k + int64_t(k) * n];
        if (!(d > 0.0)) {
            if (threadIdx.x == 0) report(st, kErrCholBreakdown, step, k);
            fail = 1;
            break;
        }
        if (threadIdx.x == 0) rkk_sh = sqrt(d);
        __syncthreads();
        const double rkk = rkk_sh;
        for (int j = k + 1 + threadIdx.x; j < n; j += blockDim.x)
            W[k + int64_t(j) * n] = W[k + int64_t(j) * n] / rkk;
        if (threadIdx.x == 0) W[k + int64_t(k) * n] = rkk;
        __syncthreads();
        const int nt = n - k - 1;
        for (int idx = threadIdx.x; idx < nt * nt; idx += blockDim.x) {
            const int i = k + 1 + idx % nt, j = k + 1 + idx / nt;
            if (i <= j)
                W[i + int64_t(j) * n] =
                    fma(-W[k + int64_t(i) * n], W[k + int64_t(j) * n], W[i + int64_t(j) * n]);
        }
        __syncthreads();
    }
    __syncthreads();
    // padded output (NaN-free even after a breakdown: entries are only copied)
    for (int idx = threadIdx.x; idx < n_pad * n_pad; idx += blockDim.x) {
        const int i = idx % n_pad, j = idx / n_pad;
        const double v = (i <= j && j < n) ? W[i + int64_t(j) * n] : 0.0;
        RP[idx] = v;
        RP[int64_t(n_pad) * n_pad + int64_t(i) * n_pad + j] = v;  // row-major copy
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n_pad; i += blockDim.x)
        rinv[i] = (i < n && !fail) ? 1.0 / RP[i + int64_t(i) * n_pad] : 0.0;
    if (R != nullptr) copy_out_upper(RP, n, n_pad, R, ldr);
}

cudaError_t launch_cholesky(const double *G, int64_t ldg, int n, double *W, double *RP,
                            double *rinv, double *R, int64_t ldr, DevStatus *st, int step_id,
                            cudaStream_t stream) {
    if (cholesky_cluster_fits(n))
        return launch_cholesky_cluster(G, ldg, n, RP, rinv, R, ldr, st, step_id, stream);
    RQ_LAUNCH(KID_CHOLESKY, stream, k_cholesky<<<1, kSmallThreads, 0, stream>>>(G, ldg, n, W, RP, rinv, R, ldr, st, step_id));
    return cudaGetLastError();
}

// C = triu(A) triu(B) (n x n), C written with zeros below the diagonal.
__global__ void k_trmm_upper(const double *__restrict__ A, int64_t lda,
                             const double *__restrict__ B, int64_t ldb, int n, double *C,
                             int64_t ldc) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= int64_t(n) * n) return;
    const int i = static_cast<int>(e % n), j = static_cast<int>(e / n);
    double acc = 0.0;
    if (i <= j)
        for (int t = i; t <= j; ++t) acc = fma(A[i + int64_t(t) * lda], B[t + int64_t(j) * ldb], acc);
    C[i + int64_t(j) * ldc] = acc;
}

cudaError_t launch_trmm_upper(const double *A, int64_t lda, const double *B, int64_t ldb, int n,
                              double *C, int64_t ldc, cudaStream_t stream) {
    const int64_t ne = int64_t(n) * n;
    RQ_LAUNCH(KID_TRMM, stream, k_trmm_upper<<<static_cast<unsigned>(ceil_div(ne, 256)), 256, 0, stream>>>(A, lda, B, ldb, n, C,
                                                                              ldc));
    return cudaGetLastError();
}

// LC2: R1 = Sc N (Sc padded, N = top of the in-place LU), signs normalised.
__global__ void __launch_bounds__(kSmallThreads)
    k_lc2_r1(const double *__restrict__ Sc, int64_t lds, const double *__restrict__ LU,
             int64_t lda, int n, double *RP, double *rinv) {
    __shared__ int sgn[256];
    small_trmm_to_padded(Sc, lds, LU, lda, n, pad16(n), RP, rinv, true, sgn);
}

cudaError_t launch_lc2_r1(const double *Sc, int64_t lds, const double *LU, int64_t lda, int n,
                          double *RP, double *rinv, cudaStream_t stream) {
    RQ_LAUNCH(KID_TRMM, stream, k_lc2_r1<<<1, kSmallThreads, 0, stream>>>(Sc, lds, LU, lda, n, RP, rinv));
    return cudaGetLastError();
}

}  // namespace rq
