/*
 * Plain FP64 CPU oracle for randomized CholeskyQR with LU partial pivoting
 * (RCLUPP, RCLUPPr) and the side-by-side paths CholeskyQR2 and LC2, with the
 * generated sketches (Gaussian, sparse-sign, subsampled randomized Hadamard).
 *
 * TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg may load this library.
 * It shares no code, header, table or helper with the CUDA library.
 *
 * Conventions
 *   - Column-major storage: element (i, j) of an m x n matrix A with leading
 *     dimension lda >= m is A[i + j*lda].
 *   - All arithmetic is IEEE binary64 with round-to-nearest; this file is
 *     compiled with -ffp-contract=off so that no multiply-add is fused.
 *   - Every sum is accumulated sequentially in increasing index order.
 *     OpenMP is used only across independent outputs (columns of a Gram,
 *     rows of a triangular solve, entries of a sketch), never inside a sum.
 *   - Unit roundoff u = 2^-53 (the paper's setting, Section 1).
 *
 * Each routine names the passage of the paper it follows (the algorithm and
 * the operation in it, or the equation).  The readings taken where the paper
 * is silent are:
 *   - LU "[M,N,P] = LU(.)" is Gaussian elimination with partial pivoting,
 *     LAPACK getf2 layout: M unit lower trapezoidal (strict lower part stored),
 *     N upper triangular, P as a sequence of row interchanges ipiv[k] (row k
 *     swapped with row ipiv[k] >= k, 0-based).  The pivot is the first row of
 *     largest magnitude in the column (smallest index on ties).  A zero pivot
 *     means rank < n and is reported, not divided by.
 *   - "HouseholderQR(L)" in Algorithms 6 and 7 is read as HouseholderQR(M)
 *     (resp. of M_s); only its R-factor is used downstream.  Reflectors use
 *     the LAPACK larfg convention: beta = -sign(alpha) * ||x||, sign(0) = +1,
 *     and no reflection (tau = 0) when the part below the diagonal is zero.
 *   - The R-factor's diagonal signs are normalised after R1 = R0 N (and after
 *     R1 = S N in LC2): rows of R1 whose diagonal entry is negative are negated.
 *     This is exact and makes the computed R positive-diagonal, so Q and R are
 *     the unique thin QR factors.
 *   - R = Z R1 is evaluated as in the proof of Theorem 4.1 (C4, C8):
 *     R3 = R2 R1, then R = R4 R3.
 *   - LC2 applies one CholeskyQR after the LU + Cholesky preconditioner, as
 *     its algorithm box states (Algorithm 4), although it is named "2".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_CHOL_BREAKDOWN (-2)
#define ORC_LU_ZERO_PIVOT (-3)
#define ORC_ERR_NOMEM (-7)

#define IDX(A, ld, i, j) ((A)[(int64_t)(i) + (int64_t)(j) * (int64_t)(ld)])

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads for the following calls (k >= 1); a timing aid, no arithmetic. */
void orc_set_num_threads(int k)
{
#ifdef _OPENMP
    if (k >= 1)
        omp_set_num_threads(k);
#else
    (void)k;
#endif
}

/* ------------------------------------------------------------------------ */
/* Dense building blocks                                                     */
/* ------------------------------------------------------------------------ */

/* G = X^T X (the Gram product of Algorithm 1; C1 and C5 in the proof of
 * Theorem 4.1).
 * G is n x n with leading dimension ldg; both triangles are written. */
void orc_gram(int64_t m, int64_t n, const double *X, int64_t ldx, double *G, int64_t ldg)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t j = 0; j < n; ++j) {
        const double *xj = X + j * ldx;
        for (int64_t k = 0; k <= j; ++k) {
            const double *xk = X + k * ldx;
            double acc = 0.0;
            for (int64_t i = 0; i < m; ++i)
                acc += xk[i] * xj[i];
            IDX(G, ldg, k, j) = acc;
            IDX(G, ldg, j, k) = acc;
        }
    }
}

/* Upper Cholesky factor R of a symmetric positive definite G = R^T R
 * (Algorithm 1; C2 and C6).  Column-by-column: for column j,
 *   R[i][j] = (G[i][j] - sum_{k<i} R[k][i] R[k][j]) / R[i][i],   i < j
 *   R[j][j] = sqrt(G[j][j] - sum_{k<j} R[k][j]^2).
 * Returns ORC_OK, or ORC_CHOL_BREAKDOWN with *info = j when the radicand of
 * column j is not positive (or not a number).  The strict lower triangle of
 * R is set to zero. */
int orc_cholesky(int64_t n, const double *G, int64_t ldg, double *R, int64_t ldr, int64_t *info)
{
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = j + 1; i < n; ++i)
            IDX(R, ldr, i, j) = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        for (int64_t i = 0; i < j; ++i) {
            double acc = IDX(G, ldg, i, j);
            for (int64_t k = 0; k < i; ++k)
                acc -= IDX(R, ldr, k, i) * IDX(R, ldr, k, j);
            IDX(R, ldr, i, j) = acc / IDX(R, ldr, i, i);
        }
        double d = IDX(G, ldg, j, j);
        for (int64_t k = 0; k < j; ++k)
            d -= IDX(R, ldr, k, j) * IDX(R, ldr, k, j);
        if (!(d > 0.0)) {
            if (info)
                *info = j;
            return ORC_CHOL_BREAKDOWN;
        }
        IDX(R, ldr, j, j) = sqrt(d);
    }
    if (info)
        *info = -1;
    return ORC_OK;
}

/* Q = X R^{-1} for upper-triangular R (the solve of Algorithm 1; eq. (es) row E_e,
 * C3 and C7).  Row-wise forward substitution:
 *   q_ij = (x_ij - sum_{k<j} q_ik r_kj) / r_jj.
 * Q may alias X (the solve is row-local and reads x_ij before writing q_ij). */
void orc_trsm_right_upper(int64_t m, int64_t n, const double *X, int64_t ldx,
                          const double *R, int64_t ldr, double *Q, int64_t ldq)
{
#pragma omp parallel
    {
        double *row = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
#pragma omp for schedule(static)
        for (int64_t i = 0; i < m; ++i) {
            for (int64_t j = 0; j < n; ++j) {
                double acc = IDX(X, ldx, i, j);
                for (int64_t k = 0; k < j; ++k)
                    acc -= row[k] * IDX(R, ldr, k, j);
                row[j] = acc / IDX(R, ldr, j, j);
            }
            for (int64_t j = 0; j < n; ++j)
                IDX(Q, ldq, i, j) = row[j];
        }
        free(row);
    }
}

/* C = A B for upper-triangular n x n A and B (eq. (ey), C4, C8):
 *   C[i][j] = sum_{k=i..j} A[i][k] B[k][j] for i <= j, 0 below the diagonal. */
void orc_trmm_upper(int64_t n, const double *A, int64_t lda, const double *B, int64_t ldb,
                    double *C, int64_t ldc)
{
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < n; ++i) {
            double acc = 0.0;
            if (i <= j)
                for (int64_t k = i; k <= j; ++k)
                    acc += IDX(A, lda, i, k) * IDX(B, ldb, k, j);
            IDX(C, ldc, i, j) = acc;
        }
}

/* Gaussian elimination with partial pivoting, in place (the LU step of
 * Algorithms 4, 6 and 7; error model eq. (elu)).  On return the strict lower
 * part of A holds M (unit diagonal implied) and the upper triangle holds N;
 * ipiv[k] is the (0-based) row swapped with row k at step k.
 * For k = 0..n-1:
 *   p = first argmax_{i>=k} |A[i][k]|; swap rows k and p (all n columns);
 *   A[i][k] /= A[k][k] for i > k;  A[i][j] -= A[i][k] A[k][j] for i, j > k.
 * Returns ORC_LU_ZERO_PIVOT (*info = k) when the pivot is zero. */
int orc_gepp(int64_t m, int64_t n, double *A, int64_t lda, int32_t *ipiv, int64_t *info)
{
    int64_t kmax = m < n ? m : n;
    for (int64_t k = 0; k < kmax; ++k) {
        int64_t p = k;
        double best = fabs(IDX(A, lda, k, k));
        for (int64_t i = k + 1; i < m; ++i) {
            double v = fabs(IDX(A, lda, i, k));
            if (v > best) {
                best = v;
                p = i;
            }
        }
        ipiv[k] = (int32_t)p;
        if (best == 0.0) {
            if (info)
                *info = k;
            return ORC_LU_ZERO_PIVOT;
        }
        if (p != k)
            for (int64_t j = 0; j < n; ++j) {
                double t = IDX(A, lda, k, j);
                IDX(A, lda, k, j) = IDX(A, lda, p, j);
                IDX(A, lda, p, j) = t;
            }
        double piv = IDX(A, lda, k, k);
        for (int64_t i = k + 1; i < m; ++i)
            IDX(A, lda, i, k) = IDX(A, lda, i, k) / piv;
#pragma omp parallel for schedule(static) if (m - k > 4096)
        for (int64_t j = k + 1; j < n; ++j) {
            double ukj = IDX(A, lda, k, j);
            for (int64_t i = k + 1; i < m; ++i)
                IDX(A, lda, i, j) -= IDX(A, lda, i, k) * ukj;
        }
    }
    if (info)
        *info = -1;
    return ORC_OK;
}

/* Copy the unit-lower trapezoidal factor M (m x n) out of an in-place GEPP
 * result: M[i][j] = A[i][j] for i > j, 1 for i == j, 0 for i < j. */
void orc_extract_unit_lower(int64_t m, int64_t n, const double *A, int64_t lda, double *M, int64_t ldm)
{
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < m; ++i)
            IDX(M, ldm, i, j) = i > j ? IDX(A, lda, i, j) : (i == j ? 1.0 : 0.0);
}

/* Copy the upper-triangular factor N (n x n) out of an in-place GEPP result. */
void orc_extract_upper(int64_t n, const double *A, int64_t lda, double *N, int64_t ldn)
{
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < n; ++i)
            IDX(N, ldn, i, j) = i <= j ? IDX(A, lda, i, j) : 0.0;
}

/* R-factor of the thin Householder QR of A (s x n, s >= n), A unchanged
 * (R0 in Algorithms 5, 6 and 7; eq. (eh)).
 * For k = 0..n-1 on the working copy W:
 *   alpha = W[k][k], sigma = sum_{i>k} W[i][k]^2;
 *   if sigma == 0: no reflection, R[k][k] = alpha;
 *   else beta = -sign(alpha) sqrt(alpha^2 + sigma) (sign(0) = +1),
 *        tau = (beta - alpha)/beta, v = (1, W[k+1..][k] / (alpha - beta)),
 *        W[k..][j] -= tau v (v^T W[k..][j]) for j > k, R[k][k] = beta.
 * R's row k is then W[k][k..n-1].  Strict lower triangle of R is zero. */
void orc_householder_r(int64_t s, int64_t n, const double *A, int64_t lda, double *R, int64_t ldr)
{
    double *W = (double *)malloc(sizeof(double) * (size_t)s * (size_t)n);
    double *v = (double *)malloc(sizeof(double) * (size_t)s);
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < s; ++i)
            W[i + j * s] = IDX(A, lda, i, j);
    for (int64_t k = 0; k < n; ++k) {
        double alpha = W[k + k * s];
        double sigma = 0.0;
        for (int64_t i = k + 1; i < s; ++i)
            sigma += W[i + k * s] * W[i + k * s];
        if (sigma == 0.0) {
            continue; /* H_k = I, R[k][k] = alpha */
        }
        double norm = sqrt(alpha * alpha + sigma);
        double beta = alpha >= 0.0 ? -norm : norm;
        double tau = (beta - alpha) / beta;
        double scal = 1.0 / (alpha - beta);
        v[k] = 1.0;
        for (int64_t i = k + 1; i < s; ++i)
            v[i] = W[i + k * s] * scal;
        W[k + k * s] = beta;
        for (int64_t i = k + 1; i < s; ++i)
            W[i + k * s] = 0.0;
        for (int64_t j = k + 1; j < n; ++j) {
            double w = 0.0;
            for (int64_t i = k; i < s; ++i)
                w += v[i] * W[i + j * s];
            double tw = tau * w;
            for (int64_t i = k; i < s; ++i)
                W[i + j * s] -= v[i] * tw;
        }
    }
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < n; ++i)
            IDX(R, ldr, i, j) = i <= j ? W[i + j * s] : 0.0;
    free(v);
    free(W);
}

/* R-factor of A (s x n, s >= n) by Givens rotations, the alternative to the
 * thin HouseholderQR that Section 1 and the remark after Algorithm 5 allow
 * for the preconditioning step.  Column by column (k = 0..n-1), the entries
 * below the diagonal are annihilated from the bottom up: rows (i-1, i) for
 * i = s-1 down to k+1 are rotated by
 *     [ c  s' ] [ a ]   [ r ]
 *     [-s' c  ] [ b ] = [ 0 ],   r = hypot(a, b), c = a / r, s' = b / r,
 * (no rotation when b = 0), applied to columns k+1..n-1 of the two rows;
 * column k becomes (r, 0).
 * r >= 0, so the diagonal is non-negative wherever the column below it was
 * not already zero.  R = the upper n x n part. */
void orc_givens_r(int64_t s, int64_t n, const double *A, int64_t lda, double *R, int64_t ldr)
{
    double *W = (double *)malloc(sizeof(double) * (size_t)s * (size_t)n);
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < s; ++i)
            W[i + j * s] = IDX(A, lda, i, j);
    for (int64_t k = 0; k < n; ++k) {
        for (int64_t i = s - 1; i > k; --i) {
            double a = W[(i - 1) + k * s], b = W[i + k * s];
            if (b == 0.0)
                continue;
            double r = hypot(a, b);
            double c = a / r, sn = b / r;
            for (int64_t j = k + 1; j < n; ++j) {
                double x = W[(i - 1) + j * s], y = W[i + j * s];
                W[(i - 1) + j * s] = c * x + sn * y;
                W[i + j * s] = c * y - sn * x;
            }
            W[(i - 1) + k * s] = r;
            W[i + k * s] = 0.0;
        }
    }
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < n; ++i)
            IDX(R, ldr, i, j) = i <= j ? W[i + j * s] : 0.0;
    free(W);
}

/* R-factor methods of the preconditioning step. */
#define ORC_R0_HOUSEHOLDER 0
#define ORC_R0_GIVENS 1

static void orc_r0(int method, int64_t s, int64_t n, const double *A, int64_t lda, double *R,
                   int64_t ldr)
{
    if (method == ORC_R0_GIVENS)
        orc_givens_r(s, n, A, lda, R, ldr);
    else
        orc_householder_r(s, n, A, lda, R, ldr);
}

/* Y = S X with an explicit dense sketch S (s x m, leading dimension lds)
 * (S X in Algorithm 6, S M in Algorithm 7; eq. (es)).
 * Y[r][j] = sum_{i=0..m-1} S[r][i] X[i][j], summed in increasing i. */
void orc_sketch_dense(int64_t s, int64_t m, int64_t n, const double *S, int64_t lds,
                      const double *X, int64_t ldx, double *Y, int64_t ldy)
{
    /* Column j of Y is owned by one thread; i runs outermost so that column i
     * of S is read contiguously.  Each Y[r][j] still receives its terms in
     * increasing i, one rounding per term, exactly as in the formula. */
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) {
        const double *xj = X + j * ldx;
        for (int64_t r = 0; r < s; ++r)
            IDX(Y, ldy, r, j) = 0.0;
        for (int64_t i = 0; i < m; ++i) {
            const double x = xj[i];
            const double *si = S + i * lds;
            for (int64_t r = 0; r < s; ++r)
                IDX(Y, ldy, r, j) += si[r] * x;
        }
    }
}

/* Y = S X for a sparse-sign sketch given column by column: column i of S has
 * nonzeros at rows rows[i*zeta + t] with values signs[i*zeta + t] / sqrt(zeta)
 * (t = 0..zeta-1, distinct rows).  Y[r][j] = sum_i S[r][i] X[i][j] in
 * increasing i, the same definition as orc_sketch_dense. */
void orc_sketch_sparse(int64_t s, int64_t m, int64_t n, int zeta, const int32_t *rows,
                       const int8_t *signs, const double *X, int64_t ldx, double *Y, int64_t ldy)
{
    double val = 1.0 / sqrt((double)zeta);
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) {
        for (int64_t r = 0; r < s; ++r)
            IDX(Y, ldy, r, j) = 0.0;
        const double *xj = X + j * ldx;
        for (int64_t i = 0; i < m; ++i)
            for (int t = 0; t < zeta; ++t) {
                int64_t r = rows[i * zeta + t];
                double sv = signs[i * zeta + t] > 0 ? val : -val;
                IDX(Y, ldy, r, j) += sv * xj[i];
            }
    }
}

/* Negate every row of the upper-triangular R whose diagonal entry is
 * negative (the sign normalisation applied to R1; exact). */
static void orc_sign_fix_rows(int64_t n, double *R, int64_t ldr)
{
    for (int64_t i = 0; i < n; ++i)
        if (IDX(R, ldr, i, i) < 0.0)
            for (int64_t j = i; j < n; ++j)
                IDX(R, ldr, i, j) = -IDX(R, ldr, i, j);
}

/* ------------------------------------------------------------------------ */
/* Algorithm drivers                                                         */
/* ------------------------------------------------------------------------ */

/* [Q, R] = CholeskyQR(X) (Algorithm 1). */
int orc_cholqr(int64_t m, int64_t n, const double *X, int64_t ldx, double *Q, int64_t ldq,
               double *R, int64_t ldr, int64_t *info)
{
    double *G = (double *)malloc(sizeof(double) * (size_t)n * (size_t)n);
    if (!G)
        return ORC_ERR_NOMEM;
    orc_gram(m, n, X, ldx, G, n);
    int st = orc_cholesky(n, G, n, R, ldr, info);
    if (st == ORC_OK)
        orc_trsm_right_upper(m, n, X, ldx, R, ldr, Q, ldq);
    free(G);
    return st;
}

/* [Q, R] = CholeskyQR2(X) (Algorithm 2): CholeskyQR of X gives (Q1, R1),
 * CholeskyQR of Q1 gives (Q, Z), then R = Z R1. */
int orc_cholqr2(int64_t m, int64_t n, const double *X, int64_t ldx, double *Q, int64_t ldq,
                double *R, int64_t ldr, int64_t *info)
{
    double *Q1 = (double *)malloc(sizeof(double) * (size_t)m * (size_t)n);
    double *R1 = (double *)malloc(sizeof(double) * (size_t)n * (size_t)n);
    double *Z = (double *)malloc(sizeof(double) * (size_t)n * (size_t)n);
    int st = ORC_ERR_NOMEM;
    if (Q1 && R1 && Z) {
        st = orc_cholqr(m, n, X, ldx, Q1, m, R1, n, info);
        if (st == ORC_OK) {
            st = orc_cholqr(m, n, Q1, m, Q, ldq, Z, n, info);
            if (st == ORC_OK)
                orc_trmm_upper(n, Z, n, R1, n, R, ldr);
        }
    }
    free(Z);
    free(R1);
    free(Q1);
    return st;
}

/* Steps shared by RCLUPP and RCLUPPr after R1 is known (the CholeskyQR2 of
 * Q1 in Algorithm 6, evaluated as C1..C8 of the proof of Theorem 4.1):
 *   Q1 = X R1^{-1}; G = Q1^T Q1; R2 = chol(G); Q2 = Q1 R2^{-1}; R3 = R2 R1;
 *   G1 = Q2^T Q2; R4 = chol(G1); Q = Q2 R4^{-1}; R = R4 R3.
 * *info encodes the failing Cholesky as 100000*pass + column (pass 1 or 2). */
static int orc_precond_then_cholqr2(int64_t m, int64_t n, const double *X, int64_t ldx,
                                    const double *R1, double *Q, int64_t ldq, double *R,
                                    int64_t ldr, int64_t *info)
{
    size_t mn = (size_t)m * (size_t)n, nn = (size_t)n * (size_t)n;
    double *Q1 = (double *)malloc(sizeof(double) * mn);
    double *Q2 = (double *)malloc(sizeof(double) * mn);
    double *G = (double *)malloc(sizeof(double) * nn);
    double *R2 = (double *)malloc(sizeof(double) * nn);
    double *R3 = (double *)malloc(sizeof(double) * nn);
    double *R4 = (double *)malloc(sizeof(double) * nn);
    int st = ORC_ERR_NOMEM;
    int64_t col = -1;
    if (Q1 && Q2 && G && R2 && R3 && R4) {
        orc_trsm_right_upper(m, n, X, ldx, R1, n, Q1, m);          /* Q1 = X R1^-1   */
        orc_gram(m, n, Q1, m, G, n);                                /* C1             */
        st = orc_cholesky(n, G, n, R2, n, &col);                    /* C2             */
        if (st != ORC_OK) {
            if (info)
                *info = 100000 + col;
        } else {
            orc_trsm_right_upper(m, n, Q1, m, R2, n, Q2, m);        /* C3             */
            orc_trmm_upper(n, R2, n, R1, n, R3, n);                 /* C4             */
            orc_gram(m, n, Q2, m, G, n);                            /* C5             */
            st = orc_cholesky(n, G, n, R4, n, &col);                /* C6             */
            if (st != ORC_OK) {
                if (info)
                    *info = 200000 + col;
            } else {
                orc_trsm_right_upper(m, n, Q2, m, R4, n, Q, ldq);   /* C7             */
                orc_trmm_upper(n, R4, n, R3, n, R, ldr);            /* C8             */
                if (info)
                    *info = -1;
            }
        }
    }
    free(R4);
    free(R3);
    free(R2);
    free(G);
    free(Q2);
    free(Q1);
    return st;
}

/* R1 from a sketched s x n matrix Y (the preconditioner of Algorithm 6):
 *   [M, N, P] = LU(Y); R0 = R-factor of HouseholderQR(M); R1 = R0 N;
 * then the diagonal sign normalisation of R1.  Y is not modified. */
int orc_sketch_precond(int64_t s, int64_t n, const double *Y, int64_t ldy, double *R1,
                       int64_t ldr, int64_t *info, int r0_method)
{
    double *A = (double *)malloc(sizeof(double) * (size_t)s * (size_t)n);
    double *M = (double *)malloc(sizeof(double) * (size_t)s * (size_t)n);
    double *N = (double *)malloc(sizeof(double) * (size_t)n * (size_t)n);
    double *R0 = (double *)malloc(sizeof(double) * (size_t)n * (size_t)n);
    int32_t *ipiv = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int st = ORC_ERR_NOMEM;
    if (A && M && N && R0 && ipiv) {
        for (int64_t j = 0; j < n; ++j)
            for (int64_t i = 0; i < s; ++i)
                A[i + j * s] = IDX(Y, ldy, i, j);
        st = orc_gepp(s, n, A, s, ipiv, info);
        if (st == ORC_OK) {
            orc_extract_unit_lower(s, n, A, s, M, s);
            orc_extract_upper(n, A, s, N, n);
            orc_r0(r0_method, s, n, M, s, R0, n);
            orc_trmm_upper(n, R0, n, N, n, R1, ldr);
            orc_sign_fix_rows(n, R1, ldr);
        }
    }
    free(ipiv);
    free(R0);
    free(N);
    free(M);
    free(A);
    return st;
}

/* Sketch kinds accepted by the drivers below. */
#define ORC_SKETCH_DENSE 0  /* explicit dense S (s x m, lds)                  */
#define ORC_SKETCH_SPARSE 1 /* sparse-sign S given by rows/signs (zeta/column) */

static void orc_apply_sketch(int kind, int64_t s, int64_t m, int64_t n, int zeta, const double *S,
                             int64_t lds, const int32_t *rows, const int8_t *signs,
                             const double *A, int64_t lda, double *Y, int64_t ldy)
{
    if (kind == ORC_SKETCH_SPARSE)
        orc_sketch_sparse(s, m, n, zeta, rows, signs, A, lda, Y, ldy);
    else
        orc_sketch_dense(s, m, n, S, lds, A, lda, Y, ldy);
}

/* [Q, R] = RCLUPP(X) (Algorithm 6):
 *   X_s = S X; [M, N, P] = LU(X_s); R0 = R of HouseholderQR(M); R1 = R0 N;
 *   Q1 = X R1^{-1}; [Q, Z] = CholeskyQR2(Q1); R = Z R1.
 * *info: LU failure -> column; Cholesky failure -> 100000*pass + column. */
int orc_rclupp(int64_t m, int64_t n, const double *X, int64_t ldx, int kind, int64_t s, int zeta,
               const double *S, int64_t lds, const int32_t *rows, const int8_t *signs, double *Q,
               int64_t ldq, double *R, int64_t ldr, int64_t *info, int r0_method)
{
    if (m < n || n < 1 || s < n)
        return ORC_ERR_ARG;
    double *Y = (double *)malloc(sizeof(double) * (size_t)s * (size_t)n);
    double *R1 = (double *)malloc(sizeof(double) * (size_t)n * (size_t)n);
    int st = ORC_ERR_NOMEM;
    if (Y && R1) {
        orc_apply_sketch(kind, s, m, n, zeta, S, lds, rows, signs, X, ldx, Y, s);
        st = orc_sketch_precond(s, n, Y, s, R1, n, info, r0_method);
        if (st == ORC_OK)
            st = orc_precond_then_cholqr2(m, n, X, ldx, R1, Q, ldq, R, ldr, info);
    }
    free(R1);
    free(Y);
    return st;
}

/* R1 of RCLUPPr (the preconditioner of Algorithm 7):
 *   [M, N, P] = LU(X); M_s = S M (M in the row order the LU leaves it);
 *   R0 = R-factor of M_s (HouseholderQR, or Givens rotations); R1 = R0 N;
 * then the diagonal sign normalisation of R1.  X is not modified; R1 is
 * n x n with leading dimension ldr.  Returns the LU's status (*info = the
 * column of a zero pivot). */
int orc_rcluppr_precond(int64_t m, int64_t n, const double *X, int64_t ldx, int kind, int64_t s,
                        int zeta, const double *S, int64_t lds, const int32_t *rows,
                        const int8_t *signs, double *R1, int64_t ldr, int64_t *info, int r0_method)
{
    if (m < n || n < 1 || s < n)
        return ORC_ERR_ARG;
    size_t mn = (size_t)m * (size_t)n, nn = (size_t)n * (size_t)n;
    double *A = (double *)malloc(sizeof(double) * mn);
    double *M = (double *)malloc(sizeof(double) * mn);
    double *N = (double *)malloc(sizeof(double) * nn);
    double *Ms = (double *)malloc(sizeof(double) * (size_t)s * (size_t)n);
    double *R0 = (double *)malloc(sizeof(double) * nn);
    int32_t *ipiv = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int st = ORC_ERR_NOMEM;
    if (A && M && N && Ms && R0 && ipiv) {
        for (int64_t j = 0; j < n; ++j)
            memcpy(A + j * m, X + j * ldx, sizeof(double) * (size_t)m);
        st = orc_gepp(m, n, A, m, ipiv, info);
        if (st == ORC_OK) {
            orc_extract_unit_lower(m, n, A, m, M, m);
            orc_extract_upper(n, A, m, N, n);
            orc_apply_sketch(kind, s, m, n, zeta, S, lds, rows, signs, M, m, Ms, s);
            orc_r0(r0_method, s, n, Ms, s, R0, n);
            orc_trmm_upper(n, R0, n, N, n, R1, ldr);
            orc_sign_fix_rows(n, R1, ldr);
        }
    }
    free(ipiv);
    free(R0);
    free(Ms);
    free(N);
    free(M);
    free(A);
    return st;
}

/* [Q, R] = RCLUPPr(X) (Algorithm 7):
 *   [M, N, P] = LU(X); M_s = S M; R0 = R of HouseholderQR(M_s); R1 = R0 N;
 *   Q1 = X R1^{-1}; [Q, Z] = CholeskyQR2(Q1); R = Z R1.
 * M is the m x n unit-lower factor in the row order GEPP leaves it. */
int orc_rcluppr(int64_t m, int64_t n, const double *X, int64_t ldx, int kind, int64_t s, int zeta,
                const double *S, int64_t lds, const int32_t *rows, const int8_t *signs, double *Q,
                int64_t ldq, double *R, int64_t ldr, int64_t *info, int r0_method)
{
    if (m < n || n < 1 || s < n)
        return ORC_ERR_ARG;
    double *R1 = (double *)malloc(sizeof(double) * (size_t)n * (size_t)n);
    int st = ORC_ERR_NOMEM;
    if (R1) {
        st = orc_rcluppr_precond(m, n, X, ldx, kind, s, zeta, S, lds, rows, signs, R1, n, info,
                                 r0_method);
        if (st == ORC_OK)
            st = orc_precond_then_cholqr2(m, n, X, ldx, R1, Q, ldq, R, ldr, info);
    }
    free(R1);
    return st;
}

/* [Q, R] = LC2(X) (Algorithm 4):
 *   [M, N, P] = LU(X); G = M^T M; S = chol(G); R1 = S N;
 *   Q1 = X R1^{-1}; [Q, Z] = CholeskyQR(Q1); R = Z R1.
 * R1's diagonal signs are normalised as in RCLUPP. */
int orc_lc2(int64_t m, int64_t n, const double *X, int64_t ldx, double *Q, int64_t ldq, double *R,
            int64_t ldr, int64_t *info)
{
    if (m < n || n < 1)
        return ORC_ERR_ARG;
    size_t mn = (size_t)m * (size_t)n, nn = (size_t)n * (size_t)n;
    double *A = (double *)malloc(sizeof(double) * mn);
    double *M = (double *)malloc(sizeof(double) * mn);
    double *Q1 = (double *)malloc(sizeof(double) * mn);
    double *N = (double *)malloc(sizeof(double) * nn);
    double *G = (double *)malloc(sizeof(double) * nn);
    double *Sc = (double *)malloc(sizeof(double) * nn);
    double *R1 = (double *)malloc(sizeof(double) * nn);
    double *Z = (double *)malloc(sizeof(double) * nn);
    int32_t *ipiv = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int st = ORC_ERR_NOMEM;
    int64_t col = -1;
    if (A && M && Q1 && N && G && Sc && R1 && Z && ipiv) {
        for (int64_t j = 0; j < n; ++j)
            memcpy(A + j * m, X + j * ldx, sizeof(double) * (size_t)m);
        st = orc_gepp(m, n, A, m, ipiv, info);
        if (st == ORC_OK) {
            orc_extract_unit_lower(m, n, A, m, M, m);
            orc_extract_upper(n, A, m, N, n);
            orc_gram(m, n, M, m, G, n);
            st = orc_cholesky(n, G, n, Sc, n, &col);
            if (st != ORC_OK) {
                if (info)
                    *info = 100000 + col;
            } else {
                orc_trmm_upper(n, Sc, n, N, n, R1, n);
                orc_sign_fix_rows(n, R1, n);
                orc_trsm_right_upper(m, n, X, ldx, R1, n, Q1, m);
                orc_gram(m, n, Q1, m, G, n);
                st = orc_cholesky(n, G, n, Z, n, &col);
                if (st != ORC_OK) {
                    if (info)
                        *info = 200000 + col;
                } else {
                    orc_trsm_right_upper(m, n, Q1, m, Z, n, Q, ldq);
                    orc_trmm_upper(n, Z, n, R1, n, R, ldr);
                    if (info)
                        *info = -1;
                }
            }
        }
    }
    free(ipiv);
    free(Z);
    free(R1);
    free(Sc);
    free(G);
    free(N);
    free(Q1);
    free(M);
    free(A);
    return st;
}

/* [Q, R] = RCholeskyQR(X) (Algorithm 5, single sketch):
 *   K = S X; R1 = R-factor of HouseholderQR(K) (diagonal signs normalised);
 *   Q1 = X R1^{-1}; [Q, Z] = CholeskyQR(Q1); R = Z R1. */
int orc_rcholqr(int64_t m, int64_t n, const double *X, int64_t ldx, int kind, int64_t s, int zeta,
                const double *S, int64_t lds, const int32_t *rows, const int8_t *signs, double *Q,
                int64_t ldq, double *R, int64_t ldr, int64_t *info, int r0_method)
{
    if (m < n || n < 1 || s < n)
        return ORC_ERR_ARG;
    size_t mn = (size_t)m * (size_t)n, nn = (size_t)n * (size_t)n;
    double *K = (double *)malloc(sizeof(double) * (size_t)s * (size_t)n);
    double *R1 = (double *)malloc(sizeof(double) * nn);
    double *Q1 = (double *)malloc(sizeof(double) * mn);
    double *G = (double *)malloc(sizeof(double) * nn);
    double *Z = (double *)malloc(sizeof(double) * nn);
    int st = ORC_ERR_NOMEM;
    int64_t col = -1;
    if (K && R1 && Q1 && G && Z) {
        orc_apply_sketch(kind, s, m, n, zeta, S, lds, rows, signs, X, ldx, K, s);
        orc_r0(r0_method, s, n, K, s, R1, n);
        orc_sign_fix_rows(n, R1, n);
        orc_trsm_right_upper(m, n, X, ldx, R1, n, Q1, m);
        orc_gram(m, n, Q1, m, G, n);
        st = orc_cholesky(n, G, n, Z, n, &col);
        if (st != ORC_OK) {
            if (info)
                *info = 100000 + col;
        } else {
            orc_trsm_right_upper(m, n, Q1, m, Z, n, Q, ldq);
            orc_trmm_upper(n, Z, n, R1, n, R, ldr);
            if (info)
                *info = -1;
        }
    }
    free(Z);
    free(G);
    free(Q1);
    free(R1);
    free(K);
    return st;
}

/* Shift of SCholeskyQR3 (Section 2.2): s = 11 (m n u + n (n+1) u) ||X||_g^2
 * with ||X||_g = max_j ||X_j||_2 (Definition 2.1), ||X_j||_2^2 = G_jj. */
double orc_scholqr3_shift(int64_t m, int64_t n, const double *G, int64_t ldg)
{
    const double u = 0x1p-53;
    double g = 0.0;
    for (int64_t j = 0; j < n; ++j)
        if (IDX(G, ldg, j, j) > g)
            g = IDX(G, ldg, j, j);
    return 11.0 * ((double)m * (double)n * u + (double)n * (double)(n + 1) * u) * g;
}

/* [Q, R] = SCholeskyQR3(X) (Algorithm 3): G = X^T X; R1 = chol(G + s I);
 * Q1 = X R1^{-1}; [Q, Z] = CholeskyQR2(Q1); R = Z R1, evaluated like the
 * randomized drivers (R3 = R2 R1, R = R4 R3). */
int orc_scholqr3(int64_t m, int64_t n, const double *X, int64_t ldx, double *Q, int64_t ldq,
                 double *R, int64_t ldr, int64_t *info)
{
    if (m < n || n < 1)
        return ORC_ERR_ARG;
    size_t nn = (size_t)n * (size_t)n;
    double *G = (double *)malloc(sizeof(double) * nn);
    double *R1 = (double *)malloc(sizeof(double) * nn);
    int st = ORC_ERR_NOMEM;
    int64_t col = -1;
    if (G && R1) {
        orc_gram(m, n, X, ldx, G, n);
        const double shift = orc_scholqr3_shift(m, n, G, n);
        for (int64_t j = 0; j < n; ++j)
            IDX(G, n, j, j) += shift;
        st = orc_cholesky(n, G, n, R1, n, &col);
        if (st != ORC_OK) {
            if (info)
                *info = col;
        } else {
            st = orc_precond_then_cholqr2(m, n, X, ldx, R1, Q, ldq, R, ldr, info);
        }
    }
    free(R1);
    free(G);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Counter-based sketch generators                                           */
/*                                                                          */
/* When the sketch is generated on the fly, both sides implement the same   */
/* published generator independently:                                       */
/*   Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers:   */
/*   as easy as 1, 2, 3", SC'11): 10 rounds, multipliers 0xD2511F53 and     */
/*   0xCD9E8D57, key increments 0x9E3779B9 and 0xBB67AE85.                   */
/* The Gaussian entries use the Box-Muller transform (Box & Muller 1958)    */
/* evaluated in binary32 with a logarithm and a sine/cosine defined below   */
/* by truncated series (only correctly rounded +, -, *, /, sqrt), so the    */
/* entries are reproducible bit for bit on any IEEE platform.               */
/* ------------------------------------------------------------------------ */

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0;
        c1 = n1;
        c2 = n2;
        c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

static float orc_f32_bits(uint32_t b)
{
    float f;
    memcpy(&f, &b, sizeof f);
    return f;
}

static uint32_t orc_bits_f32(float f)
{
    uint32_t b;
    memcpy(&b, &f, sizeof b);
    return b;
}

/* Natural logarithm of a normal binary32 x > 0, defined as
 *   x = 2^e f with f in (sqrt(2)/2, sqrt(2)],  t = (f - 1)/(f + 1),
 *   ln x = e ln2 + 2 t (1 + t^2/3 + t^4/5 + t^6/7 + t^8/9 + t^10/11)
 * (the atanh series; |t| <= 0.1716), Horner order, every operation rounded. */
float orc_ln_f32(float x)
{
    uint32_t b = orc_bits_f32(x);
    int e = (int)((b >> 23) & 0xffu) - 127;
    float f = orc_f32_bits((b & 0x7fffffu) | 0x3f800000u);
    if (f > 0x1.6a09e6p+0f) {
        f = f * 0.5f;
        e += 1;
    }
    float t = (f - 1.0f) / (f + 1.0f);
    float t2 = t * t;
    float p = 0x1.745d18p-4f;      /* 1/11 */
    p = p * t2 + 0x1.c71c72p-4f;   /* 1/9  */
    p = p * t2 + 0x1.24924ap-3f;   /* 1/7  */
    p = p * t2 + 0x1.99999ap-3f;   /* 1/5  */
    p = p * t2 + 0x1.555556p-2f;   /* 1/3  */
    p = p * t2 + 1.0f;
    float lnf = (2.0f * t) * p;
    return (float)e * 0x1.62e430p-1f + lnf; /* ln 2 */
}

/* cos(2 pi u) and sin(2 pi u) for binary32 u in [0, 1), defined by
 *   v = 4u, q = floor(v), r = v - q (exact);  a = r if r <= 1/2 else 1 - r;
 *   phi = a * (pi/2);  sin phi and cos phi by their Taylor series to phi^9 and
 *   phi^10 (Horner order); for r > 1/2 the two are exchanged; then the
 *   quadrant q rotates (c, s) -> (c, s), (-s, c), (-c, -s), (s, -c). */
void orc_cossin_2pi_f32(float u, float *cos_out, float *sin_out)
{
    float v = u * 4.0f;
    int q = (int)v;
    float r = v - (float)q;
    int refl = r > 0.5f;
    float a = refl ? (1.0f - r) : r;
    float phi = a * 0x1.921fb6p+0f; /* pi/2 */
    float p2 = phi * phi;
    float sp = 0x1.71de3ap-19f;       /*  1/9!  */
    sp = sp * p2 + -0x1.a01a02p-13f;  /* -1/7!  */
    sp = sp * p2 + 0x1.111112p-7f;    /*  1/5!  */
    sp = sp * p2 + -0x1.555556p-3f;   /* -1/3!  */
    sp = sp * p2 + 1.0f;
    float sn = phi * sp;
    float cp = -0x1.27e4fcp-22f;      /* -1/10! */
    cp = cp * p2 + 0x1.a01a02p-16f;   /*  1/8!  */
    cp = cp * p2 + -0x1.6c16c2p-10f;  /* -1/6!  */
    cp = cp * p2 + 0x1.555556p-5f;    /*  1/4!  */
    cp = cp * p2 + -0.5f;
    cp = cp * p2 + 1.0f;
    float c0 = refl ? sn : cp;
    float s0 = refl ? cp : sn;
    float c, s;
    switch (q & 3) {
    case 0: c = c0; s = s0; break;
    case 1: c = -s0; s = c0; break;
    case 2: c = -c0; s = -s0; break;
    default: c = s0; s = -c0; break;
    }
    *cos_out = c;
    *sin_out = s;
}

/* Unscaled standard-normal entry z(r, i) of the on-the-fly Gaussian sketch
 * (S = z / sqrt(s), Section 3: S = G / sqrt(s) with G standard Gaussian).
 *   counter = (i mod 2^32, i div 2^32, r div 4, 0x53474155), key = seed;
 *   (w0, w1, w2, w3) = Philox4x32-10(counter, key);
 *   lane = r mod 4 takes the pair (w0, w1) for lanes 0-1, (w2, w3) for 2-3;
 *   u1 = ((w_even >> 9) + 1) 2^-23 in (0, 1], u2 = (w_odd >> 9) 2^-23;
 *   rho = sqrt(-2 ln u1); z = rho cos(2 pi u2) (even lane), rho sin (odd). */
float orc_gauss_entry(uint64_t seed, int64_t r, int64_t i)
{
    uint32_t ctr[4] = {(uint32_t)(uint64_t)i, (uint32_t)((uint64_t)i >> 32),
                       (uint32_t)((uint64_t)r >> 2), 0x53474155u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    int lane = (int)(r & 3);
    uint32_t we = w[(lane >> 1) * 2], wo = w[(lane >> 1) * 2 + 1];
    float u1 = (float)((we >> 9) + 1u) * 0x1p-23f;
    float u2 = (float)(wo >> 9) * 0x1p-23f;
    float rho = sqrtf(-2.0f * orc_ln_f32(u1));
    float c, s;
    orc_cossin_2pi_f32(u2, &c, &s);
    return (lane & 1) ? rho * s : rho * c;
}

/* Materialise the on-the-fly Gaussian sketch: S[r][i] = z(r, i) / sqrt(s)
 * with 1/sqrt(s) rounded once in binary64. */
void orc_gaussian_sketch_matrix(int64_t s, int64_t m, uint64_t seed, double *S, int64_t lds)
{
    double scale = 1.0 / sqrt((double)s);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i)
        for (int64_t r = 0; r < s; ++r)
            IDX(S, lds, r, i) = (double)orc_gauss_entry(seed, r, i) * scale;
}

/* Nonzero pattern of column i of the on-the-fly sparse-sign sketch.
 * Words are drawn from Philox4x32-10 with counter (i mod 2^32, i div 2^32,
 * block, 0x53535047), key = seed, blocks 0, 1, ... and words 0..3 within a
 * block.  Each word w proposes row floor(w * s / 2^32) with sign - if w is
 * odd, + if even; a row already taken is skipped.  After 1024 words (never
 * reached unless zeta is close to s) the smallest untaken rows are used,
 * with sign +.  Rows are reported in the order they were taken. */
void orc_sparse_sign_column(uint64_t seed, int64_t i, int64_t s, int zeta, int32_t *rows,
                            int8_t *signs)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    int cnt = 0;
    for (uint32_t blk = 0; blk < 256u && cnt < zeta; ++blk) {
        uint32_t ctr[4] = {(uint32_t)(uint64_t)i, (uint32_t)((uint64_t)i >> 32), blk, 0x53535047u};
        uint32_t w[4];
        orc_philox4x32_10(ctr, key, w);
        for (int t = 0; t < 4 && cnt < zeta; ++t) {
            int32_t row = (int32_t)(((uint64_t)w[t] * (uint64_t)s) >> 32);
            int dup = 0;
            for (int q = 0; q < cnt; ++q)
                dup |= rows[q] == row;
            if (dup)
                continue;
            rows[cnt] = row;
            signs[cnt] = (w[t] & 1u) ? (int8_t)-1 : (int8_t)1;
            ++cnt;
        }
    }
    for (int32_t row = 0; cnt < zeta; ++row) {
        int dup = 0;
        for (int q = 0; q < cnt; ++q)
            dup |= rows[q] == row;
        if (!dup) {
            rows[cnt] = row;
            signs[cnt] = 1;
            ++cnt;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Reduced-precision sketch definition (the library's tensor-core tier)      */
/*                                                                          */
/* The sketch only has to be an embedding, so its product may run in bf16   */
/* with fp32 sums: S's entries z_b(r, i) are bf16 values of a discretised   */
/* standard normal (defined below), and each x of X is either rounded to    */
/* bf16 (one term) or split into three bf16 terms x ~ x1 + x2 + x3 with     */
/* x1 = bf16(x), x2 = bf16(x - x1), x3 = bf16(x - x1 - x2) (the differences */
/* are exact in binary64).  All roundings are to nearest, ties to even.     */
/* The result is Y = (sum_i z_b (x1 + x2 + x3)) / sqrt(s), evaluated here   */
/* in binary64.                                                             */
/* ------------------------------------------------------------------------ */

/* Round a binary64 value to the nearest bf16 value (8 significant bits,
 * ties to even), returned as a binary64 value.  Normal range only (the
 * inputs here are far from bf16's under/overflow thresholds); zero stays
 * zero. */
double orc_round_bf16(double x)
{
    uint64_t b;
    memcpy(&b, &x, sizeof b);
    const uint64_t mag = b & 0x7fffffffffffffffull;
    if (mag == 0)
        return x;
    const uint64_t lsb = (b >> 45) & 1u;
    const uint64_t rnd = (b >> 44) & 1u;
    const uint64_t sticky = (b & ((1ull << 44) - 1u)) != 0;
    if (rnd && (sticky || lsb))
        b += 1ull << 45;
    b &= ~((1ull << 45) - 1u);
    double y;
    memcpy(&y, &b, sizeof y);
    return y;
}

/* The tensor-core tiers' S is not the binary64 tier's S rounded: since only
 * an embedding is needed, its entries lie on the grid k / 32 of a 4096-level
 * quantile discretisation of the standard normal,
 *   T[j] = k_j / 32,  k_j = round(32 Phi^{-1}((j + 1/2) / 4096))  (|k_j| <= 117),
 * rounded half to even (zero as +0), so every entry is an integer k over 32 (an exact
 * bf16, and an exact digit of the integer products of the digit tier), and
 * entry (r, i) of the unscaled sketch is
 *   z_b(r, i) = T[ h >> 4 ],  h = bits 16 (t mod 2) .. 16 (t mod 2) + 15 of
 *   word w_{t div 2} of Philox4x32-10 with counter (q mod 2^32, q div 2^32,
 *   r, 0x53424631) and key = seed, where q = i div 8 and t = i mod 8
 * (eight entries of one sketch row per Philox block).  S = z_b / sqrt(s). */

/* Standard normal quantile Phi^{-1}(p), 0 < p < 1: bisection on
 * Phi(x) = erfc(-x / sqrt(2)) / 2 until the bracket [lo, hi] holds two
 * neighbouring binary64 numbers; returns hi, the smaller of the two with
 * Phi(x) >= p.  p > 1/2 by the symmetry Phi^{-1}(p) = -Phi^{-1}(1 - p). */
double orc_normal_quantile(double p)
{
    if (p > 0.5)
        return -orc_normal_quantile(1.0 - p);
    double lo = -40.0, hi = 0.0;
    for (int it = 0; it < 4000; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid == lo || mid == hi)
            break;
        const double phi = 0.5 * erfc(-mid / sqrt(2.0));
        if (phi < p)
            lo = mid;
        else
            hi = mid;
    }
    return hi;
}

/* T[j] = k_j / 32, k_j = round(32 Phi^{-1}((j + 1/2) / 4096)), j = 0 .. 4095. */
void orc_tier_levels(double *T)
{
    for (int j = 0; j < 4096; ++j)
        T[j] = nearbyint(32.0 * orc_normal_quantile(((double)j + 0.5) / 4096.0)) / 32.0 + 0.0;
}

/* z_b(r, i) of the tensor-core tiers, given the table T. */
static double orc_tier_entry_t(uint64_t seed, int64_t r, int64_t i, const double *T)
{
    const uint64_t q = (uint64_t)i >> 3;
    const int t = (int)(i & 7);
    uint32_t ctr[4] = {(uint32_t)q, (uint32_t)(q >> 32), (uint32_t)(uint64_t)r, 0x53424631u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    const uint32_t h = (w[t >> 1] >> (16 * (t & 1))) & 0xffffu;
    return T[h >> 4];
}

/* Unscaled sketch z_b of the tensor-core tiers (s x m, leading dimension ldz). */
int orc_tier_sketch_entries(int64_t s, int64_t m, uint64_t seed, double *Z, int64_t ldz)
{
    double *T = (double *)malloc(sizeof(double) * 4096);
    if (!T)
        return ORC_ERR_NOMEM;
    orc_tier_levels(T);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i)
        for (int64_t r = 0; r < s; ++r)
            IDX(Z, ldz, r, i) = orc_tier_entry_t(seed, r, i, T);
    free(T);
    return ORC_OK;
}

/* Y = (sum_i z_b(r, i) * xs(i, j)) / sqrt(s) with xs the one- or
 * three-term bf16 split of X, sums in increasing i (binary64).
 * nterms is 1 or 3. */
int orc_sketch_bf16(int64_t s, int64_t m, int64_t n, uint64_t seed, int nterms, const double *X,
                    int64_t ldx, double *Y, int64_t ldy)
{
    double *Sb = (double *)malloc(sizeof(double) * (size_t)s * (size_t)m);
    double *Xs = (double *)malloc(sizeof(double) * (size_t)m * (size_t)n);
    if (!Sb || !Xs || orc_tier_sketch_entries(s, m, seed, Sb, s) != ORC_OK) {
        free(Sb);
        free(Xs);
        return ORC_ERR_NOMEM;
    }
    /* X as the sum of its bf16 terms; x1 + x2 + x3 is exact in binary64
     * (the three terms cover disjoint runs of at most 8 bits) */
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < m; ++i) {
            const double x = IDX(X, ldx, i, j);
            const double x1 = orc_round_bf16(x);
            double xs = x1;
            if (nterms == 3) {
                const double r1 = x - x1;
                const double x2 = orc_round_bf16(r1);
                const double x3 = orc_round_bf16(r1 - x2);
                xs = x1 + x2 + x3;
            }
            Xs[i + j * m] = xs;
        }
    orc_sketch_dense(s, m, n, Sb, s, Xs, m, Y, ldy);
    const double scale = 1.0 / sqrt((double)s);
    for (int64_t j = 0; j < n; ++j)
        for (int64_t r = 0; r < s; ++r)
            IDX(Y, ldy, r, j) *= scale;
    free(Xs);
    free(Sb);
    return ORC_OK;
}

/* The digit tier: X in six balanced base-256 digits per column and exact
 * integer sums.  Column j's exponent E_j = b_j - 1022 with b_j the largest
 * biased binary64 exponent field of the column (so 2^E_j > |x_ij|; b_j = 0
 * for a column of zeros and subnormals), every x_ij is rounded to
 *   F_ij = round(x_ij 2^(47 - E_j))   (half away from zero; |F_ij| < 2^47,
 *                                      x_ij = F_ij 2^(E_j - 47) up to 2^(E_j - 48)),
 * and Y(r, j) = (sum_i k(r, i) F_ij) 2^(E_j - 52) / sqrt(s), k = 32 z_b, the
 * integer sum taken exactly (128-bit) and rounded once to binary64.  A column
 * holding a NaN or an infinity gives a NaN column. */
int orc_sketch_digits(int64_t s, int64_t m, int64_t n, uint64_t seed, const double *X, int64_t ldx,
                      double *Y, int64_t ldy)
{
    double *Z = (double *)malloc(sizeof(double) * (size_t)s * (size_t)m);
    int64_t *F = (int64_t *)malloc(sizeof(int64_t) * (size_t)m);
    if (!Z || !F || orc_tier_sketch_entries(s, m, seed, Z, s) != ORC_OK) {
        free(Z);
        free(F);
        return ORC_ERR_NOMEM;
    }
    const double scale = 1.0 / sqrt((double)s);
    for (int64_t j = 0; j < n; ++j) {
        int bmax = 0;
        for (int64_t i = 0; i < m; ++i) {
            uint64_t b;
            const double x = IDX(X, ldx, i, j);
            memcpy(&b, &x, sizeof b);
            const int e = (int)((b >> 52) & 0x7ff);
            if (e > bmax)
                bmax = e;
        }
        if (bmax == 0x7ff) {
            for (int64_t r = 0; r < s; ++r)
                IDX(Y, ldy, r, j) = NAN;
            continue;
        }
        const int E = bmax - 1022;
        for (int64_t i = 0; i < m; ++i)
            F[i] = (int64_t)round(ldexp(IDX(X, ldx, i, j), 47 - E));
#pragma omp parallel for schedule(static)
        for (int64_t r = 0; r < s; ++r) {
            __int128 acc = 0;
            for (int64_t i = 0; i < m; ++i)
                acc += (__int128)(int64_t)(32.0 * IDX(Z, s, r, i)) * F[i];
            IDX(Y, ldy, r, j) = ldexp((double)acc, E - 52) * scale;
        }
    }
    free(F);
    free(Z);
    return ORC_OK;
}

/* Patterns of all m columns: rows/signs of length m*zeta. */
void orc_sparse_sign_pattern(int64_t s, int64_t m, int zeta, uint64_t seed, int32_t *rows,
                             int8_t *signs)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i)
        orc_sparse_sign_column(seed, i, s, zeta, rows + i * zeta, signs + i * zeta);
}

/* ------------------------------------------------------------------------ */
/* Subsampled randomized Hadamard transform (SRHT), the third of the        */
/* common sketches Section 3 lists next to the Gaussian sketch and          */
/* CountSketch.  The paper gives no formula; the reading is the usual one    */
/* (Tropp 2011; Boutsidis and Gittens 2013):                                 */
/*   S = sqrt(m'/s) R (H / sqrt(m')) D = (1/sqrt(s)) R H D,                  */
/* m' = 2^b >= m the padded order (X extended by zero rows), D = diag(d_i)   */
/* with random signs d_i, H the unnormalised Sylvester-Hadamard matrix of    */
/* order m', H(p, i) = (-1)^popcount(p AND i), and R the restriction to s    */
/* distinct rows p_0 .. p_{s-1} drawn uniformly without replacement.  So     */
/*   S(r, i) = d_i (-1)^popcount(p_r AND i) / sqrt(s).                       */
/* Random draws, from Philox4x32-10 with key = seed:                        */
/*   d_i  : bit (i mod 128) of the 128 output bits for counter              */
/*          (q mod 2^32, q div 2^32, 0, 0x53524844), q = floor(i / 128);     */
/*          bit k is bit (k mod 32) of word floor(k / 32); set means -1.     */
/*   p_r  : pi(r), pi a permutation of [0, 2^b): a 4-round Feistel network   */
/*          on b bits.  x = L 2^wr + R with widths (wl, wr) = (ceil(b/2),    */
/*          floor(b/2)); round k = 0..3 replaces (L, R) by                    */
/*          (R, L XOR (w0 mod 2^wl)), w0 the first word for counter          */
/*          (R, k, b, 0x53524850), and swaps the widths.  Every round is a    */
/*          bijection of [0, 2^b), so pi is one and p_0 .. p_{s-1} are        */
/*          distinct.                                                        */
/* ------------------------------------------------------------------------ */

/* pi(x) on b bits (0 <= b <= 31, 0 <= x < 2^b). */
int64_t orc_srht_perm_one(int b, uint64_t seed, int64_t x)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    int wl = (b + 1) / 2, wr = b / 2;
    uint32_t L = (uint32_t)((uint64_t)x >> wr);
    uint32_t R = (uint32_t)((uint64_t)x & ((1u << wr) - 1u));
    for (uint32_t k = 0; k < 4; ++k) {
        uint32_t ctr[4] = {R, k, (uint32_t)b, 0x53524850u};
        uint32_t w[4];
        orc_philox4x32_10(ctr, key, w);
        uint32_t f = w[0] & ((1u << wl) - 1u);
        uint32_t newL = R, newR = L ^ f;
        int t = wl;
        wl = wr;
        wr = t;
        L = newL;
        R = newR;
    }
    return (int64_t)(((uint64_t)L << wr) | (uint64_t)R);
}

/* p[r] = pi(r), r = 0 .. s-1 (s <= 2^b): the sampled rows of H. */
void orc_srht_perm(int b, int64_t s, uint64_t seed, int64_t *p)
{
    for (int64_t r = 0; r < s; ++r)
        p[r] = orc_srht_perm_one(b, seed, r);
}

/* d[i] = d_{row0 + i}, i = 0 .. m-1 (+1 or -1). */
void orc_srht_signs(uint64_t seed, int64_t row0, int64_t m, int8_t *d)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int64_t i = 0; i < m; ++i) {
        uint64_t g = (uint64_t)(row0 + i), q = g >> 7;
        uint32_t ctr[4] = {(uint32_t)q, (uint32_t)(q >> 32), 0u, 0x53524844u};
        uint32_t w[4];
        orc_philox4x32_10(ctr, key, w);
        uint32_t k = (uint32_t)(g & 127u);
        d[i] = ((w[k >> 5] >> (k & 31u)) & 1u) ? (int8_t)-1 : (int8_t)1;
    }
}

/* k rows and columns row0 .. row0 + m - 1 of S (k x m, lds) for a sketch of
 * s rows: row t is S(r, .) for the sampled Hadamard row p[t] = p_r, so
 * S(t, i) = d_i (-1)^popcount(p[t] AND (row0 + i)) / sqrt(s), with p from
 * orc_srht_perm (all s rows, or a selection) and d from
 * orc_srht_signs(seed, row0, m, d). */
void orc_srht_dense(int64_t k, int64_t s, int64_t m, int64_t row0, const int64_t *p,
                    const int8_t *d, double *S, int64_t lds)
{
    double scale = 1.0 / sqrt((double)s);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        uint64_t g = (uint64_t)(row0 + i);
        for (int64_t r = 0; r < k; ++r) {
            int odd = __builtin_popcountll((uint64_t)p[r] & g) & 1;
            double h = odd ? -1.0 : 1.0;
            IDX(S, lds, r, i) = (d[i] < 0 ? -h : h) * scale;
        }
    }
}
