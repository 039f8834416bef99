/*
 * rclupp.h -- C ABI of the GB300 (sm_103a) library for the QR factorization
 * of tall-skinny matrices by randomized CholeskyQR with LU partial pivoting.
 *
 * Paper: "A new randomized CholeskyQR based on LU decomposition with partial
 * pivoting" (arXiv 2412.06551).  The problem (Section 1): X in R^{m x n},
 * m >= n, rank(X) = n; compute X = Q R with Q (m x n) orthonormal columns and
 * R (n x n) upper triangular.
 *
 * Conventions for every entry point
 *   - Matrices are column-major FP64: element (i, j) of a matrix A with
 *     leading dimension lda is A[i + j*lda], lda >= number of rows.
 *   - Matrix pointers are DEVICE pointers owned by the caller, unless an
 *     argument says "host".  The library never frees them.
 *   - The handle owns its stream binding and a device workspace that grows
 *     on demand (cudaMalloc) and is released by rclupp_destroy.
 *   - Every call is enqueued on the handle's stream and is synchronous with
 *     respect to its returned status: the function returns after the GPU work
 *     has finished, so a numerical status (breakdown, zero pivot) can be
 *     returned.  Entry points marked "async" only enqueue.
 *   - On any status other than RCLUPP_OK the contents of the outputs are
 *     unspecified.  Argument errors are detected before any GPU work.
 *   - Errors every entry point may return besides those it lists: ERR_ARG
 *     (a NULL pointer, a size below 1, a leading dimension below the number
 *     of rows), ERR_UNSUPPORTED (n > 256, m >= 2^31, s > 4096), ERR_NOMEM
 *     (the workspace could not grow), ERR_CUDA (a CUDA call failed) and
 *     ERR_TIMEOUT (a bounded device wait gave up after 2 s).
 *   - R outputs are n x n upper triangular with the strict lower triangle set
 *     to zero and a positive diagonal (the unique thin QR).
 *   - Q may alias X for rclupp_factor and cholqr2_factor (every tall pass is
 *     row-local).  For rclupp_r_factor and lc2_factor aliasing makes the
 *     handle allocate an m x n workspace for the LU factor.
 */
#ifndef RCLUPP_H
#define RCLUPP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rclupp_handle_s *rclupp_handle_t;

typedef enum {
    RCLUPP_OK = 0,
    RCLUPP_ERR_ARG = -1,            /* invalid argument (sizes, pointers, leading dims) */
    RCLUPP_ERR_CHOL_BREAKDOWN = -2, /* a Cholesky radicand was <= 0 or NaN (info: column) */
    RCLUPP_ERR_LU_ZERO_PIVOT = -3,  /* zero pivot in an LU factorization: rank < n */
    RCLUPP_ERR_NONFINITE = -4,      /* non-finite value met where a finite one is required */
    RCLUPP_ERR_CUDA = -5,           /* a CUDA runtime call failed */
    RCLUPP_ERR_TIMEOUT = -6,        /* a bounded device-side wait gave up */
    RCLUPP_ERR_NOMEM = -7,          /* workspace allocation failed */
    RCLUPP_ERR_UNSUPPORTED = -8     /* size or option outside what this build supports */
} rclupp_status_t;

typedef enum {
    RCLUPP_SKETCH_GAUSSIAN = 0,    /* S = G / sqrt(s), G standard Gaussian (Section 3) */
    RCLUPP_SKETCH_SPARSE_SIGN = 1, /* zeta distinct rows per column, +-1/sqrt(zeta);
                                      zeta = 1 is CountSketch (Section 3)          */
    RCLUPP_SKETCH_SRHT = 2         /* subsampled randomized Hadamard transform
                                      S = R H D / sqrt(s) (Section 3)              */
} rclupp_sketch_kind_t;

/* Precision form.  The sketch only has to be an embedding (Section 3): the
 * reduced tiers run the generated Gaussian sketch on the tensor cores
 * (tcgen05, bf16 operands, fp32 accumulation in tensor memory) with S on an
 * integer grid: z_b(r, i) = T[h >> 4] with T[j] = k_j / 32,
 * k_j = round(32 Phi^{-1}((j + 1/2) / 4096)) (half to even, |k_j| <= 117),
 * and h the 16-bit half (i mod 8) mod 2 of word (i mod 8) div 2 of
 * Philox4x32-10 at counter (i div 8 mod 2^32, i div 2^35, r, 0x53424631),
 * key = seed (so these tiers' S differs from the binary64 tier's), and
 * S = z_b / sqrt(s).  Every x of X is rounded to bf16 (BF16), split into
 * three bf16 terms x1 = bf16(x), x2 = bf16(x - x1), x3 = bf16(x - x1 - x2)
 * (FP32), or rounded to 48 bits of its column with exact integer sums
 * (DIGITS, below); per-CTA partial sums are combined in binary64.  EMULATED
 * sketches at the DIGITS tier and adds binary64-emulating tensor-core
 * products for the solves and the first Gram.  Other steps stay in binary64.
 * The sparse-sign and SRHT sketches only add and always run in binary64
 * (their results report RCLUPP_PREC_FP64 as the tier used); an explicit S
 * requires RCLUPP_PREC_FP64 or one of the emulated tiers (whose sketch is
 * then binary64). */
typedef enum {
    RCLUPP_PREC_FP64 = 0,        /* every step in binary64 */
    RCLUPP_PREC_SKETCH_BF16 = 1, /* tensor-core sketch: bf16 S, bf16 X, fp32 sums          */
    RCLUPP_PREC_SKETCH_FP32 = 2, /* tensor-core sketch: bf16 S, three-term bf16 X, fp32 sums */
    RCLUPP_PREC_EMULATED = 3,    /* the DIGITS sketch tier; the triangular solves' block products
                                    (rclupp_trsm_emulated for the first solve by R1,
                                    rclupp_trsm_emulated_wellcond for the solves by R2 and R4)
                                    and the Gram of the first CholeskyQR pass (Q1^T Q1,
                                    rclupp_gram_emulated) as binary64-emulating split-bf16
                                    products on the tensor cores; the final-pass Gram, the
                                    diagonal blocks of the first solve, the inverses of R2 and R4
                                    and the n x n factorizations stay in binary64.  An explicit S or the
                                    sparse-sign or SRHT sketch keeps a binary64 sketch. */
    RCLUPP_PREC_EMULATED_ALL = 4, /* EMULATED, and the final-pass Gram (C5; for RCholeskyQR its
                                    one Gram) emulated as well: its digit products are exact and
                                    are summed exactly in fp32 windows, then in int64 and
                                    binary64, so the accumulation stays binary64 or better */
    RCLUPP_PREC_SKETCH_DIGITS = 5 /* tensor-core sketch with the S of BF16 (the integers k on
                                    the tensor cores, 1/32 in the scale) and X rounded to 48 bits
                                    of each column's largest entry (six balanced base-256 digits
                                    of F = round(x 2^(47 - E_j)), half away from zero, 2^E_j above
                                    the column); the integer sums k F are exact on the tensor
                                    cores (fp32 windows of 1024 rows, int64 drains), then summed
                                    in binary64.  Needs no escalation up to kappa(X) ~ 1e15;
                                    the emulated tiers sketch at this tier. */
} rclupp_precision_t;

/* R-factor R0 of the preconditioning step: of M in Algorithm 6, of M_s in
 * Algorithm 7, of the sketch S X in Algorithm 5. */
typedef enum {
    RCLUPP_R0_HOUSEHOLDER = 0, /* thin HouseholderQR, LAPACK larfg signs (the paper's choice) */
    RCLUPP_R0_GIVENS = 1       /* Givens rotations, r = hypot(a, b) >= 0 (Section 1)         */
} rclupp_r0_method_t;

/* Sketch options of the randomized algorithms (RCLUPP, RCLUPPr).
 *   kind  : Gaussian, sparse-sign or SRHT.
 *   s     : sketch size, n <= s <= 4096 (the paper uses s = O(n), e.g. n+1 or 2n).
 *   zeta  : nonzeros per column for the sparse-sign sketch (1 <= zeta <= s, <= 16).
 *   seed  : key of the counter-based generator (Philox4x32-10) for S.
 *   prec  : precision of the sketch product (rclupp_precision_t).
 *   order_log2 : SRHT only: b of the Hadamard order m' = 2^b (0 <= b <= 31);
 *           0 takes the smallest power of two >= m (for rclupp_sketch_rows,
 *           >= row0 + m).  A row-sharded sketch passes the whole matrix's b.
 *           Requires m (row0 + m) <= 2^b and s <= 2^b.
 *   S/lds : optional explicit dense sketch (DEVICE, s x m, column-major); when
 *           non-NULL it replaces the generated one (kind and seed are ignored).
 *   r0_method : R-factor R0 of the preconditioning step (rclupp_r0_method_t):
 *           Householder (default, the paper's choice) or Givens rotations
 *           (the alternative of Section 1 and of the remark after Algorithm 5);
 *           Givens needs the s x n matrix to fit a cluster's shared memory
 *           (s n <= 25600 doubles per CTA, up to 8 CTAs), else
 *           RCLUPP_ERR_UNSUPPORTED.
 *   reserved : 0.
 * The generated S: entry (r, i) depends only on (seed, r, i), so S is never
 * stored.  Gaussian: Philox4x32-10 with counter (i mod 2^32, i div 2^32,
 * r div 4, 0x53474155) and key = seed; words (w0, w1) serve rows 4b, 4b+1 and
 * (w2, w3) rows 4b+2, 4b+3 by the Box-Muller transform, evaluated in binary32
 * with series for ln and sin/cos; S = z / sqrt(s).  Sparse-sign: Philox words
 * with counter (i mod 2^32, i div 2^32, block, 0x53535047) propose rows
 * floor(w s / 2^32), duplicates skipped, sign from the lowest bit.
 * SRHT: S(r, i) = d_i (-1)^popcount(p_r AND i) / sqrt(s), i.e. rows p_r of
 * the Sylvester-Hadamard matrix of order 2^b times random signs, A padded
 * with zero rows.  d_i = -1 when bit (i mod 128) of the 128 output bits of
 * Philox with counter (q mod 2^32, q div 2^32, 0, 0x53524844), q = i div 128,
 * is set (bit k = bit k mod 32 of word k div 32).  p_r = pi(r) for a keyed
 * permutation pi of [0, 2^b): four Feistel rounds on x = L 2^wr + R with
 * widths (wl, wr) = (ceil(b/2), floor(b/2)), each mapping (L, R) to
 * (R, L XOR (w0 mod 2^wl)), w0 the first Philox word for counter
 * (R, round, b, 0x53524850), then swapping the widths; so the s rows are
 * distinct.  The product runs in binary64 at every precision tier: the
 * transform of each 256-row block is exact in integers (entries rounded to
 * 53 bits relative to the block's largest), the sampled values are summed in
 * binary64. */
typedef struct {
    int32_t kind;
    int32_t zeta;
    int64_t s;
    uint64_t seed;
    int32_t prec;
    int32_t order_log2;
    const double *S;
    int64_t lds;
    int32_t r0_method;
    int32_t reserved;
} rclupp_opts_t;

/* Diagnostic output of a factorization (may be NULL). */
typedef struct {
    int32_t status;      /* same as the return value */
    int32_t failed_step; /* 0 none; 1 sketch LU; 2 tall LU; 3 first Cholesky of the
                            CholeskyQR passes; 4 second one; 6 shifted Cholesky
                            (SCholeskyQR3) */
    int64_t info;        /* failing column for breakdown / zero pivot, else -1 */
    int32_t prec_used;   /* sketch tier that produced the result (rclupp_precision_t):
                            RCLUPP/RCLUPPr escalate bf16 -> three-term bf16 -> FP64 when
                            the first Cholesky breaks down or the spread of its diagonal
                            exceeds 1e4 (Q1 too ill-conditioned for CholeskyQR2); the
                            emulated tiers report RCLUPP_PREC_SKETCH_DIGITS (FP64 with an
                            explicit, sparse-sign or SRHT sketch), which never escalates */
    int32_t emulated;    /* 1 when the solves and the first pass's Gram ran on the
                            binary64-emulating tensor-core path (RCLUPP_PREC_EMULATED), 2 when
                            every Gram did too (RCLUPP_PREC_EMULATED_ALL), else 0 */
} rclupp_info_t;

/* ---- handle (no counterpart in the paper: stream binding, workspace) ------ */

/* Create a handle bound to the CUDA stream `stream` (a cudaStream_t; NULL =
 * the legacy default stream) on the current device.  Allocates a small
 * status buffer; the workspace is allocated lazily.  A handle serves one call
 * at a time: it has one stream binding and one workspace and takes no lock,
 * so host threads that call the library concurrently each need their own
 * handle.  Errors: ERR_ARG (NULL out-pointer), ERR_CUDA, ERR_NOMEM. */
rclupp_status_t rclupp_create(rclupp_handle_t *handle, void *stream);
/* Release the handle and its workspace (synchronizes its stream first). */
rclupp_status_t rclupp_destroy(rclupp_handle_t handle);
/* Rebind the handle to another stream of the same device. */
rclupp_status_t rclupp_set_stream(rclupp_handle_t handle, void *stream);
/* Bytes of device workspace currently held by the handle. */
rclupp_status_t rclupp_workspace_bytes(rclupp_handle_t handle, size_t *bytes);
/* Bytes of device workspace one factorization of an m x n matrix by `algo`
 * (rclupp_algo_t) needs on the current device with these options (NULL =
 * defaults): partial sums, the sketch, small-factor scratch, the padded
 * triangular factors, and for RCLUPPr / LC2 an m x n copy of the LU factor
 * when q_aliases_x != 0 (or, for RCLUPPr, at a non-binary64 tier).  A handle
 * grows its workspace to this size on the first such call.  No GPU work;
 * without a visible device the size is the one a GB300 (152 SMs) needs.
 * Errors as the drivers' argument checks. */
rclupp_status_t rclupp_workspace_size(int32_t algo, int64_t m, int64_t n, const rclupp_opts_t *opts,
                                      int32_t q_aliases_x, size_t *bytes);
/* Human-readable name of a status code (static string). */
const char *rclupp_status_string(int status);

/* ---- algorithm drivers -------------------------------------------------- */

/* [Q, R] = RCLUPP(X) -- Algorithm 6 (RCLUPP), Section 1:
 *   X_s = S X; [M, N, P] = LU(X_s); R0 = R of HouseholderQR(M); R1 = R0 N
 *   (diagonal signs of R1 normalised); Q1 = X R1^{-1};
 *   [Q, Z] = CholeskyQR2(Q1); R = Z R1  (evaluated R3 = R2 R1, R = R4 R3).
 * X: m x n (ldx >= m); Q: m x n (ldq >= m), may alias X; R: n x n (ldr >= n).
 * opts: sketch options (NULL = Gaussian, s = 2n, seed 0, FP64).
 * Requires 1 <= n <= 256, n <= m, n <= s.  Errors: ERR_ARG, ERR_UNSUPPORTED,
 * ERR_LU_ZERO_PIVOT (sketch rank-deficient), ERR_NONFINITE (a column of the
 * sketch without a finite non-zero pivot candidate: the LU pivot searches
 * skip NaN), ERR_CHOL_BREAKDOWN, ERR_CUDA, ERR_NOMEM, ERR_TIMEOUT; info
 * (may be NULL) names the failing step and column.  A NaN or an infinite
 * entry of X ends in ERR_NONFINITE or ERR_CHOL_BREAKDOWN. */
rclupp_status_t rclupp_factor(rclupp_handle_t handle, int64_t m, int64_t n, const double *X,
                              int64_t ldx, const rclupp_opts_t *opts, double *Q, int64_t ldq,
                              double *R, int64_t ldr, rclupp_info_t *info);

/* [Q, R] = RCLUPPr(X) -- Algorithm 7 (RCLUPPr), Section 4.4:
 *   [M, N, P] = LU(X) (tall, partial pivoting over all m rows); M_s = S M;
 *   R0 = R of HouseholderQR(M_s); R1 = R0 N (signs normalised);
 *   Q1 = X R1^{-1}; [Q, Z] = CholeskyQR2(Q1); R = Z R1.
 * Same arguments and errors as rclupp_factor; X is not modified. */
rclupp_status_t rclupp_r_factor(rclupp_handle_t handle, int64_t m, int64_t n, const double *X,
                                int64_t ldx, const rclupp_opts_t *opts, double *Q, int64_t ldq,
                                double *R, int64_t ldr, rclupp_info_t *info);

/* [Q, R] = CholeskyQR2(X) -- Algorithm 2 (Section 2.1).  No sketch.
 * Breaks down (ERR_CHOL_BREAKDOWN) when kappa_2(X) approaches u^{-1/2}. */
rclupp_status_t cholqr2_factor(rclupp_handle_t handle, int64_t m, int64_t n, const double *X,
                               int64_t ldx, double *Q, int64_t ldq, double *R, int64_t ldr,
                               rclupp_info_t *info);

/* [Q, R] = LC2(X) -- Algorithm 4 (Section 2.3): [M, N, P] = LU(X);
 * S = chol(M^T M); R1 = S N (signs normalised); Q1 = X R1^{-1};
 * [Q, Z] = CholeskyQR(Q1); R = Z R1.  Errors as rclupp_factor; LU failures
 * come from the tall LU of X (failed_step 2). */
rclupp_status_t lc2_factor(rclupp_handle_t handle, int64_t m, int64_t n, const double *X,
                           int64_t ldx, double *Q, int64_t ldq, double *R, int64_t ldr,
                           rclupp_info_t *info);

/* [Q, R] = RCholeskyQR(X) -- Algorithm 5 (single sketch): K = S X;
 * R1 = R of HouseholderQR(K) (signs normalised); Q1 = X R1^{-1};
 * [Q, Z] = CholeskyQR(Q1); R = Z R1.  A comparison path: one CholeskyQR
 * after the preconditioner, so its orthogonality is worse than RCLUPP's on
 * ill-conditioned X (Section 5.1).  Arguments as rclupp_factor; the sketch
 * tier is used as given (no escalation). */
rclupp_status_t rcholqr_factor(rclupp_handle_t handle, int64_t m, int64_t n, const double *X,
                               int64_t ldx, const rclupp_opts_t *opts, double *Q, int64_t ldq,
                               double *R, int64_t ldr, rclupp_info_t *info);

/* [Q, R] = SCholeskyQR3(X) -- Algorithm 3 with the shift of Section 2.2,
 * s = 11 (m n u + n (n+1) u) ||X||_g^2, ||X||_g = max_j ||X_j||_2
 * (Definition 2.1): G = X^T X; R1 = chol(G + s I); Q1 = X R1^{-1};
 * [Q, Z] = CholeskyQR2(Q1); R = Z R1.  failed_step 6 marks a breakdown of
 * the shifted Cholesky. */
rclupp_status_t scholqr3_factor(rclupp_handle_t handle, int64_t m, int64_t n, const double *X,
                                int64_t ldx, double *Q, int64_t ldq, double *R, int64_t ldr,
                                rclupp_info_t *info);

/* ---- batched form (no counterpart in the paper: many independent
 * factorizations by Algorithms 2-7 in one call) ---------------------------- */

typedef enum {
    RCLUPP_ALGO_RCLUPP = 0,  /* Algorithm 6 */
    RCLUPP_ALGO_RCLUPPR = 1, /* Algorithm 7 */
    RCLUPP_ALGO_CHOLQR2 = 2, /* Algorithm 2 */
    RCLUPP_ALGO_LC2 = 3,     /* Algorithm 4 */
    RCLUPP_ALGO_RCHOLQR = 4, /* Algorithm 5 */
    RCLUPP_ALGO_SCHOLQR3 = 5 /* Algorithm 3 */
} rclupp_algo_t;

/* Many independent factorizations of uneven sizes in one call: problem i is
 * the m[i] x n[i] matrix X[i] (ldx[i]) with outputs Q[i] (ldq[i]) and R[i]
 * (ldr[i]), every pointer a DEVICE pointer; the arrays themselves (m, n, X,
 * ldx, opts, Q, ldq, R, ldr, status) are HOST arrays of length count.  opts
 * holds one rclupp_opts_t per problem (NULL = defaults) and is used by the
 * randomized algorithms.  A graph cannot escalate a sketch tier, so each
 * problem's sketch runs at one tier: binary64 for RCLUPP_PREC_FP64; the
 * three-term bf16 tensor-core sketch (FP32 level, enough for kappa(X) up to
 * about 1e12) for RCLUPP_PREC_SKETCH_FP32; the digit tier for
 * RCLUPP_PREC_SKETCH_DIGITS and for the emulated tiers, which keep their
 * emulated solves and Gram products; RCLUPP_PREC_SKETCH_BF16, which relies
 * on escalation, returns RCLUPP_ERR_UNSUPPORTED.  The sparse-sign,
 * SRHT and explicit sketches stay binary64.  Each problem obeys the
 * single-problem rules;
 * problems run concurrently, so the outputs of different problems must not
 * overlap (inputs may be shared).
 * The whole batch is enqueued as one CUDA graph: it forks into B parallel
 * branches (streams; B set by rclupp_set_batch_branches, default 16) so that
 * small problems fill the GPU together, and joins.  Problems go to branches
 * longest first, each to the branch with the least estimated work so far
 * (m n^2 plus a per-column term for the small factorizations), and each
 * branch runs its problems largest first.  The instantiated graph is cached in the handle and
 * replayed while the batch is unchanged: sizes, pointers, options, branch
 * count, launch shapes and workspace, compared byte for byte.  The
 * workspace holds B per-branch slices sized for the largest problem.
 * status[i] (may be NULL) receives problem i's status; the return value is
 * the first non-OK status, or RCLUPP_OK.  Synchronous like the other calls. */
rclupp_status_t rclupp_factor_batched(rclupp_handle_t handle, int32_t algo, int32_t count,
                                      const int64_t *m, const int64_t *n, const double *const *X,
                                      const int64_t *ldx, const rclupp_opts_t *opts,
                                      double *const *Q, const int64_t *ldq, double *const *R,
                                      const int64_t *ldr, int32_t *status);

/* The same batch enqueued on the handle's stream without waiting, for a
 * caller that captures it into a CUDA graph of its own: no graph of the
 * library's, no host synchronization, no host read-back.  The problems fork
 * into the B branch streams and join back into the handle's stream, every
 * step being a stream operation that a capture records; at the end problem
 * i's status code is written to d_status[i], a DEVICE array of count int32.
 * The arrays m .. ldr are read during the call only.  While the handle's
 * stream captures nothing may be allocated: the handle's workspace and
 * branch streams must already be large enough, from an earlier call
 * (batched or async) with the same or larger problems and branch count
 * outside the capture; otherwise RCLUPP_ERR_UNSUPPORTED.  A graph that
 * recorded this call keeps pointers into the handle's workspace, so it stays
 * valid while the handle lives and its workspace is not regrown (a later
 * call with larger problems would regrow it).  Two such graphs, or this
 * call and another call on the same handle, must not run concurrently.
 * Returns RCLUPP_OK once enqueued; argument errors as rclupp_factor_batched. */
rclupp_status_t rclupp_factor_batched_async(rclupp_handle_t handle, int32_t algo, int32_t count,
                                            const int64_t *m, const int64_t *n,
                                            const double *const *X, const int64_t *ldx,
                                            const rclupp_opts_t *opts, double *const *Q,
                                            const int64_t *ldq, double *const *R, const int64_t *ldr,
                                            int32_t *d_status);

/* Number of parallel branches of the batched graph (1 ..64). */
rclupp_status_t rclupp_set_batch_branches(rclupp_handle_t handle, int32_t branches);

/* Launch shapes of the kernels inside the batched graph: grid_div (1 ..64)
 * divides the number of CTAs each tall pass aims for (2 per SM for a single
 * call), so that concurrent problems use fewer, longer-lived CTAs;
 * fine_tiles = 1 selects the smaller row tile of the TRSM (n <= 64: 64 rows
 * instead of 128) and of the Gram (64 instead of 128 rows for n <= 64, 32
 * instead of 64 for n <= 128).  Results are the same up to the order of the
 * split-K sums.  Defaults 1 and 0. */
rclupp_status_t rclupp_set_batch_policy(rclupp_handle_t handle, int32_t grid_div, int32_t fine_tiles);

/* The handle's current branch count and launch shapes (any pointer may be NULL). */
rclupp_status_t rclupp_get_batch_policy(rclupp_handle_t handle, int32_t *branches, int32_t *grid_div,
                                        int32_t *fine_tiles);

/* Autotuner of the batched form: runs the batch (same arguments as
 * rclupp_factor_batched; outputs are overwritten) with 4, 8, 16, 32 and 64
 * branches (up to the batch size), then, at the fastest branch count, with
 * the launch shapes (grid_div, fine_tiles) = (1, 1), (2, 0), (2, 1), (4, 0),
 * (4, 1), (8, 0); it times one replay of each cached graph with CUDA events
 * on the handle's stream, keeps the fastest combination in the handle and
 * returns its branch count in *best_branches and its time in *best_ms
 * (either may be NULL; rclupp_get_batch_policy reads the rest).  A numerical
 * failure of a problem (breakdown, zero pivot, non-finite input) does not
 * stop the tuning and is not returned; any other failure stops it and is
 * returned. */
rclupp_status_t rclupp_autotune_batched(rclupp_handle_t handle, int32_t algo, int32_t count,
                                        const int64_t *m, const int64_t *n,
                                        const double *const *X, const int64_t *ldx,
                                        const rclupp_opts_t *opts, double *const *Q,
                                        const int64_t *ldq, double *const *R, const int64_t *ldr,
                                        int32_t *best_branches, float *best_ms);

/* ---- individual steps of the tall path (each is one row of the path) ---- */

/* Y = S A (s x n, ldy >= s): the sketch S X of Algorithm 6 and S M of
 * Algorithm 7.  unit_lower != 0 reads A as the unit-lower
 * trapezoidal factor of an in-place LU (ones on the diagonal, zeros above).
 * Sum order is a fixed split over row chunks and a fixed-order reduction, so
 * results are bitwise reproducible for a given device. */
rclupp_status_t rclupp_sketch(rclupp_handle_t handle, int64_t m, int64_t n, const double *A,
                              int64_t lda, int32_t unit_lower, const rclupp_opts_t *opts,
                              double *Y, int64_t ldy);

/* The sketch of a block of rows: A holds rows row0 .. row0 + m - 1 of a
 * taller matrix and Y = S[:, row0 : row0 + m] A, with the generated S's entry
 * (r, row0 + i) multiplying row i of A -- the partial that each rank of a
 * row-sharded factorization adds into the full S X (Section 3's sketch is a
 * sum over rows).  An explicit S (opts->S) is read from its column 0, i.e.
 * the caller passes the slice.  row0 >= 0; otherwise as rclupp_sketch. */
rclupp_status_t rclupp_sketch_rows(rclupp_handle_t handle, int64_t m, int64_t n, const double *A,
                                   int64_t lda, int64_t row0, int32_t unit_lower,
                                   const rclupp_opts_t *opts, double *Y, int64_t ldy);

/* G = A^T A (n x n, ldg >= n, both triangles written): the Gram product of
 * Algorithm 1, C1/C5 of Theorem 4.1; unit_lower as in rclupp_sketch (LC2's M^T M). */
rclupp_status_t rclupp_gram(rclupp_handle_t handle, int64_t m, int64_t n, const double *A,
                            int64_t lda, int32_t unit_lower, double *G, int64_t ldg);

/* G = A^T A (n x n, both triangles) as binary64-emulating products on the
 * tensor cores: the Gram product of the CholeskyQR pass (Algorithm 1,
 * C1) in the precision form RCLUPP_PREC_EMULATED.  Each element is written as
 * a_ij = 2^(E_j - 7) sum_{s=0..7} d_s 2^(-8s) with integer digits |d_s| <= 128
 * (E_j: 2^E_j exceeds every |a_ij| of column j; round to nearest, half away
 * from zero, at 2^(E_j - 63)); G sums the digit products of levels
 * s + t <= 7 exactly in fp32 over 128-row windows, then in int64 and binary64.
 * Error: about m 2^-60 2^(E_j + E_k) from the split plus binary64 sums, i.e.
 * at or below binary64's, relative to the columns' largest entries.
 * NaN in G(j, k) when column j or k holds a non-finite value.  n <= 256. */
rclupp_status_t rclupp_gram_emulated(rclupp_handle_t handle, int64_t m, int64_t n, const double *A,
                                     int64_t lda, double *G, int64_t ldg);

/* Q = A R^{-1} with the block products emulating binary64 on the tensor
 * cores: the triangular solve of eq. (ewy) (C3, C7) in the precision form
 * RCLUPP_PREC_EMULATED.  Substitution by 32-column blocks: the update
 * A_J - Q_{<J} R_{<J,J} uses the digits of rclupp_gram_emulated (one exponent
 * per row of Q over its first 32J columns, one per column of R over rows
 * < 32J; levels <= 7 summed exactly in fp32 over at most 128 K-columns, then
 * in int64), the 32 x 32 diagonal blocks are solved in binary64.  Error of
 * an update entry: about (j0 + 128) 2^-60 2^(E_i + E'_c).  R: n x n upper,
 * nonzero diagonal.  Q may alias A.  n <= 256. */
rclupp_status_t rclupp_trsm_emulated(rclupp_handle_t handle, int64_t m, int64_t n, const double *A,
                                     int64_t lda, const double *R, int64_t ldr, double *Q,
                                     int64_t ldq);

/* Q = A R^{-1} for an R expected to be well conditioned, the form the
 * emulated tiers use for the second and final solves of CholeskyQR2 (C3, C7:
 * R2 and R4 have the condition numbers of Q1 and Q2).  W = R^{-1} is formed
 * in binary64 by forward substitution along its rows, with Skeel's condition
 * number cond(R) = || |W| |R| ||_inf; if cond(R) <= max(100, n), Q = A W runs
 * as one binary64-emulating product on the tensor cores (digits of A's rows
 * with one exponent per row over all n columns, of W's columns with one per
 * column; levels <= 7 exact in fp32 over <= 128 K-columns, int64 drains),
 * whose residual |Q R - A| <= c u |A| |W| |R| then stays within the bound
 * of eq. (ewy)'s substitution (gamma_n |Q| |R|); else the substitution of
 * rclupp_trsm_emulated runs.  The choice is made on the device.  *form (may
 * be NULL) receives 1 for the product, 0 for the substitution.  Q may alias
 * A.  n <= 256. */
rclupp_status_t rclupp_trsm_emulated_wellcond(rclupp_handle_t handle, int64_t m, int64_t n,
                                              const double *A, int64_t lda, const double *R,
                                              int64_t ldr, double *Q, int64_t ldq, int32_t *form);

/* Q = A R^{-1} by substitution (eq. (ewy), C3, C7) and, when G != NULL,
 * G = Q^T Q (C1, C5) in the same pass.  R: n x n upper, nonzero diagonal.
 * Q may alias A. */
rclupp_status_t rclupp_trsm_gram(rclupp_handle_t handle, int64_t m, int64_t n, const double *A,
                                 int64_t lda, const double *R, int64_t ldr, double *Q, int64_t ldq,
                                 double *G, int64_t ldg);

/* Upper Cholesky factor of an SPD n x n G (the Cholesky factorization of Algorithm 1; C2, C6).
 * Returns ERR_CHOL_BREAKDOWN with *col (if non-NULL) = failing column. */
rclupp_status_t rclupp_cholesky(rclupp_handle_t handle, int64_t n, const double *G, int64_t ldg,
                                double *R, int64_t ldr, int64_t *col);

/* C = A B for upper-triangular n x n A, B (eq. (ey), C4, C8). */
rclupp_status_t rclupp_trmm_upper(rclupp_handle_t handle, int64_t n, const double *A, int64_t lda,
                                  const double *B, int64_t ldb, double *C, int64_t ldc);

/* Tall LU with partial pivoting, in place ([M, N, P] = LU(X) of Algorithms 4
 * and 7): on return the strict lower part of A holds M (unit diagonal
 * implied), its top n x n upper triangle holds N, and ipiv (DEVICE, n int32)
 * holds 0-based row interchanges (row k swapped with ipiv[k] >= k).  The
 * pivot is the first row of largest magnitude (smallest index on ties).
 * Returns ERR_LU_ZERO_PIVOT with *col = k for a zero pivot, ERR_NONFINITE
 * with *col = k when column k has no finite candidate (NaN candidates are
 * skipped). */
rclupp_status_t rclupp_tall_lupp(rclupp_handle_t handle, int64_t m, int64_t n, double *A,
                                 int64_t lda, int32_t *ipiv, int64_t *col);

/* R1 from a sketched s x n matrix Y (the preconditioner of Algorithm 6): LU with partial
 * pivoting of Y, R-factor of the Householder QR of M, R1 = R0 N, diagonal
 * signs normalised.  Y is not modified.  Errors: ERR_LU_ZERO_PIVOT,
 * ERR_NONFINITE (as rclupp_tall_lupp). */
rclupp_status_t rclupp_sketch_precond(rclupp_handle_t handle, int64_t s, int64_t n,
                                      const double *Y, int64_t ldy, double *R1, int64_t ldr);

/* rclupp_sketch_precond (Algorithm 6's preconditioner) with the R-factor R0
 * chosen by r0_method (rclupp_r0_method_t): Householder as in Algorithm 6, or
 * Givens rotations (Section 1; remark after Algorithm 5).  Givens: per
 * column a tree of rotations over the
 * rows (each CTA's rows, then the CTAs' head rows), r = hypot(a, b) >= 0,
 * c = a / r, s = b / r; needs the matrix to fit a cluster's shared memory
 * (else RCLUPP_ERR_UNSUPPORTED). */
rclupp_status_t rclupp_sketch_precond_r0(rclupp_handle_t handle, int64_t s, int64_t n,
                                         const double *Y, int64_t ldy, int32_t r0_method, double *R1,
                                         int64_t ldr);

/* R-factor of an s x n matrix A by Givens rotations (Section 1; remark after
 * Algorithm 5), as one cluster of CTAs: rows of R with a negative diagonal
 * entry (possible only where the subcolumn below it was already zero) are
 * negated, so R has a non-negative diagonal.  A not modified.  The matrix
 * must fit a cluster's shared memory, else RCLUPP_ERR_UNSUPPORTED. */
rclupp_status_t rclupp_givens_r(rclupp_handle_t handle, int64_t s, int64_t n, const double *A,
                                int64_t lda, double *R, int64_t ldr);

/* R-factor of the Householder QR of an s x n matrix A (R0 in Algorithms 5 and
 * 6): LAPACK larfg sign convention, A not modified. */
rclupp_status_t rclupp_householder_r(rclupp_handle_t handle, int64_t s, int64_t n,
                                     const double *A, int64_t lda, double *R, int64_t ldr);

/* ---- bounded waits and fault injection (no counterpart in the paper) -----
 * The tall LU (rclupp_r_factor, lc2_factor, rclupp_tall_lupp) runs each
 * panel's column steps in one cooperative launch whose CTAs meet at a
 * grid-wide barrier after every pivot selection; each wait there is bounded
 * and, when it runs out, the call returns RCLUPP_ERR_TIMEOUT (failed_step 2,
 * info / *col = the column whose pivot was being waited for) with the handle
 * still usable.  Under stream capture (and where the device refuses the
 * cooperative launch) every column step is its own launch and no device
 * wait exists.  These two calls let a caller (or a test of the failure path)
 * bound and exercise that wait. */

/* Limit of each grid-barrier wait of the handle's tall LUs, in nanoseconds of
 * %globaltimer time; 0 restores the default of 2 s.  Errors: ERR_ARG. */
rclupp_status_t rclupp_set_wait_limit(rclupp_handle_t handle, uint64_t limit_ns);

typedef enum {
    RCLUPP_FAULT_NONE = 0,             /* clear a pending injection */
    RCLUPP_FAULT_LU_BARRIER_STALL = 1  /* the next tall LU's first grid barrier expects one
                                          arrival more than its grid has, so its wait runs
                                          out (no device memory is touched wrongly) */
} rclupp_fault_t;

/* Arm (or clear) a one-shot fault for the handle's next tall LU; the call
 * that runs it consumes it.  Errors: ERR_ARG (unknown fault). */
rclupp_status_t rclupp_inject_fault(rclupp_handle_t handle, int32_t fault);

/* ---- allocation-free Gram (no counterpart in the paper) ------------------
 * G = A^T A (n x n, ldg >= n, both triangles), the same kernels as
 * rclupp_gram, for callers that cannot let a library allocate device memory:
 * hosts that reserve nearly all GPU memory for their own pool up front,
 * loops where cudaMalloc/cudaFree would add device-wide synchronization, and
 * callers that account for every buffer themselves.  No handle is needed and
 * nothing is allocated (no cudaMalloc, cudaFree or allocating library call):
 * the split-K partial sums and a status word live in a fixed array of
 * 8 MiB + 256 bytes inside the library, which every GPU that loads the
 * library holds until the process exits.
 *   m, n, A, lda : DEVICE matrix A (m x n, lda >= m), 1 <= n <= 128,
 *                  m < 2^31; larger n or m returns RCLUPP_ERR_UNSUPPORTED.
 *   G, ldg       : DEVICE output (caller-owned).
 *   stream       : cudaStream_t to run on (NULL = legacy default stream).
 * The call returns after its GPU work has finished (status read back).
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current) and caches it for the
 * life of the process; make that first call before any stream capture.  The
 * cache assumes the device is not reset (cudaDeviceReset) while the process
 * runs: a reset unloads the library's device image, and later calls would
 * use the stale address.  Every call on a device shares the array and
 * overwrites it: calls that overlap on the GPU race, so do not run two of
 * them concurrently on one device. */
rclupp_status_t rclupp_gram_noalloc(int64_t m, int64_t n, const double *A, int64_t lda, double *G,
                                    int64_t ldg, void *stream);

/* ---- instrumentation (no counterpart in the paper) ----------------------
 * Launch accounting and per-kernel timing for benchmarks.  Every kernel the
 * library launches increments a process-wide counter.  When profiling is
 * enabled, a CUDA event pair is recorded on the launching stream around each
 * kernel; rclupp_profile_get synchronizes on the recorded events and returns,
 * for one kernel class (0 <= kid < 19), the number of timed launches, their
 * summed duration in milliseconds and the class name (static string).
 * Classes: 0 sketch_gauss, 1 sketch_sparse, 2 gram, 3 trsm_gram (fused
 * TRSM + Gram), 4 trsm, 5 reduce, 6 lu_col, 7 lu_trailing, 8 lu_u12,
 * 9 small_precond, 10 cholesky, 11 trmm, 12 pad, 13 sketch_tc (tensor-core
 * sketch), 14 gram_emu, 15 emu_aux (exponent and digit-preparation kernels
 * of the emulated products), 16 trsm_emu, 17 sketch_srht, 18 fp64_peak
 * (the microbenchmark below).  Returns ERR_ARG
 * for an invalid class.  The open event of a launch is kept per kernel
 * class for the whole process, so enable timing only while one host thread
 * launches; the launch counter is exact with any number of threads.
 * Kernels launched inside a captured graph are counted when the graph is
 * launched and are not timed. */
void rclupp_profile_enable(int enable);
void rclupp_profile_reset(void);
int rclupp_profile_get(int kid, long long *launches, double *total_ms, const char **name);
unsigned long long rclupp_kernel_launches(void);

/* Measured FP64-pipe throughput of the current device, the denominator of
 * the binary64 kernels' roofline: 2 CTAs per SM of 256 threads, each thread
 * running 8 independent chains of 2^15 dependent DFMAs (a <- a b + c), timed
 * with CUDA events on `stream` (a cudaStream_t, NULL = legacy default); the
 * best of three launches after one warm-up.  *gflops = 2 x DFMAs / time;
 * *ms (may be NULL) its time; *sms and *clock_mhz (may be NULL) the device's
 * SM count and maximum SM clock as the runtime reports them, so a caller can
 * set the measured rate beside SMs x clock x the DFMAs per clock.  Runs for
 * about 0.1 s; synchronous.  Errors: ERR_ARG (gflops NULL), ERR_CUDA. */
rclupp_status_t rclupp_profile_fp64_peak(void *stream, double *gflops, double *ms, int32_t *sms,
                                         int32_t *clock_mhz);

#ifdef __cplusplus
}
#endif
#endif /* RCLUPP_H */
