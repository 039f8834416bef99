// Host-side launchers of the library's kernels (internal interface between
// the C-ABI layer and the kernel translation units).  All pointers are
// device pointers; every launcher enqueues on `stream` and returns the CUDA
// launch status.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace rq {

// Number of streaming multiprocessors of the current device (cached).
int num_sms();

// Builds a 2-D TMA descriptor for a column-major FP64 matrix (rows x cols,
// leading dimension ld) with a box of box_rows x box_cols.  Returns false
// when the matrix does not meet TMA's alignment rules (16-byte base address,
// 16-byte multiple stride) or the encoder is unavailable; callers then use
// plain loads.  With swizzle128 (box_rows = 16, one 128-byte line per
// column) the box lands with the 128-byte swizzle: the 16-byte chunk j of
// column c's line is stored at chunk j ^ (c % 8), so that eight threads
// reading chunk j of eight neighbouring columns hit distinct banks.
bool make_tma_map(CUtensorMap *map, const double *A, int64_t rows, int64_t cols, int64_t ld,
                  int box_rows, int box_cols, bool swizzle128 = false);

// ---- tall passes (tall.cu) ----
struct TallPlan {
    int bm;          // rows per tile
    int ncb;         // columns per tile slice (TMA box width)
    int64_t chunk;   // rows per CTA (multiple of bm)
    int grid_x;      // CTAs along the rows
};

// Launch shape of the tall passes, per host thread: `grid_div` divides the
// number of CTAs a pass aims for (grid_sms() = SMs / grid_div), `fine_tiles`
// selects the next smaller row tile of the TRSM and Gram passes where a
// variant exists.  The batched form sets it (RAII scope) while it captures a
// batch graph, so that many concurrent problems can use smaller launches;
// single calls use the default {1, 0}.
struct LaunchPolicy {
    int grid_div = 1;
    int fine_tiles = 0;
};
LaunchPolicy &launch_policy();
struct LaunchPolicyScope {
    LaunchPolicy saved;
    explicit LaunchPolicyScope(LaunchPolicy p) : saved(launch_policy()) { launch_policy() = p; }
    ~LaunchPolicyScope() { launch_policy() = saved; }
};
int grid_sms();

// Row partition of an m-row pass for a kernel with `ctas_per_sm` resident
// CTAs, rows per tile bm, and `ytiles` independent column/output tiles.
TallPlan plan_rows(int64_t m, int bm, int ctas_per_sm, int ytiles);

// Partial-sum buffer sizes (doubles).
size_t gram_partials_doubles(int64_t m, int n);
size_t sketch_partials_doubles(int64_t m, int n, int64_t s, int kind);

// G = A^T A into G (ldg), partial buffer `part` of gram_partials_doubles().
cudaError_t launch_gram(const double *A, int64_t lda, int64_t m, int n, int unit_lower, double *G,
                        int64_t ldg, double *part, DevStatus *st, cudaStream_t stream);

// G = A^T A for n <= 128 using at most max_parts CTAs; `part` holds
// max_parts x 16384 doubles.
cudaError_t launch_gram_bounded(const double *A, int64_t lda, int64_t m, int n, double *G,
                                int64_t ldg, double *part, int max_parts, DevStatus *st,
                                cudaStream_t stream);

// Q = A R^{-1} with R given as a padded upper factor RP (n_pad x n_pad,
// ld n_pad, zeros elsewhere) and rinv[n_pad] = 1 / diag; optionally G = Q^T Q.
cudaError_t launch_trsm_gram(const double *A, int64_t lda, int64_t m, int n, const double *RP,
                             const double *rinv, double *Q, int64_t ldq, double *G, int64_t ldg,
                             double *part, DevStatus *st, cudaStream_t stream);

// Y = S A (s x n, ldy); kind 0 Gaussian (generated from seed, or explicit S
// when S != nullptr), kind 1 sparse-sign, kind 2 subsampled randomized
// Hadamard of order 2^srht_b (srht_b = 0: the smallest power of two >= row0 + m).
// row0: global index of A's first row, for the generated sketches (entry
// (r, row0 + i) of S multiplies row i of A); 0 for a whole matrix.
cudaError_t launch_sketch(const double *A, int64_t lda, int64_t m, int n, int unit_lower, int kind,
                          int64_t s, int zeta, uint64_t seed, const double *S, int64_t lds,
                          double *Y, int64_t ldy, double *part, DevStatus *st,
                          cudaStream_t stream, int64_t row0 = 0, int srht_b = 0);

// The SRHT sketch (srht.cu): S = R H D / sqrt(s) with H of order 2^b,
// b >= srht_order_log2(row0 + m), s <= 2^b; partials in `part` as for
// launch_sketch, then the fixed-order reduction into Y.
int srht_order_log2(int64_t rows);
cudaError_t launch_sketch_srht(const double *A, int64_t lda, int64_t m, int n, int unit_lower, int64_t s,
                               uint64_t seed, int b, double *Y, int64_t ldy, double *part,
                               cudaStream_t stream, int64_t row0);

// Fixed-order sum of sketch partials: Y[r][c] = sum_p part[p][c*s_pad + r].
cudaError_t launch_reduce_sketch(const double *part, int nparts, int s, int n, int s_pad, int n_pad,
                                 double *Y, int64_t ldy, cudaStream_t stream);

// ---- small factorizations in one thread block cluster (small_cluster.cu) ----
// The s x n (n x n) matrix split by rows over 1..8 CTAs' shared memory.
// mode 0: R1 = R(HouseholderQR(M)) N from the LU P Y = M N (Nbuf: n x n
// scratch); mode 1: R1 = R(HouseholderQR(Y)) triu(Nsrc) (identity when
// Nsrc == nullptr).  Outputs as launch_sketch_precond / launch_cholesky.
// mode | kPrecondGivens: R0 by Givens rotations instead of Householder.
constexpr int kPrecondGivens = 2;
bool precond_cluster_fits(int s, int n, bool givens = false);
cudaError_t launch_precond_cluster(const double *Y, int64_t ldy, int s, int n, int mode,
                                   const double *Nsrc, int64_t ldn, double *Nbuf, double *RP,
                                   double *rinv, double *R1, int64_t ldr, DevStatus *st, int step,
                                   cudaStream_t stream);
bool cholesky_cluster_fits(int n);
cudaError_t launch_cholesky_cluster(const double *G, int64_t ldg, int n, double *RP, double *rinv,
                                    double *R, int64_t ldr, DevStatus *st, int step,
                                    cudaStream_t stream);

// ---- tensor-core sketch (tc_sketch.cu) ----
// Y = S X with S's entries bf16 levels of a discretised normal and X split
// into nterms (1 or 3) bf16 terms, fp32 accumulation on tcgen05 (n <= 256).
cudaError_t launch_sketch_tc(const double *X, int64_t ldx, int64_t m, int n, int unit_lower,
                             int64_t s, uint64_t seed, int nterms, double *Y, int64_t ldy,
                             double *part, DevStatus *st, cudaStream_t stream, int64_t row0 = 0);
size_t tc_sketch_smem_bytes(int n, int nterms);
// The digit tier's sketch (tc_sketch.cu): the same S, X rounded to 48 bits of
// each column (six base-256 digits), exact integer sums on the tensor cores,
// binary64 across windows and CTAs.  part: sketch_digits_partials_doubles().
cudaError_t launch_sketch_digits(const double *X, int64_t ldx, int64_t m, int n, int unit_lower,
                                 int64_t s, uint64_t seed, double *Y, int64_t ldy, double *part,
                                 DevStatus *st, cudaStream_t stream, int64_t row0 = 0);
size_t sketch_digits_partials_doubles(int64_t s, int n);
// The reduced tier's level table (bf16 levels of the discretised normal) on
// the current device, written once per device; called at handle creation.
cudaError_t ensure_sketch_levels();

// ---- binary64-emulating Gram on the tensor cores (emu_gram.cu) ----
// G = A^T A (n <= 256) from seven balanced base-256 digits of every element
// (per-column exponents), exact fp32 level sums over 128-row windows,
// int64/fp32 drains and a fixed-order binary64 reduction.  part holds the
// per-CTA partials and the column exponents (gram_emu_partials_doubles).
cudaError_t launch_gram_emu(const double *A, int64_t lda, int64_t m, int n, double *G, int64_t ldg,
                            double *part, DevStatus *st, cudaStream_t stream);
size_t gram_emu_partials_doubles(int n);

// ---- triangular solve with binary64-emulating block products (emu_trsm.cu) ----
// Q = A R^{-1} by 16-column (n <= 128) or 32-column blocks: the off-diagonal block products on the
// tensor cores (digits of Q's rows and R's columns, exact fp32 level sums,
// int64 drains), the diagonal blocks in binary64.  RP/rinv as for
// launch_trsm_gram (padded factor followed by its row-major copy); scratch
// holds R's digit tiles (trsm_emu_scratch_bytes).  Q may alias A.
// skip_if: when non-null, the kernels return at once if the estimate stored
// there selects the product form (launch_trsm_emu_wellcond).
cudaError_t launch_trsm_emu(const double *A, int64_t lda, int64_t m, int n, const double *RP,
                            const double *rinv, double *Q, int64_t ldq, void *scratch,
                            DevStatus *st, cudaStream_t stream,
                            const unsigned long long *skip_if = nullptr);
size_t trsm_emu_scratch_bytes(int n);
// The 32-column-block form (emu_trsm32.cu) that launch_trsm_emu uses for n > 160.
cudaError_t launch_trsm_emu32(const double *A, int64_t lda, int64_t m, int n, const double *RP,
                              const double *rinv, double *Q, int64_t ldq, void *scratch,
                              DevStatus *st, cudaStream_t stream,
                              const unsigned long long *skip_if = nullptr);
size_t trsm_emu32_scratch_bytes(int n);
// Q = A R^{-1} for a factor expected to be well conditioned (emu_wprod.cu):
// W = R^{-1} in binary64 and Skeel's condition number || |W| |R| ||_inf;
// then either the emulated product Q = A W (cond <= max(100, n)) or the
// substitution form, chosen on the device.  scratch: wellcond_scratch_bytes(n).
// Q may alias A.
cudaError_t launch_trsm_emu_wellcond(const double *A, int64_t lda, int64_t m, int n, const double *RP,
                                     const double *rinv, double *Q, int64_t ldq, void *scratch,
                                     DevStatus *st, cudaStream_t stream);
size_t wprod_scratch_bytes(int n);
// Which form the last launch_trsm_emu_wellcond with this scratch ran: 1 the
// product, 0 the substitution, -1 a CUDA error (synchronizes the stream).
int wellcond_used_product(const void *scratch, int n, cudaStream_t stream);
inline size_t wellcond_scratch_bytes(int n) {
    return size_t(round_up(int64_t(trsm_emu_scratch_bytes(n)), 1024)) + wprod_scratch_bytes(n);
}

// Padded upper factor: RP = triu(R) padded to n_pad with zeros, rinv = 1/diag.
cudaError_t launch_pad_upper(const double *R, int64_t ldr, int n, double *RP, double *rinv,
                             cudaStream_t stream);


// ---- tall LU with partial pivoting (lu.cu) ----
// Bounded-wait options of the panel launches: limit_ns (0 = the default
// limit) for each wait at the grid-wide barrier; stall = 1 makes the first
// barrier of the first panel launch expect one arrival more than the grid has,
// so that its wait runs out (fault injection for tests).
struct LuWaitOptions {
    uint64_t limit_ns = 0;
    int stall = 0;
};
size_t lu_scratch_bytes(int64_t m, int n);
cudaError_t launch_tall_lupp(double *A, int64_t lda, int64_t m, int n, int32_t *ipiv,
                             void *scratch, DevStatus *st, int step_id, cudaStream_t stream,
                             const LuWaitOptions *wopt = nullptr);

// ---- small dense factorizations on one CTA (small.cu) ----
// R1 from the sketch Y (s x n): LU with partial pivoting, Householder R of
// M, R1 = R0 N, diagonal signs normalised.  Writes R1 into RP/rinv (padded)
// and, when R1 != nullptr, into R1 (ld ldr).  W: s*n*2 doubles scratch.
// r0_method 1: R0 by Givens rotations (cluster form only; cudaErrorNotSupported
// when the matrix does not fit a cluster's shared memory).
cudaError_t launch_sketch_precond(const double *Y, int64_t ldy, int s, int n, double *W,
                                  double *RP, double *rinv, double *R1, int64_t ldr,
                                  DevStatus *st, int step_id, cudaStream_t stream, int r0_method = 0);

// RCLUPPr's R1 from the sketched factor M_s (s x n): Householder R of M_s,
// R1 = R0 N with N the top of the in-place tall LU (lda), signs normalised.
// W: 2*s*n scratch.
cudaError_t launch_rcluppr_r1(const double *Ms, int64_t ldm, int s, int n, const double *LU,
                              int64_t lda, double *W, double *RP, double *rinv,
                              cudaStream_t stream, int r0_method = 0);

// RCholeskyQR's R1: Householder R of the sketch K (s x n), signs normalised.
cudaError_t launch_rcholqr_r1(const double *K, int64_t ldk, int s, int n, double *W, double *RP,
                              double *rinv, cudaStream_t stream, int r0_method = 0);

// R-factor of A (s x n) by Givens rotations, rows with a negative diagonal
// negated (only where a subcolumn was already zero), into R (ldr) and the
// padded RP/rinv; cluster form only (cudaErrorNotSupported otherwise).
cudaError_t launch_givens_r(const double *A, int64_t lda, int s, int n, double *W, double *RP,
                            double *rinv, double *R, int64_t ldr, cudaStream_t stream);

// Gs = G + s I with SCholeskyQR3's shift s = 11 (mnu + n(n+1)u) max_j G_jj.
cudaError_t launch_shifted_gram(const double *G, int64_t ldg, int n, int64_t m, double *Gs,
                                cudaStream_t stream);

// R-factor of the Householder QR of A (s x n) into R (ldr); W: s*n scratch.
cudaError_t launch_householder_r(const double *A, int64_t lda, int s, int n, double *W, double *R,
                                 int64_t ldr, cudaStream_t stream);

// Upper Cholesky of G (n x n); writes padded RP/rinv and, when R != nullptr,
// R (ldr).  W: n*n scratch.  Breakdown -> status with step_id and column.
cudaError_t launch_cholesky(const double *G, int64_t ldg, int n, double *W, double *RP,
                            double *rinv, double *R, int64_t ldr, DevStatus *st, int step_id,
                            cudaStream_t stream);

// C = triu(A) triu(B) (n x n), written to C (ldc) with zeros below the diagonal.
cudaError_t launch_trmm_upper(const double *A, int64_t lda, const double *B, int64_t ldb, int n,
                              double *C, int64_t ldc, cudaStream_t stream);

// LC2's R1 = Sc N with N read from the top of an in-place LU (lda), signs
// normalised; output padded RP/rinv.
cudaError_t launch_lc2_r1(const double *Sc, int64_t lds, const double *LU, int64_t lda, int n,
                          double *RP, double *rinv, cudaStream_t stream);

}  // namespace rq

namespace rq {

// ---- launch accounting and per-kernel timing (prof.cu) ----
// Kernel classes timed by the optional profiler.
enum KernelId : int {
    KID_SKETCH_GAUSS = 0,
    KID_SKETCH_SPARSE,
    KID_GRAM,
    KID_TRSM_GRAM,
    KID_TRSM,
    KID_REDUCE,
    KID_LU_COL,
    KID_LU_TRAILING,
    KID_LU_U12,
    KID_SMALL_PRECOND,
    KID_CHOLESKY,
    KID_TRMM,
    KID_PAD,
    KID_SKETCH_TC,
    KID_GRAM_EMU,
    KID_EMU_AUX,
    KID_TRSM_EMU,
    KID_SKETCH_SRHT,
    KID_FP64_PEAK,
    KID_COUNT
};

// Every kernel launch of the library goes through these two calls: the
// launch counter is always kept; when profiling is enabled an event pair
// brackets the launch on its stream.
void prof_begin(int kid, cudaStream_t stream);
void prof_end(int kid, cudaStream_t stream);
void prof_add_launches(unsigned long long k);

#define RQ_LAUNCH(KID, STREAM, ...)       \
    do {                                  \
        ::rq::prof_begin((KID), (STREAM)); \
        __VA_ARGS__;                      \
        ::rq::prof_end((KID), (STREAM));   \
    } while (0)

}  // namespace rq
