// C ABI of the library (declared in include/rclupp.h): handles, workspace,
// argument checks, and the drivers that sequence the tall passes and the
// small factorizations in the order the algorithm boxes fix.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <utility>
#include <vector>

#include "../../include/rclupp.h"
#include "common.cuh"
#include "kernels.h"

using namespace rq;

namespace {
constexpr int kMaxBranches = 64;
}

struct rclupp_handle_s {
    cudaStream_t stream = nullptr;
    int device = 0;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    DevStatus *d_status = nullptr;
    DevStatus *h_status = nullptr;  // pinned
    // batched form: parallel branches of the batch graph and the cached graph
    int batch_branches = 16;
    int batch_grid_div = 1;    // launch policy inside the batch graph (LaunchPolicy)
    int batch_fine_tiles = 0;
    int nstreams = 0;
    cudaStream_t bstreams[kMaxBranches] = {};
    cudaEvent_t join[kMaxBranches] = {};
    cudaEvent_t fork = nullptr;
    cudaStream_t cap = nullptr;  // origin stream of the batch graph's capture
    cudaGraphExec_t graph_exec = nullptr;
    std::vector<unsigned char> graph_desc;  // description the cached graph was captured for
    unsigned long long graph_kernels = 0;
    // bounded waits of the tall LU's grid-wide barrier: limit (0 = default)
    // and the one-shot stall a test injects (rclupp_inject_fault)
    uint64_t lu_wait_limit_ns = 0;
    int lu_stall = 0;
};

namespace {

rclupp_status_t ensure_streams(rclupp_handle_t h, int k) {
    if (!h->fork && cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming) != cudaSuccess)
        return RCLUPP_ERR_CUDA;
    if (!h->cap && cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess)
        return RCLUPP_ERR_CUDA;
    while (h->nstreams < k) {
        const int i = h->nstreams;
        if (cudaStreamCreateWithFlags(&h->bstreams[i], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&h->join[i], cudaEventDisableTiming) != cudaSuccess)
            return RCLUPP_ERR_CUDA;
        ++h->nstreams;
    }
    return RCLUPP_OK;
}

// Byte image of the batch description (graph cache key): the cached graph is
// replayed only when every byte of the new description equals the stored one.
struct DescBytes {
    std::vector<unsigned char> b;
    template <class T>
    void add(const T *p, size_t count) {
        const unsigned char *q = reinterpret_cast<const unsigned char *>(p);
        b.insert(b.end(), q, q + count * sizeof(T));
    }
};

std::vector<unsigned char> batch_description(int algo, int count, const int64_t *m,
                                             const int64_t *n, const double *const *X,
                                             const int64_t *ldx, double *const *Q,
                                             const int64_t *ldq, double *const *R,
                                             const int64_t *ldr, const rclupp_opts_t *o,
                                             int branches, const void *ws,
                                             const LaunchPolicy &pol) {
    DescBytes f;
    f.add(&algo, 1);
    f.add(&count, 1);
    f.add(m, count);
    f.add(n, count);
    f.add(X, count);
    f.add(ldx, count);
    f.add(Q, count);
    f.add(ldq, count);
    f.add(R, count);
    f.add(ldr, count);
    f.add(o, count);
    f.add(&branches, 1);
    f.add(&ws, 1);
    f.add(&pol.grid_div, 1);
    f.add(&pol.fine_tiles, 1);
    return std::move(f.b);
}

constexpr int kMaxN = 256;
constexpr int64_t kMaxS = 4096;

// Carves aligned sub-buffers out of the handle's workspace.
struct Carver {
    char *base;
    size_t off = 0;
    explicit Carver(void *b) : base(static_cast<char *>(b)) {}
    template <class T>
    T *take(size_t count) {
        off = (off + 255) & ~size_t(255);
        T *p = reinterpret_cast<T *>(base ? base + off : nullptr);
        off += count * sizeof(T);
        return p;
    }
};

// Device buffers of one factorization.
struct Bufs {
    double *part;
    double *Y;
    double *W;
    double *RP[5];
    double *rinv[5];
    double *G;
    void *lu;
    int32_t *ipiv;
    double *LUbuf;
};

Bufs carve(void *base, int64_t m, int n, int64_t s, bool need_lu_copy, size_t *total) {
    Carver c(base);
    Bufs b;
    const int n_pad = pad16(n);
    const size_t part = std::max({gram_partials_doubles(m, n), sketch_partials_doubles(m, n, s, 0),
                                  sketch_digits_partials_doubles(s, n), gram_emu_partials_doubles(n),
                                  wellcond_scratch_bytes(n) / 8 + 1});
    b.part = c.take<double>(part);
    b.Y = c.take<double>(size_t(std::max<int64_t>(s, 1)) * n);
    b.W = c.take<double>(std::max(size_t(2) * std::max<int64_t>(s, n) * n, size_t(n) * n));
    for (int i = 0; i < 5; ++i) {
        b.RP[i] = c.take<double>(size_t(2) * n_pad * n_pad);  // column- then row-major
        b.rinv[i] = c.take<double>(n_pad);
    }
    b.G = c.take<double>(size_t(n) * n);
    b.lu = c.take<char>(lu_scratch_bytes(m, n));
    b.ipiv = c.take<int32_t>(n);
    b.LUbuf = need_lu_copy ? c.take<double>(size_t(m) * n) : nullptr;
    *total = c.off + 256;
    return b;
}

rclupp_status_t from_cuda(cudaError_t e) { return e == cudaSuccess ? RCLUPP_OK : RCLUPP_ERR_CUDA; }

rclupp_status_t ensure_ws(rclupp_handle_t h, size_t bytes) {
    if (h->ws_bytes >= bytes) return RCLUPP_OK;
    if (h->ws) {
        cudaStreamSynchronize(h->stream);
        if (h->graph_exec) {  // a cached batch graph points into the old workspace
            cudaGraphExecDestroy(h->graph_exec);
            h->graph_exec = nullptr;
        }
        cudaFree(h->ws);
        h->ws = nullptr;
        h->ws_bytes = 0;
    }
    if (cudaMalloc(&h->ws, bytes) != cudaSuccess) {
        cudaGetLastError();
        return RCLUPP_ERR_NOMEM;
    }
    h->ws_bytes = bytes;
    return RCLUPP_OK;
}

Bufs prepare(rclupp_handle_t h, int64_t m, int n, int64_t s, bool need_lu_copy,
             rclupp_status_t *status) {
    size_t total = 0;
    carve(nullptr, m, n, s, need_lu_copy, &total);
    *status = ensure_ws(h, total);
    Bufs b{};
    if (*status != RCLUPP_OK) return b;
    b = carve(h->ws, m, n, s, need_lu_copy, &total);
    if (cudaMemsetAsync(h->d_status, 0, sizeof(DevStatus), h->stream) != cudaSuccess)
        *status = RCLUPP_ERR_CUDA;
    return b;
}

// Waits for the stream and converts the device status.
rclupp_status_t finish(rclupp_handle_t h, rclupp_status_t launch_status, rclupp_info_t *info,
                       int64_t *col) {
    if (launch_status == RCLUPP_OK) {
        if (cudaMemcpyAsync(h->h_status, h->d_status, sizeof(DevStatus), cudaMemcpyDeviceToHost,
                            h->stream) != cudaSuccess)
            launch_status = RCLUPP_ERR_CUDA;
    }
    const cudaError_t se = cudaStreamSynchronize(h->stream);
    rclupp_status_t st = launch_status;
    int step = 0;
    long long inf = -1;
    if (st == RCLUPP_OK && se != cudaSuccess) st = RCLUPP_ERR_CUDA;
    if (st == RCLUPP_OK && h->h_status->code != 0) {
        st = static_cast<rclupp_status_t>(h->h_status->code);
        step = h->h_status->step;
        inf = h->h_status->info;
    }
    if (info) {
        info->status = st;
        info->failed_step = step;
        info->info = inf;
        info->prec_used = RCLUPP_PREC_FP64;
        info->emulated = 0;
    }
    if (col) *col = inf;
    return st;
}

bool bad_ld(int64_t ld, int64_t rows) { return ld < std::max<int64_t>(rows, 1); }

rclupp_status_t check_common(rclupp_handle_t h, int64_t m, int64_t n, const void *X, int64_t ldx,
                             const void *Q, int64_t ldq, const void *R, int64_t ldr) {
    if (!h || !X || !Q || !R) return RCLUPP_ERR_ARG;
    if (n < 1 || m < n) return RCLUPP_ERR_ARG;
    if (bad_ld(ldx, m) || bad_ld(ldq, m) || bad_ld(ldr, n)) return RCLUPP_ERR_ARG;
    if (n > kMaxN || m >= (int64_t(1) << 31)) return RCLUPP_ERR_UNSUPPORTED;
    return RCLUPP_OK;
}

rclupp_opts_t resolve_opts(const rclupp_opts_t *opts, int64_t n) {
    rclupp_opts_t o;
    std::memset(&o, 0, sizeof o);
    if (opts) o = *opts;
    else {
        o.kind = RCLUPP_SKETCH_GAUSSIAN;
        o.s = 2 * n;
        o.zeta = 8;
        o.seed = 0;
        o.prec = RCLUPP_PREC_FP64;
    }
    return o;
}

rclupp_status_t check_opts(const rclupp_opts_t &o, int64_t m, int64_t n) {
    if (o.s < n || o.s > kMaxS) return o.s < n ? RCLUPP_ERR_ARG : RCLUPP_ERR_UNSUPPORTED;
    if (o.kind != RCLUPP_SKETCH_GAUSSIAN && o.kind != RCLUPP_SKETCH_SPARSE_SIGN &&
        o.kind != RCLUPP_SKETCH_SRHT)
        return RCLUPP_ERR_ARG;
    if (o.S && o.lds < o.s) return RCLUPP_ERR_ARG;
    if (o.kind == RCLUPP_SKETCH_SRHT && !o.S) {
        // H of order 2^b must cover the rows and have s distinct rows to sample
        if (o.order_log2 < 0 || o.order_log2 > 31) return RCLUPP_ERR_ARG;
        const int b = o.order_log2 > 0 ? o.order_log2 : srht_order_log2(m);
        if (b > 31) return RCLUPP_ERR_UNSUPPORTED;
        if ((int64_t(1) << b) < m || (int64_t(1) << b) < o.s) return RCLUPP_ERR_ARG;
    }
    if (o.kind == RCLUPP_SKETCH_SPARSE_SIGN && !o.S) {
        if (o.zeta < 1 || o.zeta > o.s) return RCLUPP_ERR_ARG;
        if (o.zeta > 16) return RCLUPP_ERR_UNSUPPORTED;
        const size_t smem = size_t(round_up(o.s, 64)) * 32 * 8 + 64 * 33 * 8 + 64 * 16 * 4;
        if (smem > 220 * 1024) return RCLUPP_ERR_UNSUPPORTED;
    }
    if (o.prec != RCLUPP_PREC_FP64 && o.prec != RCLUPP_PREC_SKETCH_BF16 &&
        o.prec != RCLUPP_PREC_SKETCH_FP32 && o.prec != RCLUPP_PREC_EMULATED &&
        o.prec != RCLUPP_PREC_EMULATED_ALL && o.prec != RCLUPP_PREC_SKETCH_DIGITS)
        return RCLUPP_ERR_ARG;
    if ((o.prec == RCLUPP_PREC_SKETCH_BF16 || o.prec == RCLUPP_PREC_SKETCH_FP32 ||
         o.prec == RCLUPP_PREC_SKETCH_DIGITS) && o.S)
        return RCLUPP_ERR_UNSUPPORTED;
    if (o.r0_method != RCLUPP_R0_HOUSEHOLDER && o.r0_method != RCLUPP_R0_GIVENS) return RCLUPP_ERR_ARG;
    // the Givens R0 runs in the cluster form only (the s x n matrix in shared memory)
    if (o.r0_method == RCLUPP_R0_GIVENS && !precond_cluster_fits(int(o.s), int(n), true))
        return RCLUPP_ERR_UNSUPPORTED;
    (void)m;
    return RCLUPP_OK;
}

// The sketch product at a precision tier: the tensor-core kernel for the
// generated Gaussian sketch at the reduced tiers, the binary64 kernels
// otherwise (the sparse-sign sketch only adds, so its tier is irrelevant).
cudaError_t sketch_step(const Bufs &b, const double *A, int64_t lda, int64_t m, int n,
                        int unit_lower, const rclupp_opts_t &o, int tier, DevStatus *ds,
                        cudaStream_t s) {
    if (tier == RCLUPP_PREC_SKETCH_DIGITS && o.kind == RCLUPP_SKETCH_GAUSSIAN && !o.S)
        return launch_sketch_digits(A, lda, m, n, unit_lower, o.s, o.seed, b.Y, o.s, b.part, ds, s);
    if (tier != RCLUPP_PREC_FP64 && o.kind == RCLUPP_SKETCH_GAUSSIAN && !o.S)
        return launch_sketch_tc(A, lda, m, n, unit_lower, o.s, o.seed,
                                tier == RCLUPP_PREC_SKETCH_FP32 ? 3 : 1, b.Y, o.s, b.part, ds, s);
    return launch_sketch(A, lda, m, n, unit_lower, o.kind, o.s, o.zeta, o.seed, o.S, o.lds, b.Y, o.s,
                         b.part, ds, s, 0, o.order_log2);
}

// A reduced-precision sketch leaves Q1 = X R1^{-1} less well conditioned
// (its error acts like a perturbation of S of the sketch's relative size).
// Accept the first Cholesky only if it succeeded and the spread of R2's
// diagonal (a lower bound on kappa(Q1)) stays below this.
constexpr double kEscalateRatio = 1.0e4;

int next_tier(int tier) {
    return tier == RCLUPP_PREC_SKETCH_BF16 ? RCLUPP_PREC_SKETCH_FP32 : RCLUPP_PREC_FP64;
}

enum class FirstPassOutcome { Accept, Escalate, Fail };

// Synchronizes the stream and assesses the first Cholesky of a reduced tier.
FirstPassOutcome assess_first_pass(rclupp_handle_t h, const Bufs &b, int n) {
    const int np = pad16(n);
    double diag[256];
    if (cudaMemcpyAsync(h->h_status, h->d_status, sizeof(DevStatus), cudaMemcpyDeviceToHost,
                        h->stream) != cudaSuccess ||
        cudaMemcpy2DAsync(diag, sizeof(double), b.RP[1], size_t(np + 1) * sizeof(double),
                          sizeof(double), size_t(n), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
        return FirstPassOutcome::Fail;
    const DevStatus &ds = *h->h_status;
    if (ds.code != 0)
        return (ds.code == RCLUPP_ERR_CHOL_BREAKDOWN && ds.step == 3) ? FirstPassOutcome::Escalate
                                                                       : FirstPassOutcome::Fail;
    double lo = diag[0], hi = diag[0];
    for (int i = 1; i < n; ++i) {
        lo = std::min(lo, diag[i]);
        hi = std::max(hi, diag[i]);
    }
    return (!(lo > 0.0) || hi / lo > kEscalateRatio) ? FirstPassOutcome::Escalate
                                                      : FirstPassOutcome::Accept;
}

#define RQ_TRY(expr)                                     \
    do {                                                 \
        const cudaError_t _e = (expr);                   \
        if (_e != cudaSuccess) return RCLUPP_ERR_CUDA;   \
    } while (0)

// Where a factorization's work is enqueued: its stream and its status word.
struct Ctx {
    cudaStream_t s;
    DevStatus *st;
};

// The tall LU's wait options of a single call; consumes the one-shot stall.
LuWaitOptions take_lu_wait(rclupp_handle_t h) {
    LuWaitOptions w;
    w.limit_ns = h->lu_wait_limit_ns;
    w.stall = h->lu_stall;
    h->lu_stall = 0;
    return w;
}

Ctx ctx_of(rclupp_handle_t h) { return Ctx{h->stream, h->d_status}; }

// The CholeskyQR2 stage of Algorithms 6 and 7 (C1-C8): Q1 = X R1^{-1} with R1 in
// b.RP[0]; CholeskyQR2 of Q1 into Q (in place after the first pass);
// R = R4 (R2 R1).
// First CholeskyQR step on Q1 = X R1^{-1}: G = Q1^T Q1 (C1), R2 = chol(G) (C2).
// With `emu_solve` the triangular solve's block products run on the tensor
// cores emulating binary64, with `emu_gram` the Gram.
rclupp_status_t first_cholqr_pass(Ctx c, const Bufs &b, int64_t m, int n, const double *X,
                                  int64_t ldx, double *Q, int64_t ldq, bool emu_solve = false,
                                  bool emu_gram = false) {
    cudaStream_t s = c.s;
    DevStatus *st = c.st;
    if (emu_solve || emu_gram) {
        if (emu_solve)
            RQ_TRY(launch_trsm_emu(X, ldx, m, n, b.RP[0], b.rinv[0], Q, ldq, b.part, st, s));
        else
            RQ_TRY(launch_trsm_gram(X, ldx, m, n, b.RP[0], b.rinv[0], Q, ldq, nullptr, 0, b.part, st, s));
        if (emu_gram)
            RQ_TRY(launch_gram_emu(Q, ldq, m, n, b.G, n, b.part, st, s));
        else
            RQ_TRY(launch_gram(Q, ldq, m, n, 0, b.G, n, b.part, st, s));
    } else {
        RQ_TRY(launch_trsm_gram(X, ldx, m, n, b.RP[0], b.rinv[0], Q, ldq, b.G, n, b.part, st, s));
    }
    RQ_TRY(launch_cholesky(b.G, n, n, b.W, b.RP[1], b.rinv[1], nullptr, 0, st, 3, s));
    return RCLUPP_OK;
}

// The rest of C3-C8 after R2 is known.  With `emulated` both triangular
// solves use the emulated block products; the Gram of this final pass (C5)
// stays binary64 unless `emu_final_gram`.
rclupp_status_t rest_cholqr2(Ctx c, const Bufs &b, int64_t m, int n, double *Q, int64_t ldq,
                             double *R, int64_t ldr, bool emulated = false,
                             bool emu_final_gram = false) {
    cudaStream_t s = c.s;
    DevStatus *st = c.st;
    const int np = pad16(n);
    RQ_TRY(launch_trmm_upper(b.RP[1], np, b.RP[0], np, n, b.RP[2], np, s));  // R3 = R2 R1
    if (emulated) {
        // R2 has the condition number of Q1 (that of the sketch's embedding):
        // the product with R2^{-1} unless the estimate says otherwise
        RQ_TRY(launch_trsm_emu_wellcond(Q, ldq, m, n, b.RP[1], b.rinv[1], Q, ldq, b.part, st, s));
        if (emu_final_gram)
            RQ_TRY(launch_gram_emu(Q, ldq, m, n, b.G, n, b.part, st, s));
        else
            RQ_TRY(launch_gram(Q, ldq, m, n, 0, b.G, n, b.part, st, s));
    } else {
        RQ_TRY(launch_trsm_gram(Q, ldq, m, n, b.RP[1], b.rinv[1], Q, ldq, b.G, n, b.part, st, s));
    }
    RQ_TRY(launch_cholesky(b.G, n, n, b.W, b.RP[3], b.rinv[3], nullptr, 0, st, 4, s));
    RQ_TRY(launch_trmm_upper(b.RP[3], np, b.RP[2], np, n, R, ldr, s));  // R = R4 R3
    if (emulated)  // R4 = I + O(u kappa(Q1)^2)
        RQ_TRY(launch_trsm_emu_wellcond(Q, ldq, m, n, b.RP[3], b.rinv[3], Q, ldq, b.part, st, s));
    else
        RQ_TRY(launch_trsm_gram(Q, ldq, m, n, b.RP[3], b.rinv[3], Q, ldq, nullptr, 0, b.part, st, s));
    return RCLUPP_OK;
}

// Randomized drivers after the sketch: R1 from the sketch (the preconditioner
// `precond` of Algorithm 6 or 7), then CholeskyQR2
// of Q1 = X R1^{-1}.  At a reduced sketch tier the first Cholesky is assessed
// and, if it broke down or shows Q1 too ill-conditioned, the sketch is redone
// at the next tier (bf16 -> three-term bf16 -> binary64).  *tier_used reports
// the tier that produced the result.
template <class Precond>
rclupp_status_t randomized_tail(rclupp_handle_t h, const Bufs &b, const rclupp_opts_t &o,
                                int64_t m, int n, const double *SA, int64_t ldsa, int unit_lower,
                                Precond precond, const double *X, int64_t ldx, double *Q,
                                int64_t ldq, double *R, int64_t ldr, int *tier_used) {
    // the emulated tiers sketch at the digit tier (on the tensor cores when
    // the Gaussian sketch is generated, else in binary64)
    const bool emulated = o.prec == RCLUPP_PREC_EMULATED || o.prec == RCLUPP_PREC_EMULATED_ALL;
    int tier = o.prec;
    if (emulated) tier = RCLUPP_PREC_SKETCH_DIGITS;
    // only the generated Gaussian sketch has reduced tiers; the others are binary64
    if (o.kind != RCLUPP_SKETCH_GAUSSIAN || o.S) tier = RCLUPP_PREC_FP64;
    for (;;) {
        if (sketch_step(b, SA, ldsa, m, n, unit_lower, o, tier, h->d_status, h->stream) != cudaSuccess)
            return RCLUPP_ERR_CUDA;
        if (precond() != cudaSuccess) return RCLUPP_ERR_CUDA;
        // No a-priori test on R1 is made: a reduced-tier R1 only sees the
        // rounded X, whose condition number saturates near 1/u of the tier,
        // so R1 cannot tell an X the tier handles from one it does not.
        const rclupp_status_t st =
            first_cholqr_pass(ctx_of(h), b, m, n, X, ldx, Q, ldq, emulated, emulated);
        if (st != RCLUPP_OK) return st;
        // binary64 and the digit tier (48 bits, exact sums) are not escalated
        if (tier == RCLUPP_PREC_FP64 || tier == RCLUPP_PREC_SKETCH_DIGITS) break;
        const FirstPassOutcome v = assess_first_pass(h, b, n);
        if (v == FirstPassOutcome::Fail) break;  // the status is reported by finish()
        if (v == FirstPassOutcome::Accept) break;
        tier = next_tier(tier);
        if (cudaMemsetAsync(h->d_status, 0, sizeof(DevStatus), h->stream) != cudaSuccess)
            return RCLUPP_ERR_CUDA;
    }
    *tier_used = tier;
    return rest_cholqr2(ctx_of(h), b, m, n, Q, ldq, R, ldr, emulated,
                        o.prec == RCLUPP_PREC_EMULATED_ALL);
}

// copy an m x n matrix (device to device, possibly different leading dims)
cudaError_t copy_matrix(double *dst, int64_t ldd, const double *src, int64_t lds, int64_t m,
                        int64_t n, cudaStream_t s);

// ---- drivers as pure enqueues (no host synchronization) ----------------------
// They put the whole factorization on c.s with its status in c.st, so they
// can run several at once on different streams and be captured in a graph.
// Without a host round trip there is no escalation: the sketch runs at one
// tier, batch_sketch_tier(o).

// Sketch tier of a randomized factorization inside a batch: binary64 for
// RCLUPP_PREC_FP64, the three-term tensor-core tier (FP32 level, within
// CholeskyQR2's reach up to kappa(X) ~ 1e12) for RCLUPP_PREC_SKETCH_FP32, and
// the digit tier (48 bits, exact sums, reach ~1e15) for the digit and
// emulated tiers (the bf16 tier reaches only ~1e9 and needs the escalation a
// graph cannot make).  sketch_step() runs the sparse-sign, SRHT and explicit
// sketches in binary64 whatever the tier.
int batch_sketch_tier(const rclupp_opts_t &o) {
    if (o.prec == RCLUPP_PREC_FP64 || o.prec == RCLUPP_PREC_SKETCH_FP32) return o.prec;
    return RCLUPP_PREC_SKETCH_DIGITS;
}

// RCLUPP, Algorithm 6, sketch at batch_sketch_tier(o).
rclupp_status_t enqueue_rclupp(Ctx c, const Bufs &b, const rclupp_opts_t &o, int64_t m, int n,
                               const double *X, int64_t ldx, double *Q, int64_t ldq, double *R,
                               int64_t ldr) {
    RQ_TRY(sketch_step(b, X, ldx, m, n, 0, o, batch_sketch_tier(o), c.st, c.s));
    RQ_TRY(launch_sketch_precond(b.Y, o.s, int(o.s), n, b.W, b.RP[0], b.rinv[0], nullptr, 0, c.st, 1,
                                 c.s, o.r0_method));
    const bool emu = o.prec == RCLUPP_PREC_EMULATED || o.prec == RCLUPP_PREC_EMULATED_ALL;
    const rclupp_status_t st = first_cholqr_pass(c, b, m, n, X, ldx, Q, ldq, emu, emu);
    if (st != RCLUPP_OK) return st;
    return rest_cholqr2(c, b, m, n, Q, ldq, R, ldr, emu, o.prec == RCLUPP_PREC_EMULATED_ALL);
}

// RCLUPPr, Algorithm 7, sketch at batch_sketch_tier(o); the LU runs in L (ldl).
rclupp_status_t enqueue_rcluppr(Ctx c, const Bufs &b, const rclupp_opts_t &o, int64_t m, int n,
                                const double *X, int64_t ldx, double *L, int64_t ldl, double *Q,
                                int64_t ldq, double *R, int64_t ldr) {
    RQ_TRY(copy_matrix(L, ldl, X, ldx, m, n, c.s));
    RQ_TRY(launch_tall_lupp(L, ldl, m, n, b.ipiv, b.lu, c.st, 2, c.s));
    RQ_TRY(sketch_step(b, L, ldl, m, n, 1, o, batch_sketch_tier(o), c.st, c.s));
    RQ_TRY(launch_rcluppr_r1(b.Y, o.s, int(o.s), n, L, ldl, b.W, b.RP[0], b.rinv[0], c.s, o.r0_method));
    const bool emu = o.prec == RCLUPP_PREC_EMULATED || o.prec == RCLUPP_PREC_EMULATED_ALL;
    const rclupp_status_t st = first_cholqr_pass(c, b, m, n, X, ldx, Q, ldq, emu, emu);
    if (st != RCLUPP_OK) return st;
    return rest_cholqr2(c, b, m, n, Q, ldq, R, ldr, emu, o.prec == RCLUPP_PREC_EMULATED_ALL);
}

// CholeskyQR2, Algorithm 2.
rclupp_status_t enqueue_cholqr2(Ctx c, const Bufs &b, int64_t m, int n, const double *X,
                                int64_t ldx, double *Q, int64_t ldq, double *R, int64_t ldr) {
    const int np = pad16(n);
    // [Q1, R1] = CholeskyQR(X)
    RQ_TRY(launch_gram(X, ldx, m, n, 0, b.G, n, b.part, c.st, c.s));
    RQ_TRY(launch_cholesky(b.G, n, n, b.W, b.RP[0], b.rinv[0], nullptr, 0, c.st, 3, c.s));
    // [Q, Z] = CholeskyQR(Q1)
    RQ_TRY(launch_trsm_gram(X, ldx, m, n, b.RP[0], b.rinv[0], Q, ldq, b.G, n, b.part, c.st, c.s));
    RQ_TRY(launch_cholesky(b.G, n, n, b.W, b.RP[1], b.rinv[1], nullptr, 0, c.st, 4, c.s));
    // R = Z R1
    RQ_TRY(launch_trmm_upper(b.RP[1], np, b.RP[0], np, n, R, ldr, c.s));
    RQ_TRY(launch_trsm_gram(Q, ldq, m, n, b.RP[1], b.rinv[1], Q, ldq, nullptr, 0, b.part, c.st, c.s));
    return RCLUPP_OK;
}

// RCholeskyQR, Algorithm 5 (one sketch, one CholeskyQR), sketch at `tier`,
// emulated products as o.prec asks.
rclupp_status_t enqueue_rcholqr(Ctx c, const Bufs &b, const rclupp_opts_t &o, int tier, int64_t m,
                                int n, const double *X, int64_t ldx, double *Q, int64_t ldq,
                                double *R, int64_t ldr) {
    const int np = pad16(n);
    // K = S X; R1 = R of HouseholderQR(K)
    RQ_TRY(sketch_step(b, X, ldx, m, n, 0, o, tier, c.st, c.s));
    RQ_TRY(launch_rcholqr_r1(b.Y, o.s, int(o.s), n, b.W, b.RP[0], b.rinv[0], c.s, o.r0_method));
    // Q1 = X R1^{-1}; [Q, Z] = CholeskyQR(Q1); R = Z R1
    // the one CholeskyQR's Gram is the final-pass Gram: emulated only when
    // the caller asked for every Gram emulated (o.prec; `tier` is the sketch's)
    const bool emu = o.prec == RCLUPP_PREC_EMULATED || o.prec == RCLUPP_PREC_EMULATED_ALL;
    const rclupp_status_t st =
        first_cholqr_pass(c, b, m, n, X, ldx, Q, ldq, emu, o.prec == RCLUPP_PREC_EMULATED_ALL);
    if (st != RCLUPP_OK) return st;
    RQ_TRY(launch_trmm_upper(b.RP[1], np, b.RP[0], np, n, R, ldr, c.s));
    if (emu)
        RQ_TRY(launch_trsm_emu_wellcond(Q, ldq, m, n, b.RP[1], b.rinv[1], Q, ldq, b.part, c.st, c.s));
    else
        RQ_TRY(launch_trsm_gram(Q, ldq, m, n, b.RP[1], b.rinv[1], Q, ldq, nullptr, 0, b.part, c.st,
                                c.s));
    return RCLUPP_OK;
}

// SCholeskyQR3, Algorithm 3: G = X^T X; R1 = chol(G + s I); Q1 = X R1^{-1};
// [Q, Z] = CholeskyQR2(Q1); R = Z R1.
rclupp_status_t enqueue_scholqr3(Ctx c, const Bufs &b, int64_t m, int n, const double *X,
                                 int64_t ldx, double *Q, int64_t ldq, double *R, int64_t ldr) {
    RQ_TRY(launch_gram(X, ldx, m, n, 0, b.G, n, b.part, c.st, c.s));
    RQ_TRY(launch_shifted_gram(b.G, n, n, m, b.Y, c.s));
    RQ_TRY(launch_cholesky(b.Y, n, n, b.W, b.RP[0], b.rinv[0], nullptr, 0, c.st, 6, c.s));
    const rclupp_status_t st = first_cholqr_pass(c, b, m, n, X, ldx, Q, ldq);
    if (st != RCLUPP_OK) return st;
    return rest_cholqr2(c, b, m, n, Q, ldq, R, ldr);
}

// LC2, Algorithm 4; the LU runs in L (ldl).
rclupp_status_t enqueue_lc2(Ctx c, const Bufs &b, int64_t m, int n, const double *X, int64_t ldx,
                            double *L, int64_t ldl, double *Q, int64_t ldq, double *R,
                            int64_t ldr, const LuWaitOptions *wopt = nullptr) {
    const int np = pad16(n);
    RQ_TRY(copy_matrix(L, ldl, X, ldx, m, n, c.s));
    // [M, N, P] = LU(X)
    RQ_TRY(launch_tall_lupp(L, ldl, m, n, b.ipiv, b.lu, c.st, 2, c.s, wopt));
    // G = M^T M; S = chol(G); R1 = S N
    RQ_TRY(launch_gram(L, ldl, m, n, 1, b.G, n, b.part, c.st, c.s));
    RQ_TRY(launch_cholesky(b.G, n, n, b.W, b.RP[4], b.rinv[4], nullptr, 0, c.st, 3, c.s));
    RQ_TRY(launch_lc2_r1(b.RP[4], np, L, ldl, n, b.RP[0], b.rinv[0], c.s));
    // Q1 = X R1^{-1}; [Q, Z] = CholeskyQR(Q1); R = Z R1
    RQ_TRY(launch_trsm_gram(X, ldx, m, n, b.RP[0], b.rinv[0], Q, ldq, b.G, n, b.part, c.st, c.s));
    RQ_TRY(launch_cholesky(b.G, n, n, b.W, b.RP[1], b.rinv[1], nullptr, 0, c.st, 4, c.s));
    RQ_TRY(launch_trmm_upper(b.RP[1], np, b.RP[0], np, n, R, ldr, c.s));
    RQ_TRY(launch_trsm_gram(Q, ldq, m, n, b.RP[1], b.rinv[1], Q, ldq, nullptr, 0, b.part, c.st, c.s));
    return RCLUPP_OK;
}

// copy an m x n matrix (device to device, possibly different leading dims)
cudaError_t copy_matrix(double *dst, int64_t ldd, const double *src, int64_t lds, int64_t m,
                        int64_t n, cudaStream_t s) {
    return cudaMemcpy2DAsync(dst, size_t(ldd) * 8, src, size_t(lds) * 8, size_t(m) * 8, size_t(n),
                             cudaMemcpyDeviceToDevice, s);
}

}  // namespace

extern "C" {

rclupp_status_t rclupp_create(rclupp_handle_t *handle, void *stream) {
    if (!handle) return RCLUPP_ERR_ARG;
    *handle = nullptr;
    rclupp_handle_s *h = new (std::nothrow) rclupp_handle_s();
    if (!h) return RCLUPP_ERR_NOMEM;
    h->stream = static_cast<cudaStream_t>(stream);
    if (cudaGetDevice(&h->device) != cudaSuccess ||
        cudaMalloc(&h->d_status, sizeof(DevStatus)) != cudaSuccess ||
        cudaMallocHost(&h->h_status, sizeof(DevStatus)) != cudaSuccess) {
        cudaGetLastError();
        if (h->d_status) cudaFree(h->d_status);
        delete h;
        return RCLUPP_ERR_CUDA;
    }
    cudaMemset(h->d_status, 0, sizeof(DevStatus));
    if (ensure_sketch_levels() != cudaSuccess) {
        cudaGetLastError();
        cudaFree(h->d_status);
        cudaFreeHost(h->h_status);
        delete h;
        return RCLUPP_ERR_CUDA;
    }
    *handle = h;
    return RCLUPP_OK;
}

rclupp_status_t rclupp_destroy(rclupp_handle_t h) {
    if (!h) return RCLUPP_ERR_ARG;
    cudaStreamSynchronize(h->stream);
    if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
    for (int i = 0; i < h->nstreams; ++i) {
        cudaStreamSynchronize(h->bstreams[i]);
        cudaStreamDestroy(h->bstreams[i]);
        cudaEventDestroy(h->join[i]);
    }
    if (h->fork) cudaEventDestroy(h->fork);
    if (h->cap) cudaStreamDestroy(h->cap);
    if (h->ws) cudaFree(h->ws);
    if (h->d_status) cudaFree(h->d_status);
    if (h->h_status) cudaFreeHost(h->h_status);
    delete h;
    return RCLUPP_OK;
}

rclupp_status_t rclupp_set_stream(rclupp_handle_t h, void *stream) {
    if (!h) return RCLUPP_ERR_ARG;
    h->stream = static_cast<cudaStream_t>(stream);
    return RCLUPP_OK;
}

rclupp_status_t rclupp_workspace_size(int32_t algo, int64_t m, int64_t n, const rclupp_opts_t *opts,
                                      int32_t q_aliases_x, size_t *bytes) {
    if (!bytes || n < 1 || m < n) return RCLUPP_ERR_ARG;
    if (algo < RCLUPP_ALGO_RCLUPP || algo > RCLUPP_ALGO_SCHOLQR3) return RCLUPP_ERR_ARG;
    if (n > kMaxN || m >= (int64_t(1) << 31)) return RCLUPP_ERR_UNSUPPORTED;
    const bool randomized =
        algo == RCLUPP_ALGO_RCLUPP || algo == RCLUPP_ALGO_RCLUPPR || algo == RCLUPP_ALGO_RCHOLQR;
    const rclupp_opts_t o = resolve_opts(opts, n);
    if (randomized) {
        const rclupp_status_t st = check_opts(o, m, n);
        if (st != RCLUPP_OK) return st;
    }
    // the same rule as the drivers: RCLUPPr keeps its own LU copy when Q
    // aliases X or a non-binary64 tier may re-sketch M; LC2 when Q aliases X
    const bool lu_copy = (algo == RCLUPP_ALGO_RCLUPPR && (q_aliases_x || o.prec != RCLUPP_PREC_FP64)) ||
                         (algo == RCLUPP_ALGO_LC2 && q_aliases_x);
    size_t total = 0;
    carve(nullptr, m, int(n), randomized ? o.s : n, lu_copy, &total);
    *bytes = total;
    return RCLUPP_OK;
}

rclupp_status_t rclupp_workspace_bytes(rclupp_handle_t h, size_t *bytes) {
    if (!h || !bytes) return RCLUPP_ERR_ARG;
    *bytes = h->ws_bytes;
    return RCLUPP_OK;
}

const char *rclupp_status_string(int status) {
    switch (status) {
        case RCLUPP_OK: return "ok";
        case RCLUPP_ERR_ARG: return "invalid argument";
        case RCLUPP_ERR_CHOL_BREAKDOWN: return "Cholesky breakdown";
        case RCLUPP_ERR_LU_ZERO_PIVOT: return "zero pivot in LU";
        case RCLUPP_ERR_NONFINITE: return "non-finite value";
        case RCLUPP_ERR_CUDA: return "CUDA error";
        case RCLUPP_ERR_TIMEOUT: return "device wait timed out";
        case RCLUPP_ERR_NOMEM: return "out of device memory";
        case RCLUPP_ERR_UNSUPPORTED: return "unsupported size or option";
        default: return "unknown status";
    }
}

rclupp_status_t rclupp_factor(rclupp_handle_t h, int64_t m, int64_t n, const double *X,
                              int64_t ldx, const rclupp_opts_t *opts, double *Q, int64_t ldq,
                              double *R, int64_t ldr, rclupp_info_t *info) {
    rclupp_status_t st = check_common(h, m, n, X, ldx, Q, ldq, R, ldr);
    if (st != RCLUPP_OK) return st;
    const rclupp_opts_t o = resolve_opts(opts, n);
    if ((st = check_opts(o, m, n)) != RCLUPP_OK) return st;
    Bufs b = prepare(h, m, int(n), o.s, false, &st);
    if (st != RCLUPP_OK) return st;
    cudaStream_t s = h->stream;
    DevStatus *ds = h->d_status;
    const int ni = int(n), si = int(o.s);
    int tier = o.prec;
    // X_s = S X; [M, N, P] = LU(X_s); R0 = R of HouseholderQR(M); R1 = R0 N;
    // then CholeskyQR2 of Q1 = X R1^{-1} (Algorithm 6)
    auto precond = [&]() {
        return launch_sketch_precond(b.Y, o.s, si, ni, b.W, b.RP[0], b.rinv[0], nullptr, 0, ds, 1, s,
                                     o.r0_method);
    };
    const rclupp_status_t ls =
        randomized_tail(h, b, o, m, ni, X, ldx, 0, precond, X, ldx, Q, ldq, R, ldr, &tier);
    const rclupp_status_t r = finish(h, ls, info, nullptr);
    if (info) {
        info->prec_used = tier;
        info->emulated = o.prec == RCLUPP_PREC_EMULATED ? 1 : (o.prec == RCLUPP_PREC_EMULATED_ALL ? 2 : 0);
    }
    return r;
}

rclupp_status_t rclupp_r_factor(rclupp_handle_t h, int64_t m, int64_t n, const double *X,
                                int64_t ldx, const rclupp_opts_t *opts, double *Q, int64_t ldq,
                                double *R, int64_t ldr, rclupp_info_t *info) {
    rclupp_status_t st = check_common(h, m, n, X, ldx, Q, ldq, R, ldr);
    if (st != RCLUPP_OK) return st;
    const rclupp_opts_t o = resolve_opts(opts, n);
    if ((st = check_opts(o, m, n)) != RCLUPP_OK) return st;
    // The LU factor lives in Q unless Q aliases X or a reduced sketch tier may
    // need M again after Q1 has been written (escalation re-sketches M).
    const bool own_lu = (Q == X) || o.prec != RCLUPP_PREC_FP64;
    Bufs b = prepare(h, m, int(n), o.s, own_lu, &st);
    if (st != RCLUPP_OK) return st;
    cudaStream_t s = h->stream;
    DevStatus *ds = h->d_status;
    const int ni = int(n), si = int(o.s);
    double *L = own_lu ? b.LUbuf : Q;
    const int64_t ldl = own_lu ? m : ldq;
    rclupp_status_t ls = RCLUPP_OK;
    int tier = o.prec;
    const LuWaitOptions w = take_lu_wait(h);
    do {
        if (copy_matrix(L, ldl, X, ldx, m, n, s) != cudaSuccess) { ls = RCLUPP_ERR_CUDA; break; }
        // [M, N, P] = LU(X) (Algorithm 7)
        if (launch_tall_lupp(L, ldl, m, ni, b.ipiv, b.lu, ds, 2, s, &w) != cudaSuccess) {
            ls = RCLUPP_ERR_CUDA; break; }
        // M_s = S M; R0 = R of HouseholderQR(M_s); R1 = R0 N; then CholeskyQR2
        // of Q1 = X R1^{-1}.  Q1 overwrites the LU only after M_s is formed.
        auto precond = [&]() {
            return launch_rcluppr_r1(b.Y, o.s, si, ni, L, ldl, b.W, b.RP[0], b.rinv[0], s, o.r0_method);
        };
        ls = randomized_tail(h, b, o, m, ni, L, ldl, 1, precond, X, ldx, Q, ldq, R, ldr, &tier);
    } while (0);
    const rclupp_status_t r = finish(h, ls, info, nullptr);
    if (info) {
        info->prec_used = tier;
        info->emulated = o.prec == RCLUPP_PREC_EMULATED ? 1 : (o.prec == RCLUPP_PREC_EMULATED_ALL ? 2 : 0);
    }
    return r;
}

rclupp_status_t cholqr2_factor(rclupp_handle_t h, int64_t m, int64_t n, const double *X,
                               int64_t ldx, double *Q, int64_t ldq, double *R, int64_t ldr,
                               rclupp_info_t *info) {
    rclupp_status_t st = check_common(h, m, n, X, ldx, Q, ldq, R, ldr);
    if (st != RCLUPP_OK) return st;
    Bufs b = prepare(h, m, int(n), n, false, &st);
    if (st != RCLUPP_OK) return st;
    return finish(h, enqueue_cholqr2(ctx_of(h), b, m, int(n), X, ldx, Q, ldq, R, ldr), info,
                  nullptr);
}

rclupp_status_t lc2_factor(rclupp_handle_t h, int64_t m, int64_t n, const double *X, int64_t ldx,
                           double *Q, int64_t ldq, double *R, int64_t ldr, rclupp_info_t *info) {
    rclupp_status_t st = check_common(h, m, n, X, ldx, Q, ldq, R, ldr);
    if (st != RCLUPP_OK) return st;
    const bool alias = (Q == X);
    Bufs b = prepare(h, m, int(n), n, alias, &st);
    if (st != RCLUPP_OK) return st;
    double *L = alias ? b.LUbuf : Q;
    const int64_t ldl = alias ? m : ldq;
    const LuWaitOptions w = take_lu_wait(h);
    return finish(h, enqueue_lc2(ctx_of(h), b, m, int(n), X, ldx, L, ldl, Q, ldq, R, ldr, &w), info,
                  nullptr);
}

rclupp_status_t rcholqr_factor(rclupp_handle_t h, int64_t m, int64_t n, const double *X,
                               int64_t ldx, const rclupp_opts_t *opts, double *Q, int64_t ldq,
                               double *R, int64_t ldr, rclupp_info_t *info) {
    rclupp_status_t st = check_common(h, m, n, X, ldx, Q, ldq, R, ldr);
    if (st != RCLUPP_OK) return st;
    const rclupp_opts_t o = resolve_opts(opts, n);
    if ((st = check_opts(o, m, n)) != RCLUPP_OK) return st;
    Bufs b = prepare(h, m, int(n), o.s, false, &st);
    if (st != RCLUPP_OK) return st;
    const bool tc_sketch = o.kind == RCLUPP_SKETCH_GAUSSIAN && !o.S;
    const bool emu = o.prec == RCLUPP_PREC_EMULATED || o.prec == RCLUPP_PREC_EMULATED_ALL;
    const int tier = emu ? RCLUPP_PREC_SKETCH_DIGITS : o.prec;
    const rclupp_status_t r = finish(
        h, enqueue_rcholqr(ctx_of(h), b, o, tier, m, int(n), X, ldx, Q, ldq, R, ldr), info, nullptr);
    if (info) {
        info->prec_used = tc_sketch ? tier : RCLUPP_PREC_FP64;
        info->emulated = o.prec == RCLUPP_PREC_EMULATED ? 1 : (o.prec == RCLUPP_PREC_EMULATED_ALL ? 2 : 0);
    }
    return r;
}

rclupp_status_t scholqr3_factor(rclupp_handle_t h, int64_t m, int64_t n, const double *X,
                                int64_t ldx, double *Q, int64_t ldq, double *R, int64_t ldr,
                                rclupp_info_t *info) {
    rclupp_status_t st = check_common(h, m, n, X, ldx, Q, ldq, R, ldr);
    if (st != RCLUPP_OK) return st;
    Bufs b = prepare(h, m, int(n), n, false, &st);
    if (st != RCLUPP_OK) return st;
    return finish(h, enqueue_scholqr3(ctx_of(h), b, m, int(n), X, ldx, Q, ldq, R, ldr), info,
                  nullptr);
}

// ---- batched form ------------------------------------------------------------

}  // extern "C"

namespace {

// Branch of each problem and the order of the captures: longest processing
// time first -- problems by decreasing estimated time (m n^2 for the tall
// passes plus 4e6 n for the latency of the n-step small factorizations, in
// flop-equivalents), each to the branch with the least estimated time so far
// -- so that the branches end together and each starts with its largest
// problems.  Ties keep the problems' order.
void assign_branches(int count, const int64_t *m, const int64_t *n, int branches,
                     std::vector<int> &branch, std::vector<int> &order) {
    std::vector<double> w(count);
    for (int i = 0; i < count; ++i)
        w[i] = double(m[i]) * double(n[i]) * double(n[i]) + 4e6 * double(n[i]);
    order.resize(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return w[a] > w[b]; });
    std::vector<double> load(branches, 0.0);
    branch.assign(count, 0);
    for (int i : order) {
        const int k = int(std::min_element(load.begin(), load.end()) - load.begin());
        branch[i] = k;
        load[k] += w[i];
    }
}

// What a batch needs before anything is enqueued: every problem validated,
// its options resolved, the per-branch workspace (sized for the largest
// problem) and the branch streams.  `may_allocate` false: a workspace or
// stream set too small is RCLUPP_ERR_UNSUPPORTED instead of allocated.
struct BatchSetup {
    std::vector<rclupp_opts_t> o;
    bool randomized = false;
    size_t per_branch = 0;
    int branches = 1;
    char *base = nullptr;
    DevStatus *d_st = nullptr;
};

rclupp_status_t batch_setup(rclupp_handle_t h, int32_t algo, int32_t count, const int64_t *m,
                            const int64_t *n, const double *const *X, const int64_t *ldx,
                            const rclupp_opts_t *opts, double *const *Q, const int64_t *ldq,
                            double *const *R, const int64_t *ldr, bool may_allocate, BatchSetup &bs) {
    if (!h || count < 0 || (count > 0 && (!m || !n || !X || !ldx || !Q || !ldq || !R || !ldr)))
        return RCLUPP_ERR_ARG;
    if (algo < RCLUPP_ALGO_RCLUPP || algo > RCLUPP_ALGO_SCHOLQR3) return RCLUPP_ERR_ARG;
    bs.randomized =
        algo == RCLUPP_ALGO_RCLUPP || algo == RCLUPP_ALGO_RCLUPPR || algo == RCLUPP_ALGO_RCHOLQR;
    if (count == 0) return RCLUPP_OK;
    // validate every problem and size one branch's workspace for the largest
    bs.o.assign(count, rclupp_opts_t{});
    size_t per_branch = 0;
    for (int i = 0; i < count; ++i) {
        rclupp_status_t st = check_common(h, m[i], n[i], X[i], ldx[i], Q[i], ldq[i], R[i], ldr[i]);
        if (st != RCLUPP_OK) return st;
        bs.o[i] = resolve_opts(opts ? &opts[i] : nullptr, n[i]);
        if (bs.randomized) {
            if ((st = check_opts(bs.o[i], m[i], n[i])) != RCLUPP_OK) return st;
            // one sketch tier per problem (no escalation inside a graph):
            // binary64, or the three-term tensor-core sketch for the
            // RCLUPP_PREC_SKETCH_FP32 and emulated tiers; the bf16 tier needs
            // the escalation and is refused
            if (bs.o[i].prec == RCLUPP_PREC_SKETCH_BF16) return RCLUPP_ERR_UNSUPPORTED;
        }
        const bool own_lu = (algo == RCLUPP_ALGO_RCLUPPR || algo == RCLUPP_ALGO_LC2) && Q[i] == X[i];
        const int64_t s = bs.randomized ? bs.o[i].s : n[i];
        size_t total = 0;
        carve(nullptr, m[i], int(n[i]), s, own_lu, &total);
        per_branch = std::max(per_branch, total);
    }
    bs.per_branch = (per_branch + 255) & ~size_t(255);
    bs.branches = std::max(1, std::min<int>(count, h->batch_branches));
    const size_t status_bytes = (size_t(count) * sizeof(DevStatus) + 255) & ~size_t(255);
    const size_t need = bs.per_branch * bs.branches + status_bytes;
    if (!may_allocate && (h->ws_bytes < need || h->nstreams < bs.branches || !h->fork))
        return RCLUPP_ERR_UNSUPPORTED;
    rclupp_status_t st = ensure_ws(h, need);
    if (st != RCLUPP_OK) return st;
    if (ensure_streams(h, bs.branches) != RCLUPP_OK) return RCLUPP_ERR_CUDA;
    bs.base = static_cast<char *>(h->ws);
    bs.d_st = reinterpret_cast<DevStatus *>(bs.base + bs.per_branch * bs.branches);
    return RCLUPP_OK;
}

// The batch's work relative to `origin`: statuses cleared, a fork into the
// branch streams, each problem on the branch assign_branches gives it (each
// branch's problems largest first), a join back into `origin`.  Every call it
// makes can be captured.
rclupp_status_t enqueue_batch(rclupp_handle_t h, int32_t algo, int32_t count, const int64_t *m,
                              const int64_t *n, const double *const *X, const int64_t *ldx,
                              double *const *Q, const int64_t *ldq, double *const *R,
                              const int64_t *ldr, const BatchSetup &bs, cudaStream_t origin) {
    const int branches = bs.branches;
    rclupp_status_t ls = RCLUPP_OK;
    if (cudaMemsetAsync(bs.d_st, 0, size_t(count) * sizeof(DevStatus), origin) != cudaSuccess ||
        cudaEventRecord(h->fork, origin) != cudaSuccess)
        ls = RCLUPP_ERR_CUDA;
    for (int k = 0; k < branches && ls == RCLUPP_OK; ++k)
        if (cudaStreamWaitEvent(h->bstreams[k], h->fork, 0) != cudaSuccess) ls = RCLUPP_ERR_CUDA;
    std::vector<int> branch, order;
    assign_branches(count, m, n, branches, branch, order);
    for (int oi = 0; oi < count && ls == RCLUPP_OK; ++oi) {
        const int i = order[oi];
        const int k = branch[i];
        const Ctx c{h->bstreams[k], bs.d_st + i};
        const bool own_lu = (algo == RCLUPP_ALGO_RCLUPPR || algo == RCLUPP_ALGO_LC2) && Q[i] == X[i];
        const int64_t s = bs.randomized ? bs.o[i].s : n[i];
        size_t total = 0;
        const Bufs b = carve(bs.base + bs.per_branch * k, m[i], int(n[i]), s, own_lu, &total);
        double *L = own_lu ? b.LUbuf : Q[i];
        const int64_t ldl = own_lu ? m[i] : ldq[i];
        const int ni = int(n[i]);
        const rclupp_opts_t &oi_opts = bs.o[i];
        switch (algo) {
            case RCLUPP_ALGO_RCLUPP:
                ls = enqueue_rclupp(c, b, oi_opts, m[i], ni, X[i], ldx[i], Q[i], ldq[i], R[i], ldr[i]);
                break;
            case RCLUPP_ALGO_RCLUPPR:
                ls = enqueue_rcluppr(c, b, oi_opts, m[i], ni, X[i], ldx[i], L, ldl, Q[i], ldq[i], R[i],
                                     ldr[i]);
                break;
            case RCLUPP_ALGO_CHOLQR2:
                ls = enqueue_cholqr2(c, b, m[i], ni, X[i], ldx[i], Q[i], ldq[i], R[i], ldr[i]);
                break;
            case RCLUPP_ALGO_RCHOLQR:
                ls = enqueue_rcholqr(c, b, oi_opts, batch_sketch_tier(oi_opts), m[i], ni, X[i], ldx[i],
                                     Q[i], ldq[i], R[i], ldr[i]);
                break;
            case RCLUPP_ALGO_SCHOLQR3:
                ls = enqueue_scholqr3(c, b, m[i], ni, X[i], ldx[i], Q[i], ldq[i], R[i], ldr[i]);
                break;
            default:
                ls = enqueue_lc2(c, b, m[i], ni, X[i], ldx[i], L, ldl, Q[i], ldq[i], R[i], ldr[i]);
                break;
        }
    }
    for (int k = 0; k < branches && ls == RCLUPP_OK; ++k)
        if (cudaEventRecord(h->join[k], h->bstreams[k]) != cudaSuccess ||
            cudaStreamWaitEvent(origin, h->join[k], 0) != cudaSuccess)
            ls = RCLUPP_ERR_CUDA;
    return ls;
}

// Problem i's status code into status[i] (device memory).
__global__ void k_batch_status(const DevStatus *__restrict__ st, int count, int32_t *__restrict__ status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) status[i] = st[i].code;
}

}  // namespace

extern "C" {

rclupp_status_t rclupp_factor_batched(rclupp_handle_t h, int32_t algo, int32_t count,
                                      const int64_t *m, const int64_t *n, const double *const *X,
                                      const int64_t *ldx, const rclupp_opts_t *opts,
                                      double *const *Q, const int64_t *ldq, double *const *R,
                                      const int64_t *ldr, int32_t *status) {
    BatchSetup bs;
    rclupp_status_t st = batch_setup(h, algo, count, m, n, X, ldx, opts, Q, ldq, R, ldr, true, bs);
    if (st != RCLUPP_OK || count == 0) return st;
    const int branches = bs.branches;
    const std::vector<rclupp_opts_t> &o = bs.o;
    DevStatus *d_st = bs.d_st;

    // Graph of the whole batch: fork into `branches` streams, each problem on
    // the branch assign_branches gives it, join.  Reused while the batch is
    // unchanged.
    LaunchPolicy pol;
    pol.grid_div = h->batch_grid_div;
    pol.fine_tiles = h->batch_fine_tiles;
    std::vector<unsigned char> desc = batch_description(algo, count, m, n, X, ldx, Q, ldq, R, ldr,
                                                        o.data(), branches, h->ws, pol);
    if (!(h->graph_exec && h->graph_desc == desc)) {
        if (h->graph_exec) {
            cudaGraphExecDestroy(h->graph_exec);
            h->graph_exec = nullptr;
        }
        cudaGraph_t graph = nullptr;
        // capture on the handle's own origin stream (the caller's stream may be the
        // legacy default stream, which cannot be captured); launch on the caller's
        if (cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeRelaxed) != cudaSuccess)
            return RCLUPP_ERR_CUDA;
        rclupp_status_t ls;
        {
            const LaunchPolicyScope policy_scope(pol);  // launch shapes of the captured kernels
            ls = enqueue_batch(h, algo, count, m, n, X, ldx, Q, ldq, R, ldr, bs, h->cap);
        }
        const cudaError_t ec = cudaStreamEndCapture(h->cap, &graph);
        if (ls != RCLUPP_OK || ec != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return ls != RCLUPP_OK ? ls : RCLUPP_ERR_CUDA;
        }
        size_t nn = 0;
        cudaGraphGetNodes(graph, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        cudaGraphGetNodes(graph, nodes.data(), &nn);
        h->graph_kernels = 0;
        for (size_t j = 0; j < nn; ++j) {
            cudaGraphNodeType t;
            if (cudaGraphNodeGetType(nodes[j], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel)
                ++h->graph_kernels;
        }
        const cudaError_t ei = cudaGraphInstantiate(&h->graph_exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) {
            h->graph_exec = nullptr;
            return RCLUPP_ERR_CUDA;
        }
        h->graph_desc = std::move(desc);
    }
    if (cudaGraphLaunch(h->graph_exec, h->stream) != cudaSuccess) return RCLUPP_ERR_CUDA;
    prof_add_launches(h->graph_kernels);
    std::vector<DevStatus> hs(count);
    if (cudaMemcpyAsync(hs.data(), d_st, size_t(count) * sizeof(DevStatus), cudaMemcpyDeviceToHost,
                        h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
        return RCLUPP_ERR_CUDA;
    rclupp_status_t first = RCLUPP_OK;
    for (int i = 0; i < count; ++i) {
        if (status) status[i] = hs[i].code;
        if (first == RCLUPP_OK && hs[i].code != 0) first = static_cast<rclupp_status_t>(hs[i].code);
    }
    return first;
}

rclupp_status_t rclupp_factor_batched_async(rclupp_handle_t h, int32_t algo, int32_t count,
                                            const int64_t *m, const int64_t *n,
                                            const double *const *X, const int64_t *ldx,
                                            const rclupp_opts_t *opts, double *const *Q,
                                            const int64_t *ldq, double *const *R, const int64_t *ldr,
                                            int32_t *d_status) {
    if (count > 0 && !d_status) return RCLUPP_ERR_ARG;
    // while the caller's stream captures, nothing may be allocated
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (h && cudaStreamIsCapturing(h->stream, &cs) != cudaSuccess) {
        cudaGetLastError();
        return RCLUPP_ERR_CUDA;
    }
    BatchSetup bs;
    rclupp_status_t st = batch_setup(h, algo, count, m, n, X, ldx, opts, Q, ldq, R, ldr,
                                     cs == cudaStreamCaptureStatusNone, bs);
    if (st != RCLUPP_OK || count == 0) return st;
    LaunchPolicy pol;
    pol.grid_div = h->batch_grid_div;
    pol.fine_tiles = h->batch_fine_tiles;
    {
        const LaunchPolicyScope policy_scope(pol);
        st = enqueue_batch(h, algo, count, m, n, X, ldx, Q, ldq, R, ldr, bs, h->stream);
    }
    if (st != RCLUPP_OK) return st;
    RQ_LAUNCH(KID_REDUCE, h->stream,
              k_batch_status<<<(count + 255) / 256, 256, 0, h->stream>>>(bs.d_st, count, d_status));
    if (cudaGetLastError() != cudaSuccess) return RCLUPP_ERR_CUDA;
    return RCLUPP_OK;
}

rclupp_status_t rclupp_set_batch_branches(rclupp_handle_t h, int32_t branches) {
    if (!h || branches < 1 || branches > kMaxBranches) return RCLUPP_ERR_ARG;
    h->batch_branches = branches;
    return RCLUPP_OK;
}

rclupp_status_t rclupp_set_batch_policy(rclupp_handle_t h, int32_t grid_div, int32_t fine_tiles) {
    if (!h || grid_div < 1 || grid_div > 64 || (fine_tiles != 0 && fine_tiles != 1)) return RCLUPP_ERR_ARG;
    h->batch_grid_div = grid_div;
    h->batch_fine_tiles = fine_tiles;
    return RCLUPP_OK;
}

rclupp_status_t rclupp_get_batch_policy(rclupp_handle_t h, int32_t *branches, int32_t *grid_div,
                                        int32_t *fine_tiles) {
    if (!h) return RCLUPP_ERR_ARG;
    if (branches) *branches = h->batch_branches;
    if (grid_div) *grid_div = h->batch_grid_div;
    if (fine_tiles) *fine_tiles = h->batch_fine_tiles;
    return RCLUPP_OK;
}

rclupp_status_t rclupp_autotune_batched(rclupp_handle_t h, int32_t algo, int32_t count,
                                        const int64_t *m, const int64_t *n,
                                        const double *const *X, const int64_t *ldx,
                                        const rclupp_opts_t *opts, double *const *Q,
                                        const int64_t *ldq, double *const *R, const int64_t *ldr,
                                        int32_t *best_branches, float *best_ms) {
    if (!h) return RCLUPP_ERR_ARG;
    static const int kCandidates[] = {4, 8, 16, 32, 64};
    // launch shapes tried at the best branch count: CTA budget divisor, finer row tiles
    static const int kPolicies[][2] = {{1, 1}, {2, 0}, {2, 1}, {4, 0}, {4, 1}, {8, 0}};
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return RCLUPP_ERR_CUDA;
    int best = h->batch_branches, best_div = 1, best_fine = 0;
    float best_t = 0.f;
    rclupp_status_t st = RCLUPP_OK;
    // a problem's own numerical failure is part of the batch's result, not a
    // reason to stop tuning
    auto numerical = [](rclupp_status_t s) {
        return s == RCLUPP_ERR_CHOL_BREAKDOWN || s == RCLUPP_ERR_LU_ZERO_PIVOT ||
               s == RCLUPP_ERR_NONFINITE;
    };
    // first call builds and caches the graph; the second one is timed
    auto trial = [&](float *t) {
        st = rclupp_factor_batched(h, algo, count, m, n, X, ldx, opts, Q, ldq, R, ldr, nullptr);
        if (st != RCLUPP_OK && !numerical(st)) return false;
        cudaEventRecord(e0, h->stream);
        st = rclupp_factor_batched(h, algo, count, m, n, X, ldx, opts, Q, ldq, R, ldr, nullptr);
        cudaEventRecord(e1, h->stream);
        cudaEventSynchronize(e1);
        if (st != RCLUPP_OK && !numerical(st)) return false;
        *t = 0.f;
        cudaEventElapsedTime(t, e0, e1);
        return true;
    };
    h->batch_grid_div = 1;
    h->batch_fine_tiles = 0;
    bool ok = true;
    for (int b : kCandidates) {
        if (b > std::max<int>(count, 1) && b != kCandidates[0]) break;
        h->batch_branches = b;
        float t;
        if (!(ok = trial(&t))) break;
        if (best_t == 0.f || t < best_t) {
            best_t = t;
            best = b;
        }
    }
    h->batch_branches = best;
    for (int p = 0; ok && p < int(sizeof(kPolicies) / sizeof(kPolicies[0])); ++p) {
        h->batch_grid_div = kPolicies[p][0];
        h->batch_fine_tiles = kPolicies[p][1];
        float t;
        if (!(ok = trial(&t))) break;
        if (t < best_t) {
            best_t = t;
            best_div = kPolicies[p][0];
            best_fine = kPolicies[p][1];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->batch_grid_div = best_div;
    h->batch_fine_tiles = best_fine;
    if (best_branches) *best_branches = best;
    if (best_ms) *best_ms = best_t;
    return numerical(st) ? RCLUPP_OK : st;
}

// ---- individual steps ----

rclupp_status_t rclupp_sketch_rows(rclupp_handle_t h, int64_t m, int64_t n, const double *A,
                                   int64_t lda, int64_t row0, int32_t unit_lower,
                                   const rclupp_opts_t *opts, double *Y, int64_t ldy) {
    if (!h || !A || !Y || n < 1 || m < 1 || row0 < 0 || bad_ld(lda, m)) return RCLUPP_ERR_ARG;
    if (n > kMaxN || m >= (int64_t(1) << 31)) return RCLUPP_ERR_UNSUPPORTED;
    const rclupp_opts_t o = resolve_opts(opts, n);
    rclupp_status_t st = check_opts(o, row0 + m, n);
    if (st != RCLUPP_OK) return st;
    if (bad_ld(ldy, o.s)) return RCLUPP_ERR_ARG;
    Bufs b = prepare(h, m, int(n), o.s, false, &st);
    if (st != RCLUPP_OK) return st;
    cudaError_t e;
    // the emulated tiers sketch at the digit tier, as their drivers do
    const bool digits = o.prec == RCLUPP_PREC_SKETCH_DIGITS || o.prec == RCLUPP_PREC_EMULATED ||
                        o.prec == RCLUPP_PREC_EMULATED_ALL;
    if (digits && o.kind == RCLUPP_SKETCH_GAUSSIAN && !o.S)
        e = launch_sketch_digits(A, lda, m, int(n), unit_lower, o.s, o.seed, Y, ldy, b.part, h->d_status,
                                 h->stream, row0);
    else if (o.prec != RCLUPP_PREC_FP64 && o.kind == RCLUPP_SKETCH_GAUSSIAN && !o.S)
        e = launch_sketch_tc(A, lda, m, int(n), unit_lower, o.s, o.seed,
                             o.prec == RCLUPP_PREC_SKETCH_FP32 ? 3 : 1, Y, ldy, b.part, h->d_status,
                             h->stream, row0);
    else
        e = launch_sketch(A, lda, m, int(n), unit_lower, o.kind, o.s, o.zeta, o.seed, o.S, o.lds, Y,
                          ldy, b.part, h->d_status, h->stream, row0, o.order_log2);
    return finish(h, from_cuda(e), nullptr, nullptr);
}

rclupp_status_t rclupp_sketch(rclupp_handle_t h, int64_t m, int64_t n, const double *A, int64_t lda,
                              int32_t unit_lower, const rclupp_opts_t *opts, double *Y,
                              int64_t ldy) {
    return rclupp_sketch_rows(h, m, n, A, lda, 0, unit_lower, opts, Y, ldy);
}

rclupp_status_t rclupp_gram(rclupp_handle_t h, int64_t m, int64_t n, const double *A, int64_t lda,
                            int32_t unit_lower, double *G, int64_t ldg) {
    if (!h || !A || !G || n < 1 || m < 1 || bad_ld(lda, m) || bad_ld(ldg, n)) return RCLUPP_ERR_ARG;
    if (n > kMaxN || m >= (int64_t(1) << 31)) return RCLUPP_ERR_UNSUPPORTED;
    rclupp_status_t st;
    Bufs b = prepare(h, m, int(n), n, false, &st);
    if (st != RCLUPP_OK) return st;
    const cudaError_t e =
        launch_gram(A, lda, m, int(n), unit_lower, G, ldg, b.part, h->d_status, h->stream);
    return finish(h, from_cuda(e), nullptr, nullptr);
}

rclupp_status_t rclupp_gram_emulated(rclupp_handle_t h, int64_t m, int64_t n, const double *A,
                                     int64_t lda, double *G, int64_t ldg) {
    if (!h || !A || !G || n < 1 || m < 1 || bad_ld(lda, m) || bad_ld(ldg, n)) return RCLUPP_ERR_ARG;
    if (n > kMaxN || m >= (int64_t(1) << 31)) return RCLUPP_ERR_UNSUPPORTED;
    rclupp_status_t st;
    Bufs b = prepare(h, m, int(n), n, false, &st);
    if (st != RCLUPP_OK) return st;
    const cudaError_t e = launch_gram_emu(A, lda, m, int(n), G, ldg, b.part, h->d_status, h->stream);
    return finish(h, from_cuda(e), nullptr, nullptr);
}

rclupp_status_t rclupp_trsm_gram(rclupp_handle_t h, int64_t m, int64_t n, const double *A,
                                 int64_t lda, const double *R, int64_t ldr, double *Q, int64_t ldq,
                                 double *G, int64_t ldg) {
    if (!h || !A || !R || !Q || n < 1 || m < 1 || bad_ld(lda, m) || bad_ld(ldr, n) || bad_ld(ldq, m))
        return RCLUPP_ERR_ARG;
    if (G && bad_ld(ldg, n)) return RCLUPP_ERR_ARG;
    if (n > kMaxN || m >= (int64_t(1) << 31)) return RCLUPP_ERR_UNSUPPORTED;
    rclupp_status_t st;
    Bufs b = prepare(h, m, int(n), n, false, &st);
    if (st != RCLUPP_OK) return st;
    cudaError_t e = launch_pad_upper(R, ldr, int(n), b.RP[0], b.rinv[0], h->stream);
    if (e == cudaSuccess)
        e = launch_trsm_gram(A, lda, m, int(n), b.RP[0], b.rinv[0], Q, ldq, G, ldg, b.part,
                             h->d_status, h->stream);
    return finish(h, from_cuda(e), nullptr, nullptr);
}

rclupp_status_t rclupp_trsm_emulated(rclupp_handle_t h, int64_t m, int64_t n, const double *A,
                                     int64_t lda, const double *R, int64_t ldr, double *Q,
                                     int64_t ldq) {
    if (!h || !A || !R || !Q || n < 1 || m < 1 || bad_ld(lda, m) || bad_ld(ldr, n) || bad_ld(ldq, m))
        return RCLUPP_ERR_ARG;
    if (n > kMaxN || m >= (int64_t(1) << 31)) return RCLUPP_ERR_UNSUPPORTED;
    rclupp_status_t st;
    Bufs b = prepare(h, m, int(n), n, false, &st);
    if (st != RCLUPP_OK) return st;
    cudaError_t e = launch_pad_upper(R, ldr, int(n), b.RP[0], b.rinv[0], h->stream);
    if (e == cudaSuccess)
        e = launch_trsm_emu(A, lda, m, int(n), b.RP[0], b.rinv[0], Q, ldq, b.part, h->d_status,
                            h->stream);
    return finish(h, from_cuda(e), nullptr, nullptr);
}

rclupp_status_t rclupp_trsm_emulated_wellcond(rclupp_handle_t h, int64_t m, int64_t n, const double *A,
                                              int64_t lda, const double *R, int64_t ldr, double *Q,
                                              int64_t ldq, int32_t *form) {
    if (!h || !A || !R || !Q || n < 1 || m < 1 || bad_ld(lda, m) || bad_ld(ldr, n) || bad_ld(ldq, m))
        return RCLUPP_ERR_ARG;
    if (n > kMaxN || m >= (int64_t(1) << 31)) return RCLUPP_ERR_UNSUPPORTED;
    rclupp_status_t st;
    Bufs b = prepare(h, m, int(n), n, false, &st);
    if (st != RCLUPP_OK) return st;
    cudaError_t e = launch_pad_upper(R, ldr, int(n), b.RP[0], b.rinv[0], h->stream);
    if (e == cudaSuccess)
        e = launch_trsm_emu_wellcond(A, lda, m, int(n), b.RP[0], b.rinv[0], Q, ldq, b.part, h->d_status,
                                     h->stream);
    const rclupp_status_t r = finish(h, from_cuda(e), nullptr, nullptr);
    if (form) *form = r == RCLUPP_OK ? wellcond_used_product(b.part, int(n), h->stream) : -1;
    return r;
}

rclupp_status_t rclupp_cholesky(rclupp_handle_t h, int64_t n, const double *G, int64_t ldg,
                                double *R, int64_t ldr, int64_t *col) {
    if (!h || !G || !R || n < 1 || bad_ld(ldg, n) || bad_ld(ldr, n)) return RCLUPP_ERR_ARG;
    if (n > kMaxN) return RCLUPP_ERR_UNSUPPORTED;
    rclupp_status_t st;
    Bufs b = prepare(h, n, int(n), n, false, &st);
    if (st != RCLUPP_OK) return st;
    const cudaError_t e = launch_cholesky(G, ldg, int(n), b.W, b.RP[0], b.rinv[0], R, ldr,
                                          h->d_status, 3, h->stream);
    return finish(h, from_cuda(e), nullptr, col);
}

rclupp_status_t rclupp_trmm_upper(rclupp_handle_t h, int64_t n, const double *A, int64_t lda,
                                  const double *B, int64_t ldb, double *C, int64_t ldc) {
    if (!h || !A || !B || !C || n < 1 || bad_ld(lda, n) || bad_ld(ldb, n) || bad_ld(ldc, n))
        return RCLUPP_ERR_ARG;
    if (n > kMaxN) return RCLUPP_ERR_UNSUPPORTED;
    if (cudaMemsetAsync(h->d_status, 0, sizeof(DevStatus), h->stream) != cudaSuccess)
        return RCLUPP_ERR_CUDA;
    const cudaError_t e = launch_trmm_upper(A, lda, B, ldb, int(n), C, ldc, h->stream);
    return finish(h, from_cuda(e), nullptr, nullptr);
}

rclupp_status_t rclupp_tall_lupp(rclupp_handle_t h, int64_t m, int64_t n, double *A, int64_t lda,
                                 int32_t *ipiv, int64_t *col) {
    if (!h || !A || !ipiv || n < 1 || m < n || bad_ld(lda, m)) return RCLUPP_ERR_ARG;
    if (n > kMaxN || m >= (int64_t(1) << 31)) return RCLUPP_ERR_UNSUPPORTED;
    rclupp_status_t st;
    Bufs b = prepare(h, m, int(n), n, false, &st);
    if (st != RCLUPP_OK) return st;
    const LuWaitOptions w = take_lu_wait(h);
    const cudaError_t e = launch_tall_lupp(A, lda, m, int(n), ipiv, b.lu, h->d_status, 2, h->stream, &w);
    return finish(h, from_cuda(e), nullptr, col);
}

rclupp_status_t rclupp_set_wait_limit(rclupp_handle_t h, uint64_t limit_ns) {
    if (!h) return RCLUPP_ERR_ARG;
    h->lu_wait_limit_ns = limit_ns;
    return RCLUPP_OK;
}

rclupp_status_t rclupp_inject_fault(rclupp_handle_t h, int32_t fault) {
    if (!h || (fault != RCLUPP_FAULT_NONE && fault != RCLUPP_FAULT_LU_BARRIER_STALL)) return RCLUPP_ERR_ARG;
    h->lu_stall = fault == RCLUPP_FAULT_LU_BARRIER_STALL ? 1 : 0;
    return RCLUPP_OK;
}

rclupp_status_t rclupp_sketch_precond(rclupp_handle_t h, int64_t s, int64_t n, const double *Y,
                                      int64_t ldy, double *R1, int64_t ldr) {
    if (!h || !Y || !R1 || n < 1 || s < n || bad_ld(ldy, s) || bad_ld(ldr, n)) return RCLUPP_ERR_ARG;
    if (n > kMaxN || s > kMaxS) return RCLUPP_ERR_UNSUPPORTED;
    rclupp_status_t st;
    Bufs b = prepare(h, s, int(n), s, false, &st);
    if (st != RCLUPP_OK) return st;
    const cudaError_t e = launch_sketch_precond(Y, ldy, int(s), int(n), b.W, b.RP[0], b.rinv[0], R1,
                                                ldr, h->d_status, 1, h->stream);
    return finish(h, from_cuda(e), nullptr, nullptr);
}

rclupp_status_t rclupp_sketch_precond_r0(rclupp_handle_t h, int64_t s, int64_t n, const double *Y,
                                         int64_t ldy, int32_t r0_method, double *R1, int64_t ldr) {
    if (!h || !Y || !R1 || n < 1 || s < n || bad_ld(ldy, s) || bad_ld(ldr, n)) return RCLUPP_ERR_ARG;
    if (r0_method != RCLUPP_R0_HOUSEHOLDER && r0_method != RCLUPP_R0_GIVENS) return RCLUPP_ERR_ARG;
    if (n > kMaxN || s > kMaxS) return RCLUPP_ERR_UNSUPPORTED;
    if (r0_method == RCLUPP_R0_GIVENS && !precond_cluster_fits(int(s), int(n), true))
        return RCLUPP_ERR_UNSUPPORTED;
    rclupp_status_t st;
    Bufs b = prepare(h, s, int(n), s, false, &st);
    if (st != RCLUPP_OK) return st;
    const cudaError_t e = launch_sketch_precond(Y, ldy, int(s), int(n), b.W, b.RP[0], b.rinv[0], R1,
                                                ldr, h->d_status, 1, h->stream, r0_method);
    return finish(h, from_cuda(e), nullptr, nullptr);
}

rclupp_status_t rclupp_givens_r(rclupp_handle_t h, int64_t s, int64_t n, const double *A, int64_t lda,
                                double *R, int64_t ldr) {
    if (!h || !A || !R || n < 1 || s < n || bad_ld(lda, s) || bad_ld(ldr, n)) return RCLUPP_ERR_ARG;
    if (n > kMaxN || s > kMaxS || !precond_cluster_fits(int(s), int(n), true))
        return RCLUPP_ERR_UNSUPPORTED;
    rclupp_status_t st;
    Bufs b = prepare(h, s, int(n), s, false, &st);
    if (st != RCLUPP_OK) return st;
    const cudaError_t e = launch_givens_r(A, lda, int(s), int(n), b.W, b.RP[0], b.rinv[0], R, ldr,
                                          h->stream);
    return finish(h, from_cuda(e), nullptr, nullptr);
}

rclupp_status_t rclupp_householder_r(rclupp_handle_t h, int64_t s, int64_t n, const double *A,
                                     int64_t lda, double *R, int64_t ldr) {
    if (!h || !A || !R || n < 1 || s < n || bad_ld(lda, s) || bad_ld(ldr, n)) return RCLUPP_ERR_ARG;
    if (n > kMaxN || s > kMaxS) return RCLUPP_ERR_UNSUPPORTED;
    rclupp_status_t st;
    Bufs b = prepare(h, s, int(n), s, false, &st);
    if (st != RCLUPP_OK) return st;
    const cudaError_t e = launch_householder_r(A, lda, int(s), int(n), b.W, R, ldr, h->stream);
    return finish(h, from_cuda(e), nullptr, nullptr);
}

}  // extern "C"
