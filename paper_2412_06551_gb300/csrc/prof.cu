// Launch accounting and optional per-kernel timing with CUDA events recorded
// on the launching stream (instrumentation for benchmarks; off by default).
#include <mutex>
#include <vector>

#include "../../include/rclupp.h"
#include "kernels.h"

namespace rq {
namespace {

struct Pending {
    int kid;
    cudaEvent_t a, b;
};

struct Profiler {
    std::mutex mu;
    bool enabled = false;
    unsigned long long launches = 0;
    std::vector<cudaEvent_t> pool;
    std::vector<Pending> pending;
    cudaEvent_t open_a[KID_COUNT] = {};
    long long count[KID_COUNT] = {};
    double ms[KID_COUNT] = {};

    cudaEvent_t get_event() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
};

Profiler &prof() {
    static Profiler p;
    return p;
}

const char *kNames[KID_COUNT] = {"sketch_gauss", "sketch_sparse", "gram",       "trsm_gram",
                                 "trsm",         "reduce",        "lu_col",     "lu_trailing",
                                 "lu_u12",       "small_precond", "cholesky",   "trmm",
                                 "pad",          "sketch_tc",     "gram_emu",   "emu_aux",
                                 "trsm_emu",     "sketch_srht"};

}  // namespace

static bool capturing(cudaStream_t stream) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(stream, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
}

// Kernels inside a captured graph are counted when the graph is launched.
void prof_add_launches(unsigned long long k) {
    Profiler &p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    p.launches += k;
}

void prof_begin(int kid, cudaStream_t stream) {
    if (capturing(stream)) return;
    Profiler &p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    ++p.launches;
    if (!p.enabled) return;
    cudaEvent_t a = p.get_event();
    cudaEventRecord(a, stream);
    p.open_a[kid] = a;
}

void prof_end(int kid, cudaStream_t stream) {
    if (capturing(stream)) return;
    Profiler &p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    if (!p.enabled || p.open_a[kid] == nullptr) return;
    cudaEvent_t b = p.get_event();
    cudaEventRecord(b, stream);
    p.pending.push_back({kid, p.open_a[kid], b});
    p.open_a[kid] = nullptr;
}

}  // namespace rq

using namespace rq;

extern "C" {

void rclupp_profile_enable(int enable) {
    Profiler &p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    p.enabled = enable != 0;
}

void rclupp_profile_reset(void) {
    Profiler &p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    for (auto &q : p.pending) {
        cudaEventSynchronize(q.b);
        p.pool.push_back(q.a);
        p.pool.push_back(q.b);
    }
    p.pending.clear();
    for (int k = 0; k < KID_COUNT; ++k) {
        p.count[k] = 0;
        p.ms[k] = 0.0;
    }
    p.launches = 0;
}

int rclupp_profile_get(int kid, long long *launches, double *total_ms, const char **name) {
    if (kid < 0 || kid >= KID_COUNT) return RCLUPP_ERR_ARG;
    Profiler &p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    for (auto &q : p.pending) {
        float t = 0.f;
        if (cudaEventSynchronize(q.b) == cudaSuccess && cudaEventElapsedTime(&t, q.a, q.b) == cudaSuccess) {
            p.count[q.kid] += 1;
            p.ms[q.kid] += t;
        }
        p.pool.push_back(q.a);
        p.pool.push_back(q.b);
    }
    p.pending.clear();
    if (launches) *launches = p.count[kid];
    if (total_ms) *total_ms = p.ms[kid];
    if (name) *name = kNames[kid];
    return RCLUPP_OK;
}

unsigned long long rclupp_kernel_launches(void) {
    Profiler &p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    return p.launches;
}

}  // extern "C"
