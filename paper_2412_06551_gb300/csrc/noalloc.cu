// rclupp_gram_noalloc: the Gram product G = A^T A without any device
// allocation.
//
// Some callers cannot let a library allocate device memory: hosts that
// reserve nearly all of the GPU's memory for their own pool at start-up (a
// later cudaMalloc from a library would fail or fragment that pool),
// latency-sensitive loops where cudaMalloc/cudaFree would add implicit
// device synchronization, and code paths where the caller owns every buffer
// for accounting reasons.  For them this entry point keeps its scratch (the
// per-CTA partial sums of the split-K Gram and a status word) in one
// fixed-size array that is part of the library image: every GPU that loads
// the library holds kNoallocScratchBytes of device memory for it until the
// process exits.  The caller still supplies A and G.
//
// The array is shared by every call on a device and keeps the last call's
// contents.  The status word is cleared at the start of each call; the
// partial sums need no clearing, because every launch overwrites each slot
// it later reads.  Calls that overlap on the GPU (for instance on two
// streams at once) use the same array and race; serialize them.
#include <mutex>

#include "../../include/rclupp.h"
#include "common.cuh"
#include "kernels.h"

namespace {

constexpr int kNoallocParts = 64;                    // CTAs of the split-K Gram
constexpr size_t kNoallocPartBytes = size_t(kNoallocParts) * 16384 * sizeof(double);
constexpr size_t kNoallocStatusBytes = 256;          // DevStatus, padded
constexpr size_t kNoallocScratchBytes = kNoallocStatusBytes + kNoallocPartBytes;  // 8 MiB + 256 B
constexpr int kMaxDevices = 64;

// Host code must not use this name as an address: on the host it is only a
// stand-in.  Its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_gram_scratch[kNoallocScratchBytes];

std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

// Device address of g_gram_scratch on the current device, looked up once per
// device (with that device current) and cached for the life of the process.
// The cache assumes no cudaDeviceReset in between: a reset unloads the
// module, and the array may come back at another address.
rclupp_status_t scratch_address(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return RCLUPP_ERR_CUDA;
    }
    std::lock_guard<std::mutex> g(g_mu);
    if (g_addr[dev] == nullptr) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_gram_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return RCLUPP_ERR_CUDA;
        }
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return RCLUPP_OK;
}

}  // namespace

extern "C" rclupp_status_t rclupp_gram_noalloc(int64_t m, int64_t n, const double *A, int64_t lda,
                                               double *G, int64_t ldg, void *stream) {
    if (!A || !G || m < 1 || n < 1 || lda < m || ldg < n) return RCLUPP_ERR_ARG;
    if (n > 128 || m >= (int64_t(1) << 31)) return RCLUPP_ERR_UNSUPPORTED;
    void *base = nullptr;
    rclupp_status_t st = scratch_address(&base);
    if (st != RCLUPP_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    rq::DevStatus *ds = static_cast<rq::DevStatus *>(base);
    double *part = reinterpret_cast<double *>(static_cast<char *>(base) + kNoallocStatusBytes);
    if (cudaMemsetAsync(ds, 0, sizeof(rq::DevStatus), s) != cudaSuccess) return RCLUPP_ERR_CUDA;
    if (rq::launch_gram_bounded(A, lda, m, int(n), G, ldg, part, kNoallocParts, ds, s) !=
        cudaSuccess)
        return RCLUPP_ERR_CUDA;
    rq::DevStatus h{};
    if (cudaMemcpyAsync(&h, ds, sizeof h, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return RCLUPP_ERR_CUDA;
    return h.code == 0 ? RCLUPP_OK : static_cast<rclupp_status_t>(h.code);
}
