// Device-side helpers shared by the kernels of the tall-skinny QR library:
// status reporting, bounded waits, the TMA / mbarrier PTX wrappers, and the
// counter-based sketch generators.  sm_103a only.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace rq {

// ---------------------------------------------------------------- status ---
enum : int {
    kOk = 0,
    kErrArg = -1,
    kErrCholBreakdown = -2,
    kErrLuZeroPivot = -3,
    kErrNonfinite = -4,
    kErrCuda = -5,
    kErrTimeout = -6,
    kErrNomem = -7,
    kErrUnsupported = -8,
};

// Device status word: the first failure wins (code != 0 is never overwritten).
struct DevStatus {
    int code;
    int step;
    long long info;
};

__device__ __forceinline__ void report(DevStatus *st, int code, int step, long long info) {
    if (st == nullptr) return;
    if (atomicCAS(&st->code, 0, code) == 0) {
        st->step = step;
        st->info = info;
        __threadfence();
    }
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits are bounded: after kWaitLimitNs a waiting thread gives up and the
// kernel reports kErrTimeout and returns.
constexpr uint64_t kWaitLimitNs = 2000000000ull;

// ---------------------------------------------------------- mbarrier/TMA ---
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// Plain arrival (release: this thread's earlier shared-memory accesses are
// ordered before the phase completes).
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase.  Returns false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255u) == 0 && globaltimer_ns() - t0 > kWaitLimitNs) return false;
    }
}

// 2-D tiled TMA load global -> shared, completion signalled on `bar`.
// c0 = innermost (row) coordinate, c1 = column coordinate.
// Plain bulk copy global -> shared (both 16-byte aligned, bytes a multiple of
// 16), completing on an mbarrier that expects the bytes.
__device__ __forceinline__ void bulk_load(void *smem_dst, const void *src, uint32_t bytes,
                                          uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_2d(void *smem_dst, const CUtensorMap *map, uint64_t *bar,
                                            int32_t c0, int32_t c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
        : "memory");
}

__device__ __forceinline__ void prefetch_tensormap(const CUtensorMap *map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// ------------------------------------------------- counter-based sketches ---
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of
//   (c0, c1, c2, c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0))
// with M0 = 0xD2511F53, M1 = 0xCD9E8D57 and the key bumped by
// (0x9E3779B9, 0xBB67AE85) after each round.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        // one 32 x 32 -> 64-bit product gives both halves
        const uint64_t p0 = static_cast<uint64_t>(0xD2511F53u) * c.x;
        const uint64_t p1 = static_cast<uint64_t>(0xCD9E8D57u) * c.z;
        const uint32_t lo0 = static_cast<uint32_t>(p0), hi0 = static_cast<uint32_t>(p0 >> 32);
        const uint32_t lo1 = static_cast<uint32_t>(p1), hi1 = static_cast<uint32_t>(p1 >> 32);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Natural log of a normal positive binary32 by the atanh series,
//   x = 2^e f, f in (sqrt2/2, sqrt2], t = (f-1)/(f+1),
//   ln x = e ln2 + 2t (1 + t^2/3 + t^4/5 + t^6/7 + t^8/9 + t^10/11),
// every operation individually rounded (no contraction), so the value is
// the same on any IEEE binary32 implementation.
// Small integers as binary32 without a conversion instruction (those share
// GB300's slow FP64 pipe): 1.5 * 2^23 + k in the significand, minus 1.5 * 2^23,
// exact for |k| < 2^22; and 2^23 + k minus 2^23 for 0 <= k <= 2^23.
__device__ __forceinline__ float sk_small_int_f32(int k) {
    return __fsub_rn(__int_as_float(0x4B400000 + k), 12582912.0f);
}
__device__ __forceinline__ float sk_u23_f32(uint32_t k) {
    return __fsub_rn(__uint_as_float(0x4B000000u + k), 8388608.0f);
}

__device__ __forceinline__ float sk_ln(float x) {
    const uint32_t b = __float_as_uint(x);
    int e = static_cast<int>((b >> 23) & 0xffu) - 127;
    float f = __uint_as_float((b & 0x7fffffu) | 0x3f800000u);
    if (f > 0x1.6a09e6p+0f) {
        f = __fmul_rn(f, 0.5f);
        e += 1;
    }
    const float t = __fdiv_rn(__fsub_rn(f, 1.0f), __fadd_rn(f, 1.0f));
    const float t2 = __fmul_rn(t, t);
    float p = 0x1.745d18p-4f;
    p = __fadd_rn(__fmul_rn(p, t2), 0x1.c71c72p-4f);
    p = __fadd_rn(__fmul_rn(p, t2), 0x1.24924ap-3f);
    p = __fadd_rn(__fmul_rn(p, t2), 0x1.99999ap-3f);
    p = __fadd_rn(__fmul_rn(p, t2), 0x1.555556p-2f);
    p = __fadd_rn(__fmul_rn(p, t2), 1.0f);
    const float lnf = __fmul_rn(__fmul_rn(2.0f, t), p);
    return __fadd_rn(__fmul_rn(sk_small_int_f32(e), 0x1.62e430p-1f), lnf);
}

// cos(2 pi u), sin(2 pi u) for u in [0, 1): quadrant q = floor(4u), remainder
// r; reflect r > 1/2 to 1 - r; phi = a * pi/2; Taylor series of sin to phi^9
// and cos to phi^10 (Horner); swap for the reflected half; rotate by q.
// u = w 2^-23 is passed as the 23-bit integer w: v = 4u = w 2^-21, so
// q = floor(v) = w >> 21 and r = v - q = (w mod 2^21) 2^-21, both exact.
__device__ __forceinline__ void sk_cossin_2pi(uint32_t w, float &c, float &s) {
    const int q = static_cast<int>(w >> 21);
    const float r = __fmul_rn(sk_u23_f32(w & 0x1FFFFFu), 0x1p-21f);
    const bool refl = r > 0.5f;
    const float a = refl ? __fsub_rn(1.0f, r) : r;
    const float phi = __fmul_rn(a, 0x1.921fb6p+0f);
    const float p2 = __fmul_rn(phi, phi);
    float sp = 0x1.71de3ap-19f;
    sp = __fadd_rn(__fmul_rn(sp, p2), -0x1.a01a02p-13f);
    sp = __fadd_rn(__fmul_rn(sp, p2), 0x1.111112p-7f);
    sp = __fadd_rn(__fmul_rn(sp, p2), -0x1.555556p-3f);
    sp = __fadd_rn(__fmul_rn(sp, p2), 1.0f);
    const float sn = __fmul_rn(phi, sp);
    float cp = -0x1.27e4fcp-22f;
    cp = __fadd_rn(__fmul_rn(cp, p2), 0x1.a01a02p-16f);
    cp = __fadd_rn(__fmul_rn(cp, p2), -0x1.6c16c2p-10f);
    cp = __fadd_rn(__fmul_rn(cp, p2), 0x1.555556p-5f);
    cp = __fadd_rn(__fmul_rn(cp, p2), -0.5f);
    cp = __fadd_rn(__fmul_rn(cp, p2), 1.0f);
    const float c0 = refl ? sn : cp;
    const float s0 = refl ? cp : sn;
    switch (q & 3) {
        case 0: c = c0; s = s0; break;
        case 1: c = -s0; s = c0; break;
        case 2: c = -c0; s = -s0; break;
        default: c = s0; s = -c0; break;
    }
}

// Box-Muller pair from two Philox words: u1 = ((we >> 9) + 1) 2^-23 in (0, 1],
// u2 = (wo >> 9) 2^-23; rho = sqrt(-2 ln u1); (rho cos 2pi u2, rho sin 2pi u2).
__device__ __forceinline__ float2 sk_box_muller(uint32_t we, uint32_t wo) {
    const float u1 = __fmul_rn(sk_u23_f32((we >> 9) + 1u), 0x1p-23f);
    const float rho = __fsqrt_rn(__fmul_rn(-2.0f, sk_ln(u1)));
    float c, s;
    sk_cossin_2pi(wo >> 9, c, s);  // u2 = (wo >> 9) 2^-23
    return make_float2(__fmul_rn(rho, c), __fmul_rn(rho, s));
}

// The four unscaled normals z(4b .. 4b+3, i) of the Gaussian sketch.
__device__ __forceinline__ float4 sk_gauss4(uint64_t seed, int64_t i, int64_t rblock) {
    const uint4 w = philox4x32_10(
        make_uint4(static_cast<uint32_t>(static_cast<uint64_t>(i)),
                   static_cast<uint32_t>(static_cast<uint64_t>(i) >> 32),
                   static_cast<uint32_t>(rblock), 0x53474155u),
        static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
    const float2 a = sk_box_muller(w.x, w.y);
    const float2 b = sk_box_muller(w.z, w.w);
    return make_float4(a.x, a.y, b.x, b.y);
}

// Nonzero rows / signs of column i of the sparse-sign sketch (zeta <= 16).
// Words come from Philox4x32-10 with counter (i lo, i hi, block, 0x53535047);
// each proposes row floor(w s / 2^32), sign - for odd w; repeated rows are
// skipped; after 1024 words the smallest untaken rows fill up (sign +).
__device__ __forceinline__ void sk_sparse_column(uint64_t seed, int64_t i, int s, int zeta,
                                                 int *rows, int *sgn) {
    int cnt = 0;
    const uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
    for (uint32_t blk = 0; blk < 256u && cnt < zeta; ++blk) {
        const uint4 w4 = philox4x32_10(
            make_uint4(static_cast<uint32_t>(static_cast<uint64_t>(i)),
                       static_cast<uint32_t>(static_cast<uint64_t>(i) >> 32), blk, 0x53535047u),
            k0, k1);
        const uint32_t ws[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            if (cnt >= zeta) break;
            const int row = static_cast<int>(
                (static_cast<uint64_t>(ws[t]) * static_cast<uint64_t>(s)) >> 32);
            bool dup = false;
            for (int q = 0; q < cnt; ++q) dup |= rows[q] == row;
            if (dup) continue;
            rows[cnt] = row;
            sgn[cnt] = (ws[t] & 1u) ? -1 : 1;
            ++cnt;
        }
    }
    for (int row = 0; cnt < zeta && row < s; ++row) {
        bool dup = false;
        for (int q = 0; q < cnt; ++q) dup |= rows[q] == row;
        if (!dup) {
            rows[cnt] = row;
            sgn[cnt] = 1;
            ++cnt;
        }
    }
}

__host__ __device__ __forceinline__ int pad16(int n) { return (n + 15) / 16 * 16; }
__host__ __device__ __forceinline__ int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ __forceinline__ int64_t round_up(int64_t a, int64_t b) { return ceil_div(a, b) * b; }

// sum_p base[p * stride] for p = 0..np-1, added in increasing p (the same
// rounding as a plain loop); loads are issued eight at a time so that the
// reduction is not one memory latency per term.
__device__ __forceinline__ double ordered_sum(const double *__restrict__ base, size_t stride,
                                              int np) {
    double s = 0.0;
    int p = 0;
    for (; p + 8 <= np; p += 8) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = __ldg(base + size_t(p + u) * stride);
#pragma unroll
        for (int u = 0; u < 8; ++u) s += v[u];
    }
    for (; p < np; ++p) s += __ldg(base + size_t(p) * stride);
    return s;
}

// A padded upper factor is stored as RP (n_pad x n_pad, column-major) followed
// by the same matrix row-major (RT[i * n_pad + j] = r_ij), so that the
// substitution kernel reads a row of R with contiguous loads.  Called by one
// CTA after a barrier that completes its writes of RP.
__device__ __forceinline__ void store_r_rows(double *RP, int n_pad) {
    double *RT = RP + int64_t(n_pad) * n_pad;
    for (int idx = threadIdx.x; idx < n_pad * n_pad; idx += blockDim.x) {
        const int i = idx % n_pad, j = idx / n_pad;
        RT[int64_t(i) * n_pad + j] = RP[idx];
    }
}

}  // namespace rq
