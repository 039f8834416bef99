// Triangular solve Q = A R^{-1} with its block products emulating binary64 on
// the tensor cores (the precision form of eq. (ewy) / C3, C7), n <= 160 (the
// 32-column form of emu_trsm32.cu serves n > 160): substitution by
// 16-column blocks, the off-diagonal block products as split-bf16 products
// with exact fp32 sums, the diagonal blocks solved in binary64).
//
// For column block J (columns [16J, 16J + 16)):
//   C_J = A_J - Q_{<J} R_{<J,J}      (emulated: digits of Q's rows, R's columns)
//   Q_J = C_J R_JJ^{-1}              (binary64 substitution, as the FP64 kernel)
// Q_{<J}'s digits use one exponent per row over its first 16J columns (a
// running maximum of the row's solved exponents, so earlier blocks are
// re-split from their binary64 values in L2 when it grows), R's one per
// column over rows < 16J (precomputed by k_trsm_emu_prep).  Digits are those
// of the emulated Gram (emu.cuh); levels s + t <= 7 are kept; a level's fp32
// sum over at most 128 K-columns (8 x 128 products <= 2^14) is exact, so the
// TMEM accumulators are drained into one int64 per element (units of 2^-40
// of level 0, levels 6 and 7 rounded to that unit) after every 8 K-chunks of
// 16.  The update is then 2^(E_i + E'_c - 54) times that integer.
//
// A CTA of 128 threads walks its chunk of rows in tiles of 128: thread t owns
// row t of the tile, which is also TMEM lane t of the MMA (M = 128).  Per
// K-chunk of 16 columns each thread loads its row's 16 solved values of Q
// (L2, written by the CTA itself) and splits them into digits (K-major
// operand tiles), one thread bulk-copies R's precomputed digit tiles and
// issues eight MMAs (kind::f16, M=128, N=128 .. 16, K=16: one digit of Q
// times the side-by-side digits of R) into eight 16-column accumulators.  The drain, the binary64 update of C_J and the diagonal
// substitution all stay in the owning thread's registers: no shuffles and no
// barriers between rows.  Four CTAs share an SM (36 KB of shared memory and
// 128 TMEM columns each), so one CTA's binary64 substitution overlaps the
// others' digit splits and tensor-core work.
#include <algorithm>

#include "common.cuh"
#include "emu.cuh"
#include "kernels.h"
#include "tcgen05.cuh"

namespace rq {
namespace {

constexpr int kTeThreads = 128;
constexpr int kTeM = 128;         // rows per tile (one per thread)
constexpr int kTeB = 16;          // columns per block (= K per chunk = N of the MMA)
constexpr int kTeWinChunks = 8;   // K-chunks per exact window (128 K-columns)
constexpr int kTeCtasPerSm = 4;
constexpr int kTeTileA = kTeM * kTeB * 2;     // one digit tile of Q: 4 KB
constexpr int kTeTileB = kTeB * kTeB * 2;     // one digit tile of R: 512 B
constexpr int kTeStageA = kEmuDigits * kTeTileA;
constexpr int kTeStageB = kEmuDigits * kTeTileB;
constexpr int kTeStageBytes = kTeStageA + kTeStageB;
constexpr int kTeTmemCols = 128;              // eight 16-column accumulators
constexpr int kTeUnit = 16;                   // drain units: 2^-(24 + 16) of level 0

// Byte offset of element (row, k) of a K-major operand tile of 16 K-columns
// laid out as [row/8][k/8][row%8][k%8] (bf16).
__device__ __forceinline__ uint32_t te_off(int row, int k) {
    return static_cast<uint32_t>(((row >> 3) * 2 + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// R's digit tiles of (target block J, K-chunk kc), kc < J, stored densely.
__host__ __device__ __forceinline__ size_t te_rtile(int J, int kc) {
    return (size_t(J) * (J - 1) / 2 + kc) * kTeStageB;
}

// Column exponents of R over rows < 16J for each target block J >= 1, and the
// digit tiles of R[16 kc .. 16 kc + 15][16J .. 16J + 15].  One CTA per J.
__global__ void k_trsm_emu_prep(const double *__restrict__ RP, int ldr, int n,
                                unsigned char *__restrict__ rdig, int *__restrict__ rbits,
                                const unsigned long long *skip_if) {
    if (skip_if != nullptr && wprod_selected(skip_if)) return;
    const int J = blockIdx.x + 1;
    const int j0 = kTeB * J;
    __shared__ int cb[kTeB];
    if (threadIdx.x < kTeB) {
        const int col = j0 + threadIdx.x;
        int e = 0;
        if (col < n)
            for (int k = 0; k < j0; ++k) {
                const unsigned long long b =
                    static_cast<unsigned long long>(__double_as_longlong(RP[k + int64_t(col) * ldr]));
                e = max(e, static_cast<int>((b >> 52) & 0x7ff));
            }
        cb[threadIdx.x] = e;
        rbits[J * kTeB + threadIdx.x] = e;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < j0 * kTeB; idx += blockDim.x) {
        const int k = idx % j0, c = idx / j0;
        const int col = j0 + c;
        const double r = col < n ? RP[k + int64_t(col) * ldr] : 0.0;
        int d[kEmuDigits];
        emu_digits(r, emu_exponent(cb[c]), d);
        unsigned char *tile = rdig + te_rtile(J, k / kTeB);
#pragma unroll
        for (int s = 0; s < kEmuDigits; ++s)
            *reinterpret_cast<uint16_t *>(tile + s * kTeTileB + te_off(c, k % kTeB)) =
                static_cast<uint16_t>(small_int_bf16(d[s]));
    }
}

__global__ void __launch_bounds__(kTeThreads, kTeCtasPerSm)
    k_trsm_emu(const double *A, int64_t lda, int64_t m, int n, int n_pad, int64_t chunk,
               const double *__restrict__ RT, const double *__restrict__ rinv,
               const unsigned char *__restrict__ rdig, const int *__restrict__ rbits, double *Q,
               int64_t ldq, DevStatus *st,
               const unsigned long long *skip_if) {
    if (skip_if != nullptr && wprod_selected(skip_if)) return;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar_mma;
    __shared__ __align__(8) uint64_t bar_r;  // bulk copy of R's digit tiles
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5;
    if (warp == 0) tmem_alloc(&tmem_slot, kTeTmemCols);
    if (tid == 0) {
        mbar_init(&bar_mma, 1);
        mbar_init(&bar_r, 1);
        fence_mbar_init();
        abort_flag = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const uint32_t sa = smem_u32(smem_raw);
    const uint32_t sb = sa + kTeStageA;
    const uint32_t tl = tmem + (static_cast<uint32_t>(32 * warp) << 16);  // this warp's lanes
    const int nblk = (n + kTeB - 1) / kTeB;

    const int64_t rb = int64_t(blockIdx.x) * chunk;
    const int64_t re = std::min<int64_t>(m, rb + chunk);
    unsigned kcount = 0;  // K-chunks issued by this CTA (barrier phases)
    for (int64_t r0 = rb; r0 < re; r0 += kTeM) {
        const int64_t row = r0 + tid;
        const bool live = row < re;
        int rowbits = 0;  // running maximum of the exponents of this row's solved values
        for (int J = 0; J < nblk; ++J) {
            const int j0 = kTeB * J;
            long long acc[kTeB];
#pragma unroll
            for (int q = 0; q < kTeB; ++q) acc[q] = 0;
            // ---- update of C_J: emulated Q_{<J} R_{<J,J} over K-chunks kc < J
            for (int kc = 0; kc < J; ++kc, ++kcount) {
                double xv[kTeB];
#pragma unroll
                for (int t = 0; t < kTeB; ++t)
                    xv[t] = live ? __ldcg(Q + row + int64_t(kTeB * kc + t) * ldq) : 0.0;
                // the previous chunk's MMAs have read the stage
                if (kcount > 0 && !mbar_wait_bounded(&bar_mma, (kcount - 1) & 1u)) abort_flag = 1;
                __syncthreads();
                if (abort_flag) break;
                if (tid == 0) {
                    fence_proxy_async_smem();
                    mbar_arrive_expect_tx(&bar_r, kTeStageB);
                    bulk_load(smem_raw + kTeStageA, rdig + te_rtile(J, kc), kTeStageB, &bar_r);
                }
                const int E = emu_exponent(rowbits);
#pragma unroll
                for (int h = 0; h < 4; ++h) {  // K-columns 4h .. 4h + 3: one 8-byte piece per digit
                    uint32_t w[kEmuDigits][2];
#pragma unroll
                    for (int t = 0; t < 4; t += 2) {
                        uint32_t wp[kEmuDigits];
                        emu_digits2_packed_shift<kEmuDigits>(xv[4 * h + t], xv[4 * h + t + 1], E, wp);
#pragma unroll
                        for (int s = 0; s < kEmuDigits; ++s) w[s][t >> 1] = wp[s];
                    }
#pragma unroll
                    for (int s = 0; s < kEmuDigits; ++s)
                        *reinterpret_cast<uint2 *>(smem_raw + s * kTeTileA + te_off(tid, 4 * h)) =
                            make_uint2(w[s][0], w[s][1]);
                }
                fence_proxy_async_smem();
                __syncthreads();
                if (tid == 0) {
                    const bool have_r = mbar_wait_bounded(&bar_r, kcount & 1u);
                    if (!have_r) abort_flag = 1;
                    tc_fence_after();
                    const bool fresh = (kc % kTeWinChunks) == 0;
                    if (have_r) {
                        // R's eight digit tiles lie side by side (16 rows of the
                        // K-major operand each), so digit s of Q times digits
                        // 0 .. 7 - s of R is one MMA of N = 16 (8 - s) landing in
                        // levels s .. 7 (TMEM columns 16 s ..): eight MMAs per
                        // chunk for the 36 digit pairs; the first writes every
                        // level, so only it starts a window afresh
                        const uint64_t bd = smem_desc(sb, 128, 256);
#pragma unroll
                        for (int s = 0; s < kEmuDigits; ++s)
                            mma_bf16(tmem + static_cast<uint32_t>(s * kTeB),
                                     smem_desc(sa + s * kTeTileA, 128, 256), bd,
                                     idesc_bf16_f32(kTeM, kTeB * (kEmuDigits - s)),
                                     (fresh && s == 0) ? 0u : 1u);
                    }
                    mma_commit(&bar_mma);
                }
                if ((kc % kTeWinChunks) == kTeWinChunks - 1 || kc == J - 1) {
                    // window end: every thread drains its own TMEM lane
                    if (!mbar_wait_bounded(&bar_mma, kcount & 1u)) abort_flag = 1;
                    __syncthreads();
                    if (abort_flag) break;
                    tc_fence_after();
                    float v[kTeB];
#pragma unroll
                    for (int L = 0; L < kEmuDigits; ++L) {
                        tmem_ld16(tl + static_cast<uint32_t>(L * kTeB), v);
#pragma unroll
                        for (int q = 0; q < kTeB; ++q) {
                            switch (L) {  // compile-time after unrolling
                                case 0: acc[q] += emu_level<24 + kTeUnit>(v[q]); break;
                                case 1: acc[q] += emu_level<16 + kTeUnit>(v[q]); break;
                                case 2: acc[q] += emu_level<8 + kTeUnit>(v[q]); break;
                                case 3: acc[q] += emu_level<0 + kTeUnit>(v[q]); break;
                                case 4: acc[q] += emu_level<-8 + kTeUnit>(v[q]); break;
                                case 5: acc[q] += emu_level<-16 + kTeUnit>(v[q]); break;
                                case 6: acc[q] += emu_level<-24 + kTeUnit>(v[q]); break;
                                default: acc[q] += emu_level<-32 + kTeUnit>(v[q]); break;
                            }
                        }
                    }
                    tc_fence_before();
                    __syncthreads();  // TMEM read before the next window's MMAs overwrite it
                }
            }
            if (abort_flag) break;
            // ---- C_J = A_J - update and Q_J = C_J R_JJ^{-1}, in this thread's registers
            double x[kTeB];
#pragma unroll
            for (int q = 0; q < kTeB; ++q) {
                const int col = j0 + q;
                double a = (live && col < n) ? A[row + int64_t(col) * lda] : 0.0;
                if (J > 0 && col < n) {
                    const int cbit = __ldg(rbits + J * kTeB + q);
                    a -= (rowbits == 0x7ff || cbit == 0x7ff)
                             ? __longlong_as_double(0x7ff8000000000000ll)
                             : emu_i64_scaled(acc[q],
                                         emu_exponent(rowbits) + emu_exponent(cbit) - 14 - 24 - kTeUnit);
                }
                x[q] = a;
            }
#pragma unroll
            for (int t = 0; t < kTeB; ++t) {
                const int jt = j0 + t;
                x[t] *= (jt < n) ? __ldg(rinv + jt) : 0.0;
                if (jt < n) {
                    const double *rk = RT + int64_t(jt) * n_pad + j0;
#pragma unroll
                    for (int q = t + 1; q < kTeB; ++q)
                        if (j0 + q < n) x[q] = fma(-x[t], __ldg(rk + q), x[q]);
                }
            }
            int eb = 0;
#pragma unroll
            for (int q = 0; q < kTeB; ++q) {
                const int col = j0 + q;
                if (col < n) {
                    if (live) Q[row + int64_t(col) * ldq] = x[q];
                    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x[q]));
                    eb = max(eb, static_cast<int>((b >> 52) & 0x7ff));
                }
            }
            rowbits = max(rowbits, eb);
        }
        if (abort_flag) break;
    }
    if (abort_flag && tid == 0) report(st, kErrTimeout, 0, -1);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kTeTmemCols);
}

}  // namespace

size_t trsm_emu_scratch_bytes(int n) {
    const int nblk = (n + kTeB - 1) / kTeB;
    return std::max(te_rtile(nblk, 0) + size_t(nblk) * kTeB * sizeof(int) + 256,
                    trsm_emu32_scratch_bytes(n));
}

cudaError_t launch_trsm_emu(const double *A, int64_t lda, int64_t m, int n, const double *RP,
                            const double *rinv, double *Q, int64_t ldq, void *scratch,
                            DevStatus *st, cudaStream_t stream,
                            const unsigned long long *skip_if) {
    if (n < 1 || n > 256 || m < 1) return cudaErrorInvalidValue;
    if (n > 160)  // wide blocks: fewer re-split K-chunks per row tile (16 columns win up to n = 160)
        return launch_trsm_emu32(A, lda, m, n, RP, rinv, Q, ldq, scratch, st, stream, skip_if);
    const int n_pad = pad16(n);
    const int nblk = (n + kTeB - 1) / kTeB;
    unsigned char *rdig = static_cast<unsigned char *>(scratch);
    int *rbits = reinterpret_cast<int *>(rdig + te_rtile(nblk, 0));
    cudaError_t e;
    if (nblk > 1) {
        RQ_LAUNCH(KID_EMU_AUX, stream,
                  k_trsm_emu_prep<<<nblk - 1, 256, 0, stream>>>(RP, n_pad, n, rdig, rbits, skip_if));
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const int64_t tiles = ceil_div(m, kTeM);
    const int64_t grid = std::min<int64_t>(tiles, int64_t(kTeCtasPerSm) * grid_sms());
    const int64_t chunk = ceil_div(tiles, grid) * kTeM;
    const int g = static_cast<int>(ceil_div(m, chunk));
    const size_t smem = kTeStageBytes;
    cudaFuncSetAttribute(k_trsm_emu, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    RQ_LAUNCH(KID_TRSM_EMU, stream,
              k_trsm_emu<<<g, kTeThreads, smem, stream>>>(A, lda, m, n, n_pad, chunk,
                                                          RP + size_t(n_pad) * n_pad, rinv, rdig,
                                                          rbits, Q, ldq, st, skip_if));
    return cudaGetLastError();
}

}  // namespace rq
