// Triangular solve with binary64-emulating block products, wide-block form
// for n > 128 (the 16-column form of emu_trsm.cu serves n <= 128): the same
// substitution with 32-column blocks, so that a row tile re-splits Q's rows
// for 28 rather than 120 K-chunks at n = 256.
//
// Triangular solve Q = A R^{-1} with its block products emulating binary64 on
// the tensor cores (the precision form of eq. (ewy) / C3, C7: substitution by
// 32-column blocks, the off-diagonal block products as split-bf16 products
// with exact fp32 sums, the diagonal blocks solved in binary64).
//
// For column block J (columns [32J, 32J + 32)):
//   C_J = A_J - Q_{<J} R_{<J,J}      (emulated: digits of Q's rows, R's columns)
//   Q_J = C_J R_JJ^{-1}              (binary64 substitution, as the FP64 kernel)
// Q_{<J}'s digits use one exponent per row over its first 32J columns (from a
// running maximum of the row's solved exponents), R's one per column over
// rows < 32J (precomputed by k_trsm_emu32_prep).  Digits are those of the
// emulated Gram (emu.cuh); levels s + t <= 7 are kept; a level's fp32 sum over
// at most 128 K-columns (8 x 128 products <= 2^14) is exact, so the TMEM
// accumulators are drained into one int64 per element (units of 2^-40 of
// level 0, levels 6 and 7 rounded to that unit) after every 4 K-chunks of 32.
// The update is then 2^(E_i + E'_c - 54) times that integer.
//
// A CTA walks its chunk of rows in tiles of 128 (M = 128, one row per TMEM
// lane).  Per K-chunk the 256 threads load 128 x 32 solved values of Q (L2,
// written by the CTA itself), split them into digits (K-major operand tiles),
// copy R's precomputed digit tiles, and one thread issues 8 x 2 MMAs
// (kind::f16, M=128, N=256 .. 32, K=16: one digit of Q times the side-by-side
// digits of R) into eight 32-column accumulators.  Two CTAs
// share an SM (80 KB of shared memory and 256 TMEM columns each), so one's
// binary64 diagonal solve overlaps the other's digit split and tensor-core
// work.  The diagonal-block solve gives each row 2 adjacent lanes of a warp
// (16 interleaved columns each) and broadcasts solved values by shuffles.
#include <algorithm>

#include "common.cuh"
#include "emu.cuh"
#include "kernels.h"
#include "tcgen05.cuh"

namespace rq {
namespace {

constexpr int kTeThreads = 256;
constexpr int kTeM = 128;         // rows per tile
constexpr int kTeB = 32;          // columns per block (= K per chunk = N of the MMA)
constexpr int kTeWinChunks = 4;   // K-chunks per exact window (128 K-columns)
constexpr int kTeStages = 1;      // one stage: the second CTA on the SM covers the waits
constexpr int kTeTileA = kTeM * kEmuBK * 2;   // one digit tile of Q: 8 KB
constexpr int kTeTileB = kTeB * kEmuBK * 2;   // one digit tile of R: 2 KB
constexpr int kTeStageA = kEmuDigits * kTeTileA;
constexpr int kTeStageB = kEmuDigits * kTeTileB;
constexpr int kTeStageBytes = kTeStageA + kTeStageB;
constexpr int kTeCBytes = kTeM * kTeB * 8;    // binary64 block C_J (in the stage's Q digits)
constexpr int kTeUnit = 16;                   // drain units: 2^-(24 + 16) of level 0
static_assert(kTeCBytes <= kTeStageA, "C_J reuses the digit tiles of Q");
constexpr int kTeTmemCols = 256;
constexpr int kTeP = kTeThreads / kTeM;       // lanes per row in the diagonal solve (2)
constexpr int kTeCPT = kTeB / kTeP;           // columns per lane

// R's digit tiles of (target block J, K-chunk kc), kc < J, stored densely.
__host__ __device__ __forceinline__ size_t te_rtile(int J, int kc) {
    return (size_t(J) * (J - 1) / 2 + kc) * kTeStageB;
}

// Column exponents of R over rows < 32J for each target block J >= 1, and the
// digit tiles of R[32 kc .. 32 kc + 31][32J .. 32J + 31].  One CTA per J.
__global__ void k_trsm_emu32_prep(const double *__restrict__ RP, int ldr, int n,
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
        unsigned char *tile = rdig + te_rtile(J, k / kEmuBK);
#pragma unroll
        for (int s = 0; s < kEmuDigits; ++s)
            *reinterpret_cast<uint16_t *>(tile + s * kTeTileB + emu_off(c, k % kEmuBK)) =
                static_cast<uint16_t>(small_int_bf16(d[s]));
    }
}

__global__ void __launch_bounds__(kTeThreads, 2)
    k_trsm_emu32(const double *A, int64_t lda, int64_t m, int n, int n_pad, int64_t chunk,
               const double *__restrict__ RT, const double *__restrict__ rinv,
               const unsigned char *__restrict__ rdig, const int *__restrict__ rbits, double *Q,
               int64_t ldq, DevStatus *st,
               const unsigned long long *skip_if) {
    if (skip_if != nullptr && wprod_selected(skip_if)) return;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar_mma[kTeStages];
    __shared__ __align__(8) uint64_t bar_r;  // bulk copy of R's digit tiles
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    __shared__ int rowbits[kTeM];
    // C_J [col][row] reuses the Q digit tiles: it is written only after the
    // block's last MMAs completed and read before the next block's split
    double *Cb = reinterpret_cast<double *>(smem_raw);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) tmem_alloc(&tmem_slot, kTeTmemCols);
    if (tid == 0) {
        for (int s = 0; s < kTeStages; ++s) mbar_init(&bar_mma[s], 1);
        mbar_init(&bar_r, 1);
        fence_mbar_init();
        abort_flag = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const uint32_t smem_base = smem_u32(smem_raw);
    const int nblk = (n + kTeB - 1) / kTeB;

    // drain ownership: TMEM lanes 32 (warp % 4) .. +31 (rows), columns 16 (warp / 4) .. +15
    const int lane_base = 32 * (warp & 3);
    const int cgrp = warp >> 2;
    const int drow = lane_base + lane;
    constexpr int kDrainCols = kTeB / (kTeThreads / kTeM);  // 16
    // digit tasks: row task % 128, K-columns 8 (task / 128) .. +7 of the chunk
    constexpr int kTasks = kTeM * (kEmuBK / 8) / kTeThreads;  // 2 per thread
    // diagonal solve: row ti, lane p of 2, columns p + 2c
    const int p = tid % kTeP, ti = tid / kTeP;
    const int src0 = (tid & 31) - p;

    const int64_t rb = int64_t(blockIdx.x) * chunk;
    const int64_t re = std::min<int64_t>(m, rb + chunk);
    unsigned kcount = 0;  // K-chunks issued by this CTA (ring position and phase)
    for (int64_t r0 = rb; r0 < re; r0 += kTeM) {
        if (tid < kTeM) rowbits[tid] = 0;
        __syncthreads();
        for (int J = 0; J < nblk; ++J) {
            const int j0 = kTeB * J;
            long long acc[kDrainCols];
#pragma unroll
            for (int q = 0; q < kDrainCols; ++q) acc[q] = 0;
            // ---- C_J update: emulated Q_{<J} R_{<J,J} over K-chunks kc < J
            for (int kc = 0; kc < J; ++kc, ++kcount) {
                const int sidx = kcount % kTeStages;
                unsigned char *stage = smem_raw + sidx * kTeStageBytes;
                // loads first: in flight while the stage's previous MMAs finish
                double xv[kTasks][8];
#pragma unroll
                for (int u = 0; u < kTasks; ++u) {
                    const int task = tid + u * kTeThreads;
                    const int64_t row = r0 + task % kTeM;
#pragma unroll
                    for (int t = 0; t < 8; ++t) {
                        const int col = kEmuBK * kc + 8 * (task / kTeM) + t;
                        xv[u][t] = row < re ? __ldcg(Q + row + int64_t(col) * ldq) : 0.0;
                    }
                }
                if (kcount >= kTeStages &&
                    !mbar_wait_bounded(&bar_mma[sidx],
                                       static_cast<uint32_t>((kcount / kTeStages - 1) & 1)))
                    abort_flag = 1;
                __syncthreads();
                if (abort_flag) break;
                if (tid == 0) {  // R's digit tiles of (J, kc), one bulk copy
                    fence_proxy_async_smem();
                    mbar_arrive_expect_tx(&bar_r, kTeStageB);
                    bulk_load(stage + kTeStageA, rdig + te_rtile(J, kc), kTeStageB, &bar_r);
                }
#pragma unroll
                for (int u = 0; u < kTasks; ++u) {
                    const int task = tid + u * kTeThreads;
                    const int srow = task % kTeM, skg = task / kTeM;
                    const int E = emu_exponent(rowbits[srow]);
                    // two rows at a time: one 32-bit word (two bf16) per digit
#pragma unroll
                    for (int t = 0; t < 8; t += 2) {
                        uint32_t w[kEmuDigits];
                        emu_digits2_packed_shift<kEmuDigits>(xv[u][t], xv[u][t + 1], E, w);
#pragma unroll
                        for (int s = 0; s < kEmuDigits; ++s)
                            *reinterpret_cast<uint32_t *>(stage + s * kTeTileA +
                                                          emu_off(srow, 8 * skg + t)) = w[s];
                    }
                }
                fence_proxy_async_smem();
                __syncthreads();
                if (tid == 0) {
                    const bool have_r = mbar_wait_bounded(&bar_r, kcount & 1u);
                    if (!have_r) abort_flag = 1;
                    tc_fence_after();
                    const uint32_t sa = smem_base + sidx * kTeStageBytes;
                    const uint32_t sb = sa + kTeStageA;
                    const bool fresh = (kc % kTeWinChunks) == 0;
                    if (have_r) {
                        // R's eight digit tiles lie side by side (32 rows of the
                        // K-major operand each): digit s of Q times digits
                        // 0 .. 7 - s of R is one MMA of N = 32 (8 - s) into
                        // levels s .. 7 (TMEM columns 32 s ..), eight MMAs per
                        // 16-column k-step; those with s = 0 write every level
                        // and come first, so only they start a window afresh
#pragma unroll
                        for (int kk = 0; kk < kEmuBK / 16; ++kk) {
                            const uint64_t bd = smem_desc(sb + kk * 256, 128, (kEmuBK / 8) * 128);
#pragma unroll
                            for (int s = 0; s < kEmuDigits; ++s)
                                mma_bf16(tmem + static_cast<uint32_t>(s * kTeB),
                                         smem_desc(sa + s * kTeTileA + kk * 256, 128, (kEmuBK / 8) * 128),
                                         bd, idesc_bf16_f32(kTeM, kTeB * (kEmuDigits - s)),
                                         (fresh && s == 0 && kk == 0) ? 0u : 1u);
                        }
                    }
                    mma_commit(&bar_mma[sidx]);
                }
                if ((kc % kTeWinChunks) == kTeWinChunks - 1 || kc == J - 1) {
                    if (!mbar_wait_bounded(&bar_mma[sidx],
                                           static_cast<uint32_t>((kcount / kTeStages) & 1)))
                        abort_flag = 1;
                    __syncthreads();
                    if (abort_flag) break;
                    tc_fence_after();
                    const uint32_t tl = tmem + (static_cast<uint32_t>(lane_base) << 16) +
                                        static_cast<uint32_t>(kDrainCols * cgrp);
                    float v[kDrainCols];
#pragma unroll
                    for (int L = 0; L < kEmuDigits; ++L) {
                        tmem_ld16(tl + static_cast<uint32_t>(L * kTeB), v);
#pragma unroll
                        for (int q = 0; q < kDrainCols; ++q) {
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
                    __syncthreads();
                }
            }
            if (abort_flag) break;
            // ---- C_J = A_J - update, in shared memory [col][row]
            {
                const int64_t row = r0 + drow;
                const int rbit = rowbits[drow];
#pragma unroll
                for (int q = 0; q < kDrainCols; ++q) {
                    const int c = kDrainCols * cgrp + q, col = j0 + c;
                    double a = (row < re && col < n) ? A[row + int64_t(col) * lda] : 0.0;
                    if (J > 0 && col < n) {
                        const int cbit = __ldg(rbits + J * kTeB + c);
                        const double u = (rbit == 0x7ff || cbit == 0x7ff)
                                             ? __longlong_as_double(0x7ff8000000000000ll)
                                             : emu_i64_scaled(acc[q],
                                                         emu_exponent(rbit) + emu_exponent(cbit) -
                                                             14 - 24 - kTeUnit);
                        a -= u;
                    }
                    Cb[c * kTeM + drow] = a;
                }
            }
            __syncthreads();
            // ---- Q_J = C_J R_JJ^{-1} (binary64): column j0 + t in turn
            {
                double x[kTeCPT];
#pragma unroll
                for (int c = 0; c < kTeCPT; ++c) x[c] = Cb[(p + kTeP * c) * kTeM + ti];
#pragma unroll
                for (int t = 0; t < kTeB; ++t) {
                    const int owner = t % kTeP, lc = t / kTeP;
                    const int jt = j0 + t;
                    if (p == owner) x[lc] *= (jt < n) ? __ldg(rinv + jt) : 0.0;
                    const double q = __shfl_sync(0xffffffffu, x[lc], src0 + owner);
                    if (jt < n) {
                        const double *rk = RT + int64_t(jt) * n_pad + j0 + p;
#pragma unroll
                        for (int c = 0; c < kTeCPT; ++c) {
                            if ((kTeP - 1) + kTeP * c <= t) continue;  // no lane has a column past t
                            if (p + kTeP * c > t && j0 + p + kTeP * c < n)
                                x[c] = fma(-q, __ldg(rk + kTeP * c), x[c]);
                        }
                    }
                }
                // store Q_J and fold the row's exponents into its running maximum
                const int64_t row = r0 + ti;
                int eb = 0;
#pragma unroll
                for (int c = 0; c < kTeCPT; ++c) {
                    const int col = j0 + p + kTeP * c;
                    if (col < n) {
                        if (row < re) Q[row + int64_t(col) * ldq] = x[c];
                        const unsigned long long b =
                            static_cast<unsigned long long>(__double_as_longlong(x[c]));
                        eb = max(eb, static_cast<int>((b >> 52) & 0x7ff));
                    }
                }
#pragma unroll
                for (int off = 1; off < kTeP; off <<= 1) eb = max(eb, __shfl_xor_sync(0xffffffffu, eb, off));
                __syncthreads();  // every thread has read rowbits for this block
                if (p == 0) rowbits[ti] = max(rowbits[ti], eb);
                __syncthreads();  // Q_J stored and rowbits updated before the next block reads them
            }
        }
        if (abort_flag) break;
    }
    if (abort_flag && tid == 0) report(st, kErrTimeout, 0, -1);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kTeTmemCols);
}

}  // namespace

size_t trsm_emu32_scratch_bytes(int n) {
    const int nblk = (n + kTeB - 1) / kTeB;
    return te_rtile(nblk, 0) + size_t(nblk) * kTeB * sizeof(int) + 256;
}

cudaError_t launch_trsm_emu32(const double *A, int64_t lda, int64_t m, int n, const double *RP,
                              const double *rinv, double *Q, int64_t ldq, void *scratch,
                              DevStatus *st, cudaStream_t stream,
                            const unsigned long long *skip_if) {
    if (n < 1 || n > 256 || m < 1) return cudaErrorInvalidValue;
    const int n_pad = pad16(n);
    const int nblk = (n + kTeB - 1) / kTeB;
    unsigned char *rdig = static_cast<unsigned char *>(scratch);
    int *rbits = reinterpret_cast<int *>(rdig + te_rtile(nblk, 0));
    cudaError_t e;
    if (nblk > 1) {
        RQ_LAUNCH(KID_EMU_AUX, stream,
                  k_trsm_emu32_prep<<<nblk - 1, 256, 0, stream>>>(RP, n_pad, n, rdig, rbits, skip_if));
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const int64_t tiles = ceil_div(m, kTeM);
    const int64_t grid = std::min<int64_t>(tiles, int64_t(2) * grid_sms());
    const int64_t chunk = ceil_div(tiles, grid) * kTeM;
    const int g = static_cast<int>(ceil_div(m, chunk));
    const size_t smem = size_t(kTeStages) * kTeStageBytes;
    cudaFuncSetAttribute(k_trsm_emu32, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    RQ_LAUNCH(KID_TRSM_EMU, stream,
              k_trsm_emu32<<<g, kTeThreads, smem, stream>>>(A, lda, m, n, n_pad, chunk,
                                                          RP + size_t(n_pad) * n_pad, rinv, rdig,
                                                          rbits, Q, ldq, st, skip_if));
    return cudaGetLastError();
}

}  // namespace rq
