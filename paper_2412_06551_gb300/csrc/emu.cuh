// Digits of the binary64-emulating tensor-core products (split-bf16 with
// exact fp32 sums): an element x of a row or column with exponent E
// (2^E above every |x| of it) becomes F = round(x 2^(63 - E)) (half away
// from zero), written in eight balanced base-256 digits d_0..d_7,
// |d_s| <= 128, so that x = 2^(E - 7) sum_s d_s 2^(-8s) up to 2^(E - 64).
// Every digit is an exact bf16 and every product of two digits an integer of
// magnitude <= 2^14.  Operand tiles are K-major 8 x 8 bf16 core matrices of
// 32 K-columns.  Products keep the levels s + t <= 7 (36 digit pairs); the
// dropped ones are below 2^-61 of the scale.
#pragma once

#include <cuda_bf16.h>

#include <cstdint>

#include "common.cuh"

namespace rq {

constexpr int kEmuDigits = 8;
constexpr int kEmuBK = 32;  // K-columns of one operand tile

// Byte offset of element (row, k) of a K-major operand tile of kEmuBK
// columns laid out as [row/8][k/8][row%8][k%8] (bf16).
__device__ __forceinline__ uint32_t emu_off(int row, int k) {
    return static_cast<uint32_t>(((row >> 3) * (kEmuBK / 8) + (k >> 3)) * 128 + (row & 7) * 16 +
                                 (k & 7) * 2);
}

// Balanced base-256 digits d_0 (top) .. d_{ND-1} of F = round(x 2^(8 ND - 1 - E))
// (half away from zero), for |x| < 2^E: the digits of |F| (bytes with a carry
// into the next one when a byte is >= 128), negated for negative x.  Every
// digit lies in [-128, 128]; |F| < 2^(8 ND - 1).
template <int ND>
__device__ __forceinline__ void emu_digits_n(double x, int E, int (&d)[ND]) {
    static_assert(ND >= 2 && ND <= 8, "one to eight bytes");
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
    const int e = static_cast<int>((b >> 52) & 0x7ff);
    unsigned long long M = b & 0xFFFFFFFFFFFFFull;
    if (e != 0) M |= 1ull << 52;
    // |F| = M 2^sh; for eight digits sh <= 10 for normal x as |x| < 2^E, 11 for
    // subnormals of a column whose largest exponent is subnormal
    const int sh = (e != 0 ? e : 1) - 1076 + 8 * ND - E;
    unsigned long long F;
    if (sh >= 0)
        F = M << (sh & 15);
    else if (sh > -64)
        F = (M + (1ull << (-sh - 1))) >> (-sh);
    else
        F = 0ull;
    const uint32_t lo = static_cast<uint32_t>(F), hi = static_cast<uint32_t>(F >> 32);
    const int neg = static_cast<int>(b >> 63);
    uint32_t c = 0;
#pragma unroll
    for (int q = 0; q < ND - 1; ++q) {
        const uint32_t byte = ((q < 4 ? lo : hi) >> (8 * (q & 3))) & 0xffu;
        const uint32_t u = byte + c + 128u;
        const int dq = static_cast<int>(u & 0xffu) - 128;
        c = u >> 8;
        d[ND - 1 - q] = neg ? -dq : dq;
    }
    const int top = static_cast<int>((ND > 4 ? (hi >> (8 * (ND - 5))) : (lo >> (8 * (ND - 1)))) + c);
    d[0] = neg ? -top : top;
}

// The same digits for two values at once, as packed bf16 pairs ready for a
// K-major tile: w[s] holds digit s of x0 (low half) and of x1 (high half).
// Adding B = sum_{q < ND-1} 128 256^q to |F| gives G, whose bytes below the
// top are the balanced digits plus 128 (the carries of the digit-by-digit
// form happen in the addition) and whose top part is the top digit.  One
// byte permute places a byte of G in the low byte of the binary32 1.5 * 2^23
// (0x4B400000), which makes it the exact integer 1.5 * 2^23 + byte; one FFMA
// with the value's sign s = +-1 gives s (that - 1.5 * 2^23 - bias), the
// signed digit, exactly; two of them are packed by one bf16x2 conversion
// (every digit, |d| <= 128, is an exact bf16).
template <int ND>
__device__ __forceinline__ unsigned long long emu_biased_magnitude(double x, int E, uint32_t &sign) {
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
    const int e = static_cast<int>((b >> 52) & 0x7ff);
    unsigned long long M = b & 0xFFFFFFFFFFFFFull;
    if (e != 0) M |= 1ull << 52;
    const int sh = (e != 0 ? e : 1) - 1076 + 8 * ND - E;
    unsigned long long F;
    if (sh >= 0)
        F = M << (sh & 15);
    else if (sh > -64)
        F = (M + (1ull << (-sh - 1))) >> (-sh);
    else
        F = 0ull;
    sign = static_cast<uint32_t>(b >> 63) << 31;
    constexpr unsigned long long kBias = 0x0080808080808080ull >> (8 * (8 - ND));
    return F + kBias;
}

template <int ND>
__device__ __forceinline__ void emu_digits2_packed(double x0, double x1, int E, uint32_t (&w)[ND]) {
    uint32_t s0, s1;
    const unsigned long long g0 = emu_biased_magnitude<ND>(x0, E, s0);
    const unsigned long long g1 = emu_biased_magnitude<ND>(x1, E, s1);
    const uint32_t w0[2] = {static_cast<uint32_t>(g0), static_cast<uint32_t>(g0 >> 32)};
    const uint32_t w1[2] = {static_cast<uint32_t>(g1), static_cast<uint32_t>(g1 >> 32)};
    const float sg0 = s0 ? -1.0f : 1.0f, sg1 = s1 ? -1.0f : 1.0f;
    // -s (1.5 * 2^23 + 128) for the biased bytes, -s 1.5 * 2^23 for the top one
    const float cb0 = -12583040.0f * sg0, cb1 = -12583040.0f * sg1;
    const float ct0 = -12582912.0f * sg0, ct1 = -12582912.0f * sg1;
#pragma unroll
    for (int s = 0; s < ND; ++s) {
        const int q = ND - 1 - s;  // byte of G
        const uint32_t sel = 0x7650u | static_cast<uint32_t>(q & 3);
        const float f0 = __int_as_float(static_cast<int>(__byte_perm(w0[q >> 2], 0x4B400000u, sel)));
        const float f1 = __int_as_float(static_cast<int>(__byte_perm(w1[q >> 2], 0x4B400000u, sel)));
        const float d0 = fmaf(f0, sg0, q == ND - 1 ? ct0 : cb0);
        const float d1 = fmaf(f1, sg1, q == ND - 1 ? ct1 : cb1);
        const __nv_bfloat162 p = __floats2bfloat162_rn(d0, d1);
        w[s] = *reinterpret_cast<const uint32_t *>(&p);
    }
}

// The same digits by shifts, masks and an integer add per byte, the sign set
// by one XOR (a zero digit of a negative value is -0, which adds like +0).
// Fewer registers live than in the byte-permute form: the substitution
// kernels, capped at 128 registers per thread, run 2-8 % faster with it.
template <int ND>
__device__ __forceinline__ void emu_digits2_packed_shift(double x0, double x1, int E, uint32_t (&w)[ND]) {
    uint32_t s0, s1;
    const unsigned long long g0 = emu_biased_magnitude<ND>(x0, E, s0);
    const unsigned long long g1 = emu_biased_magnitude<ND>(x1, E, s1);
#pragma unroll
    for (int s = 0; s < ND; ++s) {
        const int q = ND - 1 - s;  // byte of G
        const uint32_t v0 = static_cast<uint32_t>(g0 >> (8 * q)), v1 = static_cast<uint32_t>(g1 >> (8 * q));
        float f0, f1;
        if (q == ND - 1) {  // the top digit, 0 .. 128, no bias
            f0 = __int_as_float(0x4B400000 + static_cast<int>(v0)) - 12582912.0f;
            f1 = __int_as_float(0x4B400000 + static_cast<int>(v1)) - 12582912.0f;
        } else {
            f0 = __int_as_float(0x4B400000 + static_cast<int>(v0 & 0xffu)) - 12583040.0f;
            f1 = __int_as_float(0x4B400000 + static_cast<int>(v1 & 0xffu)) - 12583040.0f;
        }
        f0 = __int_as_float(__float_as_int(f0) ^ static_cast<int>(s0));
        f1 = __int_as_float(__float_as_int(f1) ^ static_cast<int>(s1));
        const __nv_bfloat162 p = __floats2bfloat162_rn(f0, f1);
        w[s] = *reinterpret_cast<const uint32_t *>(&p);
    }
}

// The eight digits of the emulated Gram and solve (F = round(x 2^(63 - E))).
__device__ __forceinline__ void emu_digits(double x, int E, int (&d)[kEmuDigits]) {
    emu_digits_n<kEmuDigits>(x, E, d);
}

// bf16 bits of an integer |d| <= 256 (exact): 1.5 * 2^23 + d in binary32,
// minus 1.5 * 2^23, keeps the top 16 bits.
__device__ __forceinline__ uint32_t small_int_bf16(int d) {
    const float f = __int_as_float(0x4B400000 + d) - 12582912.0f;
    return __float_as_uint(f) >> 16;
}

// Selection between the two forms of an emulated solve by a well-conditioned
// factor: the product with R^{-1} runs when Skeel's condition number
// cond(R) = || |R^{-1}| |R| ||_inf (norms[0]) is at most the limit in
// norms[1], max(kWprodMaxCond, n) (both stored as the bits of non-negative
// doubles), the substitution otherwise.
constexpr double kWprodMaxCond = 100.0;

__device__ __forceinline__ bool wprod_selected(const unsigned long long *norms) {
    const double cond = __longlong_as_double(static_cast<long long>(norms[0]));
    const double lim = __longlong_as_double(static_cast<long long>(norms[1]));
    return cond <= lim;
}

// Exponent E with |a| < 2^E for every a of a column with largest biased exponent bits.
__device__ __forceinline__ int emu_exponent(int bits) { return bits - 1022; }

// v 2^e: one exact multiplication by a power of two built from its bits when
// 2^e is a normal number, ldexp otherwise.
__device__ __forceinline__ double emu_scale(double v, int e) {
    if (e >= -1022 && e <= 1023) return v * __longlong_as_double(static_cast<long long>(e + 1023) << 52);
    return ldexp(v, e);
}

// v 2^e as binary64, rounded to nearest (ties to even), by integer operations:
// the int64 -> binary64 conversion instruction runs on GB300's slow FP64 pipe.
// Results that would not be normal numbers take the conversion and emu_scale;
// both ways give the same bits.
__device__ __forceinline__ double emu_i64_scaled(long long v, int e) {
    if (v == 0) return 0.0;
    const unsigned long long sgn = static_cast<unsigned long long>(v) & 0x8000000000000000ull;
    const unsigned long long a = v < 0 ? 0ull - static_cast<unsigned long long>(v) : static_cast<unsigned long long>(v);
    const int lz = __clzll(static_cast<long long>(a));
    const int be = 1086 - lz + e;  // biased exponent of the leading bit of a 2^e
    if (be < 1 || be > 2045) return emu_scale(static_cast<double>(v), e);
    const unsigned long long an = a << lz;  // leading one at bit 63
    unsigned long long mant = an >> 11;     // 53 bits with the leading one
    const unsigned long long rest = an & 0x7FFull;
    mant += (rest > 0x400ull || (rest == 0x400ull && (mant & 1ull))) ? 1ull : 0ull;
    // the leading one adds 1 to the exponent field; a rounding carry adds one more
    const unsigned long long bits = (static_cast<unsigned long long>(be - 1) << 52) + mant;
    return __longlong_as_double(static_cast<long long>(bits | sgn));
}

// A level sum C (an exact integer in fp32, |C| <= 2^24) times 2^k as an
// integer: exact for k >= 0, rounded (half up) for k < 0.  A window's levels
// L = 0..7 enter one int64 accumulator with k = 24 - 8L + u, i.e. in units of
// 2^-(24 + u) of level 0.
template <int k>
__device__ __forceinline__ long long emu_level(float c) {
    const long long v = __float2int_rn(c);
    if constexpr (k >= 0)
        return v * (1ll << k);
    else
        return (v + (1ll << (-k - 1))) >> (-k);
}

}  // namespace rq
