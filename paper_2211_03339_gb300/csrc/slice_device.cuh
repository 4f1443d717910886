// slice_device.cuh -- exact splitting of FP64 values into bf16 integer digits
// (the Ozaki scheme: Ozaki, Ogita, Oishi, Rump, Numer. Algorithms 59, 2012) with
// integer operations on the FP64 bit patterns, shared by the tensor-core FP64
// sweeps (tc64_apply.cu) and the exactly split products (ozaki.cu).
//
// With E_r the largest biased exponent class of a row (exp_class), an entry x of
// the row is represented as
//
//   M = sign(x) trunc(|x| 2^(1078 - E_r)),  |M| < 2^56,  M = sum_s a_s 2^(49 - 7 s),
//   |a_0| <= 128, a_s in [-64, 63] (s = 1..7),
//
// i.e. x = 2^(E_r - 1029) sum_s a_s 2^(-7 s) up to 2^(E_r - 1078): every entry
// within 2^3 of the row maximum is represented exactly.  The digits are small
// integers, exact in bf16, and their pairwise products exact in FP32.
#pragma once

#include <cstdint>

namespace mpj {
namespace slice {

// 64 at each of the seven lower 7-bit digit positions and 256 at the top one:
// for a signed M_s (|M_s| < 2^56), M_s + kBias is positive and below 2^58; its
// base-128 digits (the top one 9 bits wide) minus 64 (minus 256 at the top) are
// the balanced digits of M_s, M_s = sum_s d_s 2^(49 - 7 s), |d_0| <= 128,
// d_s in [-64, 63].
constexpr uint64_t kBias =
    64ull * ((1ull << 42) + (1ull << 35) + (1ull << 28) + (1ull << 21) + (1ull << 14) + (1ull << 7) + 1ull) +
    (1ull << 57);

// ---------------------------------------------------------------- slicing
// Exponent class of x for a row maximum: 0 for x == 0, else max(E, 1) with E the
// biased exponent (subnormals count as 1).  Integer operations only.
__device__ __forceinline__ int exp_class(double x) {
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
    const int E = (hi >> 20) & 0x7FF;
    const int nz = ((hi & 0xFFFFFu) | lo) != 0u;
    return E ? E : nz;
}

// M_s + kBias for M_s = sign(x) trunc(|x| 2^(1078 - Er)), Er >= exp_class(x).
__device__ __forceinline__ uint64_t scaled_signed(double x, int Er) {
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    const int E = (int)((b >> 52) & 0x7FF);
    uint64_t mant = b & 0xFFFFFFFFFFFFFull;
    if (E) mant |= 1ull << 52;
    const int sh = (E ? E : 1) - Er + 3;          // <= 3
    const uint64_t M = sh >= 0 ? (mant << sh) : (sh > -64 ? (mant >> -sh) : 0ull);
    const uint64_t sm = (uint64_t)((long long)b >> 63);   // all ones for a negative x
    return ((M ^ sm) - sm) + kBias;
}

// Digit s of a biased value as an exact float: the raw field (9 bits at the top
// digit, 7 below) through the magic constant 2^23, minus 2^23 and the bias.
__device__ __forceinline__ float digit_f(uint64_t v, int s) {
    const uint32_t r = (uint32_t)(v >> (49 - 7 * s)) & (s == 0 ? 0x1FFu : 0x7Fu);
    return __fsub_rn(__uint_as_float(0x4B000000u | r), s == 0 ? 8388864.0f : 8388672.0f);
}

// bf16 pair of digit s of two elements (e0 in the low half).  Digit 0: the
// floats are small integers, so their upper halves are exact bf16.  Digits
// 1..7: the 7-bit raw fields r are placed in the mantissas of bf16 128 (0x4300
// | r = 128 + r, exact) and one bf16x2 FMA subtracts 128 + 64, exact since the
// result r - 64 is a small integer.
__device__ __forceinline__ uint32_t digit_pair(uint64_t v0, uint64_t v1, int s) {
    if (s == 0)
        return __byte_perm(__float_as_uint(digit_f(v0, 0)), __float_as_uint(digit_f(v1, 0)), 0x7632);
    const int sh = 49 - 7 * s;
    const uint32_t r = __byte_perm((uint32_t)(v0 >> sh), (uint32_t)(v1 >> sh), 0x5410);
    const uint32_t w = (r & 0x007F007Fu) | 0x43004300u;          // bf16x2 (128 + r0, 128 + r1)
    uint32_t out;
    asm("fma.rn.bf16x2 %0, %1, %2, %3;" : "=r"(out) : "r"(w), "r"(0x3F803F80u), "r"(0xC340C340u));
    return out;                                                    // (r0 - 64, r1 - 64)
}

}  // namespace slice
}  // namespace mpj
