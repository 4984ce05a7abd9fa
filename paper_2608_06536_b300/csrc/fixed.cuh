// Fixed-point conversions of the split-precision GEMM, in integer arithmetic
// only (B300's FP64 pipe runs at 1/60 of the FP32 rate):
//   exponent_of_max     the scale 2^e of a group of values (max|x| < 2^e);
//   to_fixed(48)        x under that scale as a 48-bit (or nbits-bit) signed
//                       integer;
//   i64/i128_to_f64_scaled
//                       an integer accumulator times 2^e2, rounded once to
//                       the nearest FP64 value (ties to even).
//
// Host-compilable, so that a CPU test checks this very code against exact
// integer and rational arithmetic; the device build uses the CUDA intrinsics
// for the bit casts and the leading-zero count.
#pragma once

#include <stdint.h>
#if !defined(__CUDA_ARCH__)
#include <string.h>
#endif

#if !defined(JK_HD)
#if defined(__CUDACC__)
#define JK_HD __host__ __device__ __forceinline__
#else
#define JK_HD static inline
#endif
#endif

namespace jk {
namespace fixed {

JK_HD uint64_t f64_bits(double x) {
#if defined(__CUDA_ARCH__)
    return static_cast<uint64_t>(__double_as_longlong(x));
#else
    uint64_t b;
    memcpy(&b, &x, sizeof b);
    return b;
#endif
}

JK_HD double bits_f64(uint64_t b) {
#if defined(__CUDA_ARCH__)
    return __longlong_as_double(static_cast<long long>(b));
#else
    double x;
    memcpy(&x, &b, sizeof x);
    return x;
#endif
}

// Leading zero bits of x != 0.
JK_HD int clz64(uint64_t x) {
#if defined(__CUDA_ARCH__)
    return __clzll(static_cast<long long>(x));
#else
    return __builtin_clzll(x);
#endif
}

// Exponent e with max|x| < 2^e <= 2 max|x|, from the bits of max|x| (sign
// cleared).  Zero and subnormal maxima give -1000, so an all-zero group never
// sets the scale when partial sums are aligned.
JK_HD int exponent_of_max(uint64_t maxbits) {
    const int ex = static_cast<int>((maxbits >> 52) & 0x7FF);
    return ex == 0 ? -1000 : ex - 1022;
}

// F = x * 2^(nbits - e) rounded to the nearest integer (ties away from zero),
// so |F| <= 2^nbits when |x| < 2^e (nbits <= 60).  Zero and subnormal inputs
// give 0.
JK_HD long long to_fixed(double x, int e, int nbits) {
    const uint64_t bits = f64_bits(x);
    const int ex = static_cast<int>((bits >> 52) & 0x7FF);
    if (ex == 0) return 0;
    const uint64_t m = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int r = 1075 - nbits + e - ex;   // right shift of the 53-bit significand; >= 53 - nbits when |x| < 2^e
    long long F;
    if (r <= 0) F = static_cast<long long>(m << (-r));
    else if (r >= 64) F = 0;
    else F = static_cast<long long>((m + (1ull << (r - 1))) >> r);
    return (bits >> 63) ? -F : F;
}

// The 48-bit form used by the six-slice operands.
JK_HD long long to_fixed48(double x, int e) { return to_fixed(x, e, 48); }

// The FP64 value nearest (ties to even) to (top + s) * 2^(x2 - 63), where top
// has its leading one at bit 63 and 0 <= s < 1 is nonzero exactly when
// `sticky`; negated when `neg`.  The result must be a normal double.
JK_HD double round_top(bool neg, uint64_t top, bool sticky, int x2) {
    uint64_t mant = top >> 11;                  // 53 bits including the leading one
    const uint64_t rem = top & 0x7FFull;
    if (rem > 0x400ull || (rem == 0x400ull && (sticky || (mant & 1ull)))) mant++;
    if (mant >> 53) {
        mant >>= 1;
        x2++;
    }
    return bits_f64((neg ? 0x8000000000000000ull : 0ull) | (static_cast<uint64_t>(x2 + 1023) << 52) |
                    (mant & 0xFFFFFFFFFFFFFull));
}

// v * 2^e2 rounded once to FP64 (ties to even); the result must be a normal
// double (true for every value the GEMM forms).  Branch-free: the GEMM's
// epilogue converts whole tiles with it.  With the leading one of |v| moved to
// bit 63 (top), the 53 kept bits are top >> 11 and the 11 dropped ones decide
// the rounding; adding the rounded significand (implicit bit included) to the
// exponent field one below the leading bit's carries a rounding overflow
// (2^53) into the exponent by itself.
JK_HD double i64_to_f64_scaled(long long v, int e2) {
    const uint64_t u = static_cast<uint64_t>(v);
    const uint64_t a = v < 0 ? 0ull - u : u;
    const int lz = clz64(a | 1ull);
    const uint64_t top = a << lz;
    const uint64_t mant = top >> 11;
    const uint64_t rest = top & 0x7FFull;
    const uint64_t up = (rest + (mant & 1ull)) > 0x400ull ? 1ull : 0ull;
    const uint64_t bits = (u & 0x8000000000000000ull) +
                          (static_cast<uint64_t>(e2 + 63 - lz + 1022) << 52) + mant + up;
    return a == 0 ? 0.0 : bits_f64(bits);
}

// The same for a 128-bit accumulator (the exactly aligned sum of split-K
// partials): one rounding, the bits below the leading 64 folded into `sticky`.
JK_HD double i128_to_f64_scaled(__int128 v, int e2) {
    if (v == 0) return 0.0;
    const bool neg = v < 0;
    const unsigned __int128 a = neg ? static_cast<unsigned __int128>(0) - static_cast<unsigned __int128>(v)
                                    : static_cast<unsigned __int128>(v);
    const uint64_t hi = static_cast<uint64_t>(a >> 64), lo = static_cast<uint64_t>(a);
    if (hi == 0) {
        const int lz = clz64(lo);
        return round_top(neg, lo << lz, false, e2 + 63 - lz);
    }
    const int lz = clz64(hi);
    const uint64_t top = lz ? (hi << lz) | (lo >> (64 - lz)) : hi;
    const uint64_t rest = lz ? lo << lz : lo;
    return round_top(neg, top, rest != 0, e2 + 127 - lz);
}

}  // namespace fixed
}  // namespace jk
