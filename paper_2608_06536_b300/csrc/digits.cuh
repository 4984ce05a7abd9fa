// Digit splits of a fixed-point value F into BF16 slices, the slicer's ways of
// forming them:
//   digit_values<S>   the S balanced digits of an 8S-bit F (S = 6: 48 bits,
//                     the builds; S = 7: 56 bits, the split adjoint's
//                     seven-slice operands), already scaled to their slices'
//                     values, read off the bytes of F plus a bias (the
//                     default slicer);
//   digits6 + qbf16,  the same digits by per-digit integer arithmetic and
//   digits_n<7>       one exact FP32 conversion each (a second statement of
//                     the split that the host test checks digit_values
//                     against);
//   split48           six digits of a 48-bit F by FP32 additions only
//                     (JK_OPT_SLICER = 1), below.
//
// split48: F is cut into two exact halves, lo = F mod 2^24 and
// hi = F div 2^24, each converted to FP32 exactly and pre-scaled by a power
// of two.  Each digit then costs three FP32 additions: adding and removing
// 1.5 * 2^(k+23) rounds a value to a multiple of 2^k (round to nearest even,
// exact while |value| <= 2^(k+22)), and the difference is the digit, already
// carrying its slice's scale.  The results are
//   v_j = q_j * 2^(-8(j+1)),  F * 2^-48 = v_0 + v_1 + ... + v_5  (exactly),
// with |q_0| <= 256 and |q_j| <= 128 for j >= 1 (balanced digits, ties to
// even), so every v_j has at most 8 significant bits and is an exact BF16
// value: the upper half of its FP32 word.
//
// Host-compilable (for the CPU test of these properties): the additions use
// __fadd_rn on the device, which the compiler may not contract or
// reassociate, and plain IEEE additions on the host; bit casts use the CUDA
// intrinsics on the device and memcpy on the host.
#pragma once

#include <stdint.h>
#if !defined(__CUDA_ARCH__)
#include <math.h>
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
namespace digits {

JK_HD float add_rn(float a, float b) {
#if defined(__CUDA_ARCH__)
    return __fadd_rn(a, b);
#else
    volatile float s = a + b;   // no excess precision, no reassociation
    return s;
#endif
}

// Six balanced base-256 digits of F (|F| <= 2^48) in 32-bit integer
// arithmetic: F = sum_j q_j 2^(8(5-j)), q_1..q_5 in [-128, 127] and
// |q_0| <= 256 (the integer slicer's split of the same value).
JK_HD void digits6(long long F, int q[6]) {
    int lo = static_cast<int>(F & 0xFFFFFFll);        // [0, 2^24)
    int hi = static_cast<int>(F >> 24);               // arithmetic shift
    q[5] = ((lo + 128) & 255) - 128; lo = (lo - q[5]) >> 8;
    q[4] = ((lo + 128) & 255) - 128; lo = (lo - q[4]) >> 8;
    q[3] = ((lo + 128) & 255) - 128; lo = (lo - q[3]) >> 8;
    hi += lo;
    q[2] = ((hi + 128) & 255) - 128; hi = (hi - q[2]) >> 8;
    q[1] = ((hi + 128) & 255) - 128; hi = (hi - q[1]) >> 8;
    q[0] = hi;
}

// S balanced base-256 digits of F (|F| <= 2^(8S)) in 64-bit integer
// arithmetic: F = sum_j q_j 2^(8(S-1-j)), q_1..q_{S-1} in [-128, 127] and
// |q_0| <= 256 (the seven-slice operands' split; digits6 is the same split for
// S = 6 in 32-bit arithmetic).
template <int S>
JK_HD void digits_n(long long F, int q[S]) {
    for (int j = S - 1; j >= 1; j--) {   // a constant trip count: unrolled by the compiler
        q[j] = static_cast<int>(((F + 128) & 255) - 128);
        F = (F - q[j]) >> 8;
    }
    q[0] = static_cast<int>(F);
}

JK_HD float f32_of_bits(uint32_t b) {
#if defined(__CUDA_ARCH__)
    return __uint_as_float(b);
#else
    float f;
    memcpy(&f, &b, sizeof f);
    return f;
#endif
}

JK_HD uint32_t bits_of_f32(float f) {
#if defined(__CUDA_ARCH__)
    return __float_as_uint(f);
#else
    uint32_t b;
    memcpy(&b, &f, sizeof b);
    return b;
#endif
}

// BF16 bits of q * scale for |q| <= 256 and a power-of-two scale: the integer
// is formed exactly by the 1.5*2^23 bias trick and has at most 8 significant
// bits, so after the exact scaling the low half of the FP32 word is zero.
JK_HD uint32_t qbf16(int q, float scale) {
    const float f = (f32_of_bits(static_cast<uint32_t>(0x4B400000 + q)) - 12582912.0f) * scale;
    return bits_of_f32(f) >> 16;
}

// Byte select of two words (CUDA's __byte_perm): result byte i is byte
// (s >> 4i) & 7 of the eight bytes x (0..3), y (4..7).
JK_HD uint32_t byte_perm(uint32_t x, uint32_t y, uint32_t s) {
#if defined(__CUDA_ARCH__)
    return __byte_perm(x, y, s);
#else
    const uint64_t b = (static_cast<uint64_t>(y) << 32) | x;
    uint32_t r = 0;
    for (int i = 0; i < 4; i++) r |= static_cast<uint32_t>((b >> (8 * ((s >> (4 * i)) & 7))) & 0xFF) << (8 * i);
    return r;
#endif
}

// a * b + c rounded once (fused).
JK_HD float fma_rn(float a, float b, float c) {
#if defined(__CUDA_ARCH__)
    return __fmaf_rn(a, b, c);
#else
    return fmaf(a, b, c);
#endif
}

// The S balanced base-256 digits of F (|F| <= 2^(8S)) as the values
// v_j = q_j * 2^(-8(j+1)), j = 0..S-1: the digits of digits6 / digits_n<S>.
// With the bias B = 0x80 in each of the S-1 low bytes, G = F + B holds
// q_j + 128 as its byte S-1-j for j >= 1 (balanced digits in [-128, 127] add
// no carries), and q_0 = G >> 8(S-1).  A byte dropped into the low byte of
// 0x4B400000 (1.5 * 2^23) is the FP32 value 1.5 * 2^23 + byte, so one fused
// multiply-add q_j * sc = f * sc - (1.5 * 2^23 + 128) * sc gives the slice
// value exactly (both products exact, the result an FP32 value; a zero digit
// gives +0).  biased_words forms G once per element; digit_value reads one
// slice's value off it, so a slicer keeps two words per element live, not S
// values.
template <int S>
JK_HD void biased_words(long long F, uint32_t &lo, uint32_t &hi) {
    static_assert(S == 6 || S == 7, "six or seven slices");
    constexpr unsigned long long kBias = S == 6 ? 0x8080808080ull : 0x808080808080ull;
    const unsigned long long G = static_cast<unsigned long long>(F) + kBias;
    lo = static_cast<uint32_t>(G);
    hi = static_cast<uint32_t>(G >> 32);
}

JK_HD float slice_scale(int j) {   // 2^(-8(j+1))
    float sc = 0.00390625f;
    for (int i = 0; i < j; i++) sc *= 0.00390625f;
    return sc;
}

template <int S>
JK_HD float digit_value(uint32_t lo, uint32_t hi, int j) {
    const float sc = slice_scale(j);
    if (j == 0) {
        const int q0 = static_cast<int>(hi) >> (8 * (S - 1) - 32);   // G >> 8(S-1), arithmetic
        return fma_rn(f32_of_bits(0x4B400000u + static_cast<uint32_t>(q0)), sc, -12582912.0f * sc);
    }
    const int b = S - 1 - j;   // byte of G holding q_j + 128
    const uint32_t f = byte_perm(b < 4 ? lo : hi, 0x4B400000u, 0x7650u | static_cast<uint32_t>(b & 3));
    return fma_rn(f32_of_bits(f), sc, -12583040.0f * sc);
}

template <int S>
JK_HD void digit_values(long long F, float v[S]) {
    uint32_t lo, hi;
    biased_words<S>(F, lo, hi);
    for (int j = 0; j < S; j++) v[j] = digit_value<S>(lo, hi, j);   // a constant trip count: unrolled
}

// Two exact BF16 values (FP32 v_lo, v_hi whose low 16 bits are zero) as one
// word, v_lo in the low half.
JK_HD uint32_t pack_bf16x2(float v_lo, float v_hi) {
#if defined(__CUDA_ARCH__)
    uint32_t d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(v_hi), "f"(v_lo));
    return d;
#else
    return (bits_of_f32(v_hi) & 0xFFFF0000u) | (bits_of_f32(v_lo) >> 16);
#endif
}

// x rounded to a multiple of 2^k, M = 1.5 * 2^(k+23); exact for |x| <= 2^(k+22).
JK_HD float round_to(float x, float M) { return add_rn(add_rn(x, M), -M); }

// v[j] = q_j * 2^(-8(j+1)) for j = 0..5 (see above); F = round(x * 2^(48-e)).
JK_HD void split48(long long F, float v[6]) {
    const float lo = static_cast<float>(static_cast<int>(F & 0xFFFFFFll)) * 3.5527136788005009e-15f;   // * 2^-48
    const long long hi_i = F >> 24;                                                                   // |hi| <= 2^24
    // low half: digits 5, 4, 3 (units 2^-48, 2^-40, 2^-32)
    const float r1 = round_to(lo, 1.1444091796875e-05f);     // 1.5 * 2^-17: multiple of 2^-40
    const float r2 = round_to(r1, 0.0029296875f);            // 1.5 * 2^-9:  multiple of 2^-32
    const float r3 = round_to(r2, 0.75f);                    // 1.5 * 2^-1:  multiple of 2^-24 (0 or 2^-24)
    v[5] = add_rn(lo, -r1);
    v[4] = add_rn(r1, -r2);
    v[3] = add_rn(r2, -r3);
    // high half plus the carry: digits 2, 1, 0 (units 2^-24, 2^-16, 2^-8)
    const float y = add_rn(static_cast<float>(static_cast<int>(hi_i)) * 5.9604644775390625e-08f, r3);   // * 2^-24
    const float s1 = round_to(y, 192.0f);                    // 1.5 * 2^7:  multiple of 2^-16
    const float s2 = round_to(s1, 49152.0f);                 // 1.5 * 2^15: multiple of 2^-8
    v[2] = add_rn(y, -s1);
    v[1] = add_rn(s1, -s2);
    v[0] = s2;
}

}  // namespace digits
}  // namespace jk
