// Digit splits of a fixed-point value F into BF16 slices, the slicer's ways of
// forming them:
//   digits6 + qbf16   six digits of a 48-bit F (|F| <= 2^48) in 32-bit integer
//                     arithmetic, then one exact FP32 conversion per digit
//                     (the default slicer);
//   digits_n<7>       seven digits of a 56-bit F in 64-bit arithmetic (the
//                     seven-slice operands of the split adjoint);
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
