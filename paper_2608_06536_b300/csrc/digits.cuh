// Six-digit splitting of a 48-bit fixed-point value into BF16 slices with
// FP32 additions (the slicer's alternative to integer digit extraction).
//
// F (|F| <= 2^48) is cut into two exact halves, lo = F mod 2^24 and
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
// reassociate, and plain IEEE additions on the host.
#pragma once

#include <stdint.h>

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
