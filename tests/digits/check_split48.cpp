// TEST INFRASTRUCTURE: checks both digit splits of csrc/digits.cuh (compiled
// here as host C++) against the properties the slicer relies on, for random
// and edge-case fixed-point values F, |F| <= 2^48:
//   split48: sum_j v_j * 2^48 == F exactly; |q_0| <= 256, |q_j| <= 128
//   (j >= 1) with q_j = v_j * 2^(8(j+1)) an integer; every v_j an exact BF16
//   value (the low 16 bits of its FP32 word are zero).
//   digits6 + qbf16: the same bounds and exact sum for the integer digits,
//   and qbf16(q_j, 2^-8(j+1)) is the BF16 encoding of q_j * 2^-8(j+1).
//   digits_n<7>: the same for seven digits of 56-bit values.
//   digit_values<6> / <7> (the slicer kernels' byte form): every value equal
//   to the integer path's q_j * 2^-8(j+1), bit for bit, and an exact BF16
//   value, so pack_bf16x2 of two of them is the pair of qbf16 words.
// Prints "ok <count>" and exits 0, or the first violation and exits 1.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>

#include "../../paper_2608_06536_b300/csrc/digits.cuh"

// digit_values<S>(F) against the integer digits q of the same F: equal FP32
// words (q_j * 2^-8(j+1) is exact; a zero digit is +0), low halves zero, and
// pack_bf16x2 of slices j and j+1 giving the qbf16 words of q_j and q_j+1.
template <int S>
static int check_values(long long F, const int q[S]) {
    float v[S];
    jk::digits::digit_values<S>(F, v);
    float sc = 0.00390625f;
    for (int j = 0; j < S; j++) {
        const double want = std::ldexp(static_cast<double>(q[j]), -8 * (j + 1));
        uint32_t bits;
        std::memcpy(&bits, &v[j], 4);
        if (static_cast<double>(v[j]) != want || (bits & 0xFFFFu) || bits == 0x80000000u) {
            std::printf("F=%lld: digit_values<%d> slice %d is %a, want %a\n", F, S, j, v[j], want);
            return 1;
        }
        if (j + 1 == S) break;
        const uint32_t w = jk::digits::pack_bf16x2(v[j], v[j + 1]);
        const uint32_t ref = jk::digits::qbf16(q[j], sc) | (jk::digits::qbf16(q[j + 1], sc * 0.00390625f) << 16);
        if (w != ref) {
            std::printf("F=%lld: pack_bf16x2 of slice %d is %08x, want %08x\n", F, j, w, ref);
            return 1;
        }
        sc *= 0.00390625f;
    }
    return 0;
}

static int check(long long F) {
    float v[6];
    jk::digits::split48(F, v);
    __int128 sum = 0;
    for (int j = 0; j < 6; j++) {
        uint32_t bits;
        std::memcpy(&bits, &v[j], 4);
        if (bits & 0xFFFFu) {
            std::printf("F=%lld: slice %d (%a) is not an exact BF16 value\n", F, j, v[j]);
            return 1;
        }
        const double q = std::ldexp(static_cast<double>(v[j]), 8 * (j + 1));
        if (q != std::floor(q) || std::fabs(q) > (j == 0 ? 256.0 : 128.0)) {
            std::printf("F=%lld: digit %d = %.17g out of range\n", F, j, q);
            return 1;
        }
        sum += static_cast<__int128>(static_cast<long long>(q)) << (8 * (5 - j));
    }
    if (sum != static_cast<__int128>(F)) {
        std::printf("F=%lld: digits sum to %lld\n", F, static_cast<long long>(sum));
        return 1;
    }
    // the integer path
    int q[6];
    jk::digits::digits6(F, q);
    __int128 isum = 0;
    float sc = 0.00390625f;
    for (int j = 0; j < 6; j++) {
        if (q[j] > (j == 0 ? 256 : 127) || q[j] < (j == 0 ? -256 : -128)) {
            std::printf("F=%lld: integer digit %d = %d out of range\n", F, j, q[j]);
            return 1;
        }
        const uint32_t w = jk::digits::qbf16(q[j], sc) << 16;
        float back;
        std::memcpy(&back, &w, 4);
        if (static_cast<double>(back) != std::ldexp(static_cast<double>(q[j]), -8 * (j + 1))) {
            std::printf("F=%lld: qbf16(%d) of slice %d is %a\n", F, q[j], j, back);
            return 1;
        }
        isum += static_cast<__int128>(q[j]) << (8 * (5 - j));
        sc *= 0.00390625f;
    }
    if (isum != static_cast<__int128>(F)) {
        std::printf("F=%lld: integer digits sum to %lld\n", F, static_cast<long long>(isum));
        return 1;
    }
    return check_values<6>(F, q);
}

// The seven-digit split of a 56-bit value: exact sum, digit bounds, and
// exact BF16 encodings down to the last slice's scale 2^-56.
static int check7(long long F) {
    int q[7];
    jk::digits::digits_n<7>(F, q);
    __int128 sum = 0;
    float sc = 0.00390625f;
    for (int j = 0; j < 7; j++) {
        if (q[j] > (j == 0 ? 256 : 127) || q[j] < (j == 0 ? -256 : -128)) {
            std::printf("F=%lld: seven-slice digit %d = %d out of range\n", F, j, q[j]);
            return 1;
        }
        const uint32_t w = jk::digits::qbf16(q[j], sc) << 16;
        float back;
        std::memcpy(&back, &w, 4);
        if (static_cast<double>(back) != std::ldexp(static_cast<double>(q[j]), -8 * (j + 1))) {
            std::printf("F=%lld: qbf16(%d) of seven-slice digit %d is %a\n", F, q[j], j, back);
            return 1;
        }
        sum += static_cast<__int128>(q[j]) << (8 * (6 - j));
        sc *= 0.00390625f;
    }
    if (sum != static_cast<__int128>(F)) {
        std::printf("F=%lld: seven digits sum to %lld\n", F, static_cast<long long>(sum));
        return 1;
    }
    return check_values<7>(F, q);
}

int main() {
    const long long T = 1ll << 48;
    long long n = 0;
    // edge cases: the ends of the range, carries out of the low half, ties
    const long long edges[] = {0, 1, -1, 127, 128, 129, -128, -129, 255, 256, 0x8080, 0x808080, 0xFFFFFF,
                               0x1000000, 0x1000080, 0x17FFFFF, T, -T, T - 1, -T + 1, T - 0x800000,
                               (T >> 1) + 0x808080, 0x800000, -0x800000, 0x7F7F7F7F7F7Fll, -0x7F7F7F7F7F7Fll,
                               0x808080808080ll, -0x808080808080ll};
    for (long long F : edges) {
        if (check(F)) return 1;
        n++;
    }
    // every pattern of the top and bottom digit around the half-way points
    for (long long hi = -256; hi <= 256; hi++)
        for (long long lo : {0ll, 0x7Fll, 0x80ll, 0x81ll, 0x7FFFFFll, 0x800000ll, 0x808080ll, 0xFFFFFFll}) {
            const long long F = hi * (1ll << 40) + lo;
            if (F > T || F < -T) continue;
            if (check(F)) return 1;
            n++;
        }
    // random values, uniform and with many tie digits
    std::mt19937_64 rng(12345);
    for (int i = 0; i < 4000000; i++) {
        long long F = static_cast<long long>(rng() % (2 * T + 1)) - T;
        if (i & 1) F = (F & ~0xFFll) | 0x80;                     // a tie in the lowest digit
        if ((i & 7) == 2) F = static_cast<long long>(rng() % 4096) - 2048;   // small magnitudes
        if (check(F)) return 1;
        n++;
    }
    // the seven-digit split over 56-bit values
    const long long T7 = 1ll << 56;
    for (long long F : {0ll, 1ll, -1ll, 128ll, -128ll, 0x80ll, T7, -T7, T7 - 1, -T7 + 1, 0x80808080808080ll,
                        -0x80808080808080ll, 0x7F7F7F7F7F7F7Fll, (T7 >> 1) + 0x808080ll}) {
        if (check7(F)) return 1;
        n++;
    }
    for (int i = 0; i < 2000000; i++) {
        long long F = static_cast<long long>(rng() % (2 * static_cast<unsigned long long>(T7) + 1)) - T7;
        if (i & 1) F = (F & ~0xFFll) | 0x80;
        if ((i & 7) == 2) F = static_cast<long long>(rng() % 4096) - 2048;
        if (check7(F)) return 1;
        n++;
    }
    std::printf("ok %lld\n", n);
    return 0;
}
