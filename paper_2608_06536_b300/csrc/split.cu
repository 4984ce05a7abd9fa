// Split-precision engine: FP64-accurate J/K from BF16 tensor-core products.
//
// Every dense contraction of the build (panels T = L Z and the rank update
// K_s = sum_P T_X T_Y^T) is computed as an error-free-split product:
//
//  * Slicing.  Each operand row r is scaled by 2^-e_r (e_r from the row's
//    largest magnitude) and rounded once to a 48-bit fixed-point integer F,
//    which is cut into six signed base-256 digits q_1..q_6 (|q_1| <= 256,
//    |q_j| <= 128).  Slice j stores q_j * 2^(-8j) as a BF16 value -- exact,
//    since every q_j has at most 8 significant bits.  This is done with
//    integer arithmetic only (B300 has very little FP64 throughput).
//  * Products.  The 21 slice pairs (a, b) with a + b <= 7 are multiplied on
//    tcgen05 tensor cores (kind::f16, FP32 accumulate in tensor memory).
//    Pairs on the same diagonal d = a + b - 2 share a scale 2^-(8d+16) and
//    one TMEM accumulator per diagonal (six of 80 columns, laid out by d), so
//    the pairs (a, b..b+m) of one A slice hit adjacent accumulators and run
//    as ONE MMA with N = 80(m+1): 10 MMAs per K-step instead of 21.  Over a
//    window of 128 reduction elements every partial sum of diagonals
//    d = 0..3 is an integer below 2^24 times its scale, so the FP32
//    accumulation is exact whatever the tensor core's rounding mode;
//    diagonals 4 and 5 (relative size <= 2^-32) accumulate over a whole tile
//    (<= 2048 elements) with truncation error below 2^-45.  The window
//    boundaries of the exact accumulators are staggered so their drains do
//    not coincide; the epilogue zeroes each drained accumulator.
//  * Recombination.  After each window an accumulator is
//    read from TMEM, converted to 32-bit integers in their own units and
//    shifted into a per-element int64 fixed-point accumulator with 48
//    fraction bits (exact for d <= 3).  Split-K partials are summed
//    in 128-bit integers; the only rounding to FP64 happens once per output.
//
// The representation error is below 2^-48 of each row's scale, which keeps the
// built J and K within 1e-10 absolute of the FP64 oracle on the benchmark
// workloads (see the parity tests).
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <type_traits>
#include <vector>

#include "digits.cuh"
#include "fixed.cuh"
#include "packed.cuh"
#include "jk_internal.h"
#include "tc.cuh"

namespace jk {
namespace oz {

constexpr int BM = 128;             // rows of A per tile (TMEM lanes)
constexpr int KB = 16;              // reduction elements per pipeline stage (one MMA K-step)
constexpr int KBPC = 8;             // K-blocks of a 128-element exact window
constexpr int WPERIOD = 2 * KBPC;   // the window pattern repeats every 16 K-blocks
constexpr int SUPER = 2048;         // reduction elements per int64 partial
constexpr int NSTAGE = 3;
constexpr int THREADS = 320;        // producer warp, MMA warp, 8 epilogue warps
constexpr int MAXMMA = 12;          // most merged MMAs per K-block of any configuration

// A slice configuration.  Every operand element is an S-digit fixed-point
// value (8S bits under its row's scale), cut into S BF16 slices of balanced
// 8-bit digits; the slice pairs (a, b) with a + b < S are multiplied, and the
// pairs on one diagonal d = a + b share a scale and one TMEM accumulator of BN
// columns (S accumulators, laid out by d).  Diagonals d < NEXACT accumulate in
// exact windows (128 or 256 reduction elements: every partial sum an integer
// below 2^24 in its unit) and are drained into an int64 fixed point with FRAC
// fraction bits; the two lowest diagonals, whose error is below the
// representation's, accumulate over the whole tile.
//   Cfg<6, 80>  48-bit operands, 21 pairs, 128 x 80 tiles (the default);
//   Cfg<6, 64>  the same with 128 x 64 tiles (a tuning candidate);
//   Cfg<7, 64>  56-bit operands, 28 pairs, 128 x 64 tiles (the split adjoint:
//               its chained products need the extra bits).
template <int S_, int BN_>
struct Cfg {
    static constexpr int S = S_;
    static constexpr int BN = BN_;
    static constexpr int NACC = S;
    static constexpr int NEXACT = S - 2;
    static constexpr int NPAIRS = S * (S + 1) / 2;
    static constexpr int BITS = 8 * S;
    // int64 accumulator: |sum| < K * 2^FRAC for K <= SUPER elements stays in range
    static constexpr int FRAC = S == 6 ? 48 : 51;
    static constexpr int A_BYTES = S * BM * 32;
    static constexpr int B_BYTES = S * BN * 32;
    static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    // Output staging: each epilogue warp owns 32 rows x OUT_COLS columns of
    // 64-bit words, kept as 32 x 8 blocks in the 64-byte swizzled layout of a
    // TMA store.
    static constexpr int OUT_COLS = BN / 2;
    static constexpr int OUT_BLK = 8;
    static constexpr int OUT_WARP_BYTES = 32 * OUT_COLS * 8;
    static constexpr int OUT_BYTES = 8 * OUT_WARP_BYTES;
    static constexpr int SMEM_BYTES = NSTAGE * STAGE_BYTES + OUT_BYTES + 1024 /*align slack*/ + 256 /*barriers*/;
    static_assert(S * BN <= 512, "the accumulators fit tensor memory");
    static_assert(BN % 16 == 0 && OUT_COLS % OUT_BLK == 0, "tile width");
    static_assert(NEXACT >= 1 && NEXACT <= 5, "window schedule");
    static_assert(FRAC >= 16 + 8 * (NEXACT - 1) && FRAC + 11 <= 62, "exact drains and the int64 range");
    static_assert(SMEM_BYTES <= 227 * 1024, "shared memory");
};
using Cfg6 = Cfg<6, 80>;
using Cfg6n = Cfg<6, 64>;
using Cfg7 = Cfg<7, 64>;
constexpr int OUT_BLK = 8;

// ---------------------------------------------------------------------------
// Integer helpers
// ---------------------------------------------------------------------------

using fixed::exponent_of_max;
using fixed::i128_to_f64_scaled;
using fixed::i64_to_f64_scaled;
using fixed::to_fixed;

// ---------------------------------------------------------------------------
// Slicers
// ---------------------------------------------------------------------------

// Source addressing: element (row r, reduction index kk) is at
// p + (r / rin)*sr + (r % rin)*sri + (kk / kin)*sko + (kk % kin)*ski
// (two-level row and reduction indices, e.g. rows (P, i) or K = (P, lam)).
struct Src {
    const double *p;
    long long sr, sko, ski;
    int kin;
    int rin = 1;
    long long sri = 0;
};

__device__ __forceinline__ const double *src_row(const Src &s, int r) {
    const int ro = r / s.rin, ri = r - ro * s.rin;
    return s.p + static_cast<long long>(ro) * s.sr + static_cast<long long>(ri) * s.sri;
}

// e[g * gridDim.y + z] for row groups g of `rpe` rows and super-chunks z of
// the reduction index: max|x| over the group's rows and kk in
// [z*SUPER, (z+1)*SUPER).  Each thread walks kk = k0 + tid, + 256, ... keeping
// (ko, ki) incrementally, so the hot loop has no integer division.
__global__ void __launch_bounds__(256) expo_kernel(Src src, int rows, int K, int rpe, int *e) {
    __shared__ unsigned long long red[8];
    const int g = blockIdx.x, z = blockIdx.y;
    const int r0 = g * rpe, r1 = min(rows, r0 + rpe);
    const int k0 = z * SUPER, k1 = min(K, k0 + SUPER);
    const int step_o = 256 / src.kin, step_i = 256 % src.kin;
    unsigned long long mx = 0;
    for (int r = r0; r < r1; r++) {
        const double *row = src_row(src, r);
        int ko = (k0 + threadIdx.x) / src.kin, ki = k0 + threadIdx.x - ko * src.kin;
        for (int kk = k0 + threadIdx.x; kk < k1; kk += 256) {
            const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(
                                             row[static_cast<long long>(ko) * src.sko +
                                                 static_cast<long long>(ki) * src.ski])) &
                                         0x7FFFFFFFFFFFFFFFull;
            mx = b > mx ? b : mx;
            ko += step_o;
            ki += step_i;
            if (ki >= src.kin) { ki -= src.kin; ko++; }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_down_sync(0xffffffffu, mx, o);
        mx = y > mx ? y : mx;
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long m = red[0];
        for (int i = 1; i < 8; i++) m = red[i] > m ? red[i] : m;
        e[g * gridDim.y + z] = exponent_of_max(m);
    }
}

using digits::digits6;
using digits::qbf16;

// The S digits of an element under its scale: the 32-bit split for six
// slices, the 64-bit one for seven.
template <int S>
__device__ __forceinline__ void element_digits(double x, int e, int q[S]) {
    const long long F = to_fixed(x, e, 8 * S);
    if constexpr (S == 6) digits6(F, q);
    else digits::digits_n<S>(F, q);
}

// Vector slicer: 4 consecutive reduction elements per thread.  Requires
// src.ski == 1, src.kin % 4 == 0, K % 4 == 0 and 16-byte aligned pairs
// (checked on the host).
template <int S>
__global__ void __launch_bounds__(256) slice4_kernel(Src src, int rows, int K, int Kpad, const int *e, int rpe,
                                                     int nsc, uint2 *out, long long sstride4) {
    const int kk = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (kk >= Kpad) return;
    long long koff = 0;
    if (kk < K) {
        const int ko = kk / src.kin, ki = kk - ko * src.kin;
        koff = static_cast<long long>(ko) * src.sko + ki;
    }
    for (int rb = blockIdx.y * 8; rb < rows; rb += gridDim.y * 8) {
        const int rend = min(rows, rb + 8);
        for (int r = rb; r < rend; r++) {
            int q[4][S];
            if (kk < K) {
                const double2 *p2 = reinterpret_cast<const double2 *>(src_row(src, r) + koff);
                const double2 a = p2[0], b = p2[1];
                const int er = e[(r / rpe) * nsc + kk / SUPER];
                element_digits<S>(a.x, er, q[0]);
                element_digits<S>(a.y, er, q[1]);
                element_digits<S>(b.x, er, q[2]);
                element_digits<S>(b.y, er, q[3]);
            } else {
#pragma unroll
                for (int i = 0; i < 4; i++)
#pragma unroll
                    for (int j = 0; j < S; j++) q[i][j] = 0;
            }
            const long long o = (static_cast<long long>(r) * Kpad + kk) >> 2;
            float sc = 0.00390625f;
#pragma unroll
            for (int j = 0; j < S; j++) {
                uint2 w;
                w.x = qbf16(q[0][j], sc) | (qbf16(q[1][j], sc) << 16);
                w.y = qbf16(q[2][j], sc) | (qbf16(q[3][j], sc) << 16);
                out[j * sstride4 + o] = w;
                sc *= 0.00390625f;
            }
        }
    }
}

// Vector slicer with the digits formed by FP32 additions (digits.cuh, six
// slices): the same layout and requirements as slice4_kernel; the slices are
// an equally exact split of the same 48-bit values (digits may differ from the
// integer path only where a digit rounds a tie, to even here).  The BF16 words
// are the upper halves of the FP32 digits, paired with one byte permute.
__global__ void __launch_bounds__(256) slice4f_kernel(Src src, int rows, int K, int Kpad, const int *e, int rpe,
                                                      int nsc, uint2 *out, long long sstride4) {
    constexpr int S = 6;
    const int kk = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (kk >= Kpad) return;
    long long koff = 0;
    if (kk < K) {
        const int ko = kk / src.kin, ki = kk - ko * src.kin;
        koff = static_cast<long long>(ko) * src.sko + ki;
    }
    for (int rb = blockIdx.y * 8; rb < rows; rb += gridDim.y * 8) {
        const int rend = min(rows, rb + 8);
        for (int r = rb; r < rend; r++) {
            float v[4][S];
            if (kk < K) {
                const double2 *p2 = reinterpret_cast<const double2 *>(src_row(src, r) + koff);
                const double2 a = p2[0], b = p2[1];
                const int er = e[(r / rpe) * nsc + kk / SUPER];
                digits::split48(to_fixed(a.x, er, 48), v[0]);
                digits::split48(to_fixed(a.y, er, 48), v[1]);
                digits::split48(to_fixed(b.x, er, 48), v[2]);
                digits::split48(to_fixed(b.y, er, 48), v[3]);
            } else {
#pragma unroll
                for (int i = 0; i < 4; i++)
#pragma unroll
                    for (int j = 0; j < S; j++) v[i][j] = 0.0f;
            }
            const long long o = (static_cast<long long>(r) * Kpad + kk) >> 2;
#pragma unroll
            for (int j = 0; j < S; j++) {
                uint2 w;
                w.x = __byte_perm(__float_as_uint(v[0][j]), __float_as_uint(v[1][j]), 0x7632);
                w.y = __byte_perm(__float_as_uint(v[2][j]), __float_as_uint(v[3][j]), 0x7632);
                out[j * sstride4 + o] = w;
            }
        }
    }
}

// e[g] for groups that are contiguous runs of `len` doubles starting at p + g*len
// (len even, p 16-byte aligned): 16-byte loads.
__global__ void __launch_bounds__(256) expo_flat_kernel(const double *p, long long len, int *e) {
    __shared__ unsigned long long red[8];
    const double2 *q = reinterpret_cast<const double2 *>(p + blockIdx.x * len);
    unsigned long long mx = 0;
    for (long long t = threadIdx.x; t < len / 2; t += 256) {
        const double2 v = q[t];
        const unsigned long long a = static_cast<unsigned long long>(__double_as_longlong(v.x)) & 0x7FFFFFFFFFFFFFFFull;
        const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(v.y)) & 0x7FFFFFFFFFFFFFFFull;
        mx = a > mx ? a : mx;
        mx = b > mx ? b : mx;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_down_sync(0xffffffffu, mx, o);
        mx = y > mx ? y : mx;
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long m = red[0];
        for (int i = 1; i < 8; i++) m = red[i] > m ? red[i] : m;
        e[blockIdx.x] = exponent_of_max(m);
    }
}

constexpr int SLICE_ROWS = 8;   // rows per block of the slicer

// out[j][r][kk] = q_j(r, kk) * 2^(-8(j+1)) for j = 0..S-1 (bf16), zero for kk >= K.
template <int S>
__global__ void __launch_bounds__(256) slice_kernel(Src src, int rows, int K, int Kpad, const int *e,
                                                    int rpe, int nsc, unsigned short *out, long long sstride) {
    const int kk = blockIdx.x * blockDim.x + threadIdx.x;
    if (kk >= Kpad) return;
    long long koff = 0;
    if (kk < K) {
        const int ko = kk / src.kin, ki = kk - ko * src.kin;
        koff = static_cast<long long>(ko) * src.sko + static_cast<long long>(ki) * src.ski;
    }
    for (int rb = blockIdx.y * SLICE_ROWS; rb < rows; rb += gridDim.y * SLICE_ROWS) {
        const int rend = min(rows, rb + SLICE_ROWS);
        for (int r = rb; r < rend; r++) {
            int q[S];
#pragma unroll
            for (int j = 0; j < S; j++) q[j] = 0;
            if (kk < K) element_digits<S>(src_row(src, r)[koff], e[(r / rpe) * nsc + kk / SUPER], q);
            const long long o = static_cast<long long>(r) * Kpad + kk;
            float sc = 0.00390625f;
#pragma unroll
            for (int j = 0; j < S; j++) {
                out[j * sstride + o] = static_cast<unsigned short>(qbf16(q[j], sc));
                sc *= 0.00390625f;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Grouped slicing: many operands in one launch
// ---------------------------------------------------------------------------
// A batched build slices the factor chunk and both panel operands of every
// density of every molecule in a wave; one exponent launch and one slicer
// launch take them all, their jobs carried in the parameter space (no device
// table to upload, so the launch stays capturable in a CUDA graph).  Each job
// is one operand as slice_operand would slice it; block b of a launch belongs
// to the job whose block range [b0, b0 + blocks) holds it.
struct SliceJob {
    Src src;
    int *e;                // exponents: written by the exponent launch, read by the slicer
    void *out;             // S planes, rows x Kpad each
    long long sstride;     // plane stride in units of the output words (uint2 when vec, else ushort)
    int rows, K, Kpad, rpe, nsc;
    int vec;               // 4-element vector path (alignment checked on the host)
    int flat;              // exponent groups are contiguous runs of rpe * K doubles
    int eb0, sb0;          // first block of this job in the exponent and the slicer launch
    int nbx, nby;          // slicer blocks along K (x) and rows (y)
};
constexpr int MAXJOB = 200;
struct SliceGroup {
    SliceJob j[MAXJOB];
    int njob;
};

__device__ __forceinline__ int job_of_block(const SliceGroup &g, int b, bool expo) {
    int lo = 0, hi = g.njob - 1;
    while (lo < hi) {   // the last job whose first block is <= b
        const int mid = (lo + hi + 1) >> 1;
        if ((expo ? g.j[mid].eb0 : g.j[mid].sb0) <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// The exponents of every job: expo_kernel's (or expo_flat_kernel's) work for
// the job's row group g and super-chunk z.
__global__ void __launch_bounds__(256) expo_group_kernel(const __grid_constant__ SliceGroup g) {
    __shared__ unsigned long long red[8];
    const int ji = job_of_block(g, blockIdx.x, true);
    const SliceJob &jb = g.j[ji];
    const int lb = blockIdx.x - jb.eb0;
    unsigned long long mx = 0;
    int slot;
    if (jb.flat) {
        const long long len = static_cast<long long>(jb.rpe) * jb.K;
        const double2 *q = reinterpret_cast<const double2 *>(jb.src.p + lb * len);
        for (long long t = threadIdx.x; t < len / 2; t += 256) {
            const double2 v = q[t];
            const unsigned long long a = static_cast<unsigned long long>(__double_as_longlong(v.x)) & 0x7FFFFFFFFFFFFFFFull;
            const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(v.y)) & 0x7FFFFFFFFFFFFFFFull;
            mx = a > mx ? a : mx;
            mx = b > mx ? b : mx;
        }
        slot = lb;
    } else {
        const Src src = jb.src;
        const int gi = lb / jb.nsc, z = lb - gi * jb.nsc;
        const int r0 = gi * jb.rpe, r1 = min(jb.rows, r0 + jb.rpe);
        const int k0 = z * SUPER, k1 = min(jb.K, k0 + SUPER);
        const int step_o = 256 / src.kin, step_i = 256 % src.kin;
        for (int r = r0; r < r1; r++) {
            const double *row = src_row(src, r);
            int ko = (k0 + threadIdx.x) / src.kin, ki = k0 + threadIdx.x - ko * src.kin;
            for (int kk = k0 + threadIdx.x; kk < k1; kk += 256) {
                const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(
                                                 row[static_cast<long long>(ko) * src.sko +
                                                     static_cast<long long>(ki) * src.ski])) &
                                             0x7FFFFFFFFFFFFFFFull;
                mx = b > mx ? b : mx;
                ko += step_o;
                ki += step_i;
                if (ki >= src.kin) { ki -= src.kin; ko++; }
            }
        }
        slot = gi * jb.nsc + z;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_down_sync(0xffffffffu, mx, o);
        mx = y > mx ? y : mx;
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long m = red[0];
        for (int i = 1; i < 8; i++) m = red[i] > m ? red[i] : m;
        jb.e[slot] = exponent_of_max(m);
    }
}

// The slices of every job: slice4_kernel's work (vector jobs) or
// slice_kernel's (the others) for the job's block (bx, by).
template <int S>
__global__ void __launch_bounds__(256) slice_group_kernel(const __grid_constant__ SliceGroup g) {
    const int ji = job_of_block(g, blockIdx.x, false);
    const SliceJob &jb = g.j[ji];
    const int lb = blockIdx.x - jb.sb0;
    const int by = lb / jb.nbx, bx = lb - by * jb.nbx;
    const Src src = jb.src;
    const int rows = jb.rows, K = jb.K, Kpad = jb.Kpad, rpe = jb.rpe, nsc = jb.nsc;
    const int *e = jb.e;
    if (jb.vec) {
        const int kk = 4 * (bx * 256 + threadIdx.x);
        if (kk >= Kpad) return;
        uint2 *out = static_cast<uint2 *>(jb.out);
        long long koff = 0;
        if (kk < K) {
            const int ko = kk / src.kin, ki = kk - ko * src.kin;
            koff = static_cast<long long>(ko) * src.sko + ki;
        }
        for (int rb = by * 8; rb < rows; rb += jb.nby * 8) {
            const int rend = min(rows, rb + 8);
            for (int r = rb; r < rend; r++) {
                int q[4][S];
                if (kk < K) {
                    const double2 *p2 = reinterpret_cast<const double2 *>(src_row(src, r) + koff);
                    const double2 a = p2[0], b = p2[1];
                    const int er = e[(r / rpe) * nsc + kk / SUPER];
                    element_digits<S>(a.x, er, q[0]);
                    element_digits<S>(a.y, er, q[1]);
                    element_digits<S>(b.x, er, q[2]);
                    element_digits<S>(b.y, er, q[3]);
                } else {
#pragma unroll
                    for (int i = 0; i < 4; i++)
#pragma unroll
                        for (int j = 0; j < S; j++) q[i][j] = 0;
                }
                const long long o = (static_cast<long long>(r) * Kpad + kk) >> 2;
                float sc = 0.00390625f;
#pragma unroll
                for (int j = 0; j < S; j++) {
                    uint2 w;
                    w.x = qbf16(q[0][j], sc) | (qbf16(q[1][j], sc) << 16);
                    w.y = qbf16(q[2][j], sc) | (qbf16(q[3][j], sc) << 16);
                    out[j * jb.sstride + o] = w;
                    sc *= 0.00390625f;
                }
            }
        }
    } else {
        const int kk = bx * 256 + threadIdx.x;
        if (kk >= Kpad) return;
        unsigned short *out = static_cast<unsigned short *>(jb.out);
        long long koff = 0;
        if (kk < K) {
            const int ko = kk / src.kin, ki = kk - ko * src.kin;
            koff = static_cast<long long>(ko) * src.sko + static_cast<long long>(ki) * src.ski;
        }
        for (int rb = by * SLICE_ROWS; rb < rows; rb += jb.nby * SLICE_ROWS) {
            const int rend = min(rows, rb + SLICE_ROWS);
            for (int r = rb; r < rend; r++) {
                int q[S];
#pragma unroll
                for (int j = 0; j < S; j++) q[j] = 0;
                if (kk < K) element_digits<S>(src_row(src, r)[koff], e[(r / rpe) * nsc + kk / SUPER], q);
                const long long o = static_cast<long long>(r) * Kpad + kk;
                float sc = 0.00390625f;
#pragma unroll
                for (int j = 0; j < S; j++) {
                    out[j * jb.sstride + o] = static_cast<unsigned short>(qbf16(q[j], sc));
                    sc *= 0.00390625f;
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// The tcgen05 sliced GEMM:  C[m][n] = sum_k A[m][k] B[n][k]
// ---------------------------------------------------------------------------
struct OzArgs {
    int M, N, K, nsuper;
    const int *eA;
    int a_rpe;
    const int *eB;
    int b_rpe;
    double *C;            // nsuper == 1: FP64 result, row stride ldc
    long long ldc;
    long long *P;         // nsuper > 1: int64 partial z at P + z*pz, rows of ldp words
    long long pz;
    long long ldp;
    int use_tma_store;    // output written through tmC (row stride even, 16-byte aligned)
    int *err;             // device error word (JK_ERR_TIMEOUT on a stalled pipeline)
};

// Accumulator windows.  Exactness bounds (|q_0| <= 256, |q_j| <= 128): one
// reduction element adds at most 2^16 units to diagonals 0 and 1, at most
// 2^16 + 2^14 to diagonal 2, 3 * 2^15 to diagonal 3 and 7 * 2^14 to diagonal
// 4, so windows of 256 (d = 0, 1) and 128 (d = 2, 3, 4) elements keep every
// partial sum below 2^24.  Window starts are spread over the even K-blocks of
// the 16-block period (d0: 0; d1: 8; d2: 2, 10; d3: 6, 14; d4: 4, 12) so that
// drains do not coincide and no two consecutive K-blocks both start one.
__host__ __device__ constexpr int wper(int d) { return d < 2 ? WPERIOD : KBPC; }
__host__ __device__ constexpr int woff(int d) { return d == 0 ? 0 : d == 1 ? KBPC : d == 2 ? 2 : d == 3 ? 6 : 4; }
__host__ __device__ constexpr bool ws_r(int d, int r) { return (r - woff(d) + WPERIOD) % wper(d) == 0; }
template <class C>
__host__ __device__ constexpr unsigned ws_mask(int r) {
    unsigned m = 0;
    for (int d = 0; d < C::NEXACT; d++)
        if (ws_r(d, r)) m |= 1u << d;
    return m;
}
template <class C>
__host__ __device__ constexpr unsigned we_mask(int r) { return ws_mask<C>((r + 1) % WPERIOD); }
// The window ends of K-block residue r, at run time.
template <class C>
__device__ __forceinline__ unsigned we_mask_rt(int r) {
    const int r1 = (r + 1) & (WPERIOD - 1);
    unsigned m = 0;
#pragma unroll
    for (int d = 0; d < C::NEXACT; d++)
        if (((r1 - woff(d)) & (wper(d) - 1)) == 0) m |= 1u << d;
    return m;
}

// The merged MMAs of one K-block: A slice a times B slices b0..b0+nb-1 into
// accumulators a+b0 .. a+b0+nb-1 (adjacent TMEM column blocks, since B's
// slice planes are adjacent in shared memory): one tcgen05.mma with
// N = nb * BN <= 256.
struct MmaList {
    int n;
    int a[MAXMMA], b0[MAXMMA], nb[MAXMMA];
};
template <class C>
__host__ __device__ constexpr MmaList make_mma_list() {
    MmaList L{};
    if (C::S == 6 && C::BN == 80) {
        // 21 pairs as 10 MMAs: those touching only the tile-long accumulators
        // 4, 5 first, the one touching accumulator 0 last (the accumulator
        // whose window just restarted is needed as late as possible)
        const int a[10] = {0, 1, 2, 4, 5, 3, 2, 1, 0, 0};
        const int b0[10] = {4, 3, 3, 0, 0, 0, 0, 0, 3, 0};
        const int nb[10] = {2, 2, 1, 2, 1, 3, 3, 3, 1, 3};
        L.n = 10;
        for (int i = 0; i < 10; i++) {
            L.a[i] = a[i];
            L.b0[i] = b0[i];
            L.nb[i] = nb[i];
        }
        return L;
    }
    // otherwise: each A slice's B slices in runs of at most 256 / BN, ordered
    // with the runs touching only the tile-long accumulators first, then by
    // decreasing lowest diagonal
    const int W = 256 / C::BN;
    int a[MAXMMA] = {}, b0[MAXMMA] = {}, nb[MAXMMA] = {}, key[MAXMMA] = {};
    int c = 0;
    for (int aa = 0; aa < C::S; aa++)
        for (int lo = 0; lo < C::S - aa; lo += W) {
            a[c] = aa;
            b0[c] = lo;
            nb[c] = C::S - aa - lo < W ? C::S - aa - lo : W;
            key[c] = (aa + lo >= C::NEXACT ? 1000 : 0) + 10 * (aa + lo) - aa;   // larger first
            c++;
        }
    bool used[MAXMMA] = {};
    for (int i = 0; i < c; i++) {
        int best = -1;
        for (int j = 0; j < c; j++)
            if (!used[j] && (best < 0 || key[j] > key[best])) best = j;
        used[best] = true;
        L.a[i] = a[best];
        L.b0[i] = b0[best];
        L.nb[i] = nb[best];
    }
    L.n = c;
    return L;
}

// Issue order per window residue r: the MMAs that touch an accumulator whose
// window restarts at r go last (each group keeps the list's order), so the
// MMA thread has the most work queued before it must wait for that
// accumulator's drain.
struct MmaOrder {
    int v[WPERIOD][MAXMMA];
};
template <class C>
__host__ __device__ constexpr MmaOrder make_mma_order(const MmaList &L) {
    MmaOrder t{};
    for (int r = 0; r < WPERIOD; r++) {
        const unsigned m = ws_mask<C>(r);
        int c = 0;
        for (int pass = 0; pass < 2; pass++)
            for (int j = 0; j < L.n; j++) {
                const unsigned mj = ((1u << L.nb[j]) - 1u) << (L.a[j] + L.b0[j]);
                if (((mj & m) != 0) == (pass == 1)) t.v[r][c++] = j;
            }
    }
    return t;
}

template <class C>
struct Tabs {
    static constexpr MmaList list = make_mma_list<C>();
    static constexpr MmaOrder order = make_mma_order<C>(list);
};

template <class C>
__host__ __device__ constexpr bool mma_list_covers_pairs() {
    constexpr MmaList L = Tabs<C>::list;
    int seen[8][8] = {};
    for (int i = 0; i < L.n; i++) {
        if (L.nb[i] < 1 || L.nb[i] * C::BN > 256) return false;
        for (int b = L.b0[i]; b < L.b0[i] + L.nb[i]; b++) seen[L.a[i]][b]++;
    }
    for (int a = 0; a < C::S; a++)
        for (int b = 0; b < C::S; b++)
            if (seen[a][b] != (a + b < C::S ? 1 : 0)) return false;
    return true;
}
static_assert(mma_list_covers_pairs<Cfg6>() && mma_list_covers_pairs<Cfg6n>() && mma_list_covers_pairs<Cfg7>(),
              "every slice pair with a + b < S exactly once");

// Drain order at a tile end: the first MMAs of the next tile need the
// tile-long accumulators, then the exact ones from the lowest diagonal up.
template <class C>
__host__ __device__ constexpr int drain_acc(int j) {
    return j < C::S - C::NEXACT ? C::NEXACT + j : C::NEXACT - 1 - (j - (C::S - C::NEXACT));
}

// One GEMM of a launch.  A launch carries up to MAXG of them (uneven shapes
// from many molecules and densities) in its parameter space, so a whole
// batched build is a handful of persistent launches with no device-side
// descriptor tables (and stays capturable in a CUDA graph).
struct OzProb {
    CUtensorMap tmA, tmB, tmC;
    OzArgs a;
    int tile0;          // first launch-wide work unit of this problem
    int ntn, ntm;       // output tiles along N and M
    int cfg;            // slice configuration (host side: all problems of a launch share it)
};
// Configuration ids of OzProb::cfg.
constexpr int CFG6 = 0, CFG6N = 1, CFG7 = 2;
__host__ __device__ constexpr int cfg_slices(int c) { return c == CFG7 ? 7 : 6; }
__host__ __device__ constexpr int cfg_bn(int c) { return c == CFG6 ? 80 : 64; }
__host__ __device__ constexpr int cfg_frac(int c) { return c == CFG7 ? Cfg7::FRAC : Cfg6::FRAC; }
constexpr int MAXG = 32;
struct OzGroup {
    OzProb p[MAXG];
    int nprob;
    int nunits;         // output tiles of the launch (split-K super-chunks counted apart)
    int raster;         // 0: n-tile fastest, 1: m-tile fastest
};

__device__ __forceinline__ int prob_of(const OzGroup &g, int t) {
    int i = 0;
    while (i + 1 < g.nprob && g.p[i + 1].tile0 <= t) ++i;
    return i;
}

// Work unit u of a problem: raster 0 runs the n-tiles of one A row block side
// by side (they share the A tile in L2), raster 1 the m-tiles of one B column
// block; the split-K super-chunk z varies slowest.
struct TileCoord {
    int n, m, z, kbeg, nkb;
};

__device__ __forceinline__ TileCoord tile_of(const OzProb &pr, int u, int raster) {
    TileCoord c;
    if (raster == 0) {
        c.n = u % pr.ntn;
        c.m = (u / pr.ntn) % pr.ntm;
    } else {
        c.m = u % pr.ntm;
        c.n = (u / pr.ntm) % pr.ntn;
    }
    c.z = u / (pr.ntn * pr.ntm);
    const int K = pr.a.K;
    c.kbeg = c.z * SUPER;
    const int kend = min(K, c.kbeg + SUPER);
    c.nkb = (kend - c.kbeg + KB - 1) / KB;
    return c;
}

// The MMAs of one K-block of window residue R, in the residue's issue order
// (compile-time tables): before the first MMA into an accumulator whose window
// starts here (bit set in pend), wait until the epilogue has drained and
// zeroed it.  Returns false if a wait gave up.
template <class C, int R, int I>
__device__ __forceinline__ bool issue_mmas(uint32_t tmem, uint64_t ad0, uint64_t bd0, unsigned &pend,
                                           int (&wcnt)[C::NACC], uint64_t *accempty, volatile int *abort_flag) {
    if constexpr (I == Tabs<C>::list.n) {
        return true;
    } else {
        constexpr int i = Tabs<C>::order.v[R][I];
        constexpr int a = Tabs<C>::list.a[i];
        constexpr int b0 = Tabs<C>::list.b0[i];
        constexpr int nb = Tabs<C>::list.nb[i];
        constexpr int d0 = a + b0;
        constexpr unsigned mask = ((1u << nb) - 1u) << d0;
        const unsigned need = pend & mask;
        if (need) {
#pragma unroll
            for (int d = 0; d < C::NACC; d++) {
                if (!(need & (1u << d))) continue;
                if (!tc::mbar_wait(&accempty[d], static_cast<uint32_t>(wcnt[d]) & 1u, abort_flag)) return false;
                wcnt[d]++;
            }
            pend &= ~need;
            tc::fence_after_sync();
        }
        // descriptor start addresses are in 16-byte units
        tc::mma_bf16(tmem + d0 * C::BN, ad0 + static_cast<uint64_t>(a * (BM * 32 / 16)),
                     bd0 + static_cast<uint64_t>(b0 * (C::BN * 32 / 16)), tc::idesc_bf16_f32(BM, C::BN * nb), 1u);
        return issue_mmas<C, R, I + 1>(tmem, ad0, bd0, pend, wcnt, accempty, abort_flag);
    }
}

// K-blocks kb0 + R .. kb0 + 15 of a tile (one window period, unrolled so that
// the window bookkeeping is compile-time except for the tile's first and last
// K-block).  Returns false if a wait gave up.
template <class C, int R>
__device__ __forceinline__ bool issue_period(uint8_t *smem, uint32_t tmem, int kb0, int nkb, int &stage,
                                             uint32_t &phase, int (&wcnt)[C::NACC], uint64_t *full, uint64_t *empty,
                                             uint64_t *accfull, uint64_t *accempty, volatile int *abort_flag) {
    if constexpr (R == WPERIOD) {
        return true;
    } else {
        const int kb = kb0 + R;
        if (kb >= nkb) return true;
        if (!tc::mbar_wait(&full[stage], phase, abort_flag)) return false;
        tc::fence_after_sync();
        constexpr unsigned kAll = (1u << C::NACC) - 1u;
        constexpr unsigned kStarts = ws_mask<C>(R);
        constexpr unsigned kEnds = we_mask<C>(R);
        // the tile's first K-block opens every accumulator
        unsigned pend = kStarts | ((R == 0 && kb0 == 0) ? kAll : 0u);
        const uint64_t ad0 = tc::sdesc_kmajor_sw32(tc::smem_u32(smem + stage * C::STAGE_BYTES));
        const uint64_t bd0 = ad0 + static_cast<uint64_t>(C::A_BYTES / 16);
        if (!issue_mmas<C, R, 0>(tmem, ad0, bd0, pend, wcnt, accempty, abort_flag)) return false;
        tc::mma_commit(&empty[stage]);
        const unsigned ends = kEnds | (kb == nkb - 1 ? kAll : 0u);
#pragma unroll
        for (int d = 0; d < C::NACC; d++)
            if (ends & (1u << d)) tc::mma_commit(&accfull[d]);
        if (++stage == NSTAGE) {
            stage = 0;
            phase ^= 1u;
        }
        return issue_period<C, R + 1>(smem, tmem, kb0, nkb, stage, phase, wcnt, full, empty, accfull, accempty,
                                      abort_flag);
    }
}

// Load 32 lanes x N consecutive columns (N a multiple of 8) from TMEM.
template <int N>
__device__ __forceinline__ void tmem_ld_cols(uint32_t taddr, float *v) {
#pragma unroll
    for (int c = 0; c + 16 <= N; c += 16) tc::tmem_ld16(taddr + c, v + c);
    if constexpr (N % 16 != 0) tc::tmem_ld8(taddr + (N / 16) * 16, v + (N / 16) * 16);
}
template <int N>
__device__ __forceinline__ void tmem_zero_cols(uint32_t taddr) {
#pragma unroll
    for (int c = 0; c + 16 <= N; c += 16) tc::tmem_zero16(taddr + c);
    if constexpr (N % 16 != 0) tc::tmem_zero8(taddr + (N / 16) * 16);
}

// Persistent, warp-specialized sliced GEMM.  Warp 0 streams operand stages
// with TMA, warp 1 issues the slice-pair MMAs per stage, warps 2..9 drain the
// TMEM accumulators after every window into int64 registers and write the
// finished tile while the next tile's MMAs run.
template <class C>
__global__ void __launch_bounds__(THREADS, 1)
ozgemm_kernel(const __grid_constant__ OzGroup g) {
    constexpr int NACC = C::NACC;
    constexpr int BN = C::BN;
    constexpr int OUT_COLS = C::OUT_COLS;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *outbuf = smem + NSTAGE * C::STAGE_BYTES;
    uint64_t *full = reinterpret_cast<uint64_t *>(outbuf + C::OUT_BYTES);
    uint64_t *empty = full + NSTAGE;
    uint64_t *accfull = empty + NSTAGE;
    uint64_t *accempty = accfull + NACC;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(accempty + NACC);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nunits = g.nunits;
    const int u0 = static_cast<int>(blockIdx.x);
    const int ustep = static_cast<int>(gridDim.x);

    if (threadIdx.x == 0) {
        for (int i = 0; i < NSTAGE; i++) { tc::mbar_init(&full[i], 1); tc::mbar_init(&empty[i], 1); }
        for (int i = 0; i < NACC; i++) { tc::mbar_init(&accfull[i], 1); tc::mbar_init(&accempty[i], 8); }
        *abort_flag = 0;
        tc::fence_barrier_init();
    }
    if (warp == 1) {
        tc::tmem_alloc(tmem_slot, 512);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            int last = -1;
            int stage = 0;
            uint32_t phase = 0;
            bool ok = true;
            for (int u = u0; u < nunits && ok; u += ustep) {
                const int pi = prob_of(g, u);
                const OzProb &pr = g.p[pi];
                if (pi != last) {
                    tc::prefetch_tmap(&pr.tmA);
                    tc::prefetch_tmap(&pr.tmB);
                    last = pi;
                }
                const TileCoord tc_ = tile_of(pr, u - pr.tile0, g.raster);
                for (int kb = 0; kb < tc_.nkb; kb++) {
                    if (!tc::mbar_wait(&empty[stage], phase ^ 1u, abort_flag)) { ok = false; break; }
                    const int kc = tc_.kbeg + kb * KB;
                    uint8_t *sa = smem + stage * C::STAGE_BYTES;
                    tc::mbar_expect_tx(&full[stage], C::STAGE_BYTES);
                    tc::tma_load_3d(sa, &pr.tmA, &full[stage], kc, tc_.m * BM, 0);
                    tc::tma_load_3d(sa + C::A_BYTES, &pr.tmB, &full[stage], kc, tc_.n * BN, 0);
                    if (++stage == NSTAGE) { stage = 0; phase ^= 1u; }
                }
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int wcnt[NACC];   // windows started per accumulator
#pragma unroll
            for (int d = 0; d < NACC; d++) wcnt[d] = 0;
            bool ok = true;
            for (int u = u0; u < nunits && ok; u += ustep) {
                const OzProb &pr = g.p[prob_of(g, u)];
                const TileCoord tc_ = tile_of(pr, u - pr.tile0, g.raster);
                for (int kb0 = 0; kb0 < tc_.nkb && ok; kb0 += WPERIOD)
                    ok = issue_period<C, 0>(smem, tmem, kb0, tc_.nkb, stage, phase, wcnt, full, empty, accfull,
                                            accempty, abort_flag);
            }
        }
    } else {
        // ---------------- epilogue: 8 warps, two per TMEM lane quarter ----------------
        const int ew = warp - 2;
        const int q = warp & 3;          // lane quarter this warp may access
        const int half = ew >> 2;        // which half of the tile's columns
        const uint32_t tlane = tmem + (static_cast<uint32_t>(q * 32) << 16) + half * OUT_COLS;
        // Accumulators start at zero: clear this warp's share, then open them.
#pragma unroll
        for (int d = 0; d < NACC; d++) tmem_zero_cols<OUT_COLS>(tlane + d * BN);
        tc::tmem_wait_st();
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0)
            for (int d = 0; d < NACC; d++) tc::mbar_arrive(&accempty[d]);
        uint32_t epar = 0;   // bit d: parity of the windows drained from accumulator d
        bool ok = true;
        for (int u = u0; u < nunits && ok; u += ustep) {
            // Copy the tile's problem out of parameter space once: the stores
            // below go through generic pointers and would otherwise force a
            // reload of every field per element.
            const int pi = prob_of(g, u);
            const OzArgs a = g.p[pi].a;
            const CUtensorMap *tmC = &g.p[pi].tmC;
            const TileCoord tc_ = tile_of(g.p[pi], u - g.p[pi].tile0, g.raster);
            long long acc64[OUT_COLS];
#pragma unroll
            for (int i = 0; i < OUT_COLS; i++) acc64[i] = 0;
            // Exponents of this warp's output rows and columns, fetched now so that
            // their latency hides under the tile's MMAs: lane l holds the column
            // exponents of columns l and 32 + l of its OUT_COLS (shared by shuffles).
            const int c0 = tc_.n * BN + half * OUT_COLS;
            const int row = tc_.m * BM + q * 32 + lane;
            int ea = 0, eb_lo = 0, eb_hi = 0;
            if (a.nsuper == 1) {
                if (row < a.M) ea = a.eA[row / a.a_rpe] - C::FRAC;
                if (c0 + lane < a.N) eb_lo = a.eB[(c0 + lane) / a.b_rpe];
                if (lane < OUT_COLS - 32 && c0 + 32 + lane < a.N) eb_hi = a.eB[(c0 + 32 + lane) / a.b_rpe];
            }
            for (int kb = 0; kb < tc_.nkb && ok; kb++) {
                const unsigned ends = we_mask_rt<C>(kb & (WPERIOD - 1)) | (kb == tc_.nkb - 1 ? (1u << NACC) - 1u : 0u);
                if (!ends) continue;
                // one copy of the drain-and-convert code for all accumulators
                // (per-accumulator unrolled copies cost instruction-cache misses)
#pragma unroll 1
                for (int j = 0; j < NACC; j++) {
                    const int d = drain_acc<C>(j);
                    if (!(ends & (1u << d))) continue;
                    if (!tc::mbar_wait(&accfull[d], (epar >> d) & 1u, abort_flag)) {
                        ok = false;
                        break;
                    }
                    epar ^= 1u << d;
                    __syncwarp();
                    tc::fence_after_sync();
                    float v[OUT_COLS];
                    tmem_ld_cols<OUT_COLS>(tlane + d * BN, v);
                    tc::tmem_wait_ld();
                    tmem_zero_cols<OUT_COLS>(tlane + d * BN);
                    tc::tmem_wait_st();
                    tc::fence_before_sync();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(&accempty[d]);
                    // An exact accumulator d holds integers in units of 2^-(8d+16)
                    // below 2^24; a tile-long one stays far below one unit of the
                    // output's 2^-FRAC.  Scale to the unit and convert with one
                    // FFMA against 1.5*2^23 (exact below 2^22; the rare larger
                    // value falls back to F2I), then add into the 2^-FRAC fixed
                    // point of acc64 (shifted by FRAC - 16 - 8d for the exact
                    // diagonals).  No 64-bit float conversions: those run on the
                    // scarce FP64 pipe.
                    const bool exact = d < C::NEXACT;
                    const float unit = exact ? __int_as_float((127 + 16 + 8 * d) << 23) : __int_as_float((127 + C::FRAC) << 23);
                    const float vmax = exact ? __int_as_float((127 + 22 - 16 - 8 * d) << 23)
                                             : __int_as_float((127 + 22 - C::FRAC) << 23);
                    const int sh = exact ? C::FRAC - 16 - 8 * d : 0;
#pragma unroll
                    for (int i = 0; i < OUT_COLS; i++) {
                        int xi = __float_as_int(__fmaf_rn(v[i], unit, 12582912.0f)) - 0x4B400000;
                        if (fabsf(v[i]) > vmax) xi = __float2int_rn(v[i] * unit);
                        acc64[i] += static_cast<long long>(static_cast<unsigned long long>(static_cast<long long>(xi)) << sh);
                    }
                }
            }
            if (!ok) break;
            if (a.use_tma_store) {
                // This warp's 32 x OUT_COLS block: lane = row, swizzled 32 x 8 sub-blocks.
                uint8_t *wbuf = outbuf + ew * C::OUT_WARP_BYTES;
                if (lane == 0) tc::bulk_wait_read();   // previous tile's store has read the buffer
                __syncwarp();
#pragma unroll
                for (int b = 0; b < OUT_COLS / OUT_BLK; b++) {
                    uint8_t *blk = wbuf + b * (32 * OUT_BLK * 8);
#pragma unroll
                    for (int j = 0; j < OUT_BLK / 2; j++) {   // 16-byte chunks of this row
                        const int i0 = b * OUT_BLK + 2 * j;
                        long long w0 = acc64[i0], w1 = acc64[i0 + 1];
                        if (a.nsuper == 1) {
                            const int col = c0 + i0;
                            const int eb0 = __shfl_sync(0xffffffffu, i0 < 32 ? eb_lo : eb_hi, i0 & 31);
                            const int eb1 = __shfl_sync(0xffffffffu, i0 + 1 < 32 ? eb_lo : eb_hi, (i0 + 1) & 31);
                            const double d0 = col < a.N && row < a.M ? i64_to_f64_scaled(w0, ea + eb0) : 0.0;
                            const double d1 = col + 1 < a.N && row < a.M ? i64_to_f64_scaled(w1, ea + eb1) : 0.0;
                            w0 = __double_as_longlong(d0);
                            w1 = __double_as_longlong(d1);
                        }
                        const int chunk = j ^ ((lane >> 1) & 3);   // 64-byte swizzle
                        longlong2 *dst = reinterpret_cast<longlong2 *>(blk + lane * 64 + chunk * 16);
                        *dst = make_longlong2(w0, w1);
                    }
                }
                tc::fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) {
                    const int r0 = tc_.m * BM + q * 32;
#pragma unroll
                    for (int b = 0; b < OUT_COLS / OUT_BLK; b++) {
                        const int cc = c0 + b * OUT_BLK;
                        // rows of the partial for super-chunk z follow the M rows of z-1
                        const int rr = a.nsuper == 1 ? r0 : r0 + tc_.z * static_cast<int>(a.pz / a.ldp);
                        if (cc < a.N) tc::tma_store_2d(tmC, wbuf + b * (32 * OUT_BLK * 8), cc, rr);
                    }
                    tc::bulk_commit();
                }
            } else if (row < a.M) {
                if (a.nsuper == 1) {
                    const int ear = a.eA[row / a.a_rpe] - C::FRAC;
                    double *crow = a.C + static_cast<long long>(row) * a.ldc;
#pragma unroll
                    for (int i = 0; i < OUT_COLS; i++) {
                        const int col = c0 + i;
                        if (col < a.N) crow[col] = i64_to_f64_scaled(acc64[i], ear + a.eB[col / a.b_rpe]);
                    }
                } else {
                    long long *prow = a.P + tc_.z * a.pz + static_cast<long long>(row) * a.ldp;
#pragma unroll
                    for (int i = 0; i < OUT_COLS; i++) {
                        const int col = c0 + i;
                        if (col < a.N) prow[col] = acc64[i];
                    }
                }
            }
        }
        if (lane == 0) tc::bulk_wait_all();
    }
    tc::fence_before_sync();
    __syncthreads();
    if (*abort_flag) {
        // an abandoned pipeline may still have copies in flight: let them land
        // before the shared memory is released
        const unsigned long long t0 = tc::globaltimer();
        while (tc::globaltimer() - t0 < 2000000ull) {
        }
    }
    if (warp == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, 512);
    }
    if (threadIdx.x == 0 && *abort_flag) atomicExch(g.p[0].a.err, static_cast<int>(JK_ERR_TIMEOUT));
}

// out[r][c] (+)= sum_z P[z][r][c] 2^(eA[r/arpe][z] + eB[c/brpe][z] - frac).
// The partials are aligned to the largest scale by 128-bit shifts (52 guard
// bits: a partial on a smaller scale loses only bits below 2^-52 of the
// largest scale's unit) and summed exactly; one rounding to FP64 at the end.
__global__ void __launch_bounds__(256)
reduce_partials_kernel(const long long *P, long long pz, long long ldp, int nz, int M, int N, const int *eA,
                       int arpe, const int *eB, int brpe, double *out, long long ldo, int accumulate, int frac) {
    const long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (e >= static_cast<long long>(M) * N) return;
    const int r = static_cast<int>(e / N), c = static_cast<int>(e % N);
    const long long off = static_cast<long long>(r) * ldp + c;
    const int *ea = eA + static_cast<long long>(r / arpe) * nz;
    const int *eb = eB + static_cast<long long>(c / brpe) * nz;
    int emax = -(1 << 30);
    for (int zz = 0; zz < nz; zz++) emax = max(emax, ea[zz] + eb[zz]);
    __int128 s = 0;
    for (int zz = 0; zz < nz; zz++) {
        const int d = emax - (ea[zz] + eb[zz]);
        if (d < 100) s += (static_cast<__int128>(P[zz * pz + off]) << 52) >> d;
    }
    const double v = i128_to_f64_scaled(s, emax - frac - 52);
    double *o = out + static_cast<long long>(r) * ldo + c;
    *o = accumulate ? (*o + v) : v;
}

// Many split-K reductions in one launch (the batched build's rank updates):
// each job is one reduce_partials_kernel call, its elements numbered from e0
// in the launch.
struct ReduceJob {
    const long long *P;
    long long pz, ldp;
    const int *eA, *eB;
    double *out;
    long long ldo;
    long long e0;          // first element of this job in the launch
    int nz, M, N, arpe, brpe, accumulate, frac;
};
constexpr int MAXRED = 240;
struct ReduceGroup {
    ReduceJob j[MAXRED];
    int njob;
};

__global__ void __launch_bounds__(256) reduce_group_kernel(const __grid_constant__ ReduceGroup g, long long total) {
    const long long t = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (t >= total) return;
    int lo = 0, hi = g.njob - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (g.j[mid].e0 <= t) lo = mid;
        else hi = mid - 1;
    }
    const ReduceJob &jb = g.j[lo];
    const long long e = t - jb.e0;
    const int N = jb.N, nz = jb.nz;
    const int r = static_cast<int>(e / N), c = static_cast<int>(e % N);
    const long long off = static_cast<long long>(r) * jb.ldp + c;
    const int *ea = jb.eA + static_cast<long long>(r / jb.arpe) * nz;
    const int *eb = jb.eB + static_cast<long long>(c / jb.brpe) * nz;
    int emax = -(1 << 30);
    for (int zz = 0; zz < nz; zz++) emax = max(emax, ea[zz] + eb[zz]);
    __int128 s = 0;
    for (int zz = 0; zz < nz; zz++) {
        const int d = emax - (ea[zz] + eb[zz]);
        if (d < 100) s += (static_cast<__int128>(jb.P[zz * jb.pz + off]) << 52) >> d;
    }
    const double v = i128_to_f64_scaled(s, emax - jb.frac - 52);
    double *o = jb.out + static_cast<long long>(r) * jb.ldo + c;
    *o = jb.accumulate ? (*o + v) : v;
}

// K[r][c] = K[c][r] for the entries a blocked symmetric rank update leaves
// unformed: c < bm * (r / bm), left of row r's diagonal block (those (c, r)
// all lie in the formed blocks, so no entry is both read and written).
__global__ void __launch_bounds__(256) mirror_blocks_kernel(double *K, int n, int bm) {
    const long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (e >= static_cast<long long>(n) * n) return;
    const int r = static_cast<int>(e / n), c = static_cast<int>(e - static_cast<long long>(r) * n);
    if (c < bm * (r / bm)) K[e] = K[static_cast<long long>(c) * n + r];
}

}  // namespace oz

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
namespace {

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                   CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                   CUtensorMapFloatOOBfill);

// The driver's tensor-map encoder, looked up once per process (the first
// successful lookup is published atomically, so concurrent first calls from
// several threads are safe; a failed lookup is retried on the next call).
EncodeTiledFn encode_fn() {
    static std::atomic<EncodeTiledFn> fn{nullptr};
    EncodeTiledFn f = fn.load(std::memory_order_acquire);
    if (!f) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        // the entry point as introduced with CUDA 12.0
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess) {
            f = reinterpret_cast<EncodeTiledFn>(p);
            fn.store(f, std::memory_order_release);
        }
    }
    return f;
}

// Tensor map over slices [planes][rows][Kpad] (bf16), box = {16, box_rows,
// planes}, 32-byte swizzle.  Consecutive planes lie plane_rows * Kpad elements
// apart (plane_rows >= rows: a map over a block of rows of a larger sliced
// operand).
jk_status make_slice_map(jk_ctx *h, CUtensorMap *map, const __nv_bfloat16 *base, int rows, int Kpad,
                         int box_rows, long long plane_rows, int planes) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return set_error(h, JK_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
    const int box_planes = planes;
    cuuint64_t dims[3] = {static_cast<cuuint64_t>(Kpad), static_cast<cuuint64_t>(rows),
                          static_cast<cuuint64_t>(planes)};
    cuuint64_t strides[2] = {static_cast<cuuint64_t>(Kpad) * 2, static_cast<cuuint64_t>(plane_rows) * Kpad * 2};
    cuuint32_t box[3] = {oz::KB, static_cast<cuuint32_t>(box_rows), static_cast<cuuint32_t>(box_planes)};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<__nv_bfloat16 *>(base), dims, strides,
                    box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(h, JK_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return JK_OK;
}

// Tensor map over a row-major matrix of 64-bit words (rows x cols, row stride
// ld words, ld even), box = 8 words x 32 rows, 64-byte swizzle: the layout
// the GEMM epilogue stages its output in.
jk_status make_out_map(jk_ctx *h, CUtensorMap *map, void *base, long long rows, int cols, long long ld) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return set_error(h, JK_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
    cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
    cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld) * 8};
    cuuint32_t box[2] = {static_cast<cuuint32_t>(oz::OUT_BLK), 32};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_INT64, 2, base, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(h, JK_ERR_CUDA, "cuTensorMapEncodeTiled (output) failed (%d)", (int)r);
    return JK_OK;
}

inline int kpad_of(int K) { return (K + 15) / 16 * 16; }
inline long long even_ld(long long n) { return n + (n & 1); }
// Rows reserved per split-K partial: M rounded up to whole row tiles, so a
// tile's padding rows never land in the next partial.
inline long long part_rows(long long M) { return (M + oz::BM - 1) / oz::BM * oz::BM; }

}  // namespace

// A sliced operand: S bf16 slices [S][rows][Kpad] plus per-group exponents.
// A row view (row_view) addresses rows [r0, r1) of a larger operand: its
// planes keep the parent's spacing of prows rows.
struct Sliced {
    __nv_bfloat16 *s = nullptr;
    int *e = nullptr;
    int S = 6;          // slices (6: 48-bit operand, 7: 56-bit)
    int rows = 0, K = 0, Kpad = 0, rpe = 1;
    int prows = 0;      // rows between consecutive planes (0: rows)
    long long plane_rows() const { return prows > 0 ? prows : rows; }
};

// Rows [r0, r1) of a sliced operand (r0 a multiple of its exponent group).
static Sliced row_view(const Sliced &S, int r0, int r1) {
    Sliced v = S;
    const long long nsc = (S.K + oz::SUPER - 1) / oz::SUPER;
    v.s = S.s + static_cast<long long>(r0) * S.Kpad;
    v.e = S.e + static_cast<long long>(r0 / S.rpe) * nsc;
    v.rows = r1 - r0;
    v.prows = static_cast<int>(S.plane_rows());
    return v;
}

static jk_status slice_operand(jk_ctx *h, const oz::Src &src, int rows, int K, int rpe, Sliced &out,
                               cudaStream_t st) {
    out.rows = rows;
    out.K = K;
    out.Kpad = kpad_of(K);
    out.rpe = rpe;
    const int groups = (rows + rpe - 1) / rpe;
    const int nsc = (K + oz::SUPER - 1) / oz::SUPER;   // one exponent per row group and super-chunk
    const bool aligned = (reinterpret_cast<uintptr_t>(src.p) & 15u) == 0;
    // A group of rows that is one contiguous run of doubles (e.g. one L^P).
    const bool flat = nsc == 1 && aligned && src.rin == 1 && src.ski == 1 && src.kin == K && src.sr == K &&
                      ((static_cast<long long>(rpe) * K) % 2) == 0 && rows % rpe == 0;
    {
        LaunchScope ls(h, KK_SLICE, st);
        if (flat)
            oz::expo_flat_kernel<<<groups, 256, 0, st>>>(src.p, static_cast<long long>(rpe) * K, out.e);
        else
            oz::expo_kernel<<<dim3(groups, nsc), 256, 0, st>>>(src, rows, K, rpe, out.e);
    }
    JK_LAUNCH_CHECK(h);
    const bool vec = aligned && src.ski == 1 && (src.kin % 4) == 0 && (K % 4) == 0 && (src.sr % 2) == 0 &&
                     (src.sri % 2) == 0 && (src.sko % 2) == 0;
    const int rblocks = (rows + oz::SLICE_ROWS - 1) / oz::SLICE_ROWS;
    {
        LaunchScope ls(h, KK_SLICE, st);
        if (vec) {
            dim3 grid((out.Kpad / 4 + 255) / 256, rblocks < 65535 ? rblocks : 65535);
            uint2 *o4 = reinterpret_cast<uint2 *>(out.s);
            const long long ss4 = static_cast<long long>(rows) * out.Kpad / 4;
            if (out.S == 7)
                oz::slice4_kernel<7><<<grid, 256, 0, st>>>(src, rows, K, out.Kpad, out.e, rpe, nsc, o4, ss4);
            else if (h->slicer == 1)
                oz::slice4f_kernel<<<grid, 256, 0, st>>>(src, rows, K, out.Kpad, out.e, rpe, nsc, o4, ss4);
            else
                oz::slice4_kernel<6><<<grid, 256, 0, st>>>(src, rows, K, out.Kpad, out.e, rpe, nsc, o4, ss4);
        } else {
            dim3 grid((out.Kpad + 255) / 256, rblocks < 65535 ? rblocks : 65535);
            unsigned short *o1 = reinterpret_cast<unsigned short *>(out.s);
            const long long ss1 = static_cast<long long>(rows) * out.Kpad;
            if (out.S == 7)
                oz::slice_kernel<7><<<grid, 256, 0, st>>>(src, rows, K, out.Kpad, out.e, rpe, nsc, o1, ss1);
            else
                oz::slice_kernel<6><<<grid, 256, 0, st>>>(src, rows, K, out.Kpad, out.e, rpe, nsc, o1, ss1);
        }
    }
    JK_LAUNCH_CHECK(h);
    return JK_OK;
}

static size_t sliced_bytes(int rows, int K, int rpe, int S = 6) {
    const size_t nsc = (K + oz::SUPER - 1) / oz::SUPER;
    return align_up(static_cast<size_t>(S) * rows * kpad_of(K) * 2) +
           align_up(static_cast<size_t>((rows + rpe - 1) / rpe) * nsc * 4);
}

// Workspace of an S-slice operand (S = 6 unless the call asks for 7).
static bool take_sliced(Arena &ar, int rows, int K, int rpe, Sliced &out, int S = 6) {
    out.S = S;
    out.s = ar.take<__nv_bfloat16>(static_cast<size_t>(S) * rows * kpad_of(K));
    out.e = ar.take<int>(static_cast<size_t>((rows + rpe - 1) / rpe) * ((K + oz::SUPER - 1) / oz::SUPER));
    return out.s && out.e;
}

static int nsuper_of(int K) { return (K + oz::SUPER - 1) / oz::SUPER; }

// Fill one GEMM problem C = A B^T on sliced operands.  nsuper == 1: FP64 written
// to C (row stride ldc); otherwise int64 partials go to P (padded row blocks).
static jk_status oz_problem(jk_ctx *h, const Sliced &A, const Sliced &B, double *C, long long ldc, long long *P,
                            oz::OzProb &pr) {
    if (A.K != B.K) return set_error(h, JK_ERR_ARG, "internal: sliced K mismatch");
    if (A.S != B.S) return set_error(h, JK_ERR_ARG, "internal: operands with different slice counts");
    std::memset(&pr, 0, sizeof pr);
    // seven-slice operands take 64-column tiles (seven accumulators of 80
    // columns would not fit tensor memory); six-slice ones the handle's tile width
    pr.cfg = A.S == 7 ? oz::CFG7 : (h->cur_tile == 1 ? oz::CFG6N : oz::CFG6);
    const int BN = oz::cfg_bn(pr.cfg);
    JK_TRY(make_slice_map(h, &pr.tmA, A.s, A.rows, A.Kpad, oz::BM, A.plane_rows(), A.S));
    JK_TRY(make_slice_map(h, &pr.tmB, B.s, B.rows, B.Kpad, BN, B.plane_rows(), B.S));
    oz::OzArgs &a = pr.a;
    a.M = A.rows; a.N = B.rows; a.K = A.K; a.nsuper = nsuper_of(A.K);
    a.eA = A.e; a.a_rpe = A.rpe; a.eB = B.e; a.b_rpe = B.rpe;
    a.C = C; a.ldc = ldc; a.P = P;
    a.ldp = even_ld(B.rows);
    a.pz = part_rows(A.rows) * a.ldp;
    a.err = &h->flags->error;
    if (a.nsuper > 1 && !P) return set_error(h, JK_ERR_ARG, "internal: partial buffer missing");
    a.use_tma_store = 0;
    if (a.nsuper > 1) {
        JK_TRY(make_out_map(h, &pr.tmC, P, static_cast<long long>(a.nsuper) * part_rows(a.M), a.N, a.ldp));
        a.use_tma_store = 1;
    } else if ((ldc % 2) == 0 && (reinterpret_cast<uintptr_t>(C) & 15u) == 0) {
        JK_TRY(make_out_map(h, &pr.tmC, C, a.M, a.N, ldc));
        a.use_tma_store = 1;
    }
    const long long ntn = (a.N + BN - 1) / BN, ntm = (a.M + oz::BM - 1) / oz::BM;
    if (ntn * ntm * a.nsuper > 0x3fffffffLL) return set_error(h, JK_ERR_SHAPE, "too many tiles");
    pr.ntn = static_cast<int>(ntn);
    pr.ntm = static_cast<int>(ntm);
    // Issued MMA work: every tile runs all S(S+1)/2 slice pairs over its K-blocks.
    const double tiles = static_cast<double>(ntn) * ntm;
    double kblocks = 0.0;
    for (int zz = 0; zz < a.nsuper; zz++) {
        const int kb = (a.K - zz * oz::SUPER < oz::SUPER ? a.K - zz * oz::SUPER : oz::SUPER);
        kblocks += (kb + oz::KB - 1) / oz::KB;
    }
    const int S = A.S;
    h->prof.tensor_flops += 2.0 * oz::BM * BN * oz::KB * (S * (S + 1) / 2) * kblocks * tiles;
    return JK_OK;
}

template <class C>
static jk_status oz_launch_cfg(jk_ctx *h, const oz::OzGroup &grp, int grid, int cfg, cudaStream_t st) {
    if (!(h->gemm_smem_set & (1 << cfg))) {
        // a per-device function attribute: set once per handle (a handle is bound to one device)
        JK_CUDA_TRY(h, cudaFuncSetAttribute(oz::ozgemm_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            C::SMEM_BYTES));
        h->gemm_smem_set |= 1 << cfg;
    }
    {
        LaunchScope ls(h, KK_OZGEMM, st);
        oz::ozgemm_kernel<C><<<grid, oz::THREADS, C::SMEM_BYTES, st>>>(grp);
    }
    JK_LAUNCH_CHECK(h);
    return JK_OK;
}

// Launch a list of problems: persistent grid, up to MAXG problems of one
// slice configuration per launch (a change of configuration starts a new one).
static jk_status oz_launch(jk_ctx *h, const std::vector<oz::OzProb> &probs, cudaStream_t st) {
    static thread_local oz::OzGroup grp;   // ~20 KB of launch parameters, built on the host
    for (size_t i0 = 0; i0 < probs.size();) {
        const int cfg = probs[i0].cfg;
        int np = 0;
        while (np < oz::MAXG && i0 + np < probs.size() && probs[i0 + np].cfg == cfg) np++;
        long long units = 0;
        for (int i = 0; i < np; i++) {
            grp.p[i] = probs[i0 + i];
            grp.p[i].tile0 = static_cast<int>(units);
            units += static_cast<long long>(grp.p[i].ntn) * grp.p[i].ntm * grp.p[i].a.nsuper;
        }
        if (units > 0x7fffffffLL) return set_error(h, JK_ERR_SHAPE, "too many tiles in one launch");
        grp.nprob = np;
        grp.nunits = static_cast<int>(units);
        grp.raster = h->cur_raster;
        const int grid = static_cast<int>(units < h->num_sms ? units : h->num_sms);
        if (cfg == oz::CFG7) JK_TRY(oz_launch_cfg<oz::Cfg7>(h, grp, grid, cfg, st));
        else if (cfg == oz::CFG6N) JK_TRY(oz_launch_cfg<oz::Cfg6n>(h, grp, grid, cfg, st));
        else JK_TRY(oz_launch_cfg<oz::Cfg6>(h, grp, grid, cfg, st));
        i0 += np;
    }
    return JK_OK;
}

// C = A B^T on sliced operands (one problem, one launch).
static jk_status ozgemm(jk_ctx *h, const Sliced &A, const Sliced &B, double *C, long long ldc, long long *P,
                        cudaStream_t st) {
    std::vector<oz::OzProb> v(1);
    JK_TRY(oz_problem(h, A, B, C, ldc, P, v[0]));
    return oz_launch(h, v, st);
}

static jk_status reduce_partials(jk_ctx *h, const long long *P, int nz, const Sliced &A, const Sliced &B,
                                 double *out, long long ldo, bool accumulate, cudaStream_t st) {
    const long long tot = static_cast<long long>(A.rows) * B.rows;
    const long long ldp = even_ld(B.rows);
    {
        LaunchScope ls(h, KK_OZREDUCE, st);
        oz::reduce_partials_kernel<<<static_cast<unsigned>((tot + 255) / 256), 256, 0, st>>>(
            P, part_rows(A.rows) * ldp, ldp, nz, A.rows, B.rows, A.e, A.rpe, B.e, B.rpe, out, ldo,
            accumulate ? 1 : 0, A.S == 7 ? oz::Cfg7::FRAC : oz::Cfg6::FRAC);
    }
    JK_LAUNCH_CHECK(h);
    return JK_OK;
}

// ---- grouped slicing and reductions (batched builds) -------------------------
static_assert(sizeof(oz::SliceGroup) <= 32764 && sizeof(oz::ReduceGroup) + 8 <= 32764,
              "grouped launches fit the kernel parameter space");

// Operands to slice with grouped launches: each added operand becomes one
// job of the same slicing slice_operand does (exponents, then digits).
struct SliceBatch {
    std::vector<oz::SliceJob> jobs;
};

static void slice_add(SliceBatch &sb, const oz::Src &src, int rows, int K, int rpe, Sliced &out) {
    out.rows = rows;
    out.K = K;
    out.Kpad = kpad_of(K);
    out.rpe = rpe;
    oz::SliceJob j;
    std::memset(&j, 0, sizeof j);
    j.src = src;
    j.e = out.e;
    j.out = out.s;
    j.rows = rows;
    j.K = K;
    j.Kpad = out.Kpad;
    j.rpe = rpe;
    j.nsc = (K + oz::SUPER - 1) / oz::SUPER;
    const bool aligned = (reinterpret_cast<uintptr_t>(src.p) & 15u) == 0;
    j.flat = j.nsc == 1 && aligned && src.rin == 1 && src.ski == 1 && src.kin == K && src.sr == K &&
             ((static_cast<long long>(rpe) * K) % 2) == 0 && rows % rpe == 0;
    j.vec = aligned && src.ski == 1 && (src.kin % 4) == 0 && (K % 4) == 0 && (src.sr % 2) == 0 &&
            (src.sri % 2) == 0 && (src.sko % 2) == 0;
    j.sstride = j.vec ? static_cast<long long>(rows) * out.Kpad / 4 : static_cast<long long>(rows) * out.Kpad;
    const int rblocks = (rows + oz::SLICE_ROWS - 1) / oz::SLICE_ROWS;
    j.nbx = j.vec ? (out.Kpad / 4 + 255) / 256 : (out.Kpad + 255) / 256;
    j.nby = rblocks < 65535 ? rblocks : 65535;
    sb.jobs.push_back(j);
    (void)out.S;
}

// Slice every collected operand (all six-slice) with one exponent launch and
// one slicer launch per MAXJOB jobs; the batch is emptied.
static jk_status slice_flush(jk_ctx *h, SliceBatch &sb, cudaStream_t st) {
    static thread_local oz::SliceGroup grp;
    for (size_t i0 = 0; i0 < sb.jobs.size(); i0 += oz::MAXJOB) {
        const int nj = static_cast<int>(std::min<size_t>(oz::MAXJOB, sb.jobs.size() - i0));
        long long eb = 0, sbk = 0;
        for (int i = 0; i < nj; i++) {
            oz::SliceJob &j = grp.j[i];
            j = sb.jobs[i0 + i];
            j.eb0 = static_cast<int>(eb);
            j.sb0 = static_cast<int>(sbk);
            const int groups = (j.rows + j.rpe - 1) / j.rpe;
            eb += j.flat ? groups : static_cast<long long>(groups) * j.nsc;
            sbk += static_cast<long long>(j.nbx) * j.nby;
        }
        if (eb > 0x7fffffffLL || sbk > 0x7fffffffLL) return set_error(h, JK_ERR_SHAPE, "too many slicer blocks");
        grp.njob = nj;
        {
            LaunchScope ls(h, KK_SLICE, st);
            oz::expo_group_kernel<<<static_cast<unsigned>(eb), 256, 0, st>>>(grp);
        }
        JK_LAUNCH_CHECK(h);
        {
            LaunchScope ls(h, KK_SLICE, st);
            oz::slice_group_kernel<6><<<static_cast<unsigned>(sbk), 256, 0, st>>>(grp);
        }
        JK_LAUNCH_CHECK(h);
    }
    sb.jobs.clear();
    return JK_OK;
}

// Split-K reductions collected for grouped launches (reduce_partials' work).
struct ReduceBatch {
    std::vector<oz::ReduceJob> jobs;
};

static void reduce_add(ReduceBatch &rb, const long long *P, int nz, const Sliced &A, const Sliced &B, double *out,
                       long long ldo, bool accumulate) {
    oz::ReduceJob j;
    std::memset(&j, 0, sizeof j);
    j.ldp = even_ld(B.rows);
    j.P = P;
    j.pz = part_rows(A.rows) * j.ldp;
    j.eA = A.e;
    j.eB = B.e;
    j.out = out;
    j.ldo = ldo;
    j.nz = nz;
    j.M = A.rows;
    j.N = B.rows;
    j.arpe = A.rpe;
    j.brpe = B.rpe;
    j.accumulate = accumulate ? 1 : 0;
    j.frac = A.S == 7 ? oz::Cfg7::FRAC : oz::Cfg6::FRAC;
    rb.jobs.push_back(j);
}

static jk_status reduce_flush(jk_ctx *h, ReduceBatch &rb, cudaStream_t st) {
    static thread_local oz::ReduceGroup grp;
    for (size_t i0 = 0; i0 < rb.jobs.size(); i0 += oz::MAXRED) {
        const int nj = static_cast<int>(std::min<size_t>(oz::MAXRED, rb.jobs.size() - i0));
        long long tot = 0;
        for (int i = 0; i < nj; i++) {
            grp.j[i] = rb.jobs[i0 + i];
            grp.j[i].e0 = tot;
            tot += static_cast<long long>(grp.j[i].M) * grp.j[i].N;
        }
        grp.njob = nj;
        {
            LaunchScope ls(h, KK_OZREDUCE, st);
            oz::reduce_group_kernel<<<static_cast<unsigned>((tot + 255) / 256), 256, 0, st>>>(grp, tot);
        }
        JK_LAUNCH_CHECK(h);
    }
    rb.jobs.clear();
    return JK_OK;
}

// ---- symmetric rank updates (JK_OPT_SYRK) -----------------------------------
// K_s = T_X T_X^T of a symmetric density is symmetric.  Row block i (rows
// [r0, r1) = [BM i, BM (i+1)) of T_X) is multiplied by rows [r0, n) only: one
// GEMM problem per block on row views of the same sliced operand, forming
// every entry on or above the diagonal (and the lower half of the diagonal
// blocks); mirror_blocks_kernel fills the rest from its transpose once all
// aux chunks are summed.  For n = 400 that is 12 output tiles instead of 20.
struct SymPart {
    Sliced A, B;
    long long out_off;   // offset of the block in the n x n output
    long long p_off;     // offset of its int64 partials (nsuper > 1)
};

static std::vector<SymPart> sym_parts(const Sliced &TX, int n, int nsuper) {
    std::vector<SymPart> v;
    long long p = 0;
    for (int r0 = 0; r0 < n; r0 += oz::BM) {
        const int r1 = std::min(n, r0 + oz::BM);
        SymPart sp{row_view(TX, r0, r1), row_view(TX, r0, n), static_cast<long long>(r0) * n + r0, p};
        if (nsuper > 1) p += static_cast<long long>(nsuper) * part_rows(r1 - r0) * even_ld(n - r0);
        v.push_back(sp);
    }
    return v;
}

// Partial words of one blocked symmetric rank update (at most those of the full one).
static long long sym_partial_words(int n, int nsuper) {
    long long w = 0;
    for (int r0 = 0; r0 < n; r0 += oz::BM)
        w += static_cast<long long>(nsuper) * part_rows(std::min(n, r0 + oz::BM) - r0) * even_ld(n - r0);
    return w;
}

// Append the problems of the blocked symmetric rank update of TX (nsuper ==
// 1: FP64 into C, row stride n; otherwise int64 partials from P).
static jk_status sym_rank_problems(jk_ctx *h, const Sliced &TX, int n, double *C, long long *P,
                                   std::vector<oz::OzProb> &probs) {
    const int ns = nsuper_of(TX.K);
    for (const SymPart &sp : sym_parts(TX, n, ns)) {
        probs.emplace_back();
        if (ns == 1) JK_TRY(oz_problem(h, sp.A, sp.B, C + sp.out_off, n, nullptr, probs.back()));
        else JK_TRY(oz_problem(h, sp.A, sp.B, nullptr, 0, P + sp.p_off, probs.back()));
    }
    return JK_OK;
}

// The split-K reductions of those problems into K (+= when accumulate).
static jk_status sym_rank_reduce(jk_ctx *h, const Sliced &TX, int n, const long long *P, double *K, bool accumulate,
                                 cudaStream_t st) {
    const int ns = nsuper_of(TX.K);
    for (const SymPart &sp : sym_parts(TX, n, ns))
        JK_TRY(reduce_partials(h, P + sp.p_off, ns, sp.A, sp.B, K + sp.out_off, n, accumulate, st));
    return JK_OK;
}

static_assert(kSymBlock == oz::BM, "symmetric row blocks are single GEMM row tiles");

jk_status mirror_sym_blocks(jk_ctx *h, double *K, int n, cudaStream_t st) {
    const long long n2 = static_cast<long long>(n) * n;
    {
        LaunchScope ls(h, KK_MISC, st);
        oz::mirror_blocks_kernel<<<static_cast<unsigned>((n2 + 255) / 256), 256, 0, st>>>(K, n, kSymBlock);
    }
    JK_LAUNCH_CHECK(h);
    return JK_OK;
}

// ---------------------------------------------------------------------------
// The split build
// ---------------------------------------------------------------------------

// P-chunk so that the per-chunk workspace stays below ~12 GB.
static int split_pchunk(const Problem &pb) {
    const size_t n = pb.n;
    size_t per = n * n * (6 * 2) + n * pb.ctot * 8 + n * pb.ctot * (6 * 2);
    if (pb.packed) per += n * n * 8;               // the expanded factor chunk
    size_t budget = static_cast<size_t>(12) << 30;
    size_t pc = per ? budget / per : 1;
    if (pc < 1) pc = 1;
    if (pb.aux_chunk > 0) pc = pb.aux_chunk;       // explicit or tuned chunk
    if (pc > static_cast<size_t>(pb.naux)) pc = pb.naux;
    // Keep rows of the panel GEMM within the grid limit.
    size_t maxrows = static_cast<size_t>(65535) * oz::BM;
    if (pc * n > maxrows) pc = maxrows / n;
    return static_cast<int>(pc);
}

int split_auto_pchunk(const Problem &pb) {
    Problem q = pb;
    q.aux_chunk = 0;
    return split_pchunk(q);
}

static size_t partial_count(const Problem &pb, int pc) {
    // int64 partials of all densities' rank updates for one P-chunk.
    size_t cnt = 0;
    for (int s = 0; s < pb.nd; s++) {
        int ns = nsuper_of(pc * pb.k[s]);
        if (ns > 1) cnt += static_cast<size_t>(ns) * part_rows(pb.n) * even_ld(pb.n);
    }
    return cnt;
}

size_t split_build_workspace(const Problem &pb) {
    const int pc = split_pchunk(pb);
    const size_t n = pb.n;
    size_t b = 0;
    b += align_up(n * pb.ctot * 8);                                  // Z
    b += sliced_bytes(pc * pb.n, pb.n, pb.n);                        // L chunk slices
    b += sliced_bytes(pb.ctot, pb.n, 1);                             // Z^T slices
    b += align_up(static_cast<size_t>(pc) * n * even_ld(pb.ctot) * 8);   // T chunk (FP64)
    b += align_up(static_cast<size_t>(pb.nd) * pb.naux * 8);         // gamma
    for (int s = 0; s < pb.nd; s++) {                                // T_X, T_Y slices
        b += sliced_bytes(pb.n, pc * pb.k[s], 1);
        if (!pb.sym[s]) b += sliced_bytes(pb.n, pc * pb.k[s], 1);
    }
    b += align_up(partial_count(pb, pc) * 8);
    b += align_up(static_cast<size_t>(pb.nd) * n * n * 8);           // K accumulators (if K not wanted)
    if (pb.n > oz::SUPER)
        b += align_up(static_cast<size_t>(nsuper_of(pb.n)) * part_rows(static_cast<long long>(pc) * n) * even_ld(pb.ctot) * 8);
    if (pb.packed) b += align_up(static_cast<size_t>(pc) * n * n * 8);   // expanded factor chunk
    return b;
}


jk_status split_pack_z(jk_ctx *h, const Problem &pb, double *Z, cudaStream_t st);
jk_status fp64_unpack_sym(jk_ctx *h, const double *packed, int n, long long np, double *full, cudaStream_t st);
jk_status fp64_gamma_panel(jk_ctx *h, const Problem &pb, const double *T, long long ldT, int np, double *gamma,
                           int P0, cudaStream_t st);
jk_status fp64_jstream(jk_ctx *h, const Problem &pb, const double *gamma, cudaStream_t st);

// The FP64 J back-contraction needs only the factor and gamma, and runs on the
// FP64 pipe: it is forked onto a second stream as soon as gamma is complete
// and overlaps the rank updates on the tensor pipe (join at the end of the
// build, so the call stays ordered on the caller's stream).
static jk_status fork_jstream(jk_ctx *h, cudaStream_t st) {
    if (!h->aux_stream) {
        JK_CUDA_TRY(h, cudaStreamCreateWithFlags(&h->aux_stream, cudaStreamNonBlocking));
        JK_CUDA_TRY(h, cudaEventCreateWithFlags(&h->ev_jfork, cudaEventDisableTiming));
        JK_CUDA_TRY(h, cudaEventCreateWithFlags(&h->ev_jdone, cudaEventDisableTiming));
    }
    JK_CUDA_TRY(h, cudaEventRecord(h->ev_jfork, st));
    JK_CUDA_TRY(h, cudaStreamWaitEvent(h->aux_stream, h->ev_jfork, 0));
    return JK_OK;
}

static jk_status join_jstream(jk_ctx *h, cudaStream_t st) {
    JK_CUDA_TRY(h, cudaEventRecord(h->ev_jdone, h->aux_stream));
    JK_CUDA_TRY(h, cudaStreamWaitEvent(st, h->ev_jdone, 0));
    return JK_OK;
}

jk_status split_build(jk_ctx *h, const Problem &pb, cudaStream_t st) {
    const int n = pb.n, naux = pb.naux, nd = pb.nd;
    const long long n2 = static_cast<long long>(n) * n;
    const int pc = split_pchunk(pb);
    Arena &ar = h->arena;
    double *Z = ar.take<double>(static_cast<size_t>(n) * pb.ctot);
    Sliced Ls, Zs;
    bool ok = Z && take_sliced(ar, pc * n, n, n, Ls) && take_sliced(ar, pb.ctot, n, 1, Zs);
    const long long ldT = even_ld(pb.ctot);
    double *T = ar.take<double>(static_cast<size_t>(pc) * n * ldT);
    double *gamma = ar.take<double>(static_cast<size_t>(nd) * naux);
    Sliced TX[kMaxDens], TY[kMaxDens];
    for (int s = 0; ok && s < nd; s++) {
        ok = take_sliced(ar, n, pc * pb.k[s], 1, TX[s]);
        if (ok && !pb.sym[s]) ok = take_sliced(ar, n, pc * pb.k[s], 1, TY[s]);
    }
    long long *Pbuf = ar.take<long long>(partial_count(pb, pc) > 0 ? partial_count(pb, pc) : 1);
    double *Kacc = ar.take<double>(static_cast<size_t>(nd) * n2);
    long long *Ppanel = nullptr;
    if (n > oz::SUPER)
        Ppanel = ar.take<long long>(static_cast<size_t>(nsuper_of(n)) * part_rows(static_cast<long long>(pc) * n) * ldT);
    double *Lx = pb.packed ? ar.take<double>(static_cast<size_t>(pc) * n2) : nullptr;
    if (!ok || !T || !gamma || !Pbuf || !Kacc || (n > oz::SUPER && !Ppanel) || (pb.packed && !Lx))
        return set_error(h, JK_ERR_OOM, "workspace too small for the split build");

    // Z = [X_0 | Y_0 | ...] and its transpose sliced per column (rows of Z^T).
    JK_TRY(split_pack_z(h, pb, Z, st));
    oz::Src zsrc{Z, 1, 0, pb.ctot, n};          // row c of Z^T, element lam at Z[lam][c]
    JK_TRY(slice_operand(h, zsrc, pb.ctot, n, 1, Zs, st));

    for (int P0 = 0; P0 < naux; P0 += pc) {
        const int np = naux - P0 < pc ? naux - P0 : pc;
        // a packed factor chunk is expanded first
        if (pb.packed) JK_TRY(fp64_unpack_sym(h, pb.L + P0 * packed::tri_count(n), n, np, Lx, st));
        const double *Lchunk = pb.packed ? Lx : pb.L + P0 * n2;
        // L^P rows (P, mu), reduction over lam, one exponent per P.
        oz::Src lsrc{Lchunk, n, 0, 1, n};
        Sliced Lc = Ls;
        JK_TRY(slice_operand(h, lsrc, np * n, n, n, Lc, st));
        // T[(p, mu)][c] = sum_lam L^p[mu][lam] Z[lam][c]
        if (n > oz::SUPER) {
            JK_TRY(ozgemm(h, Lc, Zs, nullptr, 0, Ppanel, st));
            JK_TRY(reduce_partials(h, Ppanel, nsuper_of(n), Lc, Zs, T, ldT, false, st));
        } else {
            JK_TRY(ozgemm(h, Lc, Zs, T, ldT, nullptr, st));
        }
        if (pb.wantJ) JK_TRY(fp64_gamma_panel(h, pb, T, ldT, np, gamma, P0, st));
        if (pb.wantJ && P0 + np >= naux) {
            JK_TRY(fork_jstream(h, st));
            JK_TRY(fp64_jstream(h, pb, gamma, h->aux_stream));
        }
        if (!pb.wantK) continue;
        // The rank-update operands of every density (grouped launches unless
        // the FP32-digit slicer is asked for), then the rank update per
        // density over this chunk's (p, i) pairs.
        {
            const bool grouped = h->slicer == 0;
            SliceBatch sb;
            for (int s = 0; s < nd; s++) {
                const int k = pb.k[s];
                const int Kr = np * k;
                oz::Src xs{T + pb.offX[s], ldT, static_cast<long long>(n) * ldT, 1, k};
                if (grouped) slice_add(sb, xs, n, Kr, 1, TX[s]);
                else JK_TRY(slice_operand(h, xs, n, Kr, 1, TX[s], st));
                if (!pb.sym[s]) {
                    oz::Src ys{T + pb.offY[s], ldT, static_cast<long long>(n) * ldT, 1, k};
                    if (grouped) slice_add(sb, ys, n, Kr, 1, TY[s]);
                    else JK_TRY(slice_operand(h, ys, n, Kr, 1, TY[s], st));
                }
            }
            JK_TRY(slice_flush(h, sb, st));
        }
        ReduceBatch rb;
        long long *Pcur = Pbuf;
        for (int s = 0; s < nd; s++) {
            const int k = pb.k[s];
            const int Kr = np * k;
            Sliced *B = pb.sym[s] ? &TX[s] : &TY[s];
            double *Kout = pb.K[s];
            const int ns = nsuper_of(Kr);
            if (pb.sym[s] && h->syrk) {
                // blocked symmetric rank update (mirrored after the last chunk)
                std::vector<oz::OzProb> probs;
                double *dst = P0 == 0 ? Kout : Kacc + s * n2;
                JK_TRY(sym_rank_problems(h, TX[s], n, dst, Pcur, probs));
                JK_TRY(oz_launch(h, probs, st));
                if (ns > 1) {
                    JK_TRY(sym_rank_reduce(h, TX[s], n, Pcur, Kout, P0 > 0, st));
                    Pcur += sym_partial_words(n, ns);
                } else if (P0 > 0) {
                    JK_TRY(fp64_axpy(h, Kout, dst, n2, st));
                }
                continue;
            }
            if (ns == 1) {
                if (P0 == 0) {
                    JK_TRY(ozgemm(h, TX[s], *B, Kout, n, nullptr, st));
                } else {
                    double *tmp = Kacc + s * n2;
                    JK_TRY(ozgemm(h, TX[s], *B, tmp, n, nullptr, st));
                    // Kout += tmp (FP64, fixed order)
                    JK_TRY(fp64_axpy(h, Kout, tmp, n2, st));
                }
            } else {
                JK_TRY(ozgemm(h, TX[s], *B, nullptr, 0, Pcur, st));
                reduce_add(rb, Pcur, ns, TX[s], *B, Kout, n, P0 > 0);
                Pcur += static_cast<size_t>(ns) * part_rows(n) * even_ld(n);
            }
        }
        JK_TRY(reduce_flush(h, rb, st));
    }
    if (pb.wantK && h->syrk)
        for (int s = 0; s < nd; s++)
            if (pb.sym[s]) JK_TRY(mirror_sym_blocks(h, pb.K[s], n, st));
    if (pb.wantJ) JK_TRY(join_jstream(h, st));
    return JK_OK;
}

// ---------------------------------------------------------------------------
// The split adjoint
// ---------------------------------------------------------------------------
namespace {

// AG[(p, mu)][col] for one density: [U^p[mu][i] | Vp^p[mu][i] | c_{P0+p,s} X[mu][i]]
// at columns off, off + k, off + 2k (U, Vp laid out [mu][(p, i)]).
__global__ void pack_ag_kernel(double *AG, long long ldag, int off, const double *U, const double *Vp,
                               const double *X, const double *cps, int P0, int n, int k, int np) {
    const long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    const long long tot = static_cast<long long>(np) * n * k;
    if (e >= tot) return;
    const int i = static_cast<int>(e % k);
    const long long pm = e / k;
    const int mu = static_cast<int>(pm % n), p = static_cast<int>(pm / n);
    double *row = AG + pm * ldag + off;
    const long long uo = static_cast<long long>(mu) * np * k + static_cast<long long>(p) * k + i;
    row[i] = U ? U[uo] : 0.0;
    row[k + i] = Vp ? Vp[uo] : 0.0;
    row[2 * k + i] = cps ? cps[P0 + p] * X[static_cast<long long>(mu) * k + i] : 0.0;
}

// BG[nu][col] = [X[nu][i] | Y[nu][i] | Y[nu][i]] at off, off + k, off + 2k.
__global__ void pack_bg_kernel(double *BG, long long ldbg, int off, const double *X, const double *Y, int n, int k) {
    const long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (e >= static_cast<long long>(n) * k) return;
    const int nu = static_cast<int>(e / k), i = static_cast<int>(e % k);
    double *row = BG + static_cast<long long>(nu) * ldbg + off;
    row[i] = X[e];
    row[k + i] = Y[e];
    row[2 * k + i] = Y[e];
}

// dL^{P0+p} = (G^p + G^p^T)/2 + (GV^p + GV^p^T)/2   (GV may be NULL)
__global__ void sym_dl_kernel(const double *G, const double *GV, int n, double *dL) {
    const long long n2 = static_cast<long long>(n) * n;
    const long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    const int p = blockIdx.y;
    if (e >= n2) return;
    const int mu = static_cast<int>(e / n), nu = static_cast<int>(e % n);
    const long long t = static_cast<long long>(nu) * n + mu;
    const double *Gp = G + p * n2;
    double v = 0.5 * (Gp[e] + Gp[t]);
    if (GV) {
        const double *Vp = GV + p * n2;
        v += 0.5 * (Vp[e] + Vp[t]);
    }
    dL[p * n2 + e] = v;
}

__global__ void fold_sym_split_kernel(double *dX, double *dY, long long cnt) {
    const long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (e >= cnt) return;
    dX[e] += dY[e];
    dY[e] = 0.0;
}

}  // namespace

jk_status fp64_frob_all(jk_ctx *h, const double *L, int n, int naux, const double *Mats, int nd, double *out,
                        cudaStream_t st, bool pk);
jk_status fp64_jstream_dense(jk_ctx *h, const double *L, int n, int naux, const double *g, int nd, double *out,
                             cudaStream_t st, bool pk);
jk_status fp64_gemm_nt(jk_ctx *h, int M, int N, int K, const double *A, long long a_sr, long long a_sk,
                       const double *B, long long b_sr, long long b_sk, double *C, long long ldc, double beta,
                       cudaStream_t st);

// out (+)= A B^T on sliced operands, FP64 out with row stride ldo.  Uses P (int64
// partials) when K spans several super-chunks, else tmp when accumulating.
static jk_status gemm_into(jk_ctx *h, const Sliced &A, const Sliced &B, double *out, long long ldo, bool accumulate,
                           long long *P, double *tmp, cudaStream_t st) {
    const int ns = nsuper_of(A.K);
    if (ns > 1) {
        JK_TRY(ozgemm(h, A, B, nullptr, 0, P, st));
        return reduce_partials(h, P, ns, A, B, out, ldo, accumulate, st);
    }
    if (!accumulate) return ozgemm(h, A, B, out, ldo, nullptr, st);
    if (ldo != B.rows) return set_error(h, JK_ERR_ARG, "internal: accumulate needs packed output");
    JK_TRY(ozgemm(h, A, B, tmp, B.rows, nullptr, st));
    return fp64_axpy(h, out, tmp, static_cast<long long>(A.rows) * B.rows, st);
}

// ---------------------------------------------------------------------------
// Dense densities on the split engine
// ---------------------------------------------------------------------------
// K_s = sum_P (L^P DK_s)(L^P)^T.  Per aux chunk: the panels
// T[(p, mu)][s*n + nu] = (L^p DK_s)[mu][nu] in one sliced GEMM (A = the L
// chunk, B = the rows (s, nu) of DK^T, sliced straight from DK), then per
// density the reduction over (p, nu) of T against L itself, sliced once per
// chunk with rows sig and reduction index (p, nu) (the layout the adjoint
// uses for dX).  J on the FP64 streams of the aux stream, overlapped.

// Aux indices per chunk: the per-index workspace (three sliced n x n blocks
// and one FP64 panel row block) within ~12 GB, panel rows within the grid.
static int dense_pchunk(const DenseProb &dp) {
    const size_t n = dp.n;
    const size_t per = n * n * (6 * 2) * 3 + n * even_ld(static_cast<long long>(dp.nd) * dp.n) * 8 +
                       (dp.packed ? n * n * 8 : 0);     // the expanded chunk of a packed factor
    size_t pc = per ? (static_cast<size_t>(12) << 30) / per : 1;
    if (pc < 1) pc = 1;
    if (dp.aux_chunk > 0) pc = dp.aux_chunk;
    if (pc > static_cast<size_t>(dp.naux)) pc = dp.naux;
    const size_t maxrows = static_cast<size_t>(65535) * oz::BM;
    if (pc * n > maxrows) pc = maxrows / n;
    return static_cast<int>(pc);
}

static size_t dense_partials(const DenseProb &dp, int pc) {
    const int ns = nsuper_of(pc * dp.n);
    return ns > 1 ? static_cast<size_t>(ns) * part_rows(dp.n) * even_ld(dp.n) : 1;
}

size_t split_dense_workspace(const DenseProb &dp) {
    const size_t n2 = static_cast<size_t>(dp.n) * dp.n, nd = dp.nd;
    size_t b = 0;
    if (dp.DJ) {
        b += align_up(nd * dp.naux * 8);                                  // gamma
        if (dp.add_j) b += align_up(nd * n2 * 8);                         // J before it joins K
    }
    if (dp.DK) {
        const int pc = dense_pchunk(dp), n = dp.n, ctot = dp.nd * dp.n;
        const long long ldT = even_ld(ctot);
        b += sliced_bytes(pc * n, n, n);                                  // L chunk, panel operand
        b += sliced_bytes(ctot, n, 1);                                    // rows (s, nu) of DK^T
        b += align_up(static_cast<size_t>(pc) * n * ldT * 8);             // FP64 panels T
        b += sliced_bytes(n, pc * n, 1);                                  // L chunk, rows sig
        b += sliced_bytes(n, pc * n, 1);                                  // one density's panels, rows mu
        b += align_up(dense_partials(dp, pc) * 8);                        // split-K partials
        b += align_up(n2 * 8);                                            // a chunk's K before it is added
        if (n > oz::SUPER)
            b += align_up(static_cast<size_t>(nsuper_of(n)) * part_rows(static_cast<long long>(pc) * n) * ldT * 8);
        if (dp.packed) b += align_up(static_cast<size_t>(pc) * n2 * 8);  // expanded factor chunk
    }
    return b;
}

jk_status split_dense(jk_ctx *h, const DenseProb &dp, cudaStream_t st) {
    const int n = dp.n, naux = dp.naux, nd = dp.nd;
    const long long n2 = static_cast<long long>(n) * n;
    Arena &ar = h->arena;
    double *gamma = nullptr, *Jt = nullptr;
    if (dp.DJ) {
        gamma = ar.take<double>(static_cast<size_t>(nd) * naux);
        if (dp.add_j) Jt = ar.take<double>(static_cast<size_t>(nd) * n2);
        if (!gamma || (dp.add_j && !Jt)) return set_error(h, JK_ERR_OOM, "workspace too small for the dense J");
    }
    const int pc = dp.DK ? dense_pchunk(dp) : 0, ctot = nd * n;
    const long long ldT = even_ld(ctot);
    Sliced Ls, Ds, LB, TS;
    double *T = nullptr, *tmp = nullptr, *Lx = nullptr;
    long long *Pbuf = nullptr, *Ppanel = nullptr;
    if (dp.DK) {
        bool ok = take_sliced(ar, pc * n, n, n, Ls) && take_sliced(ar, ctot, n, 1, Ds);
        T = ar.take<double>(static_cast<size_t>(pc) * n * ldT);
        ok = ok && T && take_sliced(ar, n, pc * n, 1, LB) && take_sliced(ar, n, pc * n, 1, TS);
        Pbuf = ar.take<long long>(dense_partials(dp, pc));
        tmp = ar.take<double>(static_cast<size_t>(n2));
        if (n > oz::SUPER)
            Ppanel = ar.take<long long>(static_cast<size_t>(nsuper_of(n)) * part_rows(static_cast<long long>(pc) * n) *
                                        ldT);
        if (dp.packed) Lx = ar.take<double>(static_cast<size_t>(pc) * n2);
        if (!ok || !Pbuf || !tmp || (n > oz::SUPER && !Ppanel) || (dp.packed && !Lx))
            return set_error(h, JK_ERR_OOM, "workspace too small for the dense split build");
    }
    if (dp.DJ) {
        JK_TRY(fork_jstream(h, st));
        JK_TRY(fp64_frob_all(h, dp.L, n, naux, dp.DJ, nd, gamma, h->aux_stream, dp.packed));
        JK_TRY(fp64_jstream_dense(h, dp.L, n, naux, gamma, nd, dp.add_j ? Jt : dp.J, h->aux_stream, dp.packed));
    }
    if (dp.DK) {
        // rows (s, nu) of DK^T, reduction over lam: element DK_s[lam][nu]
        oz::Src dsrc{dp.DK, n2, 0, n, n, n, 1};
        JK_TRY(slice_operand(h, dsrc, ctot, n, 1, Ds, st));
        for (int P0 = 0; P0 < naux; P0 += pc) {
            const int np = naux - P0 < pc ? naux - P0 : pc;
            // a packed factor chunk is expanded first
            if (dp.packed) JK_TRY(fp64_unpack_sym(h, dp.L + P0 * packed::tri_count(n), n, np, Lx, st));
            const double *Lchunk = dp.packed ? Lx : dp.L + P0 * n2;
            oz::Src lsrc{Lchunk, n, 0, 1, n};
            JK_TRY(slice_operand(h, lsrc, np * n, n, n, Ls, st));
            // T[(p, mu)][s*n + nu] = sum_lam L^p[mu][lam] DK_s[lam][nu]
            if (n > oz::SUPER) {
                JK_TRY(ozgemm(h, Ls, Ds, nullptr, 0, Ppanel, st));
                JK_TRY(reduce_partials(h, Ppanel, nsuper_of(n), Ls, Ds, T, ldT, false, st));
            } else {
                JK_TRY(ozgemm(h, Ls, Ds, T, ldT, nullptr, st));
            }
            // L with rows sig and reduction over (p, nu)
            oz::Src lm{Lchunk, n, n2, 1, n};
            JK_TRY(slice_operand(h, lm, n, np * n, 1, LB, st));
            for (int s = 0; s < nd; s++) {
                // rows mu, reduction over (p, nu): T[(p, mu)][s*n + nu]
                oz::Src ts{T + static_cast<long long>(s) * n, ldT, static_cast<long long>(n) * ldT, 1, n};
                JK_TRY(slice_operand(h, ts, n, np * n, 1, TS, st));
                // K_s (+)= sum_{p, nu} T[(p, mu)][s*n + nu] L^p[sig][nu]
                JK_TRY(gemm_into(h, TS, LB, dp.K + s * n2, n, P0 > 0, Pbuf, tmp, st));
            }
        }
    }
    if (dp.DJ) {
        JK_TRY(join_jstream(h, st));
        if (dp.add_j) JK_TRY(fp64_axpy(h, dp.K, Jt, static_cast<long long>(nd) * n2, st));
    }
    return JK_OK;
}

// Aux-index chunk of the split adjoint so that its workspace stays near 8 GB.
static int split_adj_pchunk(const Problem &pb) {
    const size_t n = pb.n, ctot = pb.ctot, ks3 = 3 * static_cast<size_t>(pb.ksum);
    const size_t sb = 2 * static_cast<size_t>(pb.slices);   // bytes of one sliced element
    size_t per = n * n * sb * 2                  // L slices: panel layout and row-mu layout
                 + n * even_ld(ctot) * 8         // T
                 + 2 * pb.kmax * n * sb          // T_X, T_Y as B operands
                 + 2 * n * pb.kmax * 8 + pb.kmax * n * sb * 2   // U, Vp and their slices
                 + n * ks3 * (8 + sb)            // AG and its slices
                 + n * n * 8 * 2                 // G, GV
                 + (pb.packed ? n * n * 8 : 0);  // the expanded chunk of a packed factor
    size_t budget = static_cast<size_t>(8) << 30;
    size_t pc = per ? budget / per : 1;
    if (pc < 1) pc = 1;
    if (pb.aux_chunk > 0) pc = pb.aux_chunk;       // explicit chunk
    if (pc > static_cast<size_t>(pb.naux)) pc = pb.naux;
    size_t maxrows = static_cast<size_t>(65535) * oz::BM;
    if (pc * n > maxrows) pc = maxrows / n;
    return static_cast<int>(pc);
}

struct AdjBufs {
    double *Z, *T, *gam, *cps, *JV, *U, *Vp, *AG, *BG, *G, *GV, *tmp;
    double *Lx = nullptr;     // packed factor: the chunk expanded to [np][n][n]
    long long *P;
    Sliced Zs, Ls, Lm, Ws[kMaxDens], WTs[kMaxDens], TXb, TYb, Ub, Vpb, AGs, BGs, Gam, Vs;
};

static size_t adj_partials(const Problem &pb, int pc) {
    const size_t n = pb.n;
    size_t m = 0;
    // dX / dY over K = pc*n, and the panel when n > SUPER
    m = std::max<size_t>(m, static_cast<size_t>(nsuper_of(pc * pb.n)) * part_rows(n) * even_ld(pb.kmax));
    if (pb.n > oz::SUPER)
        m = std::max<size_t>(m, static_cast<size_t>(nsuper_of(pb.n)) * part_rows(static_cast<long long>(pc) * n) *
                                    even_ld(pb.ctot));
    return m ? m : 1;
}

static bool adj_take(Arena &ar, const Problem &pb, int pc, bool W, bool V, bool dl, AdjBufs &b) {
    const int n = pb.n, nd = pb.nd, kmax = pb.kmax, ks3 = 3 * pb.ksum;
    const int S = pb.slices;   // every product of the adjoint on S-slice operands
    const long long n2 = static_cast<long long>(n) * n;
    bool ok = true;
    auto tk = [&](auto *&ptr, size_t cnt) {
        using T = std::remove_reference_t<decltype(*ptr)>;
        ptr = ar.take<T>(cnt ? cnt : 1);
        ok = ok && ptr;
    };
    tk(b.Z, static_cast<size_t>(n) * pb.ctot);
    tk(b.T, static_cast<size_t>(pc) * n * even_ld(pb.ctot));
    tk(b.gam, static_cast<size_t>(nd) * pb.naux);
    tk(b.cps, static_cast<size_t>(nd) * pb.naux);
    tk(b.JV, V ? static_cast<size_t>(nd) * n2 : 1);
    tk(b.U, static_cast<size_t>(n) * pc * kmax);
    tk(b.Vp, static_cast<size_t>(n) * pc * kmax);
    tk(b.AG, dl ? static_cast<size_t>(pc) * n * ks3 : 1);
    tk(b.BG, dl ? static_cast<size_t>(n) * ks3 : 1);
    tk(b.G, dl ? static_cast<size_t>(pc) * n2 : 1);
    tk(b.GV, dl && V ? static_cast<size_t>(pc) * n2 : 1);
    tk(b.tmp, static_cast<size_t>(n) * std::max(kmax, 1));
    tk(b.P, adj_partials(pb, pc));
    if (pb.packed) tk(b.Lx, static_cast<size_t>(pc) * n2);
    ok = ok && take_sliced(ar, pb.ctot, n, 1, b.Zs, S) && take_sliced(ar, pc * n, n, n, b.Ls, S) &&
         take_sliced(ar, n, pc * n, 1, b.Lm, S);
    for (int s = 0; ok && W && s < nd; s++)
        ok = take_sliced(ar, n, n, 1, b.Ws[s], S) && take_sliced(ar, n, n, 1, b.WTs[s], S);
    ok = ok && take_sliced(ar, pc * kmax, n, 1, b.TXb, S) && take_sliced(ar, pc * kmax, n, 1, b.TYb, S) &&
         take_sliced(ar, kmax, pc * n, 1, b.Ub, S) && take_sliced(ar, kmax, pc * n, 1, b.Vpb, S);
    if (ok && dl) ok = take_sliced(ar, pc * n, ks3, 1, b.AGs, S) && take_sliced(ar, n, ks3, 1, b.BGs, S);
    if (ok && dl && V)
        ok = take_sliced(ar, pc, nd, 1, b.Gam, S) && take_sliced(ar, static_cast<int>(n2), nd, 1, b.Vs, S);
    return ok;
}

size_t split_adjoint_workspace(const Problem &pb, bool want_dl) {
    // Measure with a dry-run arena (no device memory touched).
    Arena ar;
    ar.base = reinterpret_cast<char *>(static_cast<uintptr_t>(1) << 40);
    ar.bytes = static_cast<size_t>(1) << 62;
    ar.reset(0);
    AdjBufs b;
    adj_take(ar, pb, split_adj_pchunk(pb), true, true, want_dl, b);
    return ar.high + 4096;
}

jk_status split_pack_z(jk_ctx *h, const Problem &pb, double *Z, cudaStream_t st);

// ---------------------------------------------------------------------------
// Batched split build: many molecules, grouped launches
// ---------------------------------------------------------------------------
namespace {

struct MolBufs {
    double *Z = nullptr, *gamma = nullptr;
    Sliced Zs;
    int pc = 0;
};

struct ItemBufs {
    int mol = 0, P0 = 0, np = 0;
    Sliced Ls, TX[kMaxDens], TY[kMaxDens];
    double *T = nullptr, *tmp = nullptr;
    long long *P = nullptr;
    double *Lx = nullptr;     // packed factor: the chunk expanded to [np][n][n]
};

size_t item_bytes(const Problem &pb, int pc) {
    const size_t n = pb.n;
    size_t b = sliced_bytes(pc * pb.n, pb.n, pb.n) + align_up(static_cast<size_t>(pc) * n * even_ld(pb.ctot) * 8);
    for (int s = 0; s < pb.nd; s++) {
        b += sliced_bytes(pb.n, pc * pb.k[s], 1);
        if (!pb.sym[s]) b += sliced_bytes(pb.n, pc * pb.k[s], 1);
    }
    b += align_up(partial_count(pb, pc) * 8 + 8);
    b += align_up(static_cast<size_t>(pb.nd) * n * n * 8);   // per-density tmp for chunk accumulation
    if (pb.packed) b += align_up(static_cast<size_t>(pc) * n * n * 8);   // expanded factor chunk
    return b + 16 * kArenaAlign;
}

size_t mol_bytes(const Problem &pb) {
    return align_up(static_cast<size_t>(pb.n) * pb.ctot * 8) + sliced_bytes(pb.ctot, pb.n, 1) +
           align_up(static_cast<size_t>(pb.nd) * pb.naux * 8) + 4 * kArenaAlign;
}

bool take_item(Arena &ar, const Problem &pb, int pc, ItemBufs &it) {
    const int n = pb.n;
    bool ok = take_sliced(ar, pc * n, n, n, it.Ls);
    it.T = ar.take<double>(static_cast<size_t>(pc) * n * even_ld(pb.ctot));
    ok = ok && it.T;
    for (int s = 0; ok && s < pb.nd; s++) {
        ok = take_sliced(ar, n, pc * pb.k[s], 1, it.TX[s]);
        if (ok && !pb.sym[s]) ok = take_sliced(ar, n, pc * pb.k[s], 1, it.TY[s]);
    }
    it.P = ar.take<long long>(partial_count(pb, pc) + 1);
    it.tmp = ar.take<double>(static_cast<size_t>(pb.nd) * n * n);
    if (pb.packed) it.Lx = ar.take<double>(static_cast<size_t>(pc) * n * n);
    return ok && it.P && it.tmp && (!pb.packed || it.Lx);
}

}  // namespace

size_t split_batched_workspace(int nmol, const Problem *pbs) {
    size_t mols = 0, maxitem = 0, items = 0;
    for (int m = 0; m < nmol; m++) {
        const Problem &pb = pbs[m];
        mols += mol_bytes(pb);
        const int pc = split_pchunk(pb);
        const size_t ib = item_bytes(pb, pc);
        maxitem = std::max(maxitem, ib);
        items += ib * ((pb.naux + pc - 1) / pc);
    }
    // enough for every molecule's persistent buffers and at least the largest
    // work item; more (up to everything, capped at 24 GB) lets waves hold more items
    const size_t cap = static_cast<size_t>(24) << 30;
    return mols + std::max(maxitem, std::min(items, cap));
}

jk_status split_batched(jk_ctx *h, int nmol, const Problem *pbs, cudaStream_t st) {
    Arena &ar = h->arena;
    std::vector<MolBufs> mb(nmol);
    // Persistent per-molecule buffers: packed Z and its slices, gamma.
    for (int m = 0; m < nmol; m++) {
        const Problem &pb = pbs[m];
        mb[m].Z = ar.take<double>(static_cast<size_t>(pb.n) * pb.ctot);
        mb[m].gamma = ar.take<double>(static_cast<size_t>(pb.nd) * pb.naux);
        if (!mb[m].Z || !mb[m].gamma || !take_sliced(ar, pb.ctot, pb.n, 1, mb[m].Zs))
            return set_error(h, JK_ERR_OOM, "workspace too small for the batched build");
        mb[m].pc = split_pchunk(pb);
    }
    {
        // every molecule's packed densities and their slices, in grouped launches
        std::vector<double *> zs(nmol);
        for (int m = 0; m < nmol; m++) zs[m] = mb[m].Z;
        JK_TRY(pack_z_multi(h, nmol, pbs, zs.data(), st));
        SliceBatch zb;
        for (int m = 0; m < nmol; m++) {
            oz::Src zsrc{mb[m].Z, 1, 0, pbs[m].ctot, pbs[m].n};
            if (h->slicer == 0) slice_add(zb, zsrc, pbs[m].ctot, pbs[m].n, 1, mb[m].Zs);
            else JK_TRY(slice_operand(h, zsrc, pbs[m].ctot, pbs[m].n, 1, mb[m].Zs, st));
        }
        JK_TRY(slice_flush(h, zb, st));
    }
    const size_t persist = ar.off;
    bool forked = false;   // J streams running on the second stream
    // Work items (molecule, aux chunk) in order.
    std::vector<std::pair<int, int>> work;
    for (int m = 0; m < nmol; m++)
        for (int P0 = 0; P0 < pbs[m].naux; P0 += mb[m].pc) work.push_back({m, P0});
    size_t w0 = 0;
    while (w0 < work.size()) {
        ar.reset(persist);
        std::vector<ItemBufs> items;
        std::vector<char> inwave(nmol, 0);
        size_t w1 = w0;
        while (w1 < work.size()) {
            const int m = work[w1].first;
            if (inwave[m]) break;                 // one chunk per molecule per wave
            const Problem &pb = pbs[m];
            const size_t save = ar.off;
            ItemBufs it;
            it.mol = m;
            it.P0 = work[w1].second;
            it.np = std::min(mb[m].pc, pb.naux - it.P0);
            if (!take_item(ar, pb, mb[m].pc, it)) {
                ar.off = save;
                break;
            }
            items.push_back(it);
            inwave[m] = 1;
            ++w1;
        }
        if (items.empty()) return set_error(h, JK_ERR_OOM, "workspace too small for one batched work item");
        // 1. slice the factor chunks (grouped launches, unless the FP32-digit
        // slicer is asked for: that one slices operand by operand)
        const bool grouped = h->slicer == 0;
        SliceBatch sb;
        for (auto &it : items) {
            const Problem &pb = pbs[it.mol];
            const long long n2 = static_cast<long long>(pb.n) * pb.n;
            if (pb.packed)
                JK_TRY(fp64_unpack_sym(h, pb.L + it.P0 * packed::tri_count(pb.n), pb.n, it.np, it.Lx, st));
            const double *Lc = pb.packed ? it.Lx : pb.L + it.P0 * n2;
            oz::Src lsrc{Lc, pb.n, 0, 1, pb.n};
            if (grouped) slice_add(sb, lsrc, it.np * pb.n, pb.n, pb.n, it.Ls);
            else JK_TRY(slice_operand(h, lsrc, it.np * pb.n, pb.n, pb.n, it.Ls, st));
        }
        JK_TRY(slice_flush(h, sb, st));
        // 2. all panels of the wave: grouped persistent launches
        std::vector<oz::OzProb> probs;
        for (auto &it : items) {
            const Problem &pb = pbs[it.mol];
            probs.emplace_back();
            if (pb.n > oz::SUPER) return set_error(h, JK_ERR_UNSUPPORTED, "batched build needs nbf <= 2048");
            JK_TRY(oz_problem(h, it.Ls, mb[it.mol].Zs, it.T, even_ld(pb.ctot), nullptr, probs.back()));
        }
        JK_TRY(oz_launch(h, probs, st));
        // 3. gamma; the J streams of molecules whose last chunk this is go to the
        // second stream; then the rank-update operands
        bool fork = false;
        for (auto &it : items) {
            const Problem &pb = pbs[it.mol];
            if (!pb.wantJ) continue;
            JK_TRY(fp64_gamma_panel(h, pb, it.T, even_ld(pb.ctot), it.np, mb[it.mol].gamma, it.P0, st));
            fork = fork || it.P0 + it.np >= pb.naux;
        }
        if (fork) {
            JK_TRY(fork_jstream(h, st));
            forked = true;
            for (auto &it : items)
                if (pbs[it.mol].wantJ && it.P0 + it.np >= pbs[it.mol].naux)
                    JK_TRY(fp64_jstream(h, pbs[it.mol], mb[it.mol].gamma, h->aux_stream));
        }
        for (auto &it : items) {
            const Problem &pb = pbs[it.mol];
            const long long ldT = even_ld(pb.ctot);
            if (!pb.wantK) continue;
            for (int s = 0; s < pb.nd; s++) {
                const int k = pb.k[s], Kr = it.np * k;
                oz::Src xs{it.T + pb.offX[s], ldT, static_cast<long long>(pb.n) * ldT, 1, k};
                if (grouped) slice_add(sb, xs, pb.n, Kr, 1, it.TX[s]);
                else JK_TRY(slice_operand(h, xs, pb.n, Kr, 1, it.TX[s], st));
                if (!pb.sym[s]) {
                    oz::Src ys{it.T + pb.offY[s], ldT, static_cast<long long>(pb.n) * ldT, 1, k};
                    if (grouped) slice_add(sb, ys, pb.n, Kr, 1, it.TY[s]);
                    else JK_TRY(slice_operand(h, ys, pb.n, Kr, 1, it.TY[s], st));
                }
            }
        }
        JK_TRY(slice_flush(h, sb, st));
        // 4. every rank update of the wave: grouped persistent launches
        probs.clear();
        struct Red { const ItemBufs *it; int s; long long *P; double *tmp; };
        std::vector<Red> reds;
        for (auto &it : items) {
            const Problem &pb = pbs[it.mol];
            if (!pb.wantK) continue;
            const long long n2 = static_cast<long long>(pb.n) * pb.n;
            long long *Pcur = it.P;
            for (int s = 0; s < pb.nd; s++) {
                const Sliced &B = pb.sym[s] ? it.TX[s] : it.TY[s];
                const int ns = nsuper_of(it.np * pb.k[s]);
                if (pb.sym[s] && h->syrk) {
                    // blocked symmetric rank update (mirrored after the last wave)
                    double *dst = it.P0 == 0 ? pb.K[s] : it.tmp + s * n2;
                    JK_TRY(sym_rank_problems(h, it.TX[s], pb.n, dst, Pcur, probs));
                    if (ns > 1) {
                        reds.push_back({&it, s, Pcur, nullptr});
                        Pcur += sym_partial_words(pb.n, ns);
                    } else if (it.P0 > 0) {
                        reds.push_back({&it, s, nullptr, dst});
                    }
                    continue;
                }
                probs.emplace_back();
                if (ns == 1) {
                    double *out = it.P0 == 0 ? pb.K[s] : it.tmp + s * n2;
                    JK_TRY(oz_problem(h, it.TX[s], B, out, pb.n, nullptr, probs.back()));
                    if (it.P0 > 0) reds.push_back({&it, s, nullptr, it.tmp + s * n2});
                } else {
                    JK_TRY(oz_problem(h, it.TX[s], B, nullptr, 0, Pcur, probs.back()));
                    reds.push_back({&it, s, Pcur, nullptr});
                    Pcur += static_cast<size_t>(ns) * part_rows(pb.n) * even_ld(pb.n);
                }
            }
        }
        JK_TRY(oz_launch(h, probs, st));
        // 5. reductions into K (the split-K ones in grouped launches)
        ReduceBatch rb;
        for (auto &r : reds) {
            const Problem &pb = pbs[r.it->mol];
            const long long n2 = static_cast<long long>(pb.n) * pb.n;
            const Sliced &B = pb.sym[r.s] ? r.it->TX[r.s] : r.it->TY[r.s];
            if (r.P && pb.sym[r.s] && h->syrk) {
                JK_TRY(sym_rank_reduce(h, r.it->TX[r.s], pb.n, r.P, pb.K[r.s], r.it->P0 > 0, st));
            } else if (r.P) {
                reduce_add(rb, r.P, nsuper_of(r.it->np * pb.k[r.s]), r.it->TX[r.s], B, pb.K[r.s], pb.n,
                           r.it->P0 > 0);
            } else {
                JK_TRY(fp64_axpy(h, pb.K[r.s], r.tmp, n2, st));
            }
        }
        JK_TRY(reduce_flush(h, rb, st));
        w0 = w1;
    }
    if (h->syrk)
        for (int m = 0; m < nmol; m++)
            if (pbs[m].wantK)
                for (int s = 0; s < pbs[m].nd; s++)
                    if (pbs[m].sym[s]) JK_TRY(mirror_sym_blocks(h, pbs[m].K[s], pbs[m].n, st));
    if (forked) JK_TRY(join_jstream(h, st));
    return JK_OK;
}

jk_status split_adjoint(jk_ctx *h, const Problem &pb, const double *W, const double *V, double *dX, double *dY,
                        double *dL, cudaStream_t st) {
    const int n = pb.n, naux = pb.naux, nd = pb.nd;
    const long long n2 = static_cast<long long>(n) * n;
    const int pc = split_adj_pchunk(pb);
    const bool wantW = W != nullptr, wantV = V != nullptr, wantL = dL != nullptr;
    AdjBufs b;
    if (!adj_take(h->arena, pb, pc, wantW, wantV, wantL, b))
        return set_error(h, JK_ERR_OOM, "workspace too small for the split adjoint");
    const long long ldT = even_ld(pb.ctot);
    const int ks3 = 3 * pb.ksum;

    long long boff[kMaxDens + 1];
    boff[0] = 0;
    for (int s = 0; s < nd; s++) boff[s + 1] = boff[s] + static_cast<long long>(n) * pb.k[s];
    JK_CUDA_TRY(h, cudaMemsetAsync(dX, 0, boff[nd] * sizeof(double), st));
    JK_CUDA_TRY(h, cudaMemsetAsync(dY, 0, boff[nd] * sizeof(double), st));

    JK_TRY(split_pack_z(h, pb, b.Z, st));
    oz::Src zsrc{b.Z, 1, 0, pb.ctot, n};
    JK_TRY(slice_operand(h, zsrc, pb.ctot, n, 1, b.Zs, st));
    if (wantV) {
        // c_{P,s} = <V_s, L^P> and J(V_s) = sum_P c_{P,s} L^P in FP64
        JK_TRY(fp64_frob_all(h, pb.L, n, naux, V, nd, b.cps, st, pb.packed));
        JK_TRY(fp64_jstream_dense(h, pb.L, n, naux, b.cps, nd, b.JV, st, pb.packed));
    }
    if (wantW) {
        for (int s = 0; s < nd; s++) {
            const double *Wsd = W + s * n2;
            oz::Src ws{Wsd, n, 0, 1, n};          // rows mu, K = lam: W[mu][lam]
            oz::Src wt{Wsd, 1, 0, n, n};          // rows mu, K = lam: W[lam][mu]
            JK_TRY(slice_operand(h, ws, n, n, 1, b.Ws[s], st));
            JK_TRY(slice_operand(h, wt, n, n, 1, b.WTs[s], st));
        }
    }
    if (wantL) {
        int off = 0;
        for (int s = 0; s < nd; s++) {
            const int k = pb.k[s];
            const double *Ys = pb.sym[s] ? pb.X[s] : pb.Y[s];
            {
                LaunchScope ls(h, KK_PACK, st);
                pack_bg_kernel<<<static_cast<unsigned>((static_cast<long long>(n) * k + 255) / 256), 256, 0, st>>>(
                    b.BG, ks3, off, pb.X[s], Ys, n, k);
            }
            JK_LAUNCH_CHECK(h);
            off += 3 * k;
        }
        oz::Src bgs{b.BG, ks3, 0, 1, ks3};
        JK_TRY(slice_operand(h, bgs, n, ks3, 1, b.BGs, st));
        if (wantV) {
            oz::Src vsrc{V, 1, 0, n2, nd};        // rows (mu nu), K = s: V[s][mu nu]
            JK_TRY(slice_operand(h, vsrc, static_cast<int>(n2), nd, 1, b.Vs, st));
        }
    }

    for (int P0 = 0; P0 < naux; P0 += pc) {
        const int np = naux - P0 < pc ? naux - P0 : pc;
        // a packed factor chunk is expanded first
        if (pb.packed) JK_TRY(fp64_unpack_sym(h, pb.L + P0 * packed::tri_count(n), n, np, b.Lx, st));
        const double *Lchunk = pb.packed ? b.Lx : pb.L + P0 * n2;
        // Panels T^p = L^p Z (the half-transforms), as in the build
        oz::Src lsrc{Lchunk, n, 0, 1, n};
        JK_TRY(slice_operand(h, lsrc, np * n, n, n, b.Ls, st));
        if (n > oz::SUPER) {
            JK_TRY(ozgemm(h, b.Ls, b.Zs, nullptr, 0, b.P, st));
            JK_TRY(reduce_partials(h, b.P, nsuper_of(n), b.Ls, b.Zs, b.T, ldT, false, st));
        } else {
            JK_TRY(ozgemm(h, b.Ls, b.Zs, b.T, ldT, nullptr, st));
        }
        if (wantV && wantL) JK_TRY(fp64_gamma_panel(h, pb, b.T, ldT, np, b.gam, P0, st));
        if (wantW) {
            // L with rows mu and reduction over (p, lam), for dX and dY
            oz::Src lm{Lchunk, n, n2, 1, n};
            JK_TRY(slice_operand(h, lm, n, np * n, 1, b.Lm, st));
        }
        for (int s = 0; s < nd; s++) {
            const int k = pb.k[s];
            const long long npk = static_cast<long long>(np) * k;
            if (wantW) {
                // U_s = W_s T_Y^T, Vp_s = W_s^T T_X^T: rows mu, columns (p, i)
                oz::Src ty{b.T + pb.offY[s], static_cast<long long>(n) * ldT, 0, ldT, n, k, 1};
                oz::Src tx{b.T + pb.offX[s], static_cast<long long>(n) * ldT, 0, ldT, n, k, 1};
                JK_TRY(slice_operand(h, ty, static_cast<int>(npk), n, 1, b.TYb, st));
                JK_TRY(slice_operand(h, tx, static_cast<int>(npk), n, 1, b.TXb, st));
                JK_TRY(ozgemm(h, b.Ws[s], b.TYb, b.U, npk, nullptr, st));
                JK_TRY(ozgemm(h, b.WTs[s], b.TXb, b.Vp, npk, nullptr, st));
                // dX_s += sum_{p,lam} L^p[mu][lam] U[lam][(p,i)] ; dY_s likewise with Vp
                oz::Src us{b.U, 1, k, npk, n};
                oz::Src vs{b.Vp, 1, k, npk, n};
                JK_TRY(slice_operand(h, us, k, np * n, 1, b.Ub, st));
                JK_TRY(slice_operand(h, vs, k, np * n, 1, b.Vpb, st));
                JK_TRY(gemm_into(h, b.Lm, b.Ub, dX + boff[s], k, P0 > 0, b.P, b.tmp, st));
                JK_TRY(gemm_into(h, b.Lm, b.Vpb, dY + boff[s], k, P0 > 0, b.P, b.tmp, st));
            }
            if (wantL) {
                int off = 0;
                for (int t = 0; t < s; t++) off += 3 * pb.k[t];
                {
                    LaunchScope ls(h, KK_PACK, st);
                    pack_ag_kernel<<<static_cast<unsigned>((static_cast<long long>(np) * n * k + 255) / 256), 256, 0,
                                     st>>>(b.AG, ks3, off, wantW ? b.U : nullptr, wantW ? b.Vp : nullptr, pb.X[s],
                                           wantV ? b.cps + static_cast<long long>(s) * naux : nullptr, P0, n, k, np);
                }
                JK_LAUNCH_CHECK(h);
            }
        }
        if (wantL) {
            // G[(p,mu)][nu] = sum_s U X^T + Vp Y^T + c X Y^T  (sym(Vp Y^T) = sym(Y Vp^T))
            oz::Src ags{b.AG, ks3, 0, 1, ks3};
            JK_TRY(slice_operand(h, ags, np * n, ks3, 1, b.AGs, st));
            JK_TRY(ozgemm(h, b.AGs, b.BGs, b.G, n, nullptr, st));
            const double *GV = nullptr;
            if (wantV) {
                // GV[p][(mu nu)] = sum_s gamma_{P0+p,s} V_s[mu nu]
                oz::Src gsrc{b.gam + P0, 1, 0, naux, nd};
                JK_TRY(slice_operand(h, gsrc, np, nd, 1, b.Gam, st));
                JK_TRY(ozgemm(h, b.Gam, b.Vs, b.GV, n2, nullptr, st));
                GV = b.GV;
            }
            {
                LaunchScope ls(h, KK_MISC, st);
                sym_dl_kernel<<<dim3(static_cast<unsigned>((n2 + 255) / 256), np), 256, 0, st>>>(b.G, GV, n,
                                                                                                 dL + P0 * n2);
            }
            JK_LAUNCH_CHECK(h);
        }
    }
    if (wantV) {
        // dX_s += J(V_s) Y_s, dY_s += J(V_s) X_s: small (n x n by n x k) FP64 products,
        // so every J term of the adjoint stays in FP64 end to end.
        for (int s = 0; s < nd; s++) {
            const int k = pb.k[s];
            const double *Ys = pb.sym[s] ? pb.X[s] : pb.Y[s];
            JK_TRY(fp64_gemm_nt(h, n, k, n, b.JV + s * n2, n, 1, Ys, 1, k, dX + boff[s], k, 1.0, st));
            JK_TRY(fp64_gemm_nt(h, n, k, n, b.JV + s * n2, n, 1, pb.X[s], 1, k, dY + boff[s], k, 1.0, st));
        }
    }
    for (int s = 0; s < nd; s++) {
        if (!pb.sym[s]) continue;
        const long long cnt = boff[s + 1] - boff[s];
        LaunchScope ls(h, KK_MISC, st);
        fold_sym_split_kernel<<<static_cast<unsigned>((cnt + 255) / 256), 256, 0, st>>>(dX + boff[s], dY + boff[s], cnt);
        JK_LAUNCH_CHECK(h);
    }
    return JK_OK;
}

}  // namespace jk

// ---------------------------------------------------------------------------
// Test hook: the sliced tensor-core GEMM on its own (see include/jk_debug.h).
// ---------------------------------------------------------------------------
namespace jk {
// C = A B^T through the split path with S-slice operands (the test hooks below).
static jk_status debug_sliced_gemm(jk_handle h, int M, int N, int K, const double *A, const double *B, double *C,
                                   int S, cudaStream_t st) {
    if (!h) return JK_ERR_ARG;
    if (M < 1 || N < 1 || K < 1) return set_error(h, JK_ERR_SHAPE, "M, N, K must be >= 1");
    if (!A || !B || !C) return set_error(h, JK_ERR_ARG, "NULL operand");
    if (S != 6 && S != 7) return set_error(h, JK_ERR_ARG, "slices must be 6 or 7");
    h->arena.reset(align_up(sizeof(DeviceFlags)));
    // tile order and width: the handle's explicit options, else the defaults
    h->cur_raster = h->raster >= 0 ? h->raster : 0;
    h->cur_tile = h->tile >= 0 ? h->tile : 0;
    Sliced As, Bs;
    if (!take_sliced(h->arena, M, K, 1, As, S) || !take_sliced(h->arena, N, K, 1, Bs, S))
        return set_error(h, JK_ERR_OOM, "workspace too small");
    const int ns = nsuper_of(K);
    long long *P = nullptr;
    if (ns > 1) {
        P = h->arena.take<long long>(static_cast<size_t>(ns) * part_rows(M) * even_ld(N));
        if (!P) return set_error(h, JK_ERR_OOM, "workspace too small");
    }
    oz::Src sa{A, K, 0, 1, K}, sb{B, K, 0, 1, K};
    JK_TRY(slice_operand(h, sa, M, K, 1, As, st));
    JK_TRY(slice_operand(h, sb, N, K, 1, Bs, st));
    if (ns == 1) return ozgemm(h, As, Bs, C, N, nullptr, st);
    JK_TRY(ozgemm(h, As, Bs, nullptr, 0, P, st));
    return reduce_partials(h, P, ns, As, Bs, C, N, false, st);
}

static size_t debug_sliced_gemm_workspace(int M, int N, int K, int S) {
    size_t b = align_up(sizeof(DeviceFlags)) + sliced_bytes(M, K, 1, S) + sliced_bytes(N, K, 1, S);
    const int ns = nsuper_of(K);
    if (ns > 1) b += align_up(static_cast<size_t>(ns) * part_rows(M) * even_ld(N) * 8);
    return b + kArenaAlign;
}
}  // namespace jk

extern "C" jk_status jk_debug_sliced_gemm(jk_handle h, int32_t M, int32_t N, int32_t K, const double *A,
                                          const double *B, double *C, void *stream) {
    return jk::debug_sliced_gemm(h, M, N, K, A, B, C, 6, static_cast<cudaStream_t>(stream));
}

extern "C" size_t jk_debug_sliced_gemm_workspace(int32_t M, int32_t N, int32_t K) {
    return jk::debug_sliced_gemm_workspace(M, N, K, 6);
}

extern "C" jk_status jk_debug_sliced_gemm_slices(jk_handle h, int32_t M, int32_t N, int32_t K, const double *A,
                                                 const double *B, double *C, int32_t slices, void *stream) {
    return jk::debug_sliced_gemm(h, M, N, K, A, B, C, slices, static_cast<cudaStream_t>(stream));
}

extern "C" size_t jk_debug_sliced_gemm_workspace_slices(int32_t M, int32_t N, int32_t K, int32_t slices) {
    return jk::debug_sliced_gemm_workspace(M, N, K, slices == 7 ? 7 : 6);
}

namespace jk {
namespace oz {
// One thread waits on phase 0 of an mbarrier that nothing arrives on; the
// bounded wait gives up after tc::kWaitTimeoutNs and the kernel reports it.
__global__ void wait_timeout_kernel(int *err) {
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        abort_flag = 0;
        tc::fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !tc::mbar_wait(&bar, 0u, &abort_flag))
        atomicExch(err, static_cast<int>(JK_ERR_TIMEOUT));
}
}  // namespace oz
}  // namespace jk

extern "C" jk_status jk_debug_wait_timeout(jk_handle h, void *stream) {
    using namespace jk;
    if (!h) return JK_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    {
        LaunchScope ls(h, KK_MISC, st);
        oz::wait_timeout_kernel<<<1, 32, 0, st>>>(&h->flags->error);
    }
    JK_LAUNCH_CHECK(h);
    return JK_OK;
}
