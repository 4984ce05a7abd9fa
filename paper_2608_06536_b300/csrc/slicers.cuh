// Slicers of the split-precision engine: FP64 operands to S BF16 digit
// planes under a per-row (per super-chunk) power-of-two scale, one operand per
// launch or many operands per grouped launch.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "digits.cuh"
#include "fixed.cuh"
#include "ozcfg.cuh"

namespace jk {
namespace oz {

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

// max|x| bits over one row's reduction indices kk in [k0, k1) (k1 - k0 <=
// SUPER), for a block of 256 threads: thread t takes kk = k0 + t + 256 i.  The
// (ko, ki) split of kk is advanced incrementally (no integer division in the
// loop) and all of a thread's addresses are formed before any load, so its
// SUPER / 256 loads are in flight together.
__device__ __forceinline__ unsigned long long row_chunk_max(const double *row, const Src &src, int k0, int k1) {
    constexpr int U = SUPER / 256;
    const int step_o = 256 / src.kin, step_i = 256 % src.kin;
    int ko = (k0 + static_cast<int>(threadIdx.x)) / src.kin, ki = k0 + static_cast<int>(threadIdx.x) - ko * src.kin;
    long long off[U];
#pragma unroll
    for (int i = 0; i < U; i++) {
        off[i] = static_cast<long long>(ko) * src.sko + static_cast<long long>(ki) * src.ski;
        ko += step_o;
        ki += step_i;
        if (ki >= src.kin) { ki -= src.kin; ko++; }
    }
    unsigned long long v[U];
#pragma unroll
    for (int i = 0; i < U; i++)
        v[i] = k0 + static_cast<int>(threadIdx.x) + 256 * i < k1
                   ? static_cast<unsigned long long>(__double_as_longlong(row[off[i]])) & 0x7FFFFFFFFFFFFFFFull
                   : 0ull;
    unsigned long long mx = 0;
#pragma unroll
    for (int i = 0; i < U; i++) mx = v[i] > mx ? v[i] : mx;
    return mx;
}

// max|x| bits over a contiguous run of len doubles (p 16-byte aligned, len
// even), for a block of 256 threads: four 16-byte loads in flight per thread.
__device__ __forceinline__ unsigned long long run_max(const double *p, long long len) {
    const double2 *q = reinterpret_cast<const double2 *>(p);
    const long long n2 = len / 2;
    unsigned long long mx = 0;
    for (long long t = threadIdx.x; t < n2; t += 4 * 256) {
        double2 v[4];
#pragma unroll
        for (int i = 0; i < 4; i++) v[i] = t + 256 * i < n2 ? q[t + 256 * i] : make_double2(0.0, 0.0);
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const unsigned long long a = static_cast<unsigned long long>(__double_as_longlong(v[i].x)) & 0x7FFFFFFFFFFFFFFFull;
            const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(v[i].y)) & 0x7FFFFFFFFFFFFFFFull;
            mx = a > mx ? a : mx;
            mx = b > mx ? b : mx;
        }
    }
    return mx;
}

// e[g * gridDim.y + z] for row groups g of `rpe` rows and super-chunks z of
// the reduction index: max|x| over the group's rows and kk in
// [z*SUPER, (z+1)*SUPER).
__global__ void __launch_bounds__(256) expo_kernel(Src src, int rows, int K, int rpe, int *e) {
    __shared__ unsigned long long red[8];
    const int g = blockIdx.x, z = blockIdx.y;
    const int r0 = g * rpe, r1 = min(rows, r0 + rpe);
    const int k0 = z * SUPER, k1 = min(K, k0 + SUPER);
    unsigned long long mx = 0;
    for (int r = r0; r < r1; r++) {
        const unsigned long long m = row_chunk_max(src_row(src, r), src, k0, k1);
        mx = m > mx ? m : mx;
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
    unsigned long long mx = run_max(p + blockIdx.x * len, len);
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
        mx = run_max(jb.src.p + lb * len, len);
        slot = lb;
    } else {
        const Src src = jb.src;
        const int gi = lb / jb.nsc, z = lb - gi * jb.nsc;
        const int r0 = gi * jb.rpe, r1 = min(jb.rows, r0 + jb.rpe);
        const int k0 = z * SUPER, k1 = min(jb.K, k0 + SUPER);
        for (int r = r0; r < r1; r++) {
            const unsigned long long m = row_chunk_max(src_row(src, r), src, k0, k1);
            mx = m > mx ? m : mx;
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
// Exponents of the rank-update operands taken from a panel
// ---------------------------------------------------------------------------
// The split build cuts each density's rank-update operands T_X, T_Y (rows mu,
// reduction index (p, j)) out of the panel T (rows (p, mu), one column per
// column of X_s or Y_s).  Their exponent groups (row mu, super-chunk z of
// (p, j)) gather 100-element runs from rows far apart, which a per-group
// exponent pass reads as scattered short pieces.  Instead, one block reads
// one whole T row (contiguous) and each warp folds one operand's columns into
// that operand's exponents by an atomic maximum: exponents are monotone in
// |x|, so the maximum of per-element exponents is the exponent of the
// maximum, and -1000 (an all-zero group) is the neutral start.
struct PanelSeg {
    int *e;          // the operand's exponents, e[mu * nsc + z]
    int c0, k, nsc;  // its columns c0 .. c0 + k - 1 of T; super-chunks per row
    int n;           // rows mu per p of its panel
};
struct PanelItem {   // one panel: its rows (p, mu) and its operands' segments
    const double *T;
    long long ldT;
    int n, rows;
    int seg0, nseg;  // segments seg0 .. seg0 + nseg - 1
    int b0;          // first block of this panel in the launch (one block per row)
};
constexpr int MAXPITEM = 64;
constexpr int MAXSEG = 800;
struct PanelExpo {
    int nitem;
    int nseg;
    PanelItem it[MAXPITEM];
    PanelSeg s[MAXSEG];
};

// Every segment's exponents set to -1000 (blockIdx.y = segment).
__global__ void __launch_bounds__(256) int_fill_kernel(const __grid_constant__ PanelExpo g) {
    const PanelSeg &sg = g.s[blockIdx.y];
    const int cnt = sg.n * sg.nsc;
    for (int i = blockIdx.x * 256 + threadIdx.x; i < cnt; i += gridDim.x * 256) sg.e[i] = -1000;
}

// One block per panel row r = p * n + mu; warp w takes the panel's segments
// w, w + 8, ...
__global__ void __launch_bounds__(256) panel_colmax_kernel(const __grid_constant__ PanelExpo g) {
    int lo = 0, hi = g.nitem - 1;
    while (lo < hi) {   // the last panel whose first block is <= blockIdx.x
        const int mid = (lo + hi + 1) >> 1;
        if (g.it[mid].b0 <= static_cast<int>(blockIdx.x)) lo = mid;
        else hi = mid - 1;
    }
    const PanelItem &pi = g.it[lo];
    const int r = static_cast<int>(blockIdx.x) - pi.b0;
    const int p = r / pi.n, mu = r - p * pi.n;
    const double *row = pi.T + static_cast<long long>(r) * pi.ldT;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int si = pi.seg0 + warp; si < pi.seg0 + pi.nseg; si += 8) {
        const PanelSeg &sg = g.s[si];
        const int kk0 = p * sg.k;            // reduction index of the run's first element
        const int z0 = kk0 / SUPER;
        const int jb = (z0 + 1) * SUPER - kk0;   // first j of the next super-chunk
        // the exponent needs only the upper word of |x| (sign cleared)
        unsigned m0 = 0, m1 = 0;
        for (int j = lane; j < sg.k; j += 32) {
            const unsigned hw = static_cast<unsigned>(__double2hiint(row[sg.c0 + j])) & 0x7FFFFFFFu;
            if (j < jb) m0 = hw > m0 ? hw : m0;
            else m1 = hw > m1 ? hw : m1;
        }
        m0 = __reduce_max_sync(0xffffffffu, m0);
        if (jb < sg.k) m1 = __reduce_max_sync(0xffffffffu, m1);
        if (lane == 0) {
            if (m0) atomicMax(&sg.e[mu * sg.nsc + z0], exponent_of_max(static_cast<unsigned long long>(m0) << 32));
            if (jb < sg.k && m1)
                atomicMax(&sg.e[mu * sg.nsc + z0 + 1], exponent_of_max(static_cast<unsigned long long>(m1) << 32));
        }
    }
}

}  // namespace oz
}  // namespace jk
