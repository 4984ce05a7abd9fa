// Slicers of the split-precision engine: FP64 operands to S BF16 digit
// planes under a per-row (per super-chunk) power-of-two scale, one operand per
// launch or many operands per grouped launch.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "digits.cuh"
#include "fixed.cuh"
#include "ozcfg.cuh"
#include "packed.cuh"

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

// max|x| bits over a contiguous run of len doubles (p 8-byte aligned), for a
// block of 256 threads: four 16-byte loads in flight per thread over the
// 16-byte aligned body, one scalar load for an unaligned first or odd last
// element.
__device__ __forceinline__ unsigned long long run_max(const double *p, long long len) {
    constexpr unsigned long long kAbs = 0x7FFFFFFFFFFFFFFFull;
    unsigned long long mx = 0;
    if (len <= 0) return mx;
    if (reinterpret_cast<uintptr_t>(p) & 15u) {
        if (threadIdx.x == 0) mx = static_cast<unsigned long long>(__double_as_longlong(p[0])) & kAbs;
        ++p;
        --len;
    }
    if ((len & 1) && threadIdx.x == 1) {
        const unsigned long long a = static_cast<unsigned long long>(__double_as_longlong(p[len - 1])) & kAbs;
        mx = a > mx ? a : mx;
    }
    const double2 *q = reinterpret_cast<const double2 *>(p);
    const long long n2 = len / 2;
    for (long long t = threadIdx.x; t < n2; t += 4 * 256) {
        double2 v[4];
#pragma unroll
        for (int i = 0; i < 4; i++) v[i] = t + 256 * i < n2 ? q[t + 256 * i] : make_double2(0.0, 0.0);
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const unsigned long long a = static_cast<unsigned long long>(__double_as_longlong(v[i].x)) & kAbs;
            const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(v[i].y)) & kAbs;
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

// The biased words of an element under its scale (digits.cuh biased_words:
// its 8S-bit fixed-point value plus the digit bias), from which digit_value
// reads each slice's value.
template <int S>
__device__ __forceinline__ void element_words(double x, int e, uint32_t &lo, uint32_t &hi) {
    digits::biased_words<S>(to_fixed(x, e, 8 * S), lo, hi);
}

constexpr int SLICE_ROWS = 8;   // rows per block pass of the slicers

// The S digit planes of one operand's rows by*8 .. (rows step nby*8), four
// consecutive reduction indices kk .. kk+3 per thread (kk = 4 (bx*256 + tid)),
// one 8-byte word per plane and row (Kpad is a multiple of 4).  AL: the four
// sources are two 16-byte aligned pairs (src.ski == 1, src.kin % 4 == 0,
// K % 4 == 0 and even strides from a 16-byte aligned base, checked on the
// host).  Otherwise each of the four is loaded on its own, so any strides, a
// run boundary of the (ko, ki) split or the end of K may fall inside the four;
// the indices past K hold zero digits.  SUPER is a multiple of 4, so the four
// share one exponent.
template <int S, bool AL>
__device__ __forceinline__ void slice_rows4(const Src &src, int rows, int K, int Kpad, const int *e, int rpe,
                                            int nsc, uint2 *out, long long sstride4, int bx, int by, int nby) {
    const int kk = 4 * (bx * 256 + static_cast<int>(threadIdx.x));
    if (kk >= Kpad) return;
    long long off[4];
    bool ok[4];
    {
        int ko = kk / src.kin, ki = kk - ko * src.kin;
#pragma unroll
        for (int i = 0; i < 4; i++) {
            ok[i] = kk + i < K;
            off[i] = static_cast<long long>(ko) * src.sko + static_cast<long long>(ki) * src.ski;
            if (!AL && ++ki == src.kin) {
                ki = 0;
                ++ko;
            }
        }
    }
    const int zc = kk / SUPER;
    for (int rb = by * SLICE_ROWS; rb < rows; rb += nby * SLICE_ROWS) {
        const int rend = min(rows, rb + SLICE_ROWS);
        for (int r = rb; r < rend; r++) {
            uint32_t glo[4], ghi[4];   // the biased words; zero elements give zero digits
            if (kk < K) {
                const double *row = src_row(src, r);
                double x[4];
                if constexpr (AL) {
                    const double2 *p2 = reinterpret_cast<const double2 *>(row + off[0]);
                    const double2 a = p2[0], b = p2[1];
                    x[0] = a.x;
                    x[1] = a.y;
                    x[2] = b.x;
                    x[3] = b.y;
                } else {
#pragma unroll
                    for (int i = 0; i < 4; i++) x[i] = ok[i] ? row[off[i]] : 0.0;
                }
                const int er = e[(r / rpe) * nsc + zc];
#pragma unroll
                for (int i = 0; i < 4; i++) element_words<S>(x[i], er, glo[i], ghi[i]);
            } else {
#pragma unroll
                for (int i = 0; i < 4; i++) digits::biased_words<S>(0, glo[i], ghi[i]);
            }
            const long long o = (static_cast<long long>(r) * Kpad + kk) >> 2;
#pragma unroll
            for (int j = 0; j < S; j++) {
                uint2 w;
                w.x = digits::pack_bf16x2(digits::digit_value<S>(glo[0], ghi[0], j),
                                          digits::digit_value<S>(glo[1], ghi[1], j));
                w.y = digits::pack_bf16x2(digits::digit_value<S>(glo[2], ghi[2], j),
                                          digits::digit_value<S>(glo[3], ghi[3], j));
                out[j * sstride4 + o] = w;
            }
        }
    }
}

// Slicer of one operand whose rows are aligned runs (slice_rows4, AL).
template <int S>
__global__ void __launch_bounds__(256) slice4_kernel(Src src, int rows, int K, int Kpad, const int *e, int rpe,
                                                     int nsc, uint2 *out, long long sstride4) {
    slice_rows4<S, true>(src, rows, K, Kpad, e, rpe, nsc, out, sstride4, blockIdx.x, blockIdx.y, gridDim.y);
}

// Slicer of any one operand (slice_rows4, element loads).
template <int S>
__global__ void __launch_bounds__(256) slice_kernel(Src src, int rows, int K, int Kpad, const int *e, int rpe,
                                                    int nsc, uint2 *out, long long sstride4) {
    slice_rows4<S, false>(src, rows, K, Kpad, e, rpe, nsc, out, sstride4, blockIdx.x, blockIdx.y, gridDim.y);
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
    long long sstride;     // plane stride in 8-byte output words (four BF16 values)
    int rows, K, Kpad, rpe, nsc;
    int vec;               // aligned 16-byte source loads (alignment checked on the host)
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
__global__ void __launch_bounds__(256, 6) expo_group_kernel(const __grid_constant__ SliceGroup g) {
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

// The slices of every job: slice4_kernel's work (aligned jobs) or
// slice_kernel's (the others) for the job's block (bx, by).
template <int S>
__global__ void __launch_bounds__(256, 8) slice_group_kernel(const __grid_constant__ SliceGroup g) {
    const int ji = job_of_block(g, blockIdx.x, false);
    const SliceJob &jb = g.j[ji];
    const int lb = blockIdx.x - jb.sb0;
    const int by = lb / jb.nbx, bx = lb - by * jb.nbx;
    uint2 *out = static_cast<uint2 *>(jb.out);
    if (jb.vec)
        slice_rows4<S, true>(jb.src, jb.rows, jb.K, jb.Kpad, jb.e, jb.rpe, jb.nsc, out, jb.sstride, bx, by, jb.nby);
    else
        slice_rows4<S, false>(jb.src, jb.rows, jb.K, jb.Kpad, jb.e, jb.rpe, jb.nsc, out, jb.sstride, bx, by, jb.nby);
}

// ---------------------------------------------------------------------------
// Exponents of the rank-update operands taken from a panel
// ---------------------------------------------------------------------------
// The split build cuts each density's rank-update operands T_X, T_Y (rows mu,
// reduction index (p, j)) out of the panel T (rows (p, mu), one column per
// column of X_s or Y_s).  Their exponent groups (row mu, super-chunk z of
// (p, j)) gather k-element runs from rows far apart, which a per-group
// exponent pass reads as scattered short pieces.  Instead, each lane group
// reads whole T rows, and folds each operand's k columns of the row into that
// operand's exponents by an atomic maximum: exponents are monotone in |x|, so
// the maximum of per-element exponents is the exponent of the maximum, and
// -1000 (an all-zero group) is the neutral start.  Only the upper word of |x|
// is read: it fixes the exponent.  A warp splits into G = 32 / W groups of W
// lanes, one row per group, and takes PANEL_U operands of its rows at a time,
// so each lane has up to PANEL_U * PANEL_V loads in flight and a warp G rows,
// however short the rows and however small k is.
struct PanelSeg {
    int *e;          // the operand's exponents, e[mu * nsc + z]
    int c0, k, nsc;  // its columns c0 .. c0 + k - 1 of T; super-chunks per row
    int n;           // rows mu per p of its panel
};
struct PanelItem {   // one panel: its rows (p, mu) and its operands' segments
    const double *T;
    long long ldT;
    int n, rows;
    int seg0, nseg;  // segments seg0 .. seg0 + nseg - 1 (nseg <= PANEL_SEG_ITEM)
    int b0;          // first block of this panel in the launch
    int rpb;         // panel rows per block
    int lanes;       // W: lanes per operand, 4, 8, 16 or 32 (W * PANEL_V >= k where possible)
};
constexpr int MAXPITEM = 64;
constexpr int MAXSEG = 800;
constexpr int PANEL_SEG_ITEM = 128;   // operands of one panel
constexpr int PANEL_U = 4;            // operands per lane group at a time
constexpr int PANEL_V = 4;            // words per lane and operand at a time
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

// Rows r0 .. r0 + R - 1 of panel item pi with lane groups of W lanes: group
// gi of warp w takes the rows r0 + w G + gi, then 8 G rows further on.  A run
// that crosses into the next super-chunk (at j = jb) folds into two
// exponents; a batch of operands without one (the common case: a crossing
// happens once per SUPER / k rows p) keeps one maximum per operand.
template <int W>
__device__ __forceinline__ void colmax_rows(const PanelItem &pi, const int2 *sc, const int *snsc, int *const *se,
                                            int r0, int R) {
    constexpr int G = 32 / W;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gi = lane / W, sl = lane % W;
    const unsigned gmask = (W == 32 ? 0xffffffffu : (1u << W) - 1u) << (gi * W % 32);
    const int nseg = pi.nseg;
    for (int rbase = warp * G; rbase < R; rbase += 8 * G) {   // warp-uniform
        const int row = rbase + gi;
        const bool ract = row < R;
        const int r = r0 + (ract ? row : 0), p = r / pi.n, mu = r - p * pi.n;
        const unsigned *hw = reinterpret_cast<const unsigned *>(pi.T + static_cast<long long>(r) * pi.ldT) + 1;
        for (int s0 = 0; s0 < nseg; s0 += PANEL_U) {
            int c0[PANEL_U], k[PANEL_U], jb[PANEL_U], kmax = 0;
            bool cross = false;
#pragma unroll
            for (int u = 0; u < PANEL_U; u++) {
                const int2 ck = ract && s0 + u < nseg ? sc[s0 + u] : make_int2(0, 0);
                c0[u] = ck.x;
                k[u] = ck.y;
                const int kk0 = p * ck.y;                         // reduction index of the run's first element
                jb[u] = (kk0 / SUPER + 1) * SUPER - kk0;          // first j of the next super-chunk
                kmax = max(kmax, ck.y);
                cross = cross || jb[u] < ck.y;
            }
            kmax = __reduce_max_sync(0xffffffffu, kmax);
            cross = __any_sync(0xffffffffu, cross);
            unsigned m0[PANEL_U], m1[PANEL_U];
#pragma unroll
            for (int u = 0; u < PANEL_U; u++) m0[u] = m1[u] = 0;
            for (int jw = 0; jw < kmax; jw += W * PANEL_V) {   // warp-uniform
                const int j0 = jw + sl;
                unsigned x[PANEL_U][PANEL_V];
#pragma unroll
                for (int u = 0; u < PANEL_U; u++) {
                    const unsigned *q = hw + 2 * (c0[u] + j0);
#pragma unroll
                    for (int v = 0; v < PANEL_V; v++) x[u][v] = j0 + v * W < k[u] ? q[2 * v * W] : 0u;
                }
                if (!cross) {
#pragma unroll
                    for (int u = 0; u < PANEL_U; u++)
#pragma unroll
                        for (int v = 0; v < PANEL_V; v++) m0[u] = max(m0[u], x[u][v] & 0x7FFFFFFFu);
                } else {
#pragma unroll
                    for (int u = 0; u < PANEL_U; u++)
#pragma unroll
                        for (int v = 0; v < PANEL_V; v++) {
                            const unsigned a = x[u][v] & 0x7FFFFFFFu;
                            if (j0 + v * W < jb[u]) m0[u] = max(m0[u], a);
                            else m1[u] = max(m1[u], a);
                        }
                }
            }
#pragma unroll
            for (int u = 0; u < PANEL_U; u++) {
                m0[u] = __reduce_max_sync(gmask, m0[u]);
                if (cross) m1[u] = __reduce_max_sync(gmask, m1[u]);
                if (sl == 0 && k[u] > 0) {
                    const int si = s0 + u, z0 = (p * k[u]) / SUPER, nsc = snsc[si];
                    if (m0[u]) atomicMax(&se[si][mu * nsc + z0], exponent_of_max(static_cast<unsigned long long>(m0[u]) << 32));
                    if (m1[u] && jb[u] < k[u])
                        atomicMax(&se[si][mu * nsc + z0 + 1], exponent_of_max(static_cast<unsigned long long>(m1[u]) << 32));
                }
            }
        }
    }
}

// Block b of panel item i takes its rows r0 = (b - b0) rpb .. r0 + R - 1.
__global__ void __launch_bounds__(256) panel_colmax_kernel(const __grid_constant__ PanelExpo g) {
    __shared__ int2 sc[PANEL_SEG_ITEM];        // (c0, k) of the item's operands
    __shared__ int snsc[PANEL_SEG_ITEM];
    __shared__ int *se[PANEL_SEG_ITEM];
    int lo = 0, hi = g.nitem - 1;
    while (lo < hi) {   // the last panel whose first block is <= blockIdx.x
        const int mid = (lo + hi + 1) >> 1;
        if (g.it[mid].b0 <= static_cast<int>(blockIdx.x)) lo = mid;
        else hi = mid - 1;
    }
    const PanelItem &pi = g.it[lo];
    for (int i = threadIdx.x; i < pi.nseg; i += 256) {
        const PanelSeg &sg = g.s[pi.seg0 + i];
        sc[i] = make_int2(sg.c0, sg.k);
        snsc[i] = sg.nsc;
        se[i] = sg.e;
    }
    __syncthreads();
    const int r0 = (static_cast<int>(blockIdx.x) - pi.b0) * pi.rpb;
    const int R = min(pi.rpb, pi.rows - r0);
    switch (pi.lanes) {   // block-uniform
    case 4: colmax_rows<4>(pi, sc, snsc, se, r0, R); break;
    case 8: colmax_rows<8>(pi, sc, snsc, se, r0, R); break;
    case 16: colmax_rows<16>(pi, sc, snsc, se, r0, R); break;
    default: colmax_rows<32>(pi, sc, snsc, se, r0, R); break;
    }
}

// ---------------------------------------------------------------------------
// The J back-contraction's operand: the factor chunk, transposed
// ---------------------------------------------------------------------------
// J_s = sum_P gamma_{P,s} L^P is symmetric, so it is formed on the upper
// triangle as the sliced GEMM C[t][s] = sum_kk A[t][kk] G[s][kk] with
// A[t][kk] = L^{P0+kk}[mu][nu] (t = t(mu, nu), mu <= nu, the packed-triangle
// position) and G[s][kk] = gamma_{P0+kk,s}.  The factor is stored P-major, so
// A's rows are strided columns of it: an exponent pass with one thread per
// row t (the threads of a warp on consecutive positions, i.e. consecutive
// addresses of each L^P), then a slicer that stages TRI_TK x TRI_TT tiles of L in
// shared memory and writes each row's digits along kk.  PK: the factor holds
// packed upper triangles (position t is the row's offset in L^P).
constexpr int TRI_TT = 128;  // rows t per tile of the transposed slicer (a power of two, 8 .. 256)
constexpr int TRI_TK = 32;   // aux indices kk per tile (a multiple of 256 / TRI_TT and of 16)
static_assert(256 % TRI_TT == 0 && TRI_TK % (256 / TRI_TT) == 0 && TRI_TK % 16 == 0 &&
                  (TRI_TT * TRI_TK / 4) % 256 == 0, "transposed slicer tile");

template <bool PK>
__device__ __forceinline__ long long tri_offset(int n, long long t) {
    if (PK) return t;
    int mu, nu;
    packed::tri_row_col(n, t, &mu, &nu);
    return static_cast<long long>(mu) * n + nu;
}

// e[t * nsc + z] = exponent of max |A[t][kk]| over kk in super-chunk z, for
// the 256 rows t = 256 bx + thread.  pstride: doubles between consecutive L^P.
template <bool PK>
__device__ __forceinline__ void expo_tri_body(const double *L, int n, long long pstride, int P0, int np, int nsc,
                                              int *e, long long bx, int z) {
    const long long t = bx * 256 + threadIdx.x;
    if (t >= packed::tri_count(n)) return;
    const int k0 = z * SUPER, k1 = min(np, k0 + SUPER);
    const double *p = L + static_cast<long long>(P0 + k0) * pstride + tri_offset<PK>(n, t);
    constexpr unsigned long long kAbs = 0x7FFFFFFFFFFFFFFFull;
    unsigned long long mx = 0;
    int kk = 0;
    for (; kk + 8 <= k1 - k0; kk += 8) {
        unsigned long long v[8];
#pragma unroll
        for (int u = 0; u < 8; u++)
            v[u] = static_cast<unsigned long long>(__double_as_longlong(p[static_cast<long long>(kk + u) * pstride])) & kAbs;
#pragma unroll
        for (int u = 0; u < 8; u++) mx = v[u] > mx ? v[u] : mx;
    }
    for (; kk < k1 - k0; kk++) {
        const unsigned long long v = static_cast<unsigned long long>(__double_as_longlong(p[static_cast<long long>(kk) * pstride])) & kAbs;
        mx = v > mx ? v : mx;
    }
    e[t * nsc + z] = exponent_of_max(mx);
}

template <bool PK>
__global__ void __launch_bounds__(256) expo_tri_kernel(const double *L, int n, long long pstride, int P0, int np,
                                                       int nsc, int *e) {
    expo_tri_body<PK>(L, n, pstride, P0, np, nsc, e, blockIdx.x, blockIdx.y);
}

// The six digit planes of A: out[j][t][kk] (Kpad columns, zero for kk >= np),
// for rows t0 = TRI_TT bx .. t0 + TRI_TT - 1 and kk0 = TRI_TK by .. kk0 +
// TRI_TK - 1.  The tile's rows of L (one per kk, TRI_TT positions each:
// contiguous runs of the row mu) are staged in shared memory; then each
// thread forms four consecutive kk of one row t.  Consecutive blocks take
// consecutive kk tiles of the same rows t, so a row's planes are written out
// close together in time.
struct TriTile {
    double v[TRI_TK][TRI_TT + 1];   // [kk - kk0][t - t0]
    long long off[TRI_TT];
};

template <bool PK>
__device__ __forceinline__ void slice_tri_body(TriTile &sm, const double *L, int n, long long pstride, int P0, int np,
                                               int Kpad, int nsc, const int *e, uint2 *out, long long sstride4,
                                               long long bx, int by) {
    constexpr int S = 6;
    constexpr int RPP = 256 / TRI_TT;              // rows kk per load pass
    constexpr int GPR = TRI_TK / 4;                // groups of four kk per row t
    const long long ntri = packed::tri_count(n);
    const long long t0 = bx * TRI_TT;
    const int kk0 = by * TRI_TK;
    if (threadIdx.x < TRI_TT) {
        const long long t = t0 + threadIdx.x;
        sm.off[threadIdx.x] = t < ntri ? tri_offset<PK>(n, t) : -1;
    }
    __syncthreads();
    {
        const int tc = threadIdx.x % TRI_TT, kr0 = threadIdx.x / TRI_TT;
        const long long off = sm.off[tc];
        double v[TRI_TK / RPP];
#pragma unroll
        for (int i = 0; i < TRI_TK / RPP; i++) {
            const int kk = kk0 + kr0 + RPP * i;
            v[i] = kk < np && off >= 0 ? L[static_cast<long long>(P0 + kk) * pstride + off] : 0.0;
        }
#pragma unroll
        for (int i = 0; i < TRI_TK / RPP; i++) sm.v[kr0 + RPP * i][tc] = v[i];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < TRI_TT * GPR / 256; i++) {
        const int task = i * 256 + static_cast<int>(threadIdx.x), tr = task / GPR, g = task % GPR;
        const long long t = t0 + tr;
        const int kk = kk0 + 4 * g;
        if (t >= ntri || kk >= Kpad) continue;
        uint32_t glo[4], ghi[4];
        if (kk < np) {
            const int er = e[t * nsc + kk / SUPER];
#pragma unroll
            for (int u = 0; u < 4; u++) digits::biased_words<S>(to_fixed(sm.v[4 * g + u][tr], er, 8 * S), glo[u], ghi[u]);
        } else {
#pragma unroll
            for (int u = 0; u < 4; u++) digits::biased_words<S>(0, glo[u], ghi[u]);
        }
        const long long o = (t * Kpad + kk) >> 2;
#pragma unroll
        for (int j = 0; j < S; j++) {
            uint2 w;
            w.x = digits::pack_bf16x2(digits::digit_value<S>(glo[0], ghi[0], j), digits::digit_value<S>(glo[1], ghi[1], j));
            w.y = digits::pack_bf16x2(digits::digit_value<S>(glo[2], ghi[2], j), digits::digit_value<S>(glo[3], ghi[3], j));
            out[j * sstride4 + o] = w;
        }
    }
}

// One operand: a 1-D grid of sbx * sby blocks, block b at kk tile b % sby
// and row tile b / sby.
template <bool PK>
__global__ void __launch_bounds__(256) slice_tri_kernel(const double *L, int n, long long pstride, int P0, int np,
                                                        int Kpad, int nsc, const int *e, uint2 *out,
                                                        long long sstride4, int sby) {
    __shared__ TriTile sm;
    const int b = static_cast<int>(blockIdx.x), by = b % sby, bx = b / sby;
    slice_tri_body<PK>(sm, L, n, pstride, P0, np, Kpad, nsc, e, out, sstride4, bx, by);
}

// The same for many operands (the molecules of a batched build's wave) in one
// exponent and one slicer launch, the jobs in the parameter space; block b
// belongs to the job whose block range holds it.
struct TriJob {
    const double *L;
    long long pstride;
    int *e;
    uint2 *out;
    long long ss4;
    int n, P0, np, Kpad, nsc, pk;
    int ebx, sbx, sby;   // exponent blocks per super-chunk; slicer blocks along t and kk
    int eb0, sb0;        // first block of this job in the exponent and the slicer launch
};
constexpr int MAXTRI = 64;
struct TriGroup {
    TriJob j[MAXTRI];
    int njob;
};

__device__ __forceinline__ int tri_job_of_block(const TriGroup &g, int b, bool expo) {
    int lo = 0, hi = g.njob - 1;
    while (lo < hi) {   // the last job whose first block is <= b
        const int mid = (lo + hi + 1) >> 1;
        if ((expo ? g.j[mid].eb0 : g.j[mid].sb0) <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(256) expo_tri_group_kernel(const __grid_constant__ TriGroup g) {
    const TriJob &jb = g.j[tri_job_of_block(g, blockIdx.x, true)];
    const int lb = static_cast<int>(blockIdx.x) - jb.eb0, z = lb / jb.ebx, bx = lb - z * jb.ebx;
    if (jb.pk) expo_tri_body<true>(jb.L, jb.n, jb.pstride, jb.P0, jb.np, jb.nsc, jb.e, bx, z);
    else expo_tri_body<false>(jb.L, jb.n, jb.pstride, jb.P0, jb.np, jb.nsc, jb.e, bx, z);
}

__global__ void __launch_bounds__(256) slice_tri_group_kernel(const __grid_constant__ TriGroup g) {
    __shared__ TriTile sm;
    const TriJob &jb = g.j[tri_job_of_block(g, blockIdx.x, false)];
    const int lb = static_cast<int>(blockIdx.x) - jb.sb0, by = lb % jb.sby, bx = lb / jb.sby;
    if (jb.pk)
        slice_tri_body<true>(sm, jb.L, jb.n, jb.pstride, jb.P0, jb.np, jb.Kpad, jb.nsc, jb.e, jb.out, jb.ss4, bx, by);
    else
        slice_tri_body<false>(sm, jb.L, jb.n, jb.pstride, jb.P0, jb.np, jb.Kpad, jb.nsc, jb.e, jb.out, jb.ss4, bx, by);
}

}  // namespace oz
}  // namespace jk
