// The tcgen05 sliced GEMM of the split-precision engine (C = A B^T on S-slice
// operands, FP64 or int64 split-K partials out) and its split-K reductions.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "fixed.cuh"
#include "jk_internal.h"
#include "ozcfg.cuh"
#include "tc.cuh"

namespace jk {
namespace oz {

using fixed::i128_to_f64_scaled;
using fixed::i64_to_f64_scaled;

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
// Every window restarts with the tile, which would make diagonal 2's first
// window two K-blocks long and its drain due while the epilogue is still
// finishing the previous tile; instead that window runs on to the second
// one's end (K-blocks 0..9, 160 elements, still below 2^24 units).
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
// The window boundary that a tile's first period skips (see above).
constexpr int kMergedDiag = 2;
constexpr int kMergedEnd = 1;   // K-block of the skipped end; the skipped start is the next one
static_assert(woff(kMergedDiag) == kMergedEnd + 1 &&
                  (kMergedEnd + 1 + wper(kMergedDiag)) * KB * (65536 + 16384) < (1 << 24),
              "diagonal 2's merged first window stays exact");
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
        // 21 pairs as 9 MMAs, the fewest with N <= 240 (every MMA reads its
        // whole A slice from shared memory, whose bandwidth the operand
        // reads and the TMA writes share): those touching only the tile-long
        // accumulators 4, 5 first, the one touching accumulator 0 last
        const int a[9] = {1, 2, 4, 5, 0, 3, 2, 1, 0};
        const int b0[9] = {3, 3, 0, 0, 3, 0, 0, 0, 0};
        const int nb[9] = {2, 1, 2, 1, 3, 3, 3, 3, 3};
        L.n = 9;
        for (int i = 0; i < 9; i++) {
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
// window ends at r go first, so that its drain can be signalled (committed)
// as soon as they finish and overlaps the rest of the K-block; the MMAs that
// touch an accumulator whose window restarts at r go last, so the MMA thread
// has the most work queued before it must wait for that accumulator's drain
// (each group keeps the list's order; window starts and ends never share a
// residue).  nend[r] counts the first group.
struct MmaOrder {
    int v[WPERIOD][MAXMMA];
    int nend[WPERIOD];
};
template <class C>
__host__ __device__ constexpr MmaOrder make_mma_order(const MmaList &L) {
    MmaOrder t{};
    for (int r = 0; r < WPERIOD; r++) {
        const unsigned ms = ws_mask<C>(r), me = we_mask<C>(r);
        int c = 0;
        for (int pass = 0; pass < 3; pass++) {
            for (int j = 0; j < L.n; j++) {
                const unsigned mj = ((1u << L.nb[j]) - 1u) << (L.a[j] + L.b0[j]);
                const int grp = (mj & me) ? 0 : (mj & ms) ? 2 : 1;
                if (grp == pass) t.v[r][c++] = j;
            }
            if (pass == 0) t.nend[r] = c;
        }
    }
    return t;
}
template <class C>
__host__ __device__ constexpr bool starts_and_ends_apart() {
    for (int r = 0; r < WPERIOD; r++)
        if (ws_mask<C>(r) & we_mask<C>(r)) return false;
    return true;
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
static_assert(we_mask<Cfg6>(kMergedEnd) == (1u << kMergedDiag) && we_mask<Cfg7>(kMergedEnd) == (1u << kMergedDiag),
              "the skipped window end is the only one at its residue");
static_assert(starts_and_ends_apart<Cfg6>() && starts_and_ends_apart<Cfg7>(),
              "no accumulator window both starts and ends at one residue");

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
// The MMAs of one K-block of window residue R, in the residue's issue order
// (compile-time tables): before the first MMA into an accumulator whose window
// starts here (bit set in pend, a subset of PMAX), wait until the epilogue has
// drained and zeroed it.  PMAX is the residue's window starts, or every
// accumulator in a tile's first K-block, so that steady-state K-blocks carry
// no wait code for accumulators that cannot be pending.  Returns false if a
// wait gave up.
template <class C, int R, unsigned PMAX, int I>
__device__ __forceinline__ bool issue_mmas(uint32_t tmem, uint32_t a_lo, uint32_t b_lo, unsigned &pend,
                                           int (&wcnt)[C::NACC], uint64_t *accfull, uint64_t *accempty,
                                           bool early, volatile int *abort_flag) {
    if constexpr (I == Tabs<C>::order.nend[R] && I > 0) {
        // the windows ending at this residue have all their MMAs issued
        if (early) {
            constexpr unsigned kEnds = we_mask<C>(R);
#pragma unroll
            for (int d = 0; d < C::NACC; d++)
                if (kEnds & (1u << d)) tc::mma_commit(&accfull[d]);
        }
    }
    if constexpr (I == Tabs<C>::list.n) {
        return true;
    } else {
        constexpr int i = Tabs<C>::order.v[R][I];
        constexpr int a = Tabs<C>::list.a[i];
        constexpr int b0 = Tabs<C>::list.b0[i];
        constexpr int nb = Tabs<C>::list.nb[i];
        constexpr int d0 = a + b0;
        constexpr unsigned mask = (((1u << nb) - 1u) << d0) & PMAX;
        if constexpr (mask != 0) {
            const unsigned need = pend & mask;
            if (need) {
#pragma unroll
                for (int d = 0; d < C::NACC; d++) {
                    if (!(mask & (1u << d)) || !(need & (1u << d))) continue;
                    if (!tc::mbar_wait(&accempty[d], static_cast<uint32_t>(wcnt[d]) & 1u, abort_flag)) return false;
                    wcnt[d]++;
                }
                pend &= ~need;
                tc::fence_after_sync();
            }
        }
        // descriptor start addresses are in 16-byte units
        tc::mma_bf16_acc(tmem + d0 * C::BN, a_lo + a * (BM * 32 / 16), b_lo + b0 * (C::BN * 32 / 16), tc::kSw32DescHi,
                         tc::idesc_bf16_f32(BM, C::BN * nb));
        return issue_mmas<C, R, PMAX, I + 1>(tmem, a_lo, b_lo, pend, wcnt, accfull, accempty, early, abort_flag);
    }
}

// One K-block (kb) of residue R: wait for its operand stage, issue its MMAs,
// release the stage, and in the tile's last K-block signal every drain.
template <class C, int R, unsigned PMAX>
__device__ __forceinline__ bool issue_kblock(uint8_t *smem, uint32_t tmem, int kb, int nkb, unsigned pend, bool early,
                                             int &stage, uint32_t &phase, int (&wcnt)[C::NACC], uint64_t *full,
                                             uint64_t *empty, uint64_t *accfull, uint64_t *accempty,
                                             volatile int *abort_flag) {
    if (!tc::mbar_wait(&full[stage], phase, abort_flag)) return false;
    tc::fence_after_sync();
    const uint32_t a_lo = tc::sdesc_kmajor_sw32_lo(tc::smem_u32(smem + stage * C::STAGE_BYTES));
    const uint32_t b_lo = a_lo + C::A_BYTES / 16;
    // the residue's window ends are committed right after their MMAs,
    // except in the tile's last K-block, which ends every window at once
    const bool last = kb == nkb - 1;
    if (!issue_mmas<C, R, PMAX, 0>(tmem, a_lo, b_lo, pend, wcnt, accfull, accempty, early && !last, abort_flag))
        return false;
    tc::mma_commit(&empty[stage]);
    if (last) {
#pragma unroll
        for (int d = 0; d < C::NACC; d++) tc::mma_commit(&accfull[d]);
    }
    if (++stage == C::NSTAGE) {
        stage = 0;
        phase ^= 1u;
    }
    return true;
}

// A tile's first K-block: every accumulator opens a window.
template <class C>
__device__ __forceinline__ bool issue_first(uint8_t *smem, uint32_t tmem, int nkb, int &stage, uint32_t &phase,
                                            int (&wcnt)[C::NACC], uint64_t *full, uint64_t *empty, uint64_t *accfull,
                                            uint64_t *accempty, volatile int *abort_flag) {
    constexpr unsigned kAll = (1u << C::NACC) - 1u;
    static_assert(we_mask<Cfg6>(0) == 0 && we_mask<Cfg7>(0) == 0, "no window ends in a tile's first K-block");
    return issue_kblock<C, 0, kAll>(smem, tmem, 0, nkb, kAll, false, stage, phase, wcnt, full, empty, accfull,
                                    accempty, abort_flag);
}

// K-blocks kb0 + R .. kb0 + 15 of a tile (one window period, unrolled so that
// the window bookkeeping is compile-time except for the tile's first period
// and last K-block); in the first period, K-block 0 has been issued already.
// Returns false if a wait gave up.
template <class C, int R>
__device__ __forceinline__ bool issue_period(uint8_t *smem, uint32_t tmem, int kb0, int nkb, int &stage,
                                             uint32_t &phase, int (&wcnt)[C::NACC], uint64_t *full, uint64_t *empty,
                                             uint64_t *accfull, uint64_t *accempty, volatile int *abort_flag) {
    if constexpr (R == WPERIOD) {
        return true;
    } else {
        const int kb = kb0 + R;
        if (kb >= nkb) return true;
        if (R != 0 || kb0 != 0) {
            constexpr unsigned kStarts = ws_mask<C>(R);
            // the tile's first period keeps diagonal 2's first window open
            // through K-block 9
            unsigned pend = kStarts;
            if constexpr (R == kMergedEnd + 1) {
                if (kb0 == 0) pend &= ~(1u << kMergedDiag);
            }
            const bool early = !(R == kMergedEnd && kb0 == 0);
            if (!issue_kblock<C, R, kStarts>(smem, tmem, kb, nkb, pend, early, stage, phase, wcnt, full, empty,
                                             accfull, accempty, abort_flag))
                return false;
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

// A finished FP64 tile whose conversion and store are pending: its int64
// accumulators sit in this warp's staging block; the epilogue converts them
// pair by pair while it would otherwise wait for the next drain, and stores
// each 32 x 8 block as soon as it is complete.
struct PendingStore {
    int pi_i0;            // its problem in the launch (bits 8..) and the next column pair
                          // (bits 0..7; OUT_COLS when nothing is pending)
    int c0, r0;           // its first column and the warp's first row
    int ea, eb_lo, eb_hi; // row exponent (minus FRAC); column exponents of columns lane, 32 + lane
};

template <int OUT_COLS>
__device__ __forceinline__ void pending_step(PendingStore &ps, const OzGroup &g, uint8_t *wbuf, int lane) {
    const int pi = ps.pi_i0 >> 8, i0 = ps.pi_i0 & 255;
    const int N = g.p[pi].a.N, M = g.p[pi].a.M;
    const int row = ps.r0 + lane;
    const int j = (i0 % OUT_BLK) / 2;
    const int chunk = j ^ ((lane >> 1) & 3);
    longlong2 *p = reinterpret_cast<longlong2 *>(wbuf + (i0 / OUT_BLK) * (32 * OUT_BLK * 8) + lane * 64 + chunk * 16);
    const longlong2 w = *p;
    const int eb0 = __shfl_sync(0xffffffffu, i0 < 32 ? ps.eb_lo : ps.eb_hi, i0 & 31);
    const int eb1 = __shfl_sync(0xffffffffu, i0 + 1 < 32 ? ps.eb_lo : ps.eb_hi, (i0 + 1) & 31);
    const int col = ps.c0 + i0;
    const double d0 = col < N && row < M ? i64_to_f64_scaled(w.x, ps.ea + eb0) : 0.0;
    const double d1 = col + 1 < N && row < M ? i64_to_f64_scaled(w.y, ps.ea + eb1) : 0.0;
    *p = make_longlong2(__double_as_longlong(d0), __double_as_longlong(d1));
    ps.pi_i0 += 2;
    if ((i0 + 2) % OUT_BLK == 0) {
        // block complete: hand it to the TMA
        tc::fence_proxy_async_smem();
        __syncwarp();
        const int b = i0 / OUT_BLK;
        const int cc = ps.c0 + b * OUT_BLK;
        if (lane == 0 && cc < N) {
            tc::tma_store_2d(&g.p[pi].tmC, wbuf + b * (32 * OUT_BLK * 8), cc, ps.r0);
            tc::bulk_commit();
        }
    }
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
    uint8_t *outbuf = smem + C::NSTAGE * C::STAGE_BYTES;
    uint64_t *full = reinterpret_cast<uint64_t *>(outbuf + C::OUT_BYTES);
    uint64_t *empty = full + C::NSTAGE;
    uint64_t *accfull = empty + C::NSTAGE;
    uint64_t *accempty = accfull + NACC;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(accempty + NACC);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nunits = g.nunits;
    const int u0 = static_cast<int>(blockIdx.x);
    const int ustep = static_cast<int>(gridDim.x);

    if (threadIdx.x == 0) {
        for (int i = 0; i < C::NSTAGE; i++) { tc::mbar_init(&full[i], 1); tc::mbar_init(&empty[i], 1); }
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
                    if (++stage == C::NSTAGE) { stage = 0; phase ^= 1u; }
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
                if (tc_.nkb > 0)
                    ok = issue_first<C>(smem, tmem, tc_.nkb, stage, phase, wcnt, full, empty, accfull, accempty,
                                        abort_flag);
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
        uint8_t *wbuf = outbuf + ew * C::OUT_WARP_BYTES;   // this warp's staging block
        PendingStore ps;
        ps.pi_i0 = OUT_COLS;
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
            for (int kb = 0; kb < tc_.nkb && ok; kb++) {
                const unsigned wends = we_mask_rt<C>(kb & (WPERIOD - 1)) & (kb == kMergedEnd ? ~(1u << kMergedDiag) : ~0u);
                const unsigned ends = wends | (kb == tc_.nkb - 1 ? (1u << NACC) - 1u : 0u);
                if (!ends) continue;
                // one copy of the drain-and-convert code for all accumulators
                // (per-accumulator unrolled copies cost instruction-cache misses)
#pragma unroll 1
                for (int j = 0; j < NACC; j++) {
                    const int d = drain_acc<C>(j);
                    if (!(ends & (1u << d))) continue;
                    // the previous tile's pending store progresses while this
                    // accumulator is still being written
                    while ((ps.pi_i0 & 255) < OUT_COLS && !tc::mbar_test_wait(&accfull[d], (epar >> d) & 1u))
                        pending_step<OUT_COLS>(ps, g, wbuf, lane);
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
                    // below 2^24; a tile-long one stays far below 2^31 units of the
                    // output's 2^-FRAC.  Scale to the unit (exact: a power of two),
                    // convert to int32 (F2I, round to nearest: exact for the exact
                    // diagonals), then add into the 2^-FRAC fixed point of acc64
                    // (shifted by FRAC - 16 - 8d for the exact diagonals).  No
                    // branches and no 64-bit float conversions (those run on the
                    // scarce FP64 pipe).
                    const bool exact = d < C::NEXACT;
                    const float unit = exact ? __int_as_float((127 + 16 + 8 * d) << 23) : __int_as_float((127 + C::FRAC) << 23);
                    const int sh = exact ? C::FRAC - 16 - 8 * d : 0;
#pragma unroll
                    for (int i = 0; i < OUT_COLS; i++) {
                        const int xi = __float2int_rn(v[i] * unit);
                        acc64[i] += static_cast<long long>(static_cast<unsigned long long>(static_cast<long long>(xi)) << sh);
                    }
                }
            }
            if (!ok) break;
            if (a.use_tma_store) {
                // This warp's 32 x OUT_COLS block: lane = row, swizzled 32 x 8 sub-blocks.
                while ((ps.pi_i0 & 255) < OUT_COLS) pending_step<OUT_COLS>(ps, g, wbuf, lane);   // the previous tile's rest
                if (lane == 0) tc::bulk_wait_read();   // earlier stores have read the buffer
                __syncwarp();
                // the int64 accumulators as they are (the split-K partials' form)
#pragma unroll
                for (int b = 0; b < OUT_COLS / OUT_BLK; b++) {
#pragma unroll
                    for (int j = 0; j < OUT_BLK / 2; j++) {   // 16-byte chunks of this row
                        const int i0 = b * OUT_BLK + 2 * j;
                        const int chunk = j ^ ((lane >> 1) & 3);   // 64-byte swizzle
                        *reinterpret_cast<longlong2 *>(wbuf + b * (32 * OUT_BLK * 8) + lane * 64 + chunk * 16) =
                            make_longlong2(acc64[i0], acc64[i0 + 1]);
                    }
                }
                const int r0 = tc_.m * BM + q * 32;
                if (a.nsuper == 1) {
                    // FP64 out: rounding every element is deferred into the
                    // next tile's waits for its accumulators (PendingStore);
                    // the exponents' load latency hides there too
                    ps.pi_i0 = pi << 8;
                    ps.c0 = c0;
                    ps.r0 = r0;
                    ps.ea = row < a.M ? a.eA[row / a.a_rpe] - C::FRAC : 0;
                    ps.eb_lo = c0 + lane < a.N ? a.eB[(c0 + lane) / a.b_rpe] : 0;
                    ps.eb_hi = lane < OUT_COLS - 32 && c0 + 32 + lane < a.N ? a.eB[(c0 + 32 + lane) / a.b_rpe] : 0;
                } else {
                    tc::fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) {
#pragma unroll
                        for (int b = 0; b < OUT_COLS / OUT_BLK; b++) {
                            const int cc = c0 + b * OUT_BLK;
                            // rows of the partial for super-chunk z follow the M rows of z-1
                            const int rr = r0 + tc_.z * static_cast<int>(a.pz / a.ldp);
                            if (cc < a.N) tc::tma_store_2d(tmC, wbuf + b * (32 * OUT_BLK * 8), cc, rr);
                        }
                        tc::bulk_commit();
                    }
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
        if (ok)
            while ((ps.pi_i0 & 255) < OUT_COLS) pending_step<OUT_COLS>(ps, g, wbuf, lane);
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

}  // namespace oz
}  // namespace jk
