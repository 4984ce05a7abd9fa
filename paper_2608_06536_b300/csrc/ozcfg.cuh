// The sliced GEMM's configurations (slice count, tile shape) and the
// constants shared by the slicers and the GEMM of the split-precision engine.
#pragma once

#include <cuda.h>
#include <cstdint>

namespace jk {
namespace oz {

constexpr int BM = 128;             // rows of A per tile (TMEM lanes)
constexpr int KB = 16;              // reduction elements per pipeline stage (one MMA K-step)
constexpr int KBPC = 8;             // K-blocks of a 128-element exact window
constexpr int WPERIOD = 2 * KBPC;   // the window pattern repeats every 16 K-blocks
constexpr int SUPER = 2048;         // reduction elements per int64 partial
constexpr int SMEM_MAX = 227 * 1024;   // opt-in shared memory per CTA
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
    // operand stages: as many as fit beside the output staging, at most 4
    static constexpr int NST_FIT = (SMEM_MAX - OUT_BYTES - 1024 - 256) / STAGE_BYTES;
    static constexpr int NSTAGE = NST_FIT < 4 ? NST_FIT : 4;
    static constexpr int SMEM_BYTES = NSTAGE * STAGE_BYTES + OUT_BYTES + 1024 /*align slack*/ + 256 /*barriers*/;
    static_assert(S * BN <= 512, "the accumulators fit tensor memory");
    static_assert(BN % 16 == 0 && OUT_COLS % OUT_BLK == 0, "tile width");
    static_assert(NEXACT >= 1 && NEXACT <= 5, "window schedule");
    static_assert(FRAC >= 16 + 8 * (NEXACT - 1) && FRAC + 11 <= 62, "exact drains and the int64 range");
    static_assert(NSTAGE >= 2 && SMEM_BYTES <= SMEM_MAX, "shared memory");
};
using Cfg6 = Cfg<6, 80>;
using Cfg6n = Cfg<6, 64>;
using Cfg7 = Cfg<7, 64>;
constexpr int OUT_BLK = 8;

}  // namespace oz
}  // namespace jk
