// Split-precision engine: FP64-accurate J/K from BF16 tensor-core products.
//
// Every dense contraction of the build (panels T = L Z, the rank update
// K_s = sum_P T_X T_Y^T and the J back-contraction J_s = sum_P gamma_{P,s}
// L^P on the upper triangle) is computed as an error-free-split product:
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
#include "jk_internal.h"
#include "ozcfg.cuh"
#include "ozgemm.cuh"
#include "packed.cuh"
#include "slicers.cuh"
#include "tc.cuh"

namespace jk {
namespace oz {

// K[r][c] = K[c][r] for the entries a blocked symmetric rank update leaves
// unformed: c < bm * (r / bm), left of row r's diagonal block (those (c, r)
// all lie in the formed blocks, so no entry is both read and written).
__global__ void __launch_bounds__(256) mirror_blocks_kernel(double *K, int n, int bm) {
    const long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (e >= static_cast<long long>(n) * n) return;
    const int r = static_cast<int>(e / n), c = static_cast<int>(e - static_cast<long long>(r) * n);
    if (c < bm * (r / bm)) K[e] = K[static_cast<long long>(c) * n + r];
}

// J_s[mu][nu] = J_s[nu][mu] (+)= C[t][s] for every upper-triangle position
// t = t(mu, nu) (the sliced GEMM's J back-contraction of one aux chunk; acc:
// added to J, the chunks in order).
struct JOut {
    double *p[kMaxDens];
};
__global__ void __launch_bounds__(256) j_tri_add_kernel(const double *C, long long ldc, int n, int nd, int acc,
                                                        JOut J) {
    const long long t = blockIdx.x * 256LL + threadIdx.x;
    if (t >= packed::tri_count(n)) return;
    int mu, nu;
    packed::tri_row_col(n, t, &mu, &nu);
    const long long e = static_cast<long long>(mu) * n + nu, em = static_cast<long long>(nu) * n + mu;
    for (int s = 0; s < nd; s++) {
        const double v = acc ? J.p[s][e] + C[t * ldc + s] : C[t * ldc + s];
        J.p[s][e] = v;
        if (mu != nu) J.p[s][em] = v;
    }
}

// The same for many molecules in one launch (a batched build's wave): thread
// e0 + t of job i takes position t of job i's triangle; the J pointers of all
// jobs sit in one table (job i's densities at ptr[p0 ..]).
struct JAddJob {
    const double *C;
    long long ldc, e0;
    int n, nd, acc, p0;
};
constexpr int MAXJADD = 64, MAXJPTR = 1024;
struct JAddGroup {
    JAddJob j[MAXJADD];
    double *ptr[MAXJPTR];
    int njob;
};
__global__ void __launch_bounds__(256) j_tri_add_group_kernel(const __grid_constant__ JAddGroup g, long long total) {
    const long long x = blockIdx.x * 256LL + threadIdx.x;
    if (x >= total) return;
    int lo = 0, hi = g.njob - 1;
    while (lo < hi) {   // the last job whose first element is <= x
        const int mid = (lo + hi + 1) >> 1;
        if (g.j[mid].e0 <= x) lo = mid;
        else hi = mid - 1;
    }
    const JAddJob &jb = g.j[lo];
    const long long t = x - jb.e0;
    const int n = jb.n;
    int mu, nu;
    packed::tri_row_col(n, t, &mu, &nu);
    const long long e = static_cast<long long>(mu) * n + nu, em = static_cast<long long>(nu) * n + mu;
    for (int s = 0; s < jb.nd; s++) {
        double *J = g.ptr[jb.p0 + s];
        const double v = jb.acc ? J[e] + jb.C[t * jb.ldc + s] : jb.C[t * jb.ldc + s];
        J[e] = v;
        if (mu != nu) J[em] = v;
    }
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
    const bool flat = nsc == 1 && src.rin == 1 && src.ski == 1 && src.kin == K && src.sr == K && rows % rpe == 0;
    {
        LaunchScope ls(h, KK_EXPO, st);
        if (flat)
            oz::expo_flat_kernel<<<groups, 256, 0, st>>>(src.p, static_cast<long long>(rpe) * K, out.e);
        else
            oz::expo_kernel<<<dim3(groups, nsc), 256, 0, st>>>(src, rows, K, rpe, out.e);
    }
    JK_LAUNCH_CHECK(h);
    // aligned 16-byte loads of four consecutive elements, else element loads
    const bool vec = aligned && src.ski == 1 && (src.kin % 4) == 0 && (K % 4) == 0 && (src.sr % 2) == 0 &&
                     (src.sri % 2) == 0 && (src.sko % 2) == 0;
    const int rblocks = (rows + oz::SLICE_ROWS - 1) / oz::SLICE_ROWS;
    {
        LaunchScope ls(h, KK_SLICE, st);
        dim3 grid((out.Kpad / 4 + 255) / 256, rblocks < 65535 ? rblocks : 65535);
        uint2 *o4 = reinterpret_cast<uint2 *>(out.s);
        const long long ss4 = static_cast<long long>(rows) * out.Kpad / 4;
        if (vec) {
            if (out.S == 7)
                oz::slice4_kernel<7><<<grid, 256, 0, st>>>(src, rows, K, out.Kpad, out.e, rpe, nsc, o4, ss4);
            else if (h->slicer == 1)
                oz::slice4f_kernel<<<grid, 256, 0, st>>>(src, rows, K, out.Kpad, out.e, rpe, nsc, o4, ss4);
            else
                oz::slice4_kernel<6><<<grid, 256, 0, st>>>(src, rows, K, out.Kpad, out.e, rpe, nsc, o4, ss4);
        } else {
            if (out.S == 7)
                oz::slice_kernel<7><<<grid, 256, 0, st>>>(src, rows, K, out.Kpad, out.e, rpe, nsc, o4, ss4);
            else
                oz::slice_kernel<6><<<grid, 256, 0, st>>>(src, rows, K, out.Kpad, out.e, rpe, nsc, o4, ss4);
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

// ---- the J back-contraction on the tensor cores ------------------------------
// Buffers of one build's J: the transposed factor chunk's slices (rows: the
// n(n+1)/2 upper-triangle positions, K: the chunk's aux indices), gamma's
// slices, the chunk's C[t][s] and, for chunks longer than SUPER, its split-K
// partials.
struct JBufs {
    Sliced A, G;
    double *C = nullptr;
    long long ldc = 0;
    long long *P = nullptr;
};

static long long tri_rows(int n) { return packed::tri_count(n); }

static size_t jbufs_bytes(const Problem &pb, int pc) {
    const long long nt = tri_rows(pb.n);
    size_t b = sliced_bytes(static_cast<int>(nt), pc, 1) + sliced_bytes(pb.nd, pc, 1) +
               align_up(static_cast<size_t>(nt) * even_ld(pb.nd) * 8);
    if (nsuper_of(pc) > 1) b += align_up(static_cast<size_t>(nsuper_of(pc)) * part_rows(nt) * even_ld(pb.nd) * 8);
    return b + 4 * kArenaAlign;
}

static bool take_jbufs(Arena &ar, const Problem &pb, int pc, JBufs &jb) {
    const long long nt = tri_rows(pb.n);
    bool ok = take_sliced(ar, static_cast<int>(nt), pc, 1, jb.A) && take_sliced(ar, pb.nd, pc, 1, jb.G);
    jb.ldc = even_ld(pb.nd);
    jb.C = ar.take<double>(static_cast<size_t>(nt) * jb.ldc);
    if (nsuper_of(pc) > 1) jb.P = ar.take<long long>(static_cast<size_t>(nsuper_of(pc)) * part_rows(nt) * jb.ldc);
    return ok && jb.C && (nsuper_of(pc) == 1 || jb.P);
}

// J_s (+)= sum_{P in P0 .. P0+np-1} gamma_{P,s} L^P (added unless P0 == 0):
// the chunk's factor sliced transposed, gamma's chunk sliced, one sliced GEMM
// C[t][s] = sum_kk A[t][kk] G[s][kk] and its scatter onto both triangles.
static jk_status split_j_chunk(jk_ctx *h, const Problem &pb, const double *gamma, int P0, int np, JBufs &jb,
                               cudaStream_t st) {
    const int n = pb.n;
    const long long nt = tri_rows(n);
    const long long pstride = pb.packed ? nt : static_cast<long long>(n) * n;
    Sliced &A = jb.A;
    A.rows = static_cast<int>(nt);
    A.K = np;
    A.Kpad = kpad_of(np);
    A.rpe = 1;
    const int nsc = nsuper_of(np);
    {
        LaunchScope ls(h, KK_JTRI, st);
        const dim3 grid(static_cast<unsigned>((nt + 255) / 256), nsc);
        if (pb.packed) oz::expo_tri_kernel<true><<<grid, 256, 0, st>>>(pb.L, n, pstride, P0, np, nsc, A.e);
        else oz::expo_tri_kernel<false><<<grid, 256, 0, st>>>(pb.L, n, pstride, P0, np, nsc, A.e);
    }
    JK_LAUNCH_CHECK(h);
    {
        LaunchScope ls(h, KK_JTRI, st);
        const int sby = (A.Kpad + oz::TRI_TK - 1) / oz::TRI_TK;
        const long long blocks = (nt + oz::TRI_TT - 1) / oz::TRI_TT * sby;
        if (blocks > 0x7fffffffLL) return set_error(h, JK_ERR_SHAPE, "too many J slicer blocks");
        const unsigned grid = static_cast<unsigned>(blocks);
        uint2 *o4 = reinterpret_cast<uint2 *>(A.s);
        const long long ss4 = nt * A.Kpad / 4;
        if (pb.packed)
            oz::slice_tri_kernel<true><<<grid, 256, 0, st>>>(pb.L, n, pstride, P0, np, A.Kpad, nsc, A.e, o4, ss4, sby);
        else
            oz::slice_tri_kernel<false><<<grid, 256, 0, st>>>(pb.L, n, pstride, P0, np, A.Kpad, nsc, A.e, o4, ss4, sby);
    }
    JK_LAUNCH_CHECK(h);
    oz::Src gsrc{gamma + P0, pb.naux, 0, 1, np};   // row s: gamma[s][P0 ..]
    JK_TRY(slice_operand(h, gsrc, pb.nd, np, 1, jb.G, st));
    if (nsc == 1) {
        JK_TRY(ozgemm(h, A, jb.G, jb.C, jb.ldc, nullptr, st));
    } else {
        JK_TRY(ozgemm(h, A, jb.G, nullptr, 0, jb.P, st));
        JK_TRY(reduce_partials(h, jb.P, nsc, A, jb.G, jb.C, jb.ldc, false, st));
    }
    oz::JOut jo;
    for (int s = 0; s < kMaxDens; s++) jo.p[s] = s < pb.nd ? pb.J[s] : nullptr;
    {
        LaunchScope ls(h, KK_JTRI, st);
        oz::j_tri_add_kernel<<<static_cast<unsigned>((nt + 255) / 256), 256, 0, st>>>(jb.C, jb.ldc, n, pb.nd,
                                                                                       P0 > 0 ? 1 : 0, jo);
    }
    JK_LAUNCH_CHECK(h);
    return JK_OK;
}

// ---- the J back-contraction in grouped launches (batched builds) -------------
static_assert(sizeof(oz::TriGroup) <= 32764 && sizeof(oz::JAddGroup) + 8 <= 32764,
              "grouped launches fit the kernel parameter space");

struct TriBatch {
    std::vector<oz::TriJob> jobs;
};

// One operand A of split_j_chunk as a job of the grouped transposed slicing.
static void tri_add(TriBatch &tb, const Problem &pb, int P0, int np, Sliced &A) {
    const int n = pb.n;
    const long long nt = tri_rows(n);
    A.rows = static_cast<int>(nt);
    A.K = np;
    A.Kpad = kpad_of(np);
    A.rpe = 1;
    oz::TriJob j;
    std::memset(&j, 0, sizeof j);
    j.L = pb.L;
    j.pstride = pb.packed ? nt : static_cast<long long>(n) * n;
    j.e = A.e;
    j.out = reinterpret_cast<uint2 *>(A.s);
    j.ss4 = nt * A.Kpad / 4;
    j.n = n;
    j.P0 = P0;
    j.np = np;
    j.Kpad = A.Kpad;
    j.nsc = nsuper_of(np);
    j.pk = pb.packed ? 1 : 0;
    j.ebx = static_cast<int>((nt + 255) / 256);
    j.sbx = static_cast<int>((nt + oz::TRI_TT - 1) / oz::TRI_TT);
    j.sby = (A.Kpad + oz::TRI_TK - 1) / oz::TRI_TK;
    tb.jobs.push_back(j);
}

static jk_status tri_flush(jk_ctx *h, TriBatch &tb, cudaStream_t st) {
    static thread_local oz::TriGroup grp;
    for (size_t i0 = 0; i0 < tb.jobs.size(); i0 += oz::MAXTRI) {
        const int nj = static_cast<int>(std::min<size_t>(oz::MAXTRI, tb.jobs.size() - i0));
        long long eb = 0, sbk = 0;
        for (int i = 0; i < nj; i++) {
            oz::TriJob &j = grp.j[i];
            j = tb.jobs[i0 + i];
            j.eb0 = static_cast<int>(eb);
            j.sb0 = static_cast<int>(sbk);
            eb += static_cast<long long>(j.ebx) * j.nsc;
            sbk += static_cast<long long>(j.sbx) * j.sby;
            if (eb > 0x7fffffffLL || sbk > 0x7fffffffLL) return set_error(h, JK_ERR_SHAPE, "too many J slicer blocks");
        }
        grp.njob = nj;
        {
            LaunchScope ls(h, KK_JTRI, st);
            oz::expo_tri_group_kernel<<<static_cast<unsigned>(eb), 256, 0, st>>>(grp);
        }
        JK_LAUNCH_CHECK(h);
        {
            LaunchScope ls(h, KK_JTRI, st);
            oz::slice_tri_group_kernel<<<static_cast<unsigned>(sbk), 256, 0, st>>>(grp);
        }
        JK_LAUNCH_CHECK(h);
    }
    tb.jobs.clear();
    return JK_OK;
}

struct JAddBatch {
    std::vector<oz::JAddJob> jobs;
    std::vector<double *const *> outs;
};

static void jadd_add(JAddBatch &ab, const Problem &pb, const JBufs &jb, bool acc) {
    oz::JAddJob j;
    std::memset(&j, 0, sizeof j);
    j.C = jb.C;
    j.ldc = jb.ldc;
    j.n = pb.n;
    j.nd = pb.nd;
    j.acc = acc ? 1 : 0;
    ab.jobs.push_back(j);
    ab.outs.push_back(pb.J);
}

static jk_status jadd_flush(jk_ctx *h, JAddBatch &ab, cudaStream_t st) {
    static thread_local oz::JAddGroup grp;
    size_t i0 = 0;
    while (i0 < ab.jobs.size()) {
        int nj = 0, np = 0;
        long long tot = 0;
        while (i0 + nj < ab.jobs.size() && nj < oz::MAXJADD && np + ab.jobs[i0 + nj].nd <= oz::MAXJPTR) {
            oz::JAddJob &j = grp.j[nj];
            j = ab.jobs[i0 + nj];
            j.e0 = tot;
            j.p0 = np;
            for (int s = 0; s < j.nd; s++) grp.ptr[np + s] = ab.outs[i0 + nj][s];
            np += j.nd;
            tot += tri_rows(j.n);
            nj++;
        }
        grp.njob = nj;
        {
            LaunchScope ls(h, KK_JTRI, st);
            oz::j_tri_add_group_kernel<<<static_cast<unsigned>((tot + 255) / 256), 256, 0, st>>>(grp, tot);
        }
        JK_LAUNCH_CHECK(h);
        i0 += nj;
    }
    ab.jobs.clear();
    ab.outs.clear();
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
    j.flat = j.nsc == 1 && src.rin == 1 && src.ski == 1 && src.kin == K && src.sr == K && rows % rpe == 0;
    j.vec = aligned && src.ski == 1 && (src.kin % 4) == 0 && (K % 4) == 0 && (src.sr % 2) == 0 &&
            (src.sri % 2) == 0 && (src.sko % 2) == 0;
    j.sstride = static_cast<long long>(rows) * out.Kpad / 4;
    const int rblocks = (rows + oz::SLICE_ROWS - 1) / oz::SLICE_ROWS;
    j.nbx = (out.Kpad / 4 + 255) / 256;
    j.nby = rblocks < 65535 ? rblocks : 65535;
    sb.jobs.push_back(j);
    (void)out.S;
}

// Slice every collected operand (all six-slice) with one exponent launch and
// one slicer launch per MAXJOB jobs; the batch is emptied.
// expo = false: the jobs' exponents are already in place (panel_expo).
static jk_status slice_flush(jk_ctx *h, SliceBatch &sb, cudaStream_t st, bool expo = true) {
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
        if (expo) {
            LaunchScope ls(h, KK_EXPO, st);
            oz::expo_group_kernel<<<static_cast<unsigned>(eb), 256, 0, st>>>(grp);
        }
        if (expo) JK_LAUNCH_CHECK(h);
        {
            LaunchScope ls(h, KK_SLICE, st);
            oz::slice_group_kernel<6><<<static_cast<unsigned>(sbk), 256, 0, st>>>(grp);
        }
        JK_LAUNCH_CHECK(h);
    }
    sb.jobs.clear();
    return JK_OK;
}

// The exponents of the rank-update operands of whole panels (every density
// of one aux chunk of one or several molecules), from whole rows of each panel
// T (oz::panel_colmax_kernel), in grouped launches.  Usable when every k <=
// SUPER (a run of one p spans at most two super-chunks) and a panel row's
// upper words fit the block's shared memory.
static bool panel_expo_fits(const Problem &pb) {
    for (int s = 0; s < pb.nd; s++)
        if (pb.k[s] > oz::SUPER) return false;
    return 2 * pb.nd <= oz::PANEL_SEG_ITEM;
}
static_assert(2 * kMaxDens <= oz::PANEL_SEG_ITEM && oz::PANEL_SEG_ITEM <= oz::MAXSEG,
              "one panel's operands fit the row-wise exponent launch");
struct PanelBatch {
    struct Item {
        const Problem *pb;
        const double *T;
        long long ldT;
        int np;
        Sliced *TX, *TY;
    };
    std::vector<Item> items;
};
static void panel_add(PanelBatch &pbt, const Problem &pb, const double *T, long long ldT, int np, Sliced *TX,
                      Sliced *TY) {
    pbt.items.push_back({&pb, T, ldT, np, TX, TY});
}
static jk_status panel_launch(jk_ctx *h, oz::PanelExpo &g, int nscmax, long long blocks, cudaStream_t st) {
    if (blocks > 0x7fffffffLL) return set_error(h, JK_ERR_SHAPE, "too many panel rows");
    {
        LaunchScope ls(h, KK_EXPO, st);
        int nmax = 1;
        for (int i = 0; i < g.nitem; i++) nmax = std::max(nmax, g.it[i].n);
        const int bx = std::min(1024, (nmax * nscmax + 255) / 256);
        oz::int_fill_kernel<<<dim3(bx, g.nseg), 256, 0, st>>>(g);
    }
    JK_LAUNCH_CHECK(h);
    {
        LaunchScope ls(h, KK_EXPO, st);
        oz::panel_colmax_kernel<<<static_cast<unsigned>(blocks), 256, 0, st>>>(g);
    }
    JK_LAUNCH_CHECK(h);
    return JK_OK;
}
static jk_status panel_flush(jk_ctx *h, PanelBatch &pbt, cudaStream_t st) {
    static thread_local oz::PanelExpo g;
    g.nitem = 0;
    g.nseg = 0;
    int nscmax = 1;
    long long blocks = 0;
    for (const auto &itm : pbt.items) {
        const Problem &pb = *itm.pb;
        int want = 0, ncol = 1, kmax = 1;
        for (int s = 0; s < pb.nd; s++) {
            want += pb.sym[s] ? 1 : 2;
            ncol = std::max(ncol, pb.offX[s] + pb.k[s]);
            if (!pb.sym[s]) ncol = std::max(ncol, pb.offY[s] + pb.k[s]);
            kmax = std::max(kmax, pb.k[s]);
        }
        if (want > oz::PANEL_SEG_ITEM) return set_error(h, JK_ERR_SHAPE, "too many operands in one panel");
        if (g.nitem == oz::MAXPITEM || g.nseg + want > oz::MAXSEG) {
            JK_TRY(panel_launch(h, g, nscmax, blocks, st));
            g.nitem = g.nseg = 0;
            nscmax = 1;
            blocks = 0;
        }
        oz::PanelItem &pi = g.it[g.nitem++];
        pi.T = itm.T;
        pi.ldT = itm.ldT;
        pi.n = pb.n;
        pi.rows = itm.np * pb.n;
        pi.seg0 = g.nseg;
        pi.b0 = static_cast<int>(blocks);
        int lanes = 4;   // the fewest lanes (4 .. 32) that cover k in PANEL_V words each
        while (lanes < 32 && lanes * oz::PANEL_V < kmax) lanes *= 2;
        pi.lanes = lanes;
        // one row per lane group (8 warps of 32 / lanes groups), more for
        // short rows: about 8192 elements per block, at most 8 rows per group
        const int gr = 8 * (32 / lanes);
        pi.rpb = gr * std::max(1, std::min(8, 8192 / (gr * ncol)));
        for (int s = 0; s < pb.nd; s++) {
            const int nsc = (itm.np * pb.k[s] + oz::SUPER - 1) / oz::SUPER;
            nscmax = std::max(nscmax, nsc);
            g.s[g.nseg++] = oz::PanelSeg{itm.TX[s].e, pb.offX[s], pb.k[s], nsc, pb.n};
            if (!pb.sym[s]) g.s[g.nseg++] = oz::PanelSeg{itm.TY[s].e, pb.offY[s], pb.k[s], nsc, pb.n};
        }
        pi.nseg = g.nseg - pi.seg0;
        blocks += (pi.rows + pi.rpb - 1) / pi.rpb;
    }
    if (g.nitem > 0) JK_TRY(panel_launch(h, g, nscmax, blocks, st));
    pbt.items.clear();
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

// P-chunk so that the per-chunk workspace stays below ~12 GB (a single
// molecule's build) or ~6 GB (a work item of a batch of several molecules,
// so that several fit one wave of the batched arena).
static int split_pchunk(const Problem &pb, bool batched = false) {
    const size_t n = pb.n;
    size_t per = n * n * (6 * 2) + n * pb.ctot * 8 + n * pb.ctot * (6 * 2);
    if (pb.packed) per += n * n * 8;               // the expanded factor chunk
    if (j_on_tensor(pb)) per += n * (n + 1) / 2 * (6 * 2);   // the transposed chunk's slices (J)
    size_t budget = static_cast<size_t>(batched ? 6 : 12) << 30;
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
    if (j_on_tensor(pb)) b += jbufs_bytes(pb, pc);   // J on the tensor cores (counted whether or not J is asked for: queries do not say)
    return b;
}


jk_status split_pack_z(jk_ctx *h, const Problem &pb, double *Z, cudaStream_t st);
jk_status fp64_unpack_sym(jk_ctx *h, const double *packed, int n, long long np, double *full, cudaStream_t st);
jk_status fp64_gamma_panel(jk_ctx *h, const Problem &pb, const double *T, long long ldT, int np, double *gamma,
                           int P0, cudaStream_t st);
jk_status fp64_jstream(jk_ctx *h, const Problem &pb, const double *gamma, cudaStream_t st);
jk_status fp64_jstream_chunk(jk_ctx *h, const Problem &pb, const double *gamma, int P0, int np, cudaStream_t st);

// The FP64 form of J (the factored builds' J when it is small, see
// j_on_tensor; a dense-density build's metric dots and J) needs only the
// factor and gamma or the densities, and runs on the FP64 pipe: it is forked
// onto a second stream and overlaps the products on the tensor pipe (join at
// the end of the build, so the call stays ordered on the caller's stream).
// A single molecule's build forks it once per aux chunk (J accumulated chunk
// by chunk in order), a batched build once per molecule, after its last
// chunk.  Larger builds form J on the tensor cores (split_j_chunk and its
// grouped form).
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
    JBufs jb;
    const bool jt = pb.wantJ && j_on_tensor(pb);
    if (jt) ok = ok && take_jbufs(ar, pb, pc, jb);
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
        if (pb.wantJ) {
            JK_TRY(fp64_gamma_panel(h, pb, T, ldT, np, gamma, P0, st));
            if (jt) {
                JK_TRY(split_j_chunk(h, pb, gamma, P0, np, jb, st));
            } else {
                JK_TRY(fork_jstream(h, st));
                JK_TRY(fp64_jstream_chunk(h, pb, gamma, P0, np, h->aux_stream));
            }
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
            if (grouped && panel_expo_fits(pb)) {
                PanelBatch pbt;
                panel_add(pbt, pb, T, ldT, np, TX, TY);
                JK_TRY(panel_flush(h, pbt, st));
                JK_TRY(slice_flush(h, sb, st, false));
            } else {
                JK_TRY(slice_flush(h, sb, st));
            }
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
    if (pb.wantJ && !jt) JK_TRY(join_jstream(h, st));
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
    JBufs jb;                 // the chunk's J back-contraction
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
    if (j_on_tensor(pb)) b += jbufs_bytes(pb, pc);                         // J on the tensor cores
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
    ok = ok && (!(pb.wantJ && j_on_tensor(pb)) || take_jbufs(ar, pb, pc, it.jb));
    return ok && it.P && it.tmp && (!pb.packed || it.Lx);
}

}  // namespace

size_t split_batched_workspace(int nmol, const Problem *pbs) {
    size_t mols = 0, maxitem = 0, items = 0;
    for (int m = 0; m < nmol; m++) {
        const Problem &pb = pbs[m];
        mols += mol_bytes(pb);
        const int pc = split_pchunk(pb, nmol > 1);
        const size_t ib = item_bytes(pb, pc);
        maxitem = std::max(maxitem, ib);
        items += ib * ((pb.naux + pc - 1) / pc);
    }
    // enough for every molecule's persistent buffers and at least the largest
    // work item; more (up to everything, capped at 40 GB) lets waves hold more items
    const size_t cap = static_cast<size_t>(40) << 30;
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
        mb[m].pc = split_pchunk(pb, nmol > 1);
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
    bool forked = false;   // FP64 J passes running on the second stream
    // Work items (molecule, aux chunk), chunk-major: the first chunk of every
    // molecule, then the second ..., so that a wave (at most one chunk per
    // molecule, as many as the arena holds) takes many molecules at once and
    // each molecule's chunks still come in order.
    std::vector<std::pair<int, int>> work;
    for (int c = 0;; c++) {
        bool any = false;
        for (int m = 0; m < nmol; m++) {
            const long long P0 = static_cast<long long>(c) * mb[m].pc;
            if (P0 >= pbs[m].naux) continue;
            work.push_back({m, static_cast<int>(P0)});
            any = true;
        }
        if (!any) break;
    }
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
        // 3. gamma, and the J back-contraction's operands of every chunk of the
        // wave (the transposed factor chunks, gamma's chunks); then the
        // rank-update operands
        {
            std::vector<GammaItem> gi;
            for (auto &it : items)
                if (pbs[it.mol].wantJ)
                    gi.push_back({&pbs[it.mol], it.T, even_ld(pbs[it.mol].ctot), it.np, it.P0, mb[it.mol].gamma});
            JK_TRY(fp64_gamma_group(h, gi, st));
            TriBatch tb;
            SliceBatch gb;
            bool fork = false;
            for (auto &it : items) {
                const Problem &pb = pbs[it.mol];
                if (!pb.wantJ) continue;
                if (!j_on_tensor(pb)) {
                    // the FP64 form, once the molecule's gamma is complete
                    if (it.P0 + it.np >= pb.naux) {
                        if (!fork) JK_TRY(fork_jstream(h, st));
                        fork = forked = true;
                        JK_TRY(fp64_jstream(h, pb, mb[it.mol].gamma, h->aux_stream));
                    }
                    continue;
                }
                tri_add(tb, pb, it.P0, it.np, it.jb.A);
                oz::Src gsrc{mb[it.mol].gamma + it.P0, pb.naux, 0, 1, it.np};   // row s: gamma[s][P0 ..]
                slice_add(gb, gsrc, pb.nd, it.np, 1, it.jb.G);
            }
            JK_TRY(tri_flush(h, tb, st));
            JK_TRY(slice_flush(h, gb, st));
        }
        bool rowwise = grouped;   // exponents from whole panel rows when every molecule allows it
        for (auto &it : items)
            if (pbs[it.mol].wantK && !panel_expo_fits(pbs[it.mol])) rowwise = false;
        PanelBatch pbt;
        for (auto &it : items) {
            const Problem &pb = pbs[it.mol];
            const long long ldT = even_ld(pb.ctot);
            if (!pb.wantK) continue;
            if (rowwise) panel_add(pbt, pb, it.T, ldT, it.np, it.TX, it.TY);
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
        if (rowwise) JK_TRY(panel_flush(h, pbt, st));
        JK_TRY(slice_flush(h, sb, st, !rowwise));
        // 4. every rank update and J back-contraction of the wave: grouped
        // persistent launches
        probs.clear();
        ReduceBatch rb;
        JAddBatch ab;
        for (auto &it : items) {
            const Problem &pb = pbs[it.mol];
            if (!pb.wantJ || !j_on_tensor(pb)) continue;
            const int nsc = nsuper_of(it.np);
            probs.emplace_back();
            JK_TRY(oz_problem(h, it.jb.A, it.jb.G, nsc == 1 ? it.jb.C : nullptr, it.jb.ldc,
                              nsc == 1 ? nullptr : it.jb.P, probs.back()));
            if (nsc > 1) reduce_add(rb, it.jb.P, nsc, it.jb.A, it.jb.G, it.jb.C, it.jb.ldc, false);
            jadd_add(ab, pb, it.jb, it.P0 > 0);
        }
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
        // 5. reductions into K and J's C (the split-K ones in grouped launches)
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
        // 6. J_s (+)= C of every chunk of the wave (chunks of a molecule in order)
        JK_TRY(jadd_flush(h, ab, st));
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
