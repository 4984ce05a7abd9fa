// Internal declarations shared by the libjk.so translation units.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/jk.h"

namespace jk {

constexpr size_t kArenaAlign = 256;
constexpr int kMaxDens = 64;           // densities per molecule in one call

inline size_t align_up(size_t x, size_t a = kArenaAlign) { return (x + a - 1) / a * a; }

// Bump allocator over the caller's arena; reset at the start of every call.
struct Arena {
    char *base = nullptr;
    size_t bytes = 0;
    size_t off = 0;
    size_t high = 0;
    size_t floor = 0;    // buffers below this offset outlive the inner calls that reset the arena
    void reset(size_t start) { off = start > floor ? start : floor; }
    template <class T> T *take(size_t count) {
        size_t need = align_up(count * sizeof(T));
        if (off + need > bytes) return nullptr;
        T *p = reinterpret_cast<T *>(base + off);
        off += need;
        if (off > high) high = off;
        return p;
    }
};

// Device-side status words at the start of the arena.
struct DeviceFlags {
    int error;        // JK_* code raised by a kernel (0 = none)
    int where;        // kernel-specific detail
    int pad[62];
};

// Kernel kinds for launch accounting / event timing.
enum KernelKind {
    KK_DGEMM = 0, KK_JSTREAM, KK_FROB, KK_GAMMA, KK_PACK, KK_MISC,
    KK_SLICE, KK_OZGEMM, KK_OZREDUCE, KK_EXPO, KK_JTRI, KK_COUNT
};

struct Profiler {
    bool on = false;
    long long launches = 0;
    struct Rec { int kind; cudaEvent_t a, b; };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    double ms[KK_COUNT] = {};
    long long cnt[KK_COUNT] = {};
    double tensor_flops = 0.0;
};

}  // namespace jk

struct jk_ctx {
    jk::Arena arena;
    jk::DeviceFlags *flags = nullptr;    // first bytes of the arena
    std::string last_error;
    int device = -1;
    int num_sms = 148;
    int aux_chunk = -1;      // explicit options (JK_OPT_*); -1 = not set
    int schedule = -1;
    int raster = -1;
    int use_tuned = 1;
    int tile = -1;           // explicit tile width option (JK_OPT_TILE)
    int adj_slices = 7;      // slices per operand of the split adjoint (JK_OPT_ADJOINT_SLICES)
    int cur_raster = 0;      // tile order in effect for the running call
    int cur_tile = 0;        // tile width in effect for the running call: 0 80 columns, 1 64
    int gemm_smem_set = 0;   // bit c: the shared-memory attribute of slice configuration c is set
    int host_chunk = 0;      // aux indices per streamed chunk of a host-resident factor (0 = automatic)
    int slicer = 0;          // digit extraction of the vector slicer: 0 integer, 1 FP32 additions
    int syrk = 0;            // split engine: symmetric rank updates by row blocks, rest mirrored
    int packed_factor = 0;   // factors passed to builds hold packed upper triangles
    int jpath = -1;          // split J back-contraction (JK_OPT_J_PATH): -1 automatic, 0 FP64, 1 tensor
    cudaStream_t copy_stream = nullptr;   // host builds: uploads of the factor, created on first use
    cudaEvent_t ev_fork = nullptr, ev_up[2] = {nullptr, nullptr}, ev_used[2] = {nullptr, nullptr};
    cudaStream_t aux_stream = nullptr;    // FP64 J streams overlapped with the rank updates
    cudaEvent_t ev_jfork = nullptr, ev_jdone = nullptr;
    jk::Profiler prof;
};

namespace jk {

// Per-call view of one molecule's problem after validation.
struct Problem {
    int n = 0, naux = 0, nd = 0;
    const double *L = nullptr;
    int k[kMaxDens];
    int sym[kMaxDens];
    const double *X[kMaxDens];
    const double *Y[kMaxDens];
    // Column layout of the panel matrix Z = [X_0 | Y_0 | X_1 | Y_1 | ...]
    // (Y_s omitted for symmetric densities): offsets of X_s and Y_s in Z.
    int offX[kMaxDens], offY[kMaxDens];
    int ctot = 0;       // columns of Z
    int ksum = 0;       // sum of k_s
    int kmax = 0;
    // Per-density outputs ([n][n] each); NULL entries are not formed.
    double *J[kMaxDens];
    double *K[kMaxDens];
    bool wantJ = false, wantK = false;
    int aux_chunk = 0;   // at most this many aux indices per chunk (0 = automatic)
    int schedule = 0;    // split precision: 0 per-density launches, 1 grouped launches
    bool packed = false; // L holds packed upper triangles [naux][n(n+1)/2]; each aux
                         // chunk is expanded into a dense workspace copy before use
    int slices = 6;      // split adjoint: slices per operand (6: 48-bit, 7: 56-bit)
    int jpath = -1;      // split J back-contraction: -1 automatic, 0 FP64 stream, 1 tensor cores
};

// The split engine forms J on the tensor cores (sliced GEMM over the upper
// triangle) when asked, or automatically once the FP64 form's work,
// n(n+1)/2 * naux * nd multiply-adds, reaches kJTensorMin: below that the
// FP64 stream is short and overlaps the rank updates on a second stream.
constexpr double kJTensorMin = 4e9;
inline bool j_on_tensor(const Problem &pb) {
    if (pb.jpath >= 0) return pb.jpath == 1;
    return 0.5 * pb.n * (pb.n + 1.0) * pb.naux * pb.nd >= kJTensorMin;
}

jk_status set_error(jk_ctx *h, jk_status s, const char *fmt, ...);

// Rows per block of the blocked symmetric rank update (JK_OPT_SYRK): row block
// [r0, r0 + kSymBlock) of K_s is formed from column r0 on.
constexpr int kSymBlock = 128;
// K[r][c] = K[c][r] for every c < kSymBlock * (r / kSymBlock): the entries a
// blocked symmetric rank update leaves unformed.
jk_status mirror_sym_blocks(jk_ctx *h, double *K, int n, cudaStream_t st);

// The file name of a source path (messages name the file, not the directory
// it was built in).
inline const char *source_name(const char *path) {
    const char *b = path;
    for (const char *c = path; *c; ++c)
        if (*c == '/' || *c == '\\') b = c + 1;
    return b;
}

#define JK_CUDA_TRY(h, call)                                                   \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess)                                                 \
            return ::jk::set_error((h), JK_ERR_CUDA, "%s failed: %s (%s:%d)",  \
                                   #call, cudaGetErrorString(e_),              \
                                   ::jk::source_name(__FILE__),                \
                                   __LINE__);                                  \
    } while (0)

#define JK_LAUNCH_CHECK(h)                                                     \
    do {                                                                       \
        cudaError_t e_ = cudaGetLastError();                                   \
        if (e_ != cudaSuccess)                                                 \
            return ::jk::set_error((h), JK_ERR_CUDA, "launch failed: %s (%s:%d)", \
                                   cudaGetErrorString(e_),                      \
                                   ::jk::source_name(__FILE__), __LINE__);      \
    } while (0)

#define JK_TRY(expr)                                                           \
    do {                                                                       \
        jk_status s_ = (expr);                                                 \
        if (s_ != JK_OK) return s_;                                            \
    } while (0)

// ---- FP64 engine (fp64.cu) ------------------------------------------------
size_t fp64_build_workspace(const Problem &pb, int pchunk);
size_t fp64_adjoint_workspace(const Problem &pb, int pchunk, bool want_dl);
int fp64_default_pchunk(const Problem &pb);
jk_status fp64_build(jk_ctx *h, const Problem &pb, cudaStream_t st);
jk_status fp64_adjoint(jk_ctx *h, const Problem &pb, const double *W,
                       const double *V, double *dX, double *dY, double *dL,
                       cudaStream_t st);

jk_status fp64_axpy(jk_ctx *h, double *y, const double *x, long long cnt, cudaStream_t st);
// full[p] = the symmetric n x n matrix whose packed upper triangle is
// packed[p] ([np][n(n+1)/2], row-major, diagonal included).
jk_status fp64_unpack_sym(jk_ctx *h, const double *packed, int n, long long np, double *full, cudaStream_t st);
// packed[p][t(a,b)] = full[p][a][b], a <= b (the inverse of fp64_unpack_sym)
jk_status fp64_pack_sym(jk_ctx *h, const double *full, int n, long long np, double *packed_out, cudaStream_t st);

// ---- split-precision engine (split.cu) -----------------------------------
size_t split_build_workspace(const Problem &pb);
size_t split_adjoint_workspace(const Problem &pb, bool want_dl);
jk_status split_build(jk_ctx *h, const Problem &pb, cudaStream_t st);
jk_status split_adjoint(jk_ctx *h, const Problem &pb, const double *W,
                        const double *V, double *dX, double *dY, double *dL,
                        cudaStream_t st);

size_t split_batched_workspace(int nmol, const Problem *pbs);
int split_auto_pchunk(const Problem &pb);   // aux chunk chosen from the workspace budget
jk_status split_batched(jk_ctx *h, int nmol, const Problem *pbs, cudaStream_t st);

// ---- dense (general, non-symmetric) densities ------------------------------
// J(DJ_s) and K(DK_s) for dense [nd][n][n] arguments (Eq. 4 with a dense
// argument): K_s = sum_P (L^P DK_s)(L^P)^T, J_s = sum_P <L^P, DJ_s> L^P.  With
// add_j, J is formed in the workspace and added to K (the density gradient
// K(W) + J(V)); K then must not be NULL.
struct DenseProb {
    int n = 0, naux = 0, nd = 0;
    const double *L = nullptr;
    const double *DK = nullptr;   // input of K, or NULL (no K)
    const double *DJ = nullptr;   // input of J, or NULL (no J)
    double *K = nullptr;          // [nd][n][n]
    double *J = nullptr;          // [nd][n][n] (unused with add_j)
    bool add_j = false;
    int aux_chunk = 0;            // aux indices per chunk (0 = automatic)
    bool packed = false;          // L holds packed upper triangles (chunks expanded before use)
};
size_t fp64_dense_workspace(const DenseProb &dp);
jk_status fp64_dense(jk_ctx *h, const DenseProb &dp, cudaStream_t st);
size_t split_dense_workspace(const DenseProb &dp);
jk_status split_dense(jk_ctx *h, const DenseProb &dp, cudaStream_t st);

// ---- bra-ket pairings ------------------------------------------------------
// out[a*nr + b] = <A_a B_a^T, M_b> for the left densities of `left` packed in
// ZL (split_pack_z layout) and dense M_b [nr][n][n]; U: [nr][n][left.ctot].
jk_status fp64_pair_contract(jk_ctx *h, const Problem &left, const double *ZL, const double *M, int nr, double *U,
                             double *out, cudaStream_t st);
jk_status split_pack_z(jk_ctx *h, const Problem &pb, double *Z, cudaStream_t st);
// Z[m] = the packed density columns of molecule m, for nmol molecules (grouped launches).
jk_status pack_z_multi(jk_ctx *h, int nmol, const Problem *pbs, double *const *Z, cudaStream_t st);
// gamma[s][P0 + p] = sum_{sig,i} T^p[sig][offX_s + i] Y_s[sig][i], p < np, for
// panel chunks of several molecules (grouped launches).
struct GammaItem {
    const Problem *pb;
    const double *T;
    long long ldT;
    int np, P0;
    double *gamma;
};
jk_status fp64_gamma_group(jk_ctx *h, const std::vector<GammaItem> &items, cudaStream_t st);

// ---- Laplace (LT-AO) builds -------------------------------------------------
// out[k][mu][p] = C[mu][p] exp(sign alpha[k] eps[p] / 2), k < nq <= kMaxDens
// (alpha on the host); out[e] = sum_k w[k] part[k][e] (w on the host).
jk_status fp64_laplace_scale(jk_ctx *h, const double *C, const double *eps, int n, int m, int sign,
                             const double *alpha, int nq, double *out, cudaStream_t st);
jk_status fp64_weighted_sum(jk_ctx *h, double *out, const double *part, const double *w, int nq, long long cnt,
                            cudaStream_t st);

// ---- batched builds (batched.cu) ------------------------------------------
jk_status batched_build(jk_ctx *h, int nmol, const Problem *pbs, jk_precision p,
                        cudaStream_t st);


// Brackets one kernel launch: counts it and, when profiling is on, records
// CUDA events before and after it on the launch stream.
struct LaunchScope {
    jk_ctx *h;
    int kind;
    cudaStream_t st;
    cudaEvent_t b = nullptr;
    LaunchScope(jk_ctx *h_, int kind_, cudaStream_t st_);
    ~LaunchScope();
};

// ---- autotuner (tune.cu) ----------------------------------------------------
struct TuneKey {
    int op, prec, sms, nmol, nb, nauxb, nd, ksumb;
    bool operator<(const TuneKey &o) const;
};
TuneKey tune_key(jk_op op, jk_precision p, int sms, int nmol, const Problem *pbs);
bool tune_lookup(const TuneKey &k, jk_tune_config &cfg);
void tune_store(const TuneKey &k, const jk_tune_config &cfg, double ms);

}  // namespace jk
