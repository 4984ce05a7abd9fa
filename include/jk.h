/*
 * jk.h -- C ABI of libjk.so, the B300 (sm_103a) Cholesky-decomposed
 * Coulomb/exchange engine for non-symmetric densities.
 *
 * What it computes (the paper's statement of the problem, Eq. 4 and the
 * energy-level CD build of Sec. II.C; bare J and K, no factor 2, no -1/2):
 *
 *   (mu nu|lam sig) = sum_P L^P_{mu nu} L^P_{lam sig}          CD integrals
 *   D_s             = X_s Y_s^T                               factored density
 *   gamma_{P,s}     = sum_{lam sig} L^P_{lam sig} (D_s)_{lam sig}
 *   J_s             = sum_P gamma_{P,s} L^P
 *   K_s             = sum_P (L^P X_s)(L^P Y_s)^T   (= B_V^T B_U with the
 *                                                  half-transforms B_U, B_V)
 *
 * A symmetric density (D = X X^T) is the special case Y = X of the
 * non-symmetric build (Sec. II.C).
 *
 * Conventions shared by every entry point:
 *  - All arrays are row-major and live in DEVICE memory unless stated.
 *    The caller owns every input, output and the workspace arena; the
 *    library never calls cudaMalloc/cudaFree inside a build (the arena is
 *    sub-allocated by bump, as the paper's engine does, Sec. IV).
 *  - All work is enqueued asynchronously on the caller's stream
 *    (a cudaStream_t passed as void*; NULL = legacy default stream).
 *    Split builds run the FP64 form of their J back-contraction (see
 *    JK_OPT_J_PATH), and jk_build_host its uploads, on streams the handle
 *    owns; those fork from and join the caller's stream inside the call, so
 *    every result is ordered on it.
 *  - Outputs are overwritten, never accumulated into.
 *  - Arguments are validated on the host before anything is launched; a
 *    failing check returns a status and stores a message retrievable with
 *    jk_last_error(); nothing is launched in that case.
 *  - A handle must be used from one host thread and one stream at a time:
 *    successive calls reuse the same arena.
 *  - Input arrays (L, X, Y, W, V) must be 16-byte aligned; output arrays
 *    (J, K, dX, dY, dL) need only the natural 8-byte alignment of double
 *    (JK_ERR_ARG otherwise).  Outputs that are 16-byte aligned with an even
 *    row length take the bulk-store (TMA) path; others are written with
 *    plain stores.
 *  - L^P is assumed symmetric in (mu, nu); this is not checked.
 */
#ifndef JK_H
#define JK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    JK_OK = 0,
    JK_ERR_ARG = 1,          /* NULL / misaligned pointer, bad enum value     */
    JK_ERR_SHAPE = 2,        /* nbf, naux, k or counts out of range           */
    JK_ERR_OOM = 3,          /* workspace arena too small for this call       */
    JK_ERR_CUDA = 4,         /* a CUDA runtime call or launch failed          */
    JK_ERR_TIMEOUT = 5,      /* a bounded device-side wait gave up            */
    JK_ERR_UNSUPPORTED = 6   /* valid request this build does not implement   */
} jk_status;

typedef enum {
    /* Plain FP64 engine: every product and sum in IEEE double. */
    JK_FP64 = 0,
    /* Split-precision engine: FP64 operands cut into BF16 slices (error-free
     * splitting), slice products on tcgen05 tensor cores with FP32 TMEM
     * accumulators kept exact, integer/FP64 recombination; FP64-accurate. */
    JK_SPLIT_BF16 = 1
} jk_precision;

typedef struct jk_ctx *jk_handle;

/* One Cholesky factor: L is [naux][nbf][nbf] FP64 on the device (packed
 * upper triangles [naux][nbf(nbf+1)/2] under JK_OPT_PACKED_FACTOR). */
typedef struct {
    int32_t nbf;
    int32_t naux;
    const double *L;
} jk_factor;

/* One factored density D = X Y^T.  X, Y are [nbf][k] FP64 on the device,
 * 1 <= k <= 4 nbf and nbf*k <= 2^31 - 1.
 * symmetric != 0 means D = X X^T: Y is ignored (may be NULL). */
typedef struct {
    int32_t k;
    int32_t symmetric;
    const double *X;
    const double *Y;
} jk_density;

/* Which entry point a workspace query is for. */
typedef enum {
    JK_OP_BUILD = 0, JK_OP_ADJOINT = 1, JK_OP_BATCHED = 2, JK_OP_BUILD_HOST = 3,
    JK_OP_BUILD_DENSE = 4, JK_OP_DENSITY_GRAD = 5, JK_OP_PAIR = 6, JK_OP_LAPLACE = 7,
    JK_OP_BUILD_HOST_PACKED = 8
} jk_op;

/* Create a handle over a caller-owned device arena of `bytes` bytes
 * (256-byte aligned).  The arena must stay valid until jk_destroy. */
jk_status jk_create(jk_handle *h, void *workspace, size_t bytes);
jk_status jk_destroy(jk_handle h);

/* Bytes of arena a call with these shapes needs (host-only, no GPU work).
 * For JK_OP_BATCHED pass nmol factors and the concatenated densities, with
 * nd_per_mol giving the split; otherwise nmol = 1 and nd_per_mol may be NULL.
 * For JK_OP_BUILD_DENSE and JK_OP_DENSITY_GRAD only f and nd are read (d may
 * be NULL); the answer covers both maps.  For JK_OP_PAIR pass nmol = 2,
 * nd_per_mol = {nl, nr}, nd = nl + nr and d = the left densities followed by
 * the right ones (one factor); the answer covers both pairings.  For
 * JK_OP_LAPLACE pass nd = nq and d[0] with k = m and symmetric = (CY == NULL)
 * (only d[0]'s shape is read); the answer covers the weighted form.
 * Without a handle the answer covers both the default configuration and a
 * tuned one cached for these shapes (see jk_autotune); the _handle form
 * answers for the configuration that handle's options select. */
jk_status jk_workspace_query(jk_op op, int32_t nmol, const jk_factor *f,
                             const int32_t *nd_per_mol, int32_t nd,
                             const jk_density *d, jk_precision p, size_t *bytes);
jk_status jk_workspace_query_handle(jk_handle h, jk_op op, int32_t nmol, const jk_factor *f,
                                    const int32_t *nd_per_mol, int32_t nd,
                                    const jk_density *d, jk_precision p, size_t *bytes);

/* jk_build: J_s and K_s for nd densities over one factor (Eq. 4, Sec. II.C).
 *   J, K : [nd][nbf][nbf] FP64 outputs; either may be NULL (not formed).
 * Status: JK_ERR_SHAPE if nbf is outside [1, 65535], naux < 1, nd is outside
 *         [1, 64], or a density has k outside [1, 4 nbf] or nbf*k > 2^31 - 1;
 *         JK_ERR_OOM if the arena is smaller than jk_workspace_query says. */
jk_status jk_build(jk_handle h, const jk_factor *f, int32_t nd,
                   const jk_density *d, double *J, double *K,
                   jk_precision p, void *stream);

/* jk_build_host: jk_build with every array in host memory (factor, densities
 * and outputs; page-locked memory gives full copy speed and asynchrony).  The
 * factor, the bulk of the input (naux x nbf^2 doubles), is streamed to the
 * device in aux-index chunks on an internal copy stream, double-buffered and
 * overlapped with the build of the previous chunk on `stream`; J and K are
 * summed over the chunks in FP64 on the device (the build is linear in the
 * aux-index range) and copied back to the host at the end.  All work is
 * ordered on `stream` (the copy stream forks from and joins it), so the call
 * returns before the results are in host memory: synchronize `stream` (or
 * call jk_sync_status) before reading J, K.  Arena: jk_workspace_query with
 * JK_OP_BUILD_HOST.  Status as jk_build; host pointers are not checked. */
jk_status jk_build_host(jk_handle h, const jk_factor *f, int32_t nd, const jk_density *d,
                        double *J, double *K, jk_precision p, void *stream);

/* jk_build_host_packed: jk_build_host with the factor given as the packed upper
 * triangle of each (symmetric) L^P: f->L is a host array [naux][nbf(nbf+1)/2],
 * L^P_{mu nu} (mu <= nu) at index mu*nbf - mu(mu-1)/2 + (nu - mu) of block P
 * (row-major upper triangle, diagonal included).  Half the factor's bytes cross
 * the host link; each uploaded chunk is expanded to full L^P on the device
 * before its build, so results equal jk_build_host's on the same L bit for bit.
 * Arena: jk_workspace_query with JK_OP_BUILD_HOST_PACKED.  Status as jk_build_host. */
jk_status jk_build_host_packed(jk_handle h, const jk_factor *f, int32_t nd, const jk_density *d,
                               double *J, double *K, jk_precision p, void *stream);

/* jk_build_batched: many independent molecules (uneven nbf, naux, nd) in one
 * call.  f[m] is molecule m's factor, nd_per_mol[m] its density count (host
 * array), d the densities of all molecules concatenated in molecule order,
 * J[i], K[i] (host arrays of device pointers, one per density in the same
 * order) point to [nbf_m][nbf_m] FP64 outputs; J or K may be NULL.
 * In split precision the molecules' panels go into shared persistent GEMM
 * launches (up to 32 problems of different shapes each), as do their rank
 * updates; the call allocates nothing and synchronizes nothing, so it can be
 * recorded in a CUDA graph once the handle has run one eager call.
 * Status as jk_build (JK_ERR_OOM against the JK_OP_BATCHED query). */
jk_status jk_build_batched(jk_handle h, int32_t nmol, const jk_factor *f,
                           const int32_t *nd_per_mol, const jk_density *d,
                           double *const *J, double *const *K,
                           jk_precision p, void *stream);

/* jk_adjoint: gradients of E = sum_s <W_s, K_s> + <V_s, J_s> under the
 * Frobenius pairing <A,B> = Tr A^T B (the self-adjoint form of Eq. 1, Sec. II.A):
 *   dX_s = sum_P L^P W_s (L^P Y_s)   + J(V_s) Y_s
 *   dY_s = sum_P L^P W_s^T (L^P X_s) + J(V_s) X_s
 *   dL^P = sym( sum_s W_s (L^P Y_s) X_s^T + Y_s (L^P X_s)^T W_s
 *               + <V_s, L^P> D_s + gamma_{P,s} V_s ),  sym(G) = (G + G^T)/2
 * W, V : [nd][nbf][nbf] FP64 (either may be NULL = zero seeds).
 * dX, dY : [nd] blocks of [nbf][k_s] FP64, concatenated in density order.
 *          For a symmetric density Y = X, so dX receives dX_s + dY_s and the
 *          dY block is written with zeros.
 * dL : [naux][nbf][nbf] FP64, or NULL (not formed). */
jk_status jk_adjoint(jk_handle h, const jk_factor *f, int32_t nd,
                     const jk_density *d, const double *W, const double *V,
                     double *dX, double *dY, double *dL,
                     jk_precision p, void *stream);

/* ---- dense (general, non-symmetric) densities -----------------------------
 * The general primitive of Eq. 4 (Sec. II.C) takes a weight density that is
 * neither symmetric nor given in factored form.  For dense D:
 *   J(D) = sum_P <L^P, D> L^P          K(D) = sum_P L^P D L^P
 * J sees only the symmetric part of D; K(D^T) = K(D)^T.  K runs on the engine
 * `p` selects (per aux chunk: the panels L^P D for all densities in one GEMM,
 * then each K_s as the reduction of those panels against L^P itself); J runs
 * on the FP64 streams in both precisions (the metric dot <L^P, D> read from
 * D directly).  Arena: jk_workspace_query with JK_OP_BUILD_DENSE /
 * JK_OP_DENSITY_GRAD (the aux chunk follows JK_OPT_AUX_CHUNK; tuned
 * configurations do not apply).  Validation and status as jk_build.
 *
 * jk_build_dense: J_s = J(D_s), K_s = K(D_s).
 *   D    : [nd][nbf][nbf] FP64 input (16-byte aligned).
 *   J, K : [nd][nbf][nbf] FP64 outputs; either may be NULL (not formed). */
jk_status jk_build_dense(jk_handle h, const jk_factor *f, int32_t nd, const double *D,
                         double *J, double *K, jk_precision p, void *stream);

/* jk_density_grad: the density gradient of E = sum_s <W_s, K(D_s)> + <V_s, J(D_s)>
 * (Eq. 1, Sec. II.A), with D_s a free dense matrix:
 *   G_s = dE/dD_s = K(W_s) + J(V_s)
 * (K and J are self-adjoint under the Frobenius pairing).  jk_adjoint's
 * dX_s = G_s Y_s and dY_s = G_s^T X_s are this gradient carried through
 * D_s = X_s Y_s^T.  W, V: [nd][nbf][nbf] FP64 seeds, either may be NULL
 * (zero; both NULL writes G = 0).  G: [nd][nbf][nbf] FP64 output. */
jk_status jk_density_grad(jk_handle h, const jk_factor *f, int32_t nd, const double *W,
                          const double *V, double *G, jk_precision p, void *stream);

/* ---- bra-ket pairings -------------------------------------------------------
 * jk_pair: the scalar contractions of Eq. 4 (Sec. II.C) with the plain CD
 * integrals between nl left and nr right weight densities (the J and K terms
 * Eq. 5, Sec. II.D, combines):
 *   Jp[a][b] = sum W_L^{mu nu} (mu nu|lam sig) W_R^{lam sig} = <W_L^a, J(W_R^b)>
 *   Kp[a][b] = sum W_L^{mu nu} (mu lam|nu sig) W_R^{lam sig} = <W_L^a, K(W_R^b)>
 * with factored W_L^a = X_a Y_a^T (left[a]) and W_R^b = X_b Y_b^T (right[b]),
 * one factor.  Both scalars are invariant under W_L <-> W_R (bra-ket
 * symmetry): jk_pair(right, left) gives the transposes.
 *   Jp, Kp : [nl][nr] FP64 device outputs; either may be NULL (not formed).
 * The right densities' J_b, K_b are built as by jk_build (engine `p`, tuned
 * configuration of that build) into the workspace, then each pairing is
 * <X_a Y_a^T, M_b> = sum (X_a . M_b Y_a) in FP64.  Arena: jk_workspace_query
 * with JK_OP_PAIR.  Validation and status as jk_build (nl, nr in [1, 64]). */
jk_status jk_pair(jk_handle h, const jk_factor *f, int32_t nl, const jk_density *left, int32_t nr,
                  const jk_density *right, double *Jp, double *Kp, jk_precision p, void *stream);

/* ---- Laplace (LT-AO) builds -------------------------------------------------
 * jk_build_laplace: the nq builds of the Laplace representation (Eq. 3,
 * Sec. II.B), each on energy-scaled coefficients
 *   X_k[mu][p] = CX[mu][p] exp(sx alpha_k epsX[p] / 2)
 *   Y_k[mu][p] = CY[mu][p] exp(sy alpha_k epsY[p] / 2)        D_k = X_k Y_k^T
 * (sx = +1 for occupied, -1 for virtual orbital energies, so that each
 * column pair carries the factorized exp(-alpha_k D) of the denominator).
 *   alpha, w : host arrays of nq quadrature exponents and weights (w may be
 *              NULL); nq in [1, 64], all finite.
 *   CX, CY   : [nbf][m] FP64 device; epsX, epsY: [m] FP64 device.  CY and
 *              epsY NULL: Y_k = X_k (CY = CX, epsY = epsX, sy = sx), a
 *              symmetric density per point, built at half the K cost.
 *   J, K     : without weights [nq][nbf][nbf] (J_k = J(D_k), K_k = K(D_k));
 *              with weights [nbf][nbf]: sum_k w_k J_k and sum_k w_k K_k,
 *              summed in FP64 in increasing k.  Either may be NULL.
 * The scaling is one elementwise kernel; the nq points are the densities of
 * one ordinary build (engine `p`, the tuned configuration of that build).
 * Arena: jk_workspace_query with JK_OP_LAPLACE.  Status as jk_build; m must
 * lie in [1, 4 nbf]. */
jk_status jk_build_laplace(jk_handle h, const jk_factor *f, int32_t nq, const double *alpha, const double *w,
                           int32_t m, const double *CX, const double *epsX, int32_t sx, const double *CY,
                           const double *epsY, int32_t sy, double *J, double *K, jk_precision p, void *stream);

/* ---- building without a caller arena -------------------------------------
 * The paper has no counterpart of this entry point; it serves callers that
 * cannot allocate device memory at all -- e.g. code running inside a CUDA
 * graph stream capture (where cudaMalloc is illegal), plugins or callbacks
 * whose host application forbids them to grow the device memory footprint,
 * or tight loops where an allocation could synchronize the device.
 *
 * jk_build_noalloc computes exactly what jk_build(..., JK_FP64, ...) computes
 * (plain FP64 engine; same kernels, so the same bits) without a handle or an
 * arena: its workspace is one file-scope device array of
 * JK_STATIC_SCRATCH_BYTES that every GPU which loads the library holds until
 * the process exits.  It calls no cudaMalloc, cudaFree or other allocating
 * routine.  The caller passes inputs and outputs as for jk_build.
 *  - Returns JK_ERR_OOM, before launching anything, if the problem's FP64
 *    workspace would exceed JK_STATIC_SCRATCH_BYTES (roughly: the panel
 *    buffer naux*nbf*ctot*8 bytes, ctot = sum of X and Y widths, plus small
 *    terms); use jk_build for larger problems.
 *  - The first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before starting any stream capture.
 *  - All calls on a device share the one array and it keeps the last call's
 *    contents: calls whose work overlaps on the GPU (different streams, or
 *    different host threads) race on it and must be serialized by the caller.
 *  - Pointers are taken to be device memory (not checked).  Shapes are
 *    checked as in jk_build (JK_ERR_SHAPE); every pointer, outputs included,
 *    must be 16-byte aligned (JK_ERR_ARG).  All these checks, and the size
 *    check above, come before any CUDA call. */
#define JK_STATIC_SCRATCH_BYTES ((size_t)32 << 20)
jk_status jk_build_noalloc(const jk_factor *f, int32_t nd, const jk_density *d,
                           double *J, double *K, void *stream);

/* Handle options.  JK_OPT_AUX_CHUNK: this many aux indices P per internal
 * chunk, the last one smaller (0 = automatic, chosen from a workspace budget;
 * a larger chunk needs a larger workspace, see jk_workspace_query).  Chunking
 * over P is a pure memory knob (the paper's aux-index blocking, Table
 * "precision", Sec. V.F): FP64 results change only by summation order. */
typedef enum {
    JK_OPT_AUX_CHUNK = 0,   /* >= 0; 0 = automatic                                */
    JK_OPT_SCHEDULE = 1,    /* -1 = tuned/default, 0 = per-density launches,
                               1 = grouped persistent launches (split precision)  */
    JK_OPT_RASTER = 2,      /* -1 = tuned/default, 0 = n-tile fastest,
                               1 = m-tile fastest (tile order of the sliced GEMM) */
    JK_OPT_USE_TUNED = 3,   /* 1 (default) = apply autotuned configurations,
                               0 = ignore them                                    */
    /* 4 is unused */
    JK_OPT_HOST_CHUNK = 5,  /* jk_build_host: aux indices per streamed chunk of
                               the factor, 0 = automatic (about 12 chunks)         */
    JK_OPT_SLICER = 6,      /* digit extraction of the split engine's vector
                               slicer: 0 (default) integer arithmetic, 1 FP32
                               additions (fewer instructions per element; an
                               equally exact split, digits differ only where a
                               digit rounds a tie)                               */
    JK_OPT_SYRK = 7,        /* symmetric densities (both engines): 0 (default)
                               full rank update, 1 only the row blocks of
                               128 rows from their diagonal on (K of the
                               symmetric build, the U = V case of Sec. II.C,
                               is symmetric), the rest mirrored; results
                               within rounding of those of 0                  */
    JK_OPT_PACKED_FACTOR = 8, /* 0 (default) dense factor; 1 every factor passed
                               to jk_build, jk_build_batched, jk_adjoint,
                               jk_build_dense, jk_density_grad, jk_pair,
                               jk_build_laplace and jk_autotune* on this handle
                               holds packed upper triangles, L = [naux]
                               [nbf(nbf+1)/2] row-major, diagonal included
                               (position a*nbf - a(a-1)/2 + b - a for a <= b):
                               half the device memory.  Each aux chunk is
                               expanded into the workspace before its
                               products; the J back-contraction reads the
                               packed form (both of its forms, JK_OPT_J_PATH;
                               and so do the dense calls' metric dots).  Results equal the dense factor's
                               bit for bit at the same aux chunk (the automatic
                               chunk can be smaller, as the expanded copy counts
                               against its budget: then they differ by
                               summation order only).  Size the arena with
                               jk_workspace_query_handle (the handle-free query
                               assumes a dense factor).  The host builds (their
                               factor is in host memory) return
                               JK_ERR_UNSUPPORTED while it is 1; dL of the
                               adjoint stays dense [naux][nbf][nbf]            */
    JK_OPT_TILE = 9,      /* split engine, six-slice products: -1 = tuned/
                               default, 0 = output tiles of 128 x 80, 1 = 128 x
                               64 (more, narrower tiles; a tuning candidate).
                               Results are identical: the tile only changes
                               which outputs a CTA forms, not how            */
    JK_OPT_ADJOINT_SLICES = 10, /* split jk_adjoint: BF16 slices per operand of
                               every product, 7 (default: 56-bit operands, 28
                               slice pairs, 128 x 64 tiles) or 6 (48-bit, 21
                               pairs, about a quarter fewer tensor-core flops).
                               The adjoint's dX, dY are sums over aux indices
                               and basis functions of three chained products,
                               where 48-bit operands leave errors of ~1e-14
                               relative to max |dX|; 56 bits bring them below
                               the FP64 engine's own                          */
    JK_OPT_J_PATH = 11      /* split builds: how J_s = sum_P gamma_{P,s} L^P is
                               formed (Eq. 4's J term; every value gives the
                               same J to within the split engine's error).
                               -1 (default) = automatic: on the tensor cores
                               when n(n+1)/2 * naux * nd >= 4e9, else as 0;
                               0 = an FP64 pass over the factor on a second
                               stream, overlapping the rank updates; 1 = on the
                               tensor cores: each aux chunk of the factor
                               sliced transposed over the upper triangle and
                               multiplied by gamma's slices (one sliced GEMM),
                               the result added onto both triangles in chunk
                               order                                           */
} jk_option;
/* Options set explicitly on a handle override tuned configurations. */
jk_status jk_set_option(jk_handle h, jk_option opt, int64_t value);

/* jk_pack_factor: the packed form of a symmetric factor, for
 * JK_OPT_PACKED_FACTOR (L^P = L^P^T, Sec. II.C's CD vectors; only the upper
 * triangle is read).  P[p][a*nbf - a(a-1)/2 + b - a] = L[p][a][b], a <= b.
 *   L : [naux][nbf][nbf] FP64 device input (16-byte aligned).
 *   P : [naux][nbf(nbf+1)/2] FP64 device output, caller-owned, not
 *       overlapping L (16-byte aligned for use as a factor).
 * One kernel on `stream`, no workspace.  Status: JK_ERR_SHAPE if nbf is
 * outside [1, 65535] or naux < 1; JK_ERR_ARG for a NULL, misaligned,
 * non-device or overlapping pointer (nothing is launched). */
jk_status jk_pack_factor(jk_handle h, int32_t nbf, int32_t naux, const double *L, double *P, void *stream);

/* ---------------------------------------------------------------------------
 * Autotuner.  A configuration is the set of run-time choices a build makes
 * (aux-index chunk, launch schedule, GEMM tile order and tile width).  jk_autotune times the
 * candidate configurations of one problem with CUDA events on `stream` (it
 * synchronizes the stream, so it must not be called during stream capture),
 * keeps the fastest in a process-wide cache keyed by a shape bucket (op,
 * precision, SM count, nbf, naux, densities, total width, molecules) and
 * returns it.  Later jk_build / jk_build_batched calls whose shapes fall in a
 * cached bucket use that configuration (unless the handle sets the option
 * explicitly or JK_OPT_USE_TUNED is 0); jk_workspace_query accounts for it.
 * Candidates that do not fit the handle's arena are skipped.  J and K are
 * overwritten with the result of the last candidate run (all candidates agree
 * to the precision's tolerance).  reps >= 1 timed builds per candidate.
 * ------------------------------------------------------------------------- */
typedef struct {
    int32_t aux_chunk;   /* aux indices per chunk, 0 = automatic */
    int32_t schedule;    /* 0 per-density launches, 1 grouped persistent launches */
    int32_t raster;      /* 0 n-tile fastest, 1 m-tile fastest */
    int32_t tile;        /* sliced GEMM output tiles: 0 128 x 80, 1 128 x 64 */
} jk_tune_config;

jk_status jk_autotune(jk_handle h, const jk_factor *f, int32_t nd, const jk_density *d,
                      double *J, double *K, jk_precision p, void *stream, int32_t reps,
                      jk_tune_config *best, double *best_ms);
jk_status jk_autotune_batched(jk_handle h, int32_t nmol, const jk_factor *f,
                              const int32_t *nd_per_mol, const jk_density *d,
                              double *const *J, double *const *K, jk_precision p,
                              void *stream, int32_t reps, jk_tune_config *best,
                              double *best_ms);
/* Cached configuration for a problem's bucket (host only: pointers are not
 * dereferenced or checked).  JK_OK if found, JK_ERR_UNSUPPORTED if not. */
jk_status jk_tune_lookup(jk_op op, int32_t nmol, const jk_factor *f, const int32_t *nd_per_mol,
                         int32_t nd, const jk_density *d, jk_precision p, int32_t num_sms,
                         jk_tune_config *cfg);
/* The cache as text, one entry per line, for saving between processes.
 * export: writes at most cap bytes (NUL-terminated) and the full length
 * (without the NUL) to *len; import merges lines (later entries win) and
 * returns JK_ERR_ARG on a malformed line (entries before it are kept);
 * clear empties the cache. */
jk_status jk_tune_export(char *buf, size_t cap, size_t *len);
jk_status jk_tune_import(const char *text);
jk_status jk_tune_clear(void);

/* Wait for the stream and report any device-side error flag raised by this
 * handle's kernels (e.g. JK_ERR_TIMEOUT from a bounded wait); clears it. */
jk_status jk_sync_status(jk_handle h, void *stream);

const char *jk_status_string(jk_status s);
/* Message of the last failing call on this handle ("" if none). */
const char *jk_last_error(jk_handle h);
/* Library version string. */
const char *jk_version(void);

/* ---- instrumentation (does not change results) ---------------------------
 * Kernels launched by this handle since creation or the last reset. */
int64_t jk_launch_count(jk_handle h);
/* on != 0: bracket every launch with CUDA events on the call's stream and
 * accumulate per-kernel-kind device time.  Costs two event records per launch. */
jk_status jk_profile_enable(jk_handle h, int32_t on);
/* Zero the launch count and the accumulated times. */
jk_status jk_profile_reset(jk_handle h);
/* Dense tensor-core flops issued by this handle's kernels since the last reset
 * (2*M*N*K per MMA instruction, over the padded tiles actually issued). */
double jk_issued_tensor_flops(jk_handle h);
/* Number of kernel kinds and the name of kind i (NULL if out of range). */
int32_t jk_profile_kinds(void);
const char *jk_profile_kind_name(int32_t kind);
/* Total device time (ms) and launches of one kind since the last reset;
 * waits for the recorded events. */
jk_status jk_profile_read(jk_handle h, int32_t kind, double *ms, int64_t *launches);

#ifdef __cplusplus
}
#endif
#endif /* JK_H */
