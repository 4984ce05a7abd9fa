// Plain FP64 engine: every product and every sum in IEEE double.
//
// This is the reference GPU engine the split-precision path is measured
// against.  Data flow of one build (Sec. II.C, Eq. 4):
//   Z      = [X_0 | Y_0 | X_1 | Y_1 | ...]             (nbf x ctot, packed)
//   for each chunk of pc aux indices P:
//     T^P  = L^P Z                                     panels (half-transforms)
//     gamma_{P,s} = sum_{sig,i} T^P[sig][X_s col i] Y_s[sig][i]
//     K_s += sum_{P in chunk} T^P_X (T^P_Y)^T          rank update, fixed order
//   J_s = sum_P gamma_{P,s} L^P                         one L stream, all s
// B300's FP64 units are few, so this engine is bound by FP64 issue rate, not
// by HBM; it exists to be correct, deterministic and a fair baseline.
#include <cstdarg>

#include <algorithm>
#include <vector>

#include "jk_internal.h"
#include "packed.cuh"

namespace jk {

// Generic operand addressing: element (row r, reduction index kk) of batch b
// lives at p + b*sb + r*sr + (kk / kin)*sko + (kk % kin)*ski.  A two-level
// reduction index lets one kernel sum over (P, i) pairs without repacking.
struct GOp {
    const double *p;
    long long sb, sr, sko, ski;
    int kin;
};

static GOp gop(const double *p, long long sb, long long sr, long long sko,
               long long ski, int kin) {
    GOp g;
    g.p = p; g.sb = sb; g.sr = sr; g.sko = sko; g.ski = ski; g.kin = kin;
    return g;
}

constexpr int GBM = 64, GBN = 64, GBK = 16;
constexpr int kMaxRankSplit = 8;   // most aux-index groups one FP64 rank update is split into
constexpr int kMaxAdjSplit = 16;   // the same for the adjoint's n x k products

// C_b[m][n] = alpha * sum_kk A_b(m,kk) B_b(n,kk) + beta * C_b[m][n]
// 64x64 tile per CTA, 256 threads, 4x4 outputs per thread; sums run in
// increasing kk, so results are bit-reproducible for fixed shapes.
__global__ void __launch_bounds__(256)
dgemm_nt_kernel(int M, int N, int K, GOp A, GOp B, double *C, long long ldc,
                long long scb, double alpha, double beta) {
    __shared__ double As[GBK][GBM];
    __shared__ double Bs[GBK][GBN];
    const int b = blockIdx.z;
    const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const double *Ab = A.p + (long long)b * A.sb;
    const double *Bb = B.p + (long long)b * B.sb;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = 0.0;

    for (int k0 = 0; k0 < K; k0 += GBK) {
        for (int e = threadIdx.x; e < GBM * GBK; e += 256) {
            int r, c;
            if (A.ski == 1) { r = e / GBK; c = e % GBK; } else { r = e % GBM; c = e / GBM; }
            int m = m0 + r, kk = k0 + c;
            double v = 0.0;
            if (m < M && kk < K) {
                int ko = kk / A.kin, ki = kk - ko * A.kin;
                v = Ab[(long long)m * A.sr + (long long)ko * A.sko + (long long)ki * A.ski];
            }
            As[c][r] = v;
        }
        for (int e = threadIdx.x; e < GBN * GBK; e += 256) {
            int r, c;
            if (B.ski == 1) { r = e / GBK; c = e % GBK; } else { r = e % GBN; c = e / GBN; }
            int nn = n0 + r, kk = k0 + c;
            double v = 0.0;
            if (nn < N && kk < K) {
                int ko = kk / B.kin, ki = kk - ko * B.kin;
                v = Bb[(long long)nn * B.sr + (long long)ko * B.sko + (long long)ki * B.ski];
            }
            Bs[c][r] = v;
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < GBK; c++) {
            double a[4], bb[4];
#pragma unroll
            for (int i = 0; i < 4; i++) a[i] = As[c][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; j++) bb[j] = Bs[c][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
        }
        __syncthreads();
    }
    double *Cb = C + (long long)b * scb;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        int m = m0 + ty + 16 * i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            int nn = n0 + tx + 16 * j;
            if (nn >= N) continue;
            double *c = Cb + (long long)m * ldc + nn;
            double v = alpha * acc[i][j];
            if (beta != 0.0) v = fma(beta, *c, v);
            *c = v;
        }
    }
}

static jk_status dgemm(jk_ctx *h, int batch, int M, int N, int K, GOp A, GOp B,
                       double *C, long long ldc, long long scb, double alpha,
                       double beta, cudaStream_t st) {
    if (M <= 0 || N <= 0 || batch <= 0) return JK_OK;
    dim3 grid((N + GBN - 1) / GBN, (M + GBM - 1) / GBM, batch);
    {
        LaunchScope ls(h, KK_DGEMM, st);
        dgemm_nt_kernel<<<grid, 256, 0, st>>>(M, N, K, A, B, C, ldc, scb, alpha, beta);
    }
    JK_LAUNCH_CHECK(h);
    return JK_OK;
}

// Z[lam][off + i] = src[lam][i] for one density block.
__global__ void pack_cols_kernel(const double *src, int n, int k, double *Z,
                                 int ctot, int off) {
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= (long long)n * k) return;
    int lam = (int)(e / k), i = (int)(e % k);
    Z[(long long)lam * ctot + off + i] = src[e];
}

// Block-wide sum of one double per thread (256 threads), fixed order.
__device__ __forceinline__ double block_sum_256(double v, double *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) red[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < 8; i++) t += red[i];
    __syncthreads();
    return t;
}

// gamma[s*ldg + P0 + p] = <L^{P0+p}, M_s> for dense n x n matrices M_s
// (M = D_s for the Coulomb dot, M = V_s for the adjoint's <V_s, L^P>).
// One CTA per (p, group of up to 4 densities); L^P is read once per group.
__global__ void __launch_bounds__(256)
frob_stream_kernel(const double *L, long long n2, const double *Mats, int nd,
                   double *gamma, int ldg, int P0) {
    __shared__ double red[8];
    const int p = blockIdx.x;
    const int s0 = blockIdx.y * 4;
    const int ns = min(4, nd - s0);
    const double *LP = L + (long long)(P0 + p) * n2;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (long long e = threadIdx.x; e < n2; e += 256) {
        double l = LP[e];
#pragma unroll
        for (int j = 0; j < 4; j++)
            if (j < ns) acc[j] = fma(l, Mats[(long long)(s0 + j) * n2 + e], acc[j]);
    }
    for (int j = 0; j < ns; j++) {
        double t = block_sum_256(acc[j], red);
        if (threadIdx.x == 0) gamma[(long long)(s0 + j) * ldg + P0 + p] = t;
    }
}

// The same metric dots from packed upper triangles ([naux][n(n+1)/2]):
// <L^P, M> = sum_{a <= b} L^P_t(a,b) (M_ab + M_ba), the diagonal once.  Each
// thread walks its packed positions t, t + 256, ... keeping (a, b)
// incrementally (no square root per element).
__global__ void __launch_bounds__(256)
frob_packed_kernel(const double *L, int n, const double *Mats, int nd, double *gamma, int ldg, int P0) {
    __shared__ double red[8];
    const int p = blockIdx.x;
    const int s0 = blockIdx.y * 4;
    const int ns = min(4, nd - s0);
    const long long ntri = packed::tri_count(n), n2 = (long long)n * n;
    const double *LP = L + (long long)(P0 + p) * ntri;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    int a = 0, b = 0;
    if (threadIdx.x < ntri) packed::tri_row_col(n, threadIdx.x, &a, &b);
    for (long long t = threadIdx.x; t < ntri; t += 256) {
        const double l = LP[t];
        const long long ab = (long long)a * n + b, ba = (long long)b * n + a;
#pragma unroll
        for (int j = 0; j < 4; j++)
            if (j < ns) {
                const double *M = Mats + (long long)(s0 + j) * n2;
                acc[j] = fma(l, a == b ? M[ab] : M[ab] + M[ba], acc[j]);
            }
        packed::tri_advance(n, 256, &a, &b);   // the next position of this thread
    }
    for (int j = 0; j < ns; j++) {
        double t = block_sum_256(acc[j], red);
        if (threadIdx.x == 0) gamma[(long long)(s0 + j) * ldg + P0 + p] = t;
    }
}

// gamma[s*ldg + P0 + p] = sum_{sig,i} T^p[sig][offX_s + i] * Y_s[sig][i]
// (= <L^P, X_s Y_s^T>, from the panel already formed for K).
struct DensTab {
    const double *Y[kMaxDens];
    int offX[kMaxDens];
    int k[kMaxDens];
};

__device__ __forceinline__ double gamma_dot(const double *Tp, int n, long long ctot, const double *Ys, int off, int k,
                                            double *red) {
    double acc = 0.0;
    for (int e = threadIdx.x; e < n * k; e += 256) {
        int sig = e / k, i = e - sig * k;
        acc = fma(Tp[(long long)sig * ctot + off + i], Ys[e], acc);
    }
    return block_sum_256(acc, red);
}

__global__ void __launch_bounds__(256)
gamma_panel_kernel(const double *T, int n, long long ctot, DensTab tab,
                   double *gamma, int ldg, int P0) {
    __shared__ double red[8];
    const int p = blockIdx.x, s = blockIdx.y;
    const double t = gamma_dot(T + (long long)p * n * ctot, n, ctot, tab.Y[s], tab.offX[s], tab.k[s], red);
    if (threadIdx.x == 0) gamma[(long long)s * ldg + P0 + p] = t;
}

// The same for the chunks of many molecules (a batched build's wave) in one
// launch: job i covers blocks b0 .. b0 + np nd - 1 (block (p, s) at
// b0 + s np + p); the densities of all jobs in one table (job i's at d0 ..).
struct GammaJob {
    const double *T;
    double *gamma;
    long long ldT;
    int n, np, nd, P0, ldg, d0, b0;
};
constexpr int MAXGJOB = 64, MAXGDENS = 1024;
struct GammaGroup {
    GammaJob j[MAXGJOB];
    const double *Y[MAXGDENS];
    int offX[MAXGDENS], k[MAXGDENS];
    int njob;
};
__global__ void __launch_bounds__(256) gamma_group_kernel(const __grid_constant__ GammaGroup g) {
    __shared__ double red[8];
    int lo = 0, hi = g.njob - 1;
    while (lo < hi) {   // the last job whose first block is <= blockIdx.x
        const int mid = (lo + hi + 1) >> 1;
        if (g.j[mid].b0 <= static_cast<int>(blockIdx.x)) lo = mid;
        else hi = mid - 1;
    }
    const GammaJob &jb = g.j[lo];
    const int lb = static_cast<int>(blockIdx.x) - jb.b0, s = lb / jb.np, p = lb - s * jb.np;
    const int d = jb.d0 + s;
    const double t = gamma_dot(jb.T + (long long)p * jb.n * jb.ldT, jb.n, jb.ldT, g.Y[d], g.offX[d], g.k[d], red);
    if (threadIdx.x == 0) jb.gamma[(long long)s * jb.ldg + jb.P0 + p] = t;
}

// Out_s[e] = sum_P g[s][P] L^P[e]: one pass over L for up to 8 densities.
// Each thread owns two consecutive entries (16-byte loads); the sum over P
// runs in increasing P.
struct OutTab {
    double *p[8];
};

template <int NS>
__global__ void __launch_bounds__(256)
jstream_kernel(const double *L, long long n2, int naux, const double *g,
               int ldg, OutTab Out) {
    long long e = 2 * (blockIdx.x * (long long)blockDim.x + threadIdx.x);
    if (e >= n2) return;
    const bool pair = (e + 1 < n2) && ((n2 & 1) == 0);
    double a0[NS], a1[NS];
#pragma unroll
    for (int j = 0; j < NS; j++) { a0[j] = 0.0; a1[j] = 0.0; }
    for (int P = 0; P < naux; P++) {
        const double *LP = L + (long long)P * n2 + e;
        double l0, l1 = 0.0;
        if (pair) {
            double2 v = __ldg(reinterpret_cast<const double2 *>(LP));
            l0 = v.x; l1 = v.y;
        } else {
            l0 = __ldg(LP);
            if (e + 1 < n2) l1 = __ldg(LP + 1);
        }
#pragma unroll
        for (int j = 0; j < NS; j++) {
            double gg = __ldg(g + (long long)j * ldg + P);
            a0[j] = fma(gg, l0, a0[j]);
            a1[j] = fma(gg, l1, a1[j]);
        }
    }
#pragma unroll
    for (int j = 0; j < NS; j++) {
        Out.p[j][e] = a0[j];
        if (e + 1 < n2) Out.p[j][e + 1] = a1[j];
    }
}

// Symmetric form: L^P = L^P^T, so J = sum_P g_P L^P is symmetric and only the
// n(n+1)/2 upper-triangle entries are formed (one per thread, consecutive
// threads on consecutive columns of a row), then mirrored: half the FP64 work.
// PK: L is stored as packed upper triangles ([naux][n(n+1)/2]), read at the
// thread's own position t (contiguous across the threads of a warp).  The
// sum runs over P = P0 .. P0 + np - 1 in order; acc adds it to Out (a build
// that takes the aux indices chunk by chunk), else Out is overwritten.
template <int NS, bool PK>
__global__ void __launch_bounds__(64)
jstream_sym_kernel(const double *L, int n, int P0, int np, const double *g, int ldg, int acc, OutTab Out) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= packed::tri_count(n)) return;
    int mu, nu;
    packed::tri_row_col(n, t, &mu, &nu);
    const long long n2 = (long long)n * n;
    const long long e = (long long)mu * n + nu;
    double a[NS];
#pragma unroll
    for (int j = 0; j < NS; j++) a[j] = 0.0;
    const double *Lp = PK ? L + t : L + e;
    const long long pstride = PK ? packed::tri_count(n) : n2;
    for (int P = P0; P < P0 + np; P++) {
        const double l = __ldg(Lp + (long long)P * pstride);
#pragma unroll
        for (int j = 0; j < NS; j++) a[j] = fma(__ldg(g + (long long)j * ldg + P), l, a[j]);
    }
#pragma unroll
    for (int j = 0; j < NS; j++) {
        const double v = acc ? Out.p[j][e] + a[j] : a[j];
        Out.p[j][e] = v;
        if (nu != mu) Out.p[j][(long long)nu * n + mu] = v;
    }
}

// Out[s] (+)= sum_P g[s][P] L^P, P = P0 .. P0 + np - 1, for s < nd (Out[s]
// are [n][n] device arrays; acc: added to them); pk: L holds packed upper
// triangles.
static jk_status jstream(jk_ctx *h, const double *L, int n, int P0, int np,
                         const double *g, int ldg, int nd, double *const *Out,
                         cudaStream_t st, bool pk = false, bool acc = false) {
    const long long ntri = (long long)n * (n + 1) / 2;
    const int blocks = (int)((ntri + 63) / 64);
    for (int s0 = 0; s0 < nd; s0 += 8) {
        int ns = nd - s0 < 8 ? nd - s0 : 8;
        const double *gs = g + (long long)s0 * ldg;
        OutTab o;
        for (int j = 0; j < 8; j++) o.p[j] = j < ns ? Out[s0 + j] : nullptr;
        LaunchScope ls(h, KK_JSTREAM, st);
        switch (ns) {
#define JS(N)                                                                              \
    case N:                                                                                \
        if (pk) jstream_sym_kernel<N, true><<<blocks, 64, 0, st>>>(L, n, P0, np, gs, ldg, acc, o);  \
        else jstream_sym_kernel<N, false><<<blocks, 64, 0, st>>>(L, n, P0, np, gs, ldg, acc, o);    \
        break;
            JS(1) JS(2) JS(3) JS(4) JS(5) JS(6) JS(7) JS(8)
#undef JS
        }
        JK_LAUNCH_CHECK(h);
    }
    return JK_OK;
}

// G^p += sum_s c[s][P0+p] D_s + g[s][P0+p] V_s   (the J terms of dL)
__global__ void gterms_kernel(double *G, long long n2, int pc, int nd,
                              const double *D, const double *V, const double *c,
                              const double *g, int ldg, int P0) {
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    int p = blockIdx.y;
    if (e >= n2) return;
    double acc = G[(long long)p * n2 + e];
    for (int s = 0; s < nd; s++) {
        if (D) acc = fma(c[(long long)s * ldg + P0 + p], D[(long long)s * n2 + e], acc);
        if (V) acc = fma(g[(long long)s * ldg + P0 + p], V[(long long)s * n2 + e], acc);
    }
    G[(long long)p * n2 + e] = acc;
}

// dL^P = (G^p + G^p^T) / 2
__global__ void symmetrize_kernel(const double *G, int n, double *dL) {
    long long n2 = (long long)n * n;
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    int p = blockIdx.y;
    if (e >= n2) return;
    int mu = (int)(e / n), nu = (int)(e % n);
    const double *Gp = G + (long long)p * n2;
    dL[(long long)p * n2 + e] = 0.5 * (Gp[e] + Gp[(long long)nu * n + mu]);
}

// For symmetric densities (Y = X): dX += dY, dY = 0.
__global__ void fold_sym_kernel(double *dX, double *dY, long long cnt) {
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= cnt) return;
    dX[e] += dY[e];
    dY[e] = 0.0;
}

// Many column blocks packed by one launch: job j copies src [n][k] into the
// columns off..off+k-1 of Z [n][ctot]; its elements are numbered from e0 in
// the launch.  The jobs travel in the parameter space.
struct PackJob {
    const double *src;
    double *Z;
    long long e0;
    int n, k, ctot, off;
};
constexpr int MAXPACK = 600;
struct PackGroup {
    PackJob j[MAXPACK];
    int njob;
};
static_assert(sizeof(PackGroup) + 8 <= 32764, "the pack group fits the kernel parameter space");

__global__ void __launch_bounds__(256) pack_group_kernel(const __grid_constant__ PackGroup g, long long total) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= total) return;
    int lo = 0, hi = g.njob - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (g.j[mid].e0 <= t) lo = mid;
        else hi = mid - 1;
    }
    const PackJob &jb = g.j[lo];
    const long long e = t - jb.e0;
    const int lam = (int)(e / jb.k), i = (int)(e % jb.k);
    jb.Z[(long long)lam * jb.ctot + jb.off + i] = jb.src[e];
}

// Z_m = [X_0 | Y_0 | X_1 | ...] of every molecule m (Y omitted for symmetric
// densities): every density block of every molecule in grouped launches.
jk_status pack_z_multi(jk_ctx *h, int nmol, const Problem *pbs, double *const *Z, cudaStream_t st) {
    static thread_local PackGroup grp;
    std::vector<PackJob> jobs;
    for (int m = 0; m < nmol; m++) {
        const Problem &pb = pbs[m];
        for (int s = 0; s < pb.nd; s++) {
            jobs.push_back(PackJob{pb.X[s], Z[m], 0, pb.n, pb.k[s], pb.ctot, pb.offX[s]});
            if (!pb.sym[s]) jobs.push_back(PackJob{pb.Y[s], Z[m], 0, pb.n, pb.k[s], pb.ctot, pb.offY[s]});
        }
    }
    for (size_t i0 = 0; i0 < jobs.size(); i0 += MAXPACK) {
        const int nj = (int)std::min<size_t>(MAXPACK, jobs.size() - i0);
        long long tot = 0;
        for (int i = 0; i < nj; i++) {
            grp.j[i] = jobs[i0 + i];
            grp.j[i].e0 = tot;
            tot += (long long)grp.j[i].n * grp.j[i].k;
        }
        grp.njob = nj;
        {
            LaunchScope ls(h, KK_PACK, st);
            pack_group_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(grp, tot);
        }
        JK_LAUNCH_CHECK(h);
    }
    return JK_OK;
}

static jk_status pack_z(jk_ctx *h, const Problem &pb, double *Z, cudaStream_t st) {
    return pack_z_multi(h, 1, &pb, &Z, st);
}

// F[p][mu][nu] = P[p][t(min(mu,nu), max(mu,nu))] for p < np: symmetric L^P
// expanded from its packed upper triangle (packed.cuh: row-major, diagonal
// included).  One thread per full entry.
__global__ void unpack_sym_kernel(const double *P, int n, long long np, double *F) {
    const long long n2 = (long long)n * n;
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= np * n2) return;
    const long long p = e / n2, r = e - p * n2;
    const int mu = (int)(r / n), nu = (int)(r - (long long)mu * n);
    const long long a = mu < nu ? mu : nu, b = mu < nu ? nu : mu;
    F[e] = P[p * packed::tri_count(n) + packed::tri_index(n, a, b)];
}

jk_status fp64_unpack_sym(jk_ctx *h, const double *packed, int n, long long np, double *full, cudaStream_t st) {
    const long long tot = np * n * n;
    {
        LaunchScope ls(h, KK_PACK, st);
        unpack_sym_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(packed, n, np, full);
    }
    JK_LAUNCH_CHECK(h);
    return JK_OK;
}

// P[p][t] = F[p][a][b] for the packed position t of (a, b), a <= b: the upper
// triangles of np symmetric n x n matrices (packed.cuh layout).  One thread per
// packed entry; consecutive threads read consecutive columns of a row.
__global__ void pack_sym_kernel(const double *F, int n, long long np, double *P) {
    const long long ntri = packed::tri_count(n);
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= np * ntri) return;
    const long long p = e / ntri, t = e - p * ntri;
    int a, b;
    packed::tri_row_col(n, t, &a, &b);
    P[e] = F[p * (long long)n * n + (long long)a * n + b];
}

jk_status fp64_pack_sym(jk_ctx *h, const double *full, int n, long long np, double *packed_out, cudaStream_t st) {
    const long long tot = np * packed::tri_count(n);
    {
        LaunchScope ls(h, KK_PACK, st);
        pack_sym_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(full, n, np, packed_out);
    }
    JK_LAUNCH_CHECK(h);
    return JK_OK;
}

// y += x (FP64, elementwise)
__global__ void axpy_kernel(double *y, const double *x, long long cnt) {
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e < cnt) y[e] += x[e];
}

jk_status fp64_axpy(jk_ctx *h, double *y, const double *x, long long cnt, cudaStream_t st) {
    LaunchScope ls(h, KK_MISC, st);
    axpy_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(y, x, cnt);
    JK_LAUNCH_CHECK(h);
    return JK_OK;
}

// C[m][n] = sum_kk A[m*a_sr + kk*a_sk] B[n*b_sr + kk*b_sk] + beta C[m][n], in FP64.
jk_status fp64_gemm_nt(jk_ctx *h, int M, int N, int K, const double *A, long long a_sr, long long a_sk,
                       const double *B, long long b_sr, long long b_sk, double *C, long long ldc, double beta,
                       cudaStream_t st) {
    return dgemm(h, 1, M, N, K, gop(A, 0, a_sr, 0, a_sk, K), gop(B, 0, b_sr, 0, b_sk, K), C, ldc, 0, 1.0, beta, st);
}

jk_status split_pack_z(jk_ctx *h, const Problem &pb, double *Z, cudaStream_t st) {
    return pack_z(h, pb, Z, st);
}

static_assert(sizeof(GammaGroup) <= 32764, "grouped launches fit the kernel parameter space");

// gamma of every listed panel chunk (fp64_gamma_panel's work) in grouped
// launches of up to MAXGJOB chunks and MAXGDENS densities.
jk_status fp64_gamma_group(jk_ctx *h, const std::vector<GammaItem> &items, cudaStream_t st) {
    static thread_local GammaGroup grp;
    size_t i0 = 0;
    while (i0 < items.size()) {
        int nj = 0, nden = 0;
        long long blocks = 0;
        while (i0 + nj < items.size() && nj < MAXGJOB && nden + items[i0 + nj].pb->nd <= MAXGDENS) {
            const GammaItem &it = items[i0 + nj];
            const Problem &pb = *it.pb;
            GammaJob &j = grp.j[nj];
            j.T = it.T;
            j.gamma = it.gamma;
            j.ldT = it.ldT;
            j.n = pb.n;
            j.np = it.np;
            j.nd = pb.nd;
            j.P0 = it.P0;
            j.ldg = pb.naux;
            j.d0 = nden;
            j.b0 = static_cast<int>(blocks);
            for (int s = 0; s < pb.nd; s++) {
                grp.Y[nden + s] = pb.sym[s] ? pb.X[s] : pb.Y[s];
                grp.offX[nden + s] = pb.offX[s];
                grp.k[nden + s] = pb.k[s];
            }
            nden += pb.nd;
            blocks += static_cast<long long>(it.np) * pb.nd;
            if (blocks > 0x7fffffffLL) return set_error(h, JK_ERR_SHAPE, "too many gamma blocks");
            nj++;
        }
        if (nj == 0) return set_error(h, JK_ERR_SHAPE, "a molecule with more densities than one gamma launch takes");
        grp.njob = nj;
        {
            LaunchScope ls(h, KK_GAMMA, st);
            gamma_group_kernel<<<static_cast<unsigned>(blocks), 256, 0, st>>>(grp);
        }
        JK_LAUNCH_CHECK(h);
        i0 += nj;
    }
    return JK_OK;
}

// gamma[s][P0 + p] = sum_{sig,i} T^p[sig][offX_s + i] Y_s[sig][i] for p < np.
jk_status fp64_gamma_panel(jk_ctx *h, const Problem &pb, const double *T, long long ldT, int np, double *gamma,
                           int P0, cudaStream_t st) {
    DensTab tab;
    for (int s = 0; s < pb.nd; s++) {
        tab.Y[s] = pb.sym[s] ? pb.X[s] : pb.Y[s];
        tab.offX[s] = pb.offX[s];
        tab.k[s] = pb.k[s];
    }
    LaunchScope ls(h, KK_GAMMA, st);
    gamma_panel_kernel<<<dim3(np, pb.nd), 256, 0, st>>>(T, pb.n, ldT, tab, gamma, pb.naux, P0);
    JK_LAUNCH_CHECK(h);
    return JK_OK;
}

// out[s*naux + P] = <L^P, M_s> for dense n x n matrices M_s (s < nd); pk: L
// holds packed upper triangles.
jk_status fp64_frob_all(jk_ctx *h, const double *L, int n, int naux, const double *Mats, int nd, double *out,
                        cudaStream_t st, bool pk) {
    const long long n2 = (long long)n * n;
    {
        LaunchScope ls(h, KK_FROB, st);
        if (pk)
            frob_packed_kernel<<<dim3(naux, (nd + 3) / 4), 256, 0, st>>>(L, n, Mats, nd, out, naux, 0);
        else
            frob_stream_kernel<<<dim3(naux, (nd + 3) / 4), 256, 0, st>>>(L, n2, Mats, nd, out, naux, 0);
    }
    JK_LAUNCH_CHECK(h);
    return JK_OK;
}

// out[s] = sum_P g[s*naux + P] L^P (dense [nd][n][n] output); pk as above.
jk_status fp64_jstream_dense(jk_ctx *h, const double *L, int n, int naux, const double *g, int nd, double *out,
                             cudaStream_t st, bool pk) {
    double *ptrs[kMaxDens];
    for (int s = 0; s < nd; s++) ptrs[s] = out + (long long)s * n * n;
    return jstream(h, L, n, 0, naux, g, naux, nd, ptrs, st, pk);
}

jk_status fp64_jstream(jk_ctx *h, const Problem &pb, const double *gamma, cudaStream_t st) {
    return jstream(h, pb.L, pb.n, 0, pb.naux, gamma, pb.naux, pb.nd, pb.J, st, pb.packed);
}

// J_s (+)= sum_P gamma_{P,s} L^P over the aux chunk P0 .. P0 + np - 1 (added
// to J unless P0 == 0): a split build's FP64 J, one chunk at a time.
jk_status fp64_jstream_chunk(jk_ctx *h, const Problem &pb, const double *gamma, int P0, int np, cudaStream_t st) {
    return jstream(h, pb.L, pb.n, P0, np, gamma, pb.naux, pb.nd, pb.J, st, pb.packed, P0 > 0);
}


int fp64_default_pchunk(const Problem &pb) {
    // Panel chunk of at most ~256 MB of FP64 (T^P for pc aux indices, and the
    // expanded factor chunk of a packed factor).
    size_t per = (size_t)pb.n * (size_t)pb.ctot * 8 + (pb.packed ? (size_t)pb.n * pb.n * 8 : 0);
    size_t pc = (size_t)256 << 20;
    pc = per ? pc / per : 1;
    if (pc < 1) pc = 1;
    if (pb.aux_chunk > 0) pc = pb.aux_chunk;       // explicit or tuned chunk
    if (pc > (size_t)pb.naux) pc = pb.naux;
    return (int)pc;
}

size_t fp64_build_workspace(const Problem &pb, int pc) {
    size_t n = pb.n, nd = pb.nd;
    size_t b = 0;
    b += align_up(n * pb.ctot * 8);                 // Z
    b += align_up((size_t)pc * n * pb.ctot * 8);    // T chunk
    b += align_up(nd * (size_t)pb.naux * 8);        // gamma
    b += align_up(nd * n * n * 8);                  // dense D (J-only path)
    b += align_up((size_t)kMaxRankSplit * n * n * 8);   // split rank-update partials
    if (pb.packed) b += align_up((size_t)pc * n * n * 8);   // expanded factor chunk
    return b;
}

// out[e] = (accumulate ? out[e] : 0) + sum_b part[b][e], b in increasing order.
__global__ void sum_parts_kernel(double *out, const double *part, int nb, long long cnt, int accumulate) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= cnt) return;
    double acc = accumulate ? out[e] : 0.0;
    for (int b = 0; b < nb; b++) acc += part[(long long)b * cnt + e];
    out[e] = acc;
}

// out[r*ldo + c] (+)= sum_b part[b][r*N + c] for r < M, c < N, b in increasing
// order: the same sum into a block of a larger matrix.
__global__ void sum_parts_ld_kernel(double *out, long long ldo, const double *part, int nb, int M, int N,
                                    int accumulate) {
    const long long MN = (long long)M * N;
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= MN) return;
    const long long r = e / N, c = e - r * N;
    double *o = out + r * ldo + c;
    double acc = accumulate ? *o : 0.0;
    for (int b = 0; b < nb; b++) acc += part[(long long)b * MN + e];
    *o = acc;
}

// C (+)= sum over q in [0, nq) and inner index t in [0, kin) of
// A[m][q][t] B[n][q][t]  (element (m, q, t) of A at A + m*a_sr + q*a_sq + t*a_st,
// likewise B), with C M x N of row stride ldc (0: dense, ldc = N).  A small
// output (few 64 x 64 tiles) would leave most SMs idle for a long reduction,
// so the reduction is split over groups of q: one batched launch of partial
// products (plus one for a remainder group), then their sum into C in a fixed
// order.
static jk_status dgemm_split_q(jk_ctx *h, int M, int N, int nq, int kin, const double *A, long long a_sr,
                               long long a_sq, long long a_st, const double *B, long long b_sr, long long b_sq,
                               long long b_st, double *C, bool accumulate, double *part, int max_split,
                               cudaStream_t st, long long ldc = 0) {
    const long long MN = (long long)M * N;
    const int tiles = ((N + GBN - 1) / GBN) * ((M + GBM - 1) / GBM);
    int ns = (h->num_sms + tiles - 1) / tiles;
    if (ns > max_split) ns = max_split;
    if (ns > nq) ns = nq;
    if (ns < 1) ns = 1;
    const int qb = (nq + ns - 1) / ns;
    const int nfull = nq / qb, rem = nq - nfull * qb;
    if (nfull > 0)
        JK_TRY(dgemm(h, nfull, M, N, qb * kin, gop(A, qb * a_sq, a_sr, a_sq, a_st, kin),
                     gop(B, qb * b_sq, b_sr, b_sq, b_st, kin), part, N, MN, 1.0, 0.0, st));
    if (rem > 0)
        JK_TRY(dgemm(h, 1, M, N, rem * kin, gop(A + (long long)nfull * qb * a_sq, 0, a_sr, a_sq, a_st, kin),
                     gop(B + (long long)nfull * qb * b_sq, 0, b_sr, b_sq, b_st, kin), part + nfull * MN, N, 0,
                     1.0, 0.0, st));
    {
        LaunchScope ls(h, KK_MISC, st);
        if (ldc == 0 || ldc == N)
            sum_parts_kernel<<<(unsigned)((MN + 255) / 256), 256, 0, st>>>(C, part, nfull + (rem > 0), MN,
                                                                          accumulate ? 1 : 0);
        else
            sum_parts_ld_kernel<<<(unsigned)((MN + 255) / 256), 256, 0, st>>>(C, ldc, part, nfull + (rem > 0), M, N,
                                                                             accumulate ? 1 : 0);
    }
    JK_LAUNCH_CHECK(h);
    return JK_OK;
}

// K_s (+)= sum over the chunk's (p, i) of T[p][mu][offX+i] T[p][nu][offY+i].
// A symmetric density under JK_OPT_SYRK forms only row blocks of kSymBlock
// rows from their diagonal on (the rest is mirrored after the last chunk).
static jk_status rank_update_fp64(jk_ctx *h, const Problem &pb, const double *T, int np, int s, bool accumulate,
                                  double *part, cudaStream_t st) {
    const long long sp = (long long)pb.n * pb.ctot;
    const int n = pb.n;
    if (!(pb.sym[s] && h->syrk))
        return dgemm_split_q(h, n, n, np, pb.k[s], T + pb.offX[s], pb.ctot, sp, 1, T + pb.offY[s], pb.ctot, sp, 1,
                             pb.K[s], accumulate, part, kMaxRankSplit, st);
    for (int r0 = 0; r0 < n; r0 += kSymBlock) {
        const int m = n - r0 < kSymBlock ? n - r0 : kSymBlock;
        const long long ro = (long long)r0 * pb.ctot;
        JK_TRY(dgemm_split_q(h, m, n - r0, np, pb.k[s], T + pb.offX[s] + ro, pb.ctot, sp, 1, T + pb.offY[s] + ro,
                             pb.ctot, sp, 1, pb.K[s] + (long long)r0 * n + r0, accumulate, part, kMaxRankSplit, st,
                             n));
    }
    return JK_OK;
}

jk_status fp64_build(jk_ctx *h, const Problem &pb, cudaStream_t st) {
    const bool J = pb.wantJ, K = pb.wantK;
    const int n = pb.n, naux = pb.naux, nd = pb.nd;
    const long long n2 = (long long)n * n;
    const int pc = fp64_default_pchunk(pb);
    Arena &ar = h->arena;
    double *Z = ar.take<double>((size_t)n * pb.ctot);
    double *T = ar.take<double>((size_t)pc * n * pb.ctot);
    double *gamma = ar.take<double>((size_t)nd * naux);
    double *D = ar.take<double>((size_t)nd * n2);
    double *part = ar.take<double>((size_t)kMaxRankSplit * n2);
    double *Lx = pb.packed ? ar.take<double>((size_t)pc * n2) : nullptr;
    if (!Z || !T || !gamma || !D || !part || (pb.packed && !Lx))
        return set_error(h, JK_ERR_OOM, "workspace too small for the FP64 build");
    const long long ntri = packed::tri_count(n);
    // L^{P0..P0+np-1} as dense [np][n][n]: the factor itself, or its packed
    // triangles expanded into Lx.
    auto chunk_of = [&](int P0, int np, const double **out) -> jk_status {
        if (!pb.packed) {
            *out = pb.L + (long long)P0 * n2;
            return JK_OK;
        }
        JK_TRY(fp64_unpack_sym(h, pb.L + (long long)P0 * ntri, n, np, Lx, st));
        *out = Lx;
        return JK_OK;
    };

    if (K) {
        JK_TRY(pack_z(h, pb, Z, st));
        DensTab tab;
        for (int s = 0; s < nd; s++) {
            tab.Y[s] = pb.sym[s] ? pb.X[s] : pb.Y[s];
            tab.offX[s] = pb.offX[s];
            tab.k[s] = pb.k[s];
        }
        for (int P0 = 0; P0 < naux; P0 += pc) {
            const int np = naux - P0 < pc ? naux - P0 : pc;
            const double *Lc;
            JK_TRY(chunk_of(P0, np, &Lc));
            // T[(p,mu)][c] = sum_lam L^{P0+p}[mu][lam] Z[lam][c]
            JK_TRY(dgemm(h, 1, np * n, pb.ctot, n,
                         gop(Lc, 0, n, 0, 1, n),
                         gop(Z, 0, 1, 0, pb.ctot, n),
                         T, pb.ctot, 0, 1.0, 0.0, st));
            if (J) {
                LaunchScope ls(h, KK_GAMMA, st);
                gamma_panel_kernel<<<dim3(np, nd), 256, 0, st>>>(T, n, pb.ctot, tab, gamma, naux, P0);
                JK_LAUNCH_CHECK(h);
            }
            // K_s (+)= sum_{p,i} T[p][mu][offX+i] T[p][nu][offY+i]
            for (int s = 0; s < nd; s++) JK_TRY(rank_update_fp64(h, pb, T, np, s, P0 > 0, part, st));
        }
    } else if (J) {
        // J only: gamma from the dense densities D_s = X_s Y_s^T.
        for (int s = 0; s < nd; s++) {
            const double *Ys = pb.sym[s] ? pb.X[s] : pb.Y[s];
            JK_TRY(dgemm(h, 1, n, n, pb.k[s], gop(pb.X[s], 0, pb.k[s], 0, 1, pb.k[s]),
                         gop(Ys, 0, pb.k[s], 0, 1, pb.k[s]), D + (long long)s * n2, n, 0,
                         1.0, 0.0, st));
        }
        if (!pb.packed) {
            LaunchScope ls_f(h, KK_FROB, st);
            frob_stream_kernel<<<dim3(naux, (nd + 3) / 4), 256, 0, st>>>(pb.L, n2, D, nd, gamma, naux, 0);
        }
        JK_LAUNCH_CHECK(h);
        // packed factor: the same metric dots chunk by chunk on the expanded copy
        for (int P0 = 0; pb.packed && P0 < naux; P0 += pc) {
            const int np = naux - P0 < pc ? naux - P0 : pc;
            const double *Lc;
            JK_TRY(chunk_of(P0, np, &Lc));
            {
                LaunchScope ls_f(h, KK_FROB, st);
                frob_stream_kernel<<<dim3(np, (nd + 3) / 4), 256, 0, st>>>(Lc, n2, D, nd, gamma + P0, naux, 0);
            }
            JK_LAUNCH_CHECK(h);
        }
    }
    if (K && h->syrk)
        for (int s = 0; s < nd; s++)
            if (pb.sym[s]) JK_TRY(mirror_sym_blocks(h, pb.K[s], n, st));
    if (J) JK_TRY(jstream(h, pb.L, n, 0, naux, gamma, naux, nd, pb.J, st, pb.packed));
    return JK_OK;
}

// ---- dense densities -----------------------------------------------------
// K_s = sum_P (L^P DK_s)(L^P)^T: per aux chunk one batched GEMM forms the
// panels T[(p, mu)][s*n + nu] = (L^p DK_s)[mu][nu] for every density, then
// each K_s is the reduction over (p, nu) of T against L^p itself (the second
// factor needs no panel).  J_s = sum_P <L^P, DJ_s> L^P on the FP64 streams.

// Aux indices per chunk: the panel chunk (pc x n x nd*n doubles) within
// ~256 MB unless a chunk is set, and its rows within the GEMM grid's limit.
static int fp64_dense_pchunk(const DenseProb &dp) {
    const size_t per = (size_t)dp.n * dp.n * dp.nd * 8 + (dp.packed ? (size_t)dp.n * dp.n * 8 : 0);
    size_t pc = per ? ((size_t)256 << 20) / per : 1;
    if (pc < 1) pc = 1;
    if (dp.aux_chunk > 0) pc = dp.aux_chunk;
    if (pc > (size_t)dp.naux) pc = dp.naux;
    const size_t maxrows = (size_t)65535 * GBM;
    if (pc * dp.n > maxrows) pc = maxrows / dp.n;
    return (int)pc;
}

size_t fp64_dense_workspace(const DenseProb &dp) {
    const size_t n2 = (size_t)dp.n * dp.n, nd = dp.nd;
    size_t b = 0;
    if (dp.DK) {
        b += align_up((size_t)fp64_dense_pchunk(dp) * n2 * nd * 8);   // panels T
        b += align_up((size_t)kMaxRankSplit * n2 * 8);               // rank-update partials
        if (dp.packed) b += align_up((size_t)fp64_dense_pchunk(dp) * n2 * 8);   // expanded factor chunk
    }
    if (dp.DJ) {
        b += align_up(nd * (size_t)dp.naux * 8);                     // gamma
        if (dp.add_j) b += align_up(nd * n2 * 8);                    // J before it joins K
    }
    return b;
}

jk_status fp64_dense(jk_ctx *h, const DenseProb &dp, cudaStream_t st) {
    const int n = dp.n, naux = dp.naux, nd = dp.nd;
    const long long n2 = (long long)n * n, ctot = (long long)nd * n;
    const int pc = fp64_dense_pchunk(dp);
    Arena &ar = h->arena;
    double *T = nullptr, *part = nullptr, *gamma = nullptr, *Jt = nullptr, *Lx = nullptr;
    if (dp.DK) {
        T = ar.take<double>((size_t)pc * n2 * nd);
        part = ar.take<double>((size_t)kMaxRankSplit * n2);
        if (dp.packed) Lx = ar.take<double>((size_t)pc * n2);
        if (!T || !part || (dp.packed && !Lx))
            return set_error(h, JK_ERR_OOM, "workspace too small for the dense FP64 build");
    }
    if (dp.DJ) {
        gamma = ar.take<double>((size_t)nd * naux);
        if (dp.add_j) Jt = ar.take<double>((size_t)nd * n2);
        if (!gamma || (dp.add_j && !Jt)) return set_error(h, JK_ERR_OOM, "workspace too small for the dense J");
    }
    if (dp.DK) {
        for (int P0 = 0; P0 < naux; P0 += pc) {
            const int np = naux - P0 < pc ? naux - P0 : pc;
            // a packed factor chunk is expanded first
            if (dp.packed) JK_TRY(fp64_unpack_sym(h, dp.L + (long long)P0 * packed::tri_count(n), n, np, Lx, st));
            const double *Lc = dp.packed ? Lx : dp.L + (long long)P0 * n2;
            // T[(p, mu)][s*n + nu] = sum_lam L^{P0+p}[mu][lam] DK_s[lam][nu]  (batch s)
            JK_TRY(dgemm(h, nd, np * n, n, n, gop(Lc, 0, n, 0, 1, n), gop(dp.DK, n2, 1, 0, n, n), T, ctot, n,
                         1.0, 0.0, st));
            // K_s (+)= sum_{p, nu} T[(p, mu)][s*n + nu] L^{P0+p}[sig][nu]
            for (int s = 0; s < nd; s++)
                JK_TRY(dgemm_split_q(h, n, n, np, n, T + (long long)s * n, ctot, (long long)n * ctot, 1, Lc, n,
                                     n2, 1, dp.K + s * n2, P0 > 0, part, kMaxRankSplit, st));
        }
    }
    if (dp.DJ) {
        JK_TRY(fp64_frob_all(h, dp.L, n, naux, dp.DJ, nd, gamma, st, dp.packed));
        JK_TRY(fp64_jstream_dense(h, dp.L, n, naux, gamma, nd, dp.add_j ? Jt : dp.J, st, dp.packed));
        if (dp.add_j) JK_TRY(fp64_axpy(h, dp.K, Jt, nd * n2, st));
    }
    return JK_OK;
}

// ---- bra-ket pairings -----------------------------------------------------
// out[a*nr + b] = <A_a B_a^T, M_b> = sum_{mu, i} A_a[mu][i] (M_b B_a)[mu][i]
// for left densities packed as ZL = [A_0 | B_0 | A_1 | ...] (n x ctotL; a
// symmetric density has one block, B = A) and dense M_b ([nr][n][n]): one
// batched GEMM U_b = M_b ZL, then one CTA per (a, b) sums A_a . U_b over the
// (mu, i) of density a in a fixed order.
struct PairTab {
    int offA[kMaxDens], offB[kMaxDens], k[kMaxDens];
};

__global__ void __launch_bounds__(256)
pair_dot_kernel(const double *ZL, const double *U, int n, int ctotL, PairTab tab, double *out, int nr) {
    __shared__ double red[8];
    const int a = blockIdx.x, b = blockIdx.y;
    const int k = tab.k[a], oa = tab.offA[a], ob = tab.offB[a];
    const double *Ub = U + (long long)b * n * ctotL;
    double acc = 0.0;
    const long long nk = (long long)n * k;
    for (long long e = threadIdx.x; e < nk; e += 256) {
        const long long mu = e / k;
        const int i = (int)(e - mu * k);
        acc = fma(ZL[mu * ctotL + oa + i], Ub[mu * ctotL + ob + i], acc);
    }
    const double t = block_sum_256(acc, red);
    if (threadIdx.x == 0) out[(long long)a * nr + b] = t;
}

jk_status fp64_pair_contract(jk_ctx *h, const Problem &left, const double *ZL, const double *M, int nr, double *U,
                             double *out, cudaStream_t st) {
    const int n = left.n, ctotL = left.ctot;
    const long long n2 = (long long)n * n;
    // U_b[mu][c] = sum_nu M_b[mu][nu] ZL[nu][c]   (batch b)
    JK_TRY(dgemm(h, nr, n, ctotL, n, gop(M, n2, n, 0, 1, n), gop(ZL, 0, 1, 0, ctotL, n), U, ctotL,
                 (long long)n * ctotL, 1.0, 0.0, st));
    PairTab tab;
    for (int a = 0; a < left.nd; a++) {
        tab.offA[a] = left.offX[a];
        tab.offB[a] = left.offY[a];
        tab.k[a] = left.k[a];
    }
    {
        LaunchScope ls(h, KK_MISC, st);
        pair_dot_kernel<<<dim3(left.nd, nr), 256, 0, st>>>(ZL, U, n, ctotL, tab, out, nr);
    }
    JK_LAUNCH_CHECK(h);
    return JK_OK;
}

// ---- Laplace (LT-AO) energy scaling ------------------------------------------
// out[k][mu][p] = C[mu][p] exp(s alpha_k eps[p] / 2) for the nq quadrature
// points (Eq. 3): the energy-scaled coefficients each point's build runs on.
struct LapAlpha {
    double a[kMaxDens];
};

__global__ void laplace_scale_kernel(const double *C, const double *eps, int n, int m, double s, LapAlpha al,
                                     int nq, double *out) {
    const long long nm = (long long)n * m;
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= nm * nq) return;
    const int k = (int)(e / nm);
    const long long r = e - (long long)k * nm;
    const int p = (int)(r % m);
    out[e] = C[r] * exp(s * al.a[k] * eps[p] * 0.5);
}

jk_status fp64_laplace_scale(jk_ctx *h, const double *C, const double *eps, int n, int m, int sign,
                             const double *alpha, int nq, double *out, cudaStream_t st) {
    LapAlpha al;
    for (int k = 0; k < nq; k++) al.a[k] = alpha[k];
    const long long tot = (long long)n * m * nq;
    {
        LaunchScope ls(h, KK_PACK, st);
        laplace_scale_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(C, eps, n, m, (double)sign, al, nq, out);
    }
    JK_LAUNCH_CHECK(h);
    return JK_OK;
}

// out[e] = sum_k w_k part[k][e], k in increasing order (weighted Laplace sums).
__global__ void weighted_sum_kernel(double *out, const double *part, LapAlpha w, int nq, long long cnt) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= cnt) return;
    double acc = 0.0;
    for (int k = 0; k < nq; k++) acc = fma(w.a[k], part[(long long)k * cnt + e], acc);
    out[e] = acc;
}

jk_status fp64_weighted_sum(jk_ctx *h, double *out, const double *part, const double *w, int nq, long long cnt,
                            cudaStream_t st) {
    LapAlpha wt;
    for (int k = 0; k < nq; k++) wt.a[k] = w[k];
    {
        LaunchScope ls(h, KK_MISC, st);
        weighted_sum_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(out, part, wt, nq, cnt);
    }
    JK_LAUNCH_CHECK(h);
    return JK_OK;
}

size_t fp64_adjoint_workspace(const Problem &pb, int pc, bool want_dl) {
    size_t n = pb.n, nd = pb.nd, A = pb.naux;
    size_t b = 0;
    b += align_up(n * pb.ctot * 8);                 // Z
    b += align_up((size_t)pc * n * pb.ctot * 8);    // T chunk
    b += 2 * align_up(nd * A * 8);                  // gamma, c
    b += 2 * align_up(nd * n * n * 8);              // D, J(V)
    b += 2 * align_up((size_t)pc * n * pb.kmax * 8);  // U, Vp
    if (want_dl) b += align_up((size_t)pc * n * n * 8);  // G chunk
    b += align_up((size_t)kMaxAdjSplit * n * pb.kmax * 8);   // split dX / dY partials
    if (pb.packed) b += align_up((size_t)pc * n * n * 8);     // expanded factor chunk
    return b;
}

jk_status fp64_adjoint(jk_ctx *h, const Problem &pb, const double *W,
                       const double *V, double *dX, double *dY, double *dL,
                       cudaStream_t st) {
    const int n = pb.n, naux = pb.naux, nd = pb.nd;
    const long long n2 = (long long)n * n;
    const int pc = fp64_default_pchunk(pb);
    Arena &ar = h->arena;
    double *Z = ar.take<double>((size_t)n * pb.ctot);
    double *T = ar.take<double>((size_t)pc * n * pb.ctot);
    double *gamma = ar.take<double>((size_t)nd * naux);
    double *cps = ar.take<double>((size_t)nd * naux);
    double *D = ar.take<double>((size_t)nd * n2);
    double *JV = ar.take<double>((size_t)nd * n2);
    double *U = ar.take<double>((size_t)pc * n * pb.kmax);
    double *Vp = ar.take<double>((size_t)pc * n * pb.kmax);
    double *G = dL ? ar.take<double>((size_t)pc * n2) : nullptr;
    double *part = ar.take<double>((size_t)kMaxAdjSplit * n * pb.kmax);
    double *Lx = pb.packed ? ar.take<double>((size_t)pc * n2) : nullptr;
    if (!Z || !T || !gamma || !cps || !D || !JV || !U || !Vp || (dL && !G) || !part || (pb.packed && !Lx))
        return set_error(h, JK_ERR_OOM, "workspace too small for the FP64 adjoint");

    // Offsets of each density's block in dX / dY.
    long long boff[kMaxDens + 1];
    boff[0] = 0;
    for (int s = 0; s < nd; s++) boff[s + 1] = boff[s] + (long long)n * pb.k[s];
    JK_CUDA_TRY(h, cudaMemsetAsync(dX, 0, boff[nd] * sizeof(double), st));
    JK_CUDA_TRY(h, cudaMemsetAsync(dY, 0, boff[nd] * sizeof(double), st));

    JK_TRY(pack_z(h, pb, Z, st));
    for (int s = 0; s < nd; s++) {
        const double *Ys = pb.sym[s] ? pb.X[s] : pb.Y[s];
        JK_TRY(dgemm(h, 1, n, n, pb.k[s], gop(pb.X[s], 0, pb.k[s], 0, 1, pb.k[s]),
                     gop(Ys, 0, pb.k[s], 0, 1, pb.k[s]), D + (long long)s * n2, n, 0,
                     1.0, 0.0, st));
    }
    if (V) {
        // c_{P,s} = <V_s, L^P>, J(V_s) = sum_P c_{P,s} L^P
        if (pb.packed) {
            JK_TRY(fp64_frob_all(h, pb.L, n, naux, V, nd, cps, st, true));
        } else {
            { LaunchScope ls_f(h, KK_FROB, st);
            frob_stream_kernel<<<dim3(naux, (nd + 3) / 4), 256, 0, st>>>(pb.L, n2, V, nd, cps, naux, 0);
            }
            JK_LAUNCH_CHECK(h);
        }
        double *jv[kMaxDens];
        for (int s = 0; s < nd; s++) jv[s] = JV + (long long)s * n2;
        JK_TRY(jstream(h, pb.L, n, 0, naux, cps, naux, nd, jv, st, pb.packed));
        if (dL && pb.packed) {
            JK_TRY(fp64_frob_all(h, pb.L, n, naux, D, nd, gamma, st, true));
        } else if (dL) {
            { LaunchScope ls_f(h, KK_FROB, st);
            frob_stream_kernel<<<dim3(naux, (nd + 3) / 4), 256, 0, st>>>(pb.L, n2, D, nd, gamma, naux, 0);
            }
            JK_LAUNCH_CHECK(h);
        }
    }
    const bool need_chunks = (W != nullptr) || (dL != nullptr);
    for (int P0 = 0; need_chunks && P0 < naux; P0 += pc) {
        const int np = naux - P0 < pc ? naux - P0 : pc;
        const long long sp = (long long)n * pb.ctot;
        // a packed factor chunk is expanded first
        if (pb.packed) JK_TRY(fp64_unpack_sym(h, pb.L + (long long)P0 * packed::tri_count(n), n, np, Lx, st));
        const double *Lc = pb.packed ? Lx : pb.L + (long long)P0 * n2;
        if (W)
            JK_TRY(dgemm(h, 1, np * n, pb.ctot, n,
                         gop(Lc, 0, n, 0, 1, n),
                         gop(Z, 0, 1, 0, pb.ctot, n), T, pb.ctot, 0, 1.0, 0.0, st));
        if (dL) JK_CUDA_TRY(h, cudaMemsetAsync(G, 0, (size_t)np * n2 * sizeof(double), st));
        for (int s = 0; W && s < nd; s++) {
            const int k = pb.k[s];
            const double *Ws = W + (long long)s * n2;
            const double *Xs = pb.X[s];
            const double *Ys = pb.sym[s] ? pb.X[s] : pb.Y[s];
            const long long nk = (long long)n * k;
            // U^p = W_s T_Y^p ; Vp^p = W_s^T T_X^p     (batched over p)
            JK_TRY(dgemm(h, np, n, k, n, gop(Ws, 0, n, 0, 1, n),
                         gop(T + pb.offY[s], sp, 1, 0, pb.ctot, n), U, k, nk, 1.0, 0.0, st));
            JK_TRY(dgemm(h, np, n, k, n, gop(Ws, 0, 1, 0, n, n),
                         gop(T + pb.offX[s], sp, 1, 0, pb.ctot, n), Vp, k, nk, 1.0, 0.0, st));
            // dX_s += sum_{p,lam} L^p[mu][lam] U^p[lam][i]; dY_s likewise with Vp
            // (an n x k output: split over groups of p)
            JK_TRY(dgemm_split_q(h, n, k, np, n, Lc, n, n2, 1, U, 1, nk, k, dX + boff[s],
                                 true, part, kMaxAdjSplit, st));
            JK_TRY(dgemm_split_q(h, n, k, np, n, Lc, n, n2, 1, Vp, 1, nk, k, dY + boff[s],
                                 true, part, kMaxAdjSplit, st));
            if (dL) {
                // G^p += U^p X_s^T + Y_s Vp^p^T
                JK_TRY(dgemm(h, np, n, n, k, gop(U, nk, k, 0, 1, k), gop(Xs, 0, k, 0, 1, k),
                             G, n, n2, 1.0, 1.0, st));
                JK_TRY(dgemm(h, np, n, n, k, gop(Ys, 0, k, 0, 1, k), gop(Vp, nk, k, 0, 1, k),
                             G, n, n2, 1.0, 1.0, st));
            }
        }
        if (dL) {
            dim3 g2((unsigned)((n2 + 255) / 256), np);
            if (V) {
                { LaunchScope ls_m(h, KK_MISC, st);
                gterms_kernel<<<g2, 256, 0, st>>>(G, n2, np, nd, D, V, cps, gamma, naux, P0);
                }
                JK_LAUNCH_CHECK(h);
            }
            { LaunchScope ls_m(h, KK_MISC, st);
            symmetrize_kernel<<<g2, 256, 0, st>>>(G, n, dL + (long long)P0 * n2);
            }
            JK_LAUNCH_CHECK(h);
        }
    }
    if (V) {
        for (int s = 0; s < nd; s++) {
            const int k = pb.k[s];
            const double *Xs = pb.X[s];
            const double *Ys = pb.sym[s] ? pb.X[s] : pb.Y[s];
            const double *JVs = JV + (long long)s * n2;
            // dX_s += J(V_s) Y_s ; dY_s += J(V_s) X_s
            JK_TRY(dgemm(h, 1, n, k, n, gop(JVs, 0, n, 0, 1, n), gop(Ys, 0, 1, 0, k, n),
                         dX + boff[s], k, 0, 1.0, 1.0, st));
            JK_TRY(dgemm(h, 1, n, k, n, gop(JVs, 0, n, 0, 1, n), gop(Xs, 0, 1, 0, k, n),
                         dY + boff[s], k, 0, 1.0, 1.0, st));
        }
    }
    for (int s = 0; s < nd; s++) {
        if (!pb.sym[s]) continue;
        long long cnt = boff[s + 1] - boff[s];
        { LaunchScope ls_m(h, KK_MISC, st);
        fold_sym_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(dX + boff[s], dY + boff[s], cnt);
        }
        JK_LAUNCH_CHECK(h);
    }
    return JK_OK;
}

}  // namespace jk
