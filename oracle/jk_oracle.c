/*
 * jk_oracle.c -- TEST INFRASTRUCTURE ONLY, not part of the product path.
 *
 * A plain, slow, obviously correct CPU reference for the Cholesky-decomposed
 * Coulomb/exchange (J/K) build of the paper (Eq. 4, Sec. II.C) and for its
 * adjoint (Eq. 1, Sec. II.A).  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline leg of bench.py may load it.  It shares no source with the
 * CUDA path.
 *
 * Precision: inputs and outputs are IEEE double; every product is formed and
 * every sum is accumulated in long double (x87 extended, 64-bit significand),
 * and each output is rounded to double exactly once.  The oracle's own error is
 * therefore far below the 1e-12 relative / 1e-10 absolute parity gates.
 *
 * Conventions (all row-major):
 *   L    [naux][n][n]     Cholesky vectors L^P, symmetric in (mu,nu)
 *   X, Y per density s a block [n][k_s], blocks concatenated in s order
 *   D    [n][n]           dense density (brute-force entry only)
 *   J, K [nd][n][n]       outputs (bare J and K: no factor 2, no -1/2)
 *   W, V [nd][n][n]       adjoint seeds (cotangents of K_s and J_s)
 *
 * Parallelism: OpenMP only over output rows; every sum runs in a fixed order,
 * so results do not depend on the thread count.
 */
#include <stdlib.h>
#include <string.h>

typedef long double ld;

#define IDX2(i, j, ld_) ((size_t)(i) * (size_t)(ld_) + (size_t)(j))

/* ------------------------------------------------------------------------
 * O1: brute force through the explicit four-index tensor.
 * The CD representation (Sec. II.C): (mu nu|lam sig) = sum_P L^P_{mu nu} L^P_{lam sig}.
 * Coulomb:  J_{mu nu} = sum_{lam sig} (mu nu|lam sig) D_{lam sig}
 * Exchange: K_{mu nu} = sum_{lam sig} (mu lam|nu sig) D_{lam sig}
 * (the textbook real-orbital definitions; Eq. 4 with W_R = D).
 * Intended for n <= 24.
 * ---------------------------------------------------------------------- */
int jko_brute(int n, int naux, const double *L, const double *D,
              double *J, double *K)
{
    if (n < 1 || naux < 1 || n > 32) return 1;
    size_t n2 = (size_t)n * n;
    ld *eri = (ld *)calloc(n2 * n2, sizeof(ld));
    if (!eri) return 2;
    for (int a = 0; a < n; a++)
        for (int b = 0; b < n; b++)
            for (int c = 0; c < n; c++)
                for (int d = 0; d < n; d++) {
                    ld s = 0.0L;
                    for (int P = 0; P < naux; P++)
                        s += (ld)L[(size_t)P * n2 + IDX2(a, b, n)] *
                             (ld)L[(size_t)P * n2 + IDX2(c, d, n)];
                    eri[IDX2(IDX2(a, b, n), IDX2(c, d, n), n2)] = s;
                }
    for (int mu = 0; mu < n; mu++)
        for (int nu = 0; nu < n; nu++) {
            ld j = 0.0L, k = 0.0L;
            for (int lam = 0; lam < n; lam++)
                for (int sig = 0; sig < n; sig++) {
                    ld dls = (ld)D[IDX2(lam, sig, n)];
                    j += eri[IDX2(IDX2(mu, nu, n), IDX2(lam, sig, n), n2)] * dls;
                    k += eri[IDX2(IDX2(mu, lam, n), IDX2(nu, sig, n), n2)] * dls;
                }
            J[IDX2(mu, nu, n)] = (double)j;
            K[IDX2(mu, nu, n)] = (double)k;
        }
    free(eri);
    return 0;
}

/* T = L^P Z for one P: T[mu][i] = sum_lam L^P[mu][lam] Z[lam][i]. */
static void panel(int n, int k, const double *LP, const double *Z, ld *T)
{
    #pragma omp parallel for schedule(static)
    for (int mu = 0; mu < n; mu++) {
        for (int i = 0; i < k; i++) {
            ld s = 0.0L;
            for (int lam = 0; lam < n; lam++)
                s += (ld)LP[IDX2(mu, lam, n)] * (ld)Z[IDX2(lam, i, k)];
            T[IDX2(mu, i, k)] = s;
        }
    }
}

/* <A, B> = sum_{ij} A_ij B_ij with B given in long double; fixed order. */
static ld frob_dl(int n, const double *A, const ld *B)
{
    ld s = 0.0L;
    for (size_t e = 0; e < (size_t)n * n; e++) s += (ld)A[e] * B[e];
    return s;
}

static ld frob_dd(int n, const double *A, const double *B)
{
    ld s = 0.0L;
    for (size_t e = 0; e < (size_t)n * n; e++) s += (ld)A[e] * (ld)B[e];
    return s;
}

/* D = X Y^T in long double. */
static void dense_density(int n, int k, const double *X, const double *Y, ld *D)
{
    #pragma omp parallel for schedule(static)
    for (int lam = 0; lam < n; lam++)
        for (int sig = 0; sig < n; sig++) {
            ld s = 0.0L;
            for (int i = 0; i < k; i++)
                s += (ld)X[IDX2(lam, i, k)] * (ld)Y[IDX2(sig, i, k)];
            D[IDX2(lam, sig, n)] = s;
        }
}

/* ------------------------------------------------------------------------
 * O2: the factored build, following the engine's statement of the problem:
 *   gamma_{P,s} = sum_{lam sig} L^P_{lam sig} (X_s Y_s^T)_{lam sig}
 *   J_s         = sum_P gamma_{P,s} L^P
 *   K_s         = sum_P (L^P X_s)(L^P Y_s)^T        (= B_V^T B_U, Sec. II.C)
 * J or K may be NULL.
 * ---------------------------------------------------------------------- */
int jko_build(int n, int naux, const double *L, int nd, const int *k,
              const double *X, const double *Y, double *J, double *K)
{
    if (n < 1 || naux < 0 || nd < 0) return 1;
    size_t n2 = (size_t)n * n;
    int kmax = 1;
    for (int s = 0; s < nd; s++) {
        if (k[s] < 1) return 1;
        if (k[s] > kmax) kmax = k[s];
    }
    ld *D = (ld *)malloc(n2 * sizeof(ld));
    ld *Jacc = (ld *)malloc(n2 * sizeof(ld));
    ld *Kacc = (ld *)malloc(n2 * sizeof(ld));
    ld *TX = (ld *)malloc((size_t)n * kmax * sizeof(ld));
    ld *TY = (ld *)malloc((size_t)n * kmax * sizeof(ld));
    if (!D || !Jacc || !Kacc || !TX || !TY) {
        free(D); free(Jacc); free(Kacc); free(TX); free(TY);
        return 2;
    }
    size_t off = 0;
    for (int s = 0; s < nd; s++) {
        int ks = k[s];
        const double *Xs = X + off, *Ys = Y + off;
        off += (size_t)n * ks;
        dense_density(n, ks, Xs, Ys, D);
        memset(Jacc, 0, n2 * sizeof(ld));
        memset(Kacc, 0, n2 * sizeof(ld));
        for (int P = 0; P < naux; P++) {
            const double *LP = L + (size_t)P * n2;
            ld gamma = frob_dl(n, LP, D);
            panel(n, ks, LP, Xs, TX);
            panel(n, ks, LP, Ys, TY);
            #pragma omp parallel for schedule(static)
            for (int mu = 0; mu < n; mu++)
                for (int nu = 0; nu < n; nu++) {
                    ld kk = 0.0L;
                    for (int i = 0; i < ks; i++)
                        kk += TX[IDX2(mu, i, ks)] * TY[IDX2(nu, i, ks)];
                    Kacc[IDX2(mu, nu, n)] += kk;
                    Jacc[IDX2(mu, nu, n)] += gamma * (ld)LP[IDX2(mu, nu, n)];
                }
        }
        for (size_t e = 0; e < n2; e++) {
            if (J) J[(size_t)s * n2 + e] = (double)Jacc[e];
            if (K) K[(size_t)s * n2 + e] = (double)Kacc[e];
        }
    }
    free(D); free(Jacc); free(Kacc); free(TX); free(TY);
    return 0;
}

/* ------------------------------------------------------------------------
 * O2 sampled: single entries J_s[mu][nu], K_s[mu][nu] for a list of
 * (s, mu, nu), for sizes where the full build is too slow on the host.
 *   J_s[mu][nu] = sum_P gamma_{P,s} L^P[mu][nu]
 *   K_s[mu][nu] = sum_P sum_i (L^P[mu,:] . X_s[:,i]) (L^P[nu,:] . Y_s[:,i])
 * ---------------------------------------------------------------------- */
int jko_sample(int n, int naux, const double *L, int nd, const int *k,
               const double *X, const double *Y, int nsamp, const int *ss,
               const int *mus, const int *nus, double *Jout, double *Kout)
{
    if (n < 1 || naux < 0 || nd < 0 || nsamp < 0) return 1;
    size_t n2 = (size_t)n * n;
    size_t *offs = (size_t *)malloc((nd + 1) * sizeof(size_t));
    int *need = (int *)calloc(nd > 0 ? nd : 1, sizeof(int));
    ld *gamma = (ld *)calloc((size_t)(nd > 0 ? nd : 1) * (naux > 0 ? naux : 1), sizeof(ld));
    ld *D = (ld *)malloc(n2 * sizeof(ld));
    if (!offs || !need || !gamma || !D) {
        free(offs); free(need); free(gamma); free(D);
        return 2;
    }
    offs[0] = 0;
    for (int s = 0; s < nd; s++) offs[s + 1] = offs[s] + (size_t)n * k[s];
    for (int q = 0; q < nsamp; q++) {
        if (ss[q] < 0 || ss[q] >= nd || mus[q] < 0 || mus[q] >= n ||
            nus[q] < 0 || nus[q] >= n) {
            free(offs); free(need); free(gamma); free(D);
            return 1;
        }
        need[ss[q]] = 1;
    }
    for (int s = 0; s < nd; s++) {
        if (!need[s]) continue;
        dense_density(n, k[s], X + offs[s], Y + offs[s], D);
        #pragma omp parallel for schedule(static)
        for (int P = 0; P < naux; P++)
            gamma[(size_t)s * naux + P] = frob_dl(n, L + (size_t)P * n2, D);
    }
    #pragma omp parallel for schedule(dynamic)
    for (int q = 0; q < nsamp; q++) {
        int s = ss[q], mu = mus[q], nu = nus[q], ks = k[s];
        const double *Xs = X + offs[s], *Ys = Y + offs[s];
        ld jv = 0.0L, kv = 0.0L;
        for (int P = 0; P < naux; P++) {
            const double *LP = L + (size_t)P * n2;
            jv += gamma[(size_t)s * naux + P] * (ld)LP[IDX2(mu, nu, n)];
            for (int i = 0; i < ks; i++) {
                ld tx = 0.0L, ty = 0.0L;
                for (int lam = 0; lam < n; lam++) {
                    tx += (ld)LP[IDX2(mu, lam, n)] * (ld)Xs[IDX2(lam, i, ks)];
                    ty += (ld)LP[IDX2(nu, lam, n)] * (ld)Ys[IDX2(lam, i, ks)];
                }
                kv += tx * ty;
            }
        }
        if (Jout) Jout[q] = (double)jv;
        if (Kout) Kout[q] = (double)kv;
    }
    free(offs); free(need); free(gamma); free(D);
    return 0;
}

/* ------------------------------------------------------------------------
 * O3: the adjoint of E = sum_s <W_s, K_s> + <V_s, J_s> under the Frobenius
 * pairing <A,B> = Tr A^T B (Eq. 1, Sec. II.A), written out by hand:
 *
 *   dE/dX_s = sum_P L^P W_s (L^P Y_s)   + J(V_s) Y_s
 *   dE/dY_s = sum_P L^P W_s^T (L^P X_s) + J(V_s) X_s
 *   G^P     = sum_s [ W_s (L^P Y_s) X_s^T + Y_s (L^P X_s)^T W_s
 *                     + c_{P,s} X_s Y_s^T + gamma_{P,s} V_s ]
 *   dE/dL^P = (G^P + G^P^T) / 2     (gradient on the symmetric subspace)
 * with c_{P,s} = <V_s, L^P>, gamma_{P,s} = <L^P, X_s Y_s^T> and
 * J(V) = sum_P <L^P, V> L^P.  W or V may be NULL (taken as zero); dL may be
 * NULL (not formed).  dX, dY are [n][k_s] blocks concatenated like X.
 * ---------------------------------------------------------------------- */
int jko_adjoint(int n, int naux, const double *L, int nd, const int *k,
                const double *X, const double *Y, const double *W,
                const double *V, double *dX, double *dY, double *dL)
{
    if (n < 1 || naux < 0 || nd < 0) return 1;
    size_t n2 = (size_t)n * n;
    int kmax = 1;
    size_t ktot = 0;
    for (int s = 0; s < nd; s++) {
        if (k[s] < 1) return 1;
        if (k[s] > kmax) kmax = k[s];
        ktot += (size_t)k[s];
    }
    size_t *offs = (size_t *)malloc((nd + 1) * sizeof(size_t));
    ld *aX = (ld *)calloc((size_t)n * (ktot ? ktot : 1), sizeof(ld));
    ld *aY = (ld *)calloc((size_t)n * (ktot ? ktot : 1), sizeof(ld));
    ld *JV = (ld *)calloc(n2 * (nd ? nd : 1), sizeof(ld));
    ld *TX = (ld *)malloc((size_t)n * kmax * sizeof(ld));
    ld *TY = (ld *)malloc((size_t)n * kmax * sizeof(ld));
    ld *U = (ld *)malloc((size_t)n * kmax * sizeof(ld));
    ld *Vp = (ld *)malloc((size_t)n * kmax * sizeof(ld));
    ld *G = (ld *)malloc(n2 * sizeof(ld));
    ld *D = (ld *)malloc(n2 * (nd ? nd : 1) * sizeof(ld));
    if (!offs || !aX || !aY || !JV || !TX || !TY || !U || !Vp || !G || !D) {
        free(offs); free(aX); free(aY); free(JV); free(TX); free(TY);
        free(U); free(Vp); free(G); free(D);
        return 2;
    }
    offs[0] = 0;
    for (int s = 0; s < nd; s++) offs[s + 1] = offs[s] + (size_t)n * k[s];
    for (int s = 0; s < nd; s++)
        dense_density(n, k[s], X + offs[s], Y + offs[s], D + (size_t)s * n2);

    for (int P = 0; P < naux; P++) {
        const double *LP = L + (size_t)P * n2;
        memset(G, 0, n2 * sizeof(ld));
        for (int s = 0; s < nd; s++) {
            int ks = k[s];
            const double *Xs = X + offs[s], *Ys = Y + offs[s];
            const double *Ws = W ? W + (size_t)s * n2 : NULL;
            const double *Vs = V ? V + (size_t)s * n2 : NULL;
            ld gam = frob_dl(n, LP, D + (size_t)s * n2);
            ld cps = Vs ? frob_dd(n, Vs, LP) : 0.0L;
            if (Ws) {
                panel(n, ks, LP, Xs, TX);
                panel(n, ks, LP, Ys, TY);
                /* U = W_s T_Y, Vp = W_s^T T_X */
                #pragma omp parallel for schedule(static)
                for (int mu = 0; mu < n; mu++)
                    for (int i = 0; i < ks; i++) {
                        ld u = 0.0L, v = 0.0L;
                        for (int lam = 0; lam < n; lam++) {
                            u += (ld)Ws[IDX2(mu, lam, n)] * TY[IDX2(lam, i, ks)];
                            v += (ld)Ws[IDX2(lam, mu, n)] * TX[IDX2(lam, i, ks)];
                        }
                        U[IDX2(mu, i, ks)] = u;
                        Vp[IDX2(mu, i, ks)] = v;
                    }
                /* dX_s += L^P U, dY_s += L^P Vp */
                #pragma omp parallel for schedule(static)
                for (int mu = 0; mu < n; mu++)
                    for (int i = 0; i < ks; i++) {
                        ld a = 0.0L, b = 0.0L;
                        for (int lam = 0; lam < n; lam++) {
                            a += (ld)LP[IDX2(mu, lam, n)] * U[IDX2(lam, i, ks)];
                            b += (ld)LP[IDX2(mu, lam, n)] * Vp[IDX2(lam, i, ks)];
                        }
                        aX[offs[s] + IDX2(mu, i, ks)] += a;
                        aY[offs[s] + IDX2(mu, i, ks)] += b;
                    }
            }
            if (dL) {
                #pragma omp parallel for schedule(static)
                for (int mu = 0; mu < n; mu++)
                    for (int nu = 0; nu < n; nu++) {
                        ld g = 0.0L;
                        if (Ws)
                            for (int i = 0; i < ks; i++)
                                g += U[IDX2(mu, i, ks)] * (ld)Xs[IDX2(nu, i, ks)] +
                                     (ld)Ys[IDX2(mu, i, ks)] * Vp[IDX2(nu, i, ks)];
                        g += cps * D[(size_t)s * n2 + IDX2(mu, nu, n)];
                        if (Vs) g += gam * (ld)Vs[IDX2(mu, nu, n)];
                        G[IDX2(mu, nu, n)] += g;
                    }
            }
            if (Vs) {
                ld *JVs = JV + (size_t)s * n2;
                for (size_t e = 0; e < n2; e++) JVs[e] += cps * (ld)LP[e];
            }
        }
        if (dL) {
            double *dLP = dL + (size_t)P * n2;
            for (int mu = 0; mu < n; mu++)
                for (int nu = 0; nu < n; nu++)
                    dLP[IDX2(mu, nu, n)] =
                        (double)(0.5L * (G[IDX2(mu, nu, n)] + G[IDX2(nu, mu, n)]));
        }
    }
    /* J(V_s) terms: dX_s += J(V_s) Y_s, dY_s += J(V_s) X_s */
    if (V) {
        for (int s = 0; s < nd; s++) {
            int ks = k[s];
            const double *Xs = X + offs[s], *Ys = Y + offs[s];
            const ld *JVs = JV + (size_t)s * n2;
            #pragma omp parallel for schedule(static)
            for (int mu = 0; mu < n; mu++)
                for (int i = 0; i < ks; i++) {
                    ld a = 0.0L, b = 0.0L;
                    for (int nu = 0; nu < n; nu++) {
                        a += JVs[IDX2(mu, nu, n)] * (ld)Ys[IDX2(nu, i, ks)];
                        b += JVs[IDX2(mu, nu, n)] * (ld)Xs[IDX2(nu, i, ks)];
                    }
                    aX[offs[s] + IDX2(mu, i, ks)] += a;
                    aY[offs[s] + IDX2(mu, i, ks)] += b;
                }
        }
    }
    for (size_t e = 0; e < (size_t)n * ktot; e++) {
        if (dX) dX[e] = (double)aX[e];
        if (dY) dY[e] = (double)aY[e];
    }
    free(offs); free(aX); free(aY); free(JV); free(TX); free(TY);
    free(U); free(Vp); free(G); free(D);
    return 0;
}

/* ------------------------------------------------------------------------
 * O3 sampled: the adjoint formulas above at single entries, for sizes where
 * the full adjoint is too slow on the host.
 *   dX_s[mu][i] = sum_P (L^P W_s L^P Y_s)[mu][i] + (J(V_s) Y_s)[mu][i]
 *   dY_s[mu][i] = sum_P (L^P W_s^T L^P X_s)[mu][i] + (J(V_s) X_s)[mu][i]
 *   dL^P[mu][nu] = (G^P[mu][nu] + G^P[nu][mu]) / 2, G^P as in O3.
 * Each dX/dY entry is evaluated right to left (a column of L^P Y_s, then
 * W_s times it, then row mu of L^P); each dL entry forms the panels of its P.
 * W or V may be NULL (zero).  Samples: (xs, xmu, xi) for dX and dY, and
 * (lP, lmu, lnu) for dL; either list may be empty.
 * ---------------------------------------------------------------------- */
int jko_adjoint_sample(int n, int naux, const double *L, int nd, const int *k,
                       const double *X, const double *Y, const double *W,
                       const double *V, int nx, const int *xs, const int *xmu,
                       const int *xi, double *dXout, double *dYout, int nl,
                       const int *lP, const int *lmu, const int *lnu,
                       double *dLout)
{
    if (n < 1 || naux < 0 || nd < 0 || nx < 0 || nl < 0) return 1;
    size_t n2 = (size_t)n * n;
    size_t *offs = (size_t *)malloc((nd + 1) * sizeof(size_t));
    ld *c = (ld *)calloc((size_t)(nd ? nd : 1) * (naux ? naux : 1), sizeof(ld));
    int *needc = (int *)calloc(nd ? nd : 1, sizeof(int));
    if (!offs || !c || !needc) { free(offs); free(c); free(needc); return 2; }
    offs[0] = 0;
    for (int s = 0; s < nd; s++) {
        if (k[s] < 1) { free(offs); free(c); free(needc); return 1; }
        offs[s + 1] = offs[s] + (size_t)n * k[s];
    }
    for (int q = 0; q < nx; q++)
        if (xs[q] < 0 || xs[q] >= nd || xmu[q] < 0 || xmu[q] >= n || xi[q] < 0 || xi[q] >= k[xs[q]]) {
            free(offs); free(c); free(needc); return 1;
        }
    for (int q = 0; q < nl; q++)
        if (lP[q] < 0 || lP[q] >= naux || lmu[q] < 0 || lmu[q] >= n || lnu[q] < 0 || lnu[q] >= n) {
            free(offs); free(c); free(needc); return 1;
        }
    /* c_{P,s} = <V_s, L^P> for the densities the dX/dY samples touch */
    if (V) {
        for (int q = 0; q < nx; q++) needc[xs[q]] = 1;
        for (int s = 0; s < nd; s++) {
            if (!needc[s]) continue;
            #pragma omp parallel for schedule(static)
            for (int P = 0; P < naux; P++)
                c[(size_t)s * naux + P] = frob_dd(n, V + (size_t)s * n2, L + (size_t)P * n2);
        }
    }
    int fail = 0;
    #pragma omp parallel for schedule(dynamic)
    for (int q = 0; q < nx; q++) {
        int s = xs[q], mu = xmu[q], i = xi[q], ks = k[s];
        const double *Xs = X + offs[s], *Ys = Y + offs[s];
        const double *Ws = W ? W + (size_t)s * n2 : NULL;
        ld *ty = (ld *)malloc(n * sizeof(ld)), *tx = (ld *)malloc(n * sizeof(ld));
        ld *u = (ld *)malloc(n * sizeof(ld)), *v = (ld *)malloc(n * sizeof(ld));
        if (!ty || !tx || !u || !v) {
            free(ty); free(tx); free(u); free(v);
            #pragma omp atomic write
            fail = 1;
            continue;
        }
        ld ax = 0.0L, ay = 0.0L;
        for (int P = 0; P < naux; P++) {
            const double *LP = L + (size_t)P * n2;
            if (Ws) {
                /* columns i of L^P Y_s and L^P X_s */
                for (int rho = 0; rho < n; rho++) {
                    ld a = 0.0L, b = 0.0L;
                    for (int sig = 0; sig < n; sig++) {
                        a += (ld)LP[IDX2(rho, sig, n)] * (ld)Ys[IDX2(sig, i, ks)];
                        b += (ld)LP[IDX2(rho, sig, n)] * (ld)Xs[IDX2(sig, i, ks)];
                    }
                    ty[rho] = a;
                    tx[rho] = b;
                }
                /* u = W_s ty, v = W_s^T tx */
                for (int lam = 0; lam < n; lam++) {
                    ld a = 0.0L, b = 0.0L;
                    for (int rho = 0; rho < n; rho++) {
                        a += (ld)Ws[IDX2(lam, rho, n)] * ty[rho];
                        b += (ld)Ws[IDX2(rho, lam, n)] * tx[rho];
                    }
                    u[lam] = a;
                    v[lam] = b;
                }
                for (int lam = 0; lam < n; lam++) {
                    ax += (ld)LP[IDX2(mu, lam, n)] * u[lam];
                    ay += (ld)LP[IDX2(mu, lam, n)] * v[lam];
                }
            }
            if (V) {
                /* (J(V_s) Y_s)[mu][i] = sum_P c_{P,s} (L^P Y_s)[mu][i] */
                ld py = 0.0L, px = 0.0L;
                for (int nu = 0; nu < n; nu++) {
                    py += (ld)LP[IDX2(mu, nu, n)] * (ld)Ys[IDX2(nu, i, ks)];
                    px += (ld)LP[IDX2(mu, nu, n)] * (ld)Xs[IDX2(nu, i, ks)];
                }
                ax += c[(size_t)s * naux + P] * py;
                ay += c[(size_t)s * naux + P] * px;
            }
        }
        if (dXout) dXout[q] = (double)ax;
        if (dYout) dYout[q] = (double)ay;
        free(ty); free(tx); free(u); free(v);
    }
    /* dL entries: G^P[a][b] = sum_s [U[a,:].X_s[b,:] + Y_s[a,:].Vp[b,:]
     *                                + c_{P,s} D_s[a][b] + gamma_{P,s} V_s[a][b]]
     * with U = W_s (L^P Y_s), Vp = W_s^T (L^P X_s). */
    #pragma omp parallel for schedule(dynamic)
    for (int q = 0; q < nl; q++) {
        int P = lP[q], mu = lmu[q], nu = lnu[q];
        const double *LP = L + (size_t)P * n2;
        ld g = 0.0L;
        for (int s = 0; s < nd; s++) {
            int ks = k[s];
            const double *Xs = X + offs[s], *Ys = Y + offs[s];
            const double *Ws = W ? W + (size_t)s * n2 : NULL;
            const double *Vs = V ? V + (size_t)s * n2 : NULL;
            ld gam = 0.0L, cps = Vs ? frob_dd(n, Vs, LP) : 0.0L;
            for (int lam = 0; lam < n; lam++)
                for (int sig = 0; sig < n; sig++) {
                    ld d = 0.0L;
                    for (int i = 0; i < ks; i++) d += (ld)Xs[IDX2(lam, i, ks)] * (ld)Ys[IDX2(sig, i, ks)];
                    gam += (ld)LP[IDX2(lam, sig, n)] * d;
                }
            for (int pass = 0; pass < 2; pass++) {   /* G[mu][nu], then G[nu][mu] */
                int a = pass ? nu : mu, b = pass ? mu : nu;
                ld Dab = 0.0L;
                for (int i = 0; i < ks; i++) Dab += (ld)Xs[IDX2(a, i, ks)] * (ld)Ys[IDX2(b, i, ks)];
                ld term = cps * Dab + (Vs ? gam * (ld)Vs[IDX2(a, b, n)] : 0.0L);
                if (Ws) {
                    for (int i = 0; i < ks; i++) {
                        /* U[a][i] = sum_lam W[a][lam] (L^P Y_s)[lam][i];
                         * Vp[b][i] = sum_lam W[lam][b] (L^P X_s)[lam][i] */
                        ld ua = 0.0L, vb = 0.0L;
                        for (int lam = 0; lam < n; lam++) {
                            ld tyl = 0.0L, txl = 0.0L;
                            for (int sig = 0; sig < n; sig++) {
                                tyl += (ld)LP[IDX2(lam, sig, n)] * (ld)Ys[IDX2(sig, i, ks)];
                                txl += (ld)LP[IDX2(lam, sig, n)] * (ld)Xs[IDX2(sig, i, ks)];
                            }
                            ua += (ld)Ws[IDX2(a, lam, n)] * tyl;
                            vb += (ld)Ws[IDX2(lam, b, n)] * txl;
                        }
                        term += ua * (ld)Xs[IDX2(b, i, ks)] + (ld)Ys[IDX2(a, i, ks)] * vb;
                    }
                }
                g += term;
            }
        }
        if (dLout) dLout[q] = (double)(0.5L * g);
    }
    free(offs); free(c); free(needc);
    return fail ? 2 : 0;
}

/* E = sum_s <W_s, K_s> + <V_s, J_s>, evaluated from the O2 build in long
 * double (for finite-difference checks of the adjoint). */
int jko_energy(int n, int naux, const double *L, int nd, const int *k,
               const double *X, const double *Y, const double *W,
               const double *V, long double *E)
{
    size_t n2 = (size_t)n * n;
    double *J = (double *)malloc(n2 * (nd ? nd : 1) * sizeof(double));
    double *K = (double *)malloc(n2 * (nd ? nd : 1) * sizeof(double));
    if (!J || !K) { free(J); free(K); return 2; }
    int rc = jko_build(n, naux, L, nd, k, X, Y, J, K);
    if (rc) { free(J); free(K); return rc; }
    ld e = 0.0L;
    for (int s = 0; s < nd; s++) {
        if (W) e += frob_dd(n, W + (size_t)s * n2, K + (size_t)s * n2);
        if (V) e += frob_dd(n, V + (size_t)s * n2, J + (size_t)s * n2);
    }
    *E = e;
    free(J); free(K);
    return 0;
}

/* ------------------------------------------------------------------------
 * O4: dense (general, non-symmetric) densities, the general primitive of
 * Eq. 4 (Sec. II.C) with a dense argument instead of a factored one:
 *   J(D)_{mu nu} = sum_P <L^P, D> L^P_{mu nu}
 *   K(D)_{mu nu} = sum_P sum_{lam sig} L^P_{mu lam} D_{lam sig} L^P_{nu sig}
 * (the CD form of the O1 definitions).  K is formed per P as T = L^P D
 * followed by T (L^P)^T, so the transpose on the right factor is explicit
 * and no symmetry of L^P is assumed.  DJ feeds J, DK feeds K; either side may
 * be skipped (NULL input or NULL output).  With add != 0 the two results are
 * summed into one output, J: the density gradient dE/dD_s = K(W_s) + J(V_s)
 * of E = sum_s <W_s, K(D_s)> + <V_s, J(D_s)> (Eq. 1, Sec. II.A), each entry
 * rounded to double once.
 * ---------------------------------------------------------------------- */
static int dense_maps(int n, int naux, const double *L, int nd, const double *DJ,
                      const double *DK, double *J, double *K, int add)
{
    if (n < 1 || naux < 0 || nd < 0) return 1;
    size_t n2 = (size_t)n * n;
    ld *Jacc = (ld *)malloc(n2 * sizeof(ld));
    ld *Kacc = (ld *)malloc(n2 * sizeof(ld));
    ld *T = (ld *)malloc(n2 * sizeof(ld));
    if (!Jacc || !Kacc || !T) {
        free(Jacc); free(Kacc); free(T);
        return 2;
    }
    const int doJ = DJ && (J || add), doK = DK && (add ? J != NULL : K != NULL);
    for (int s = 0; s < nd; s++) {
        const double *Ds_J = DJ ? DJ + (size_t)s * n2 : NULL;
        const double *Ds_K = DK ? DK + (size_t)s * n2 : NULL;
        memset(Jacc, 0, n2 * sizeof(ld));
        memset(Kacc, 0, n2 * sizeof(ld));
        for (int P = 0; P < naux; P++) {
            const double *LP = L + (size_t)P * n2;
            if (doJ) {
                ld gamma = frob_dd(n, LP, Ds_J);
                for (size_t e = 0; e < n2; e++) Jacc[e] += gamma * (ld)LP[e];
            }
            if (doK) {
                #pragma omp parallel for schedule(static)
                for (int mu = 0; mu < n; mu++)
                    for (int sig = 0; sig < n; sig++) {
                        ld t = 0.0L;
                        for (int lam = 0; lam < n; lam++)
                            t += (ld)LP[IDX2(mu, lam, n)] * (ld)Ds_K[IDX2(lam, sig, n)];
                        T[IDX2(mu, sig, n)] = t;
                    }
                #pragma omp parallel for schedule(static)
                for (int mu = 0; mu < n; mu++)
                    for (int nu = 0; nu < n; nu++) {
                        ld kk = 0.0L;
                        for (int sig = 0; sig < n; sig++)
                            kk += T[IDX2(mu, sig, n)] * (ld)LP[IDX2(nu, sig, n)];
                        Kacc[IDX2(mu, nu, n)] += kk;
                    }
            }
        }
        for (size_t e = 0; e < n2; e++) {
            if (add) {
                J[(size_t)s * n2 + e] = (double)(Jacc[e] + Kacc[e]);
            } else {
                if (J) J[(size_t)s * n2 + e] = (double)Jacc[e];
                if (K) K[(size_t)s * n2 + e] = (double)Kacc[e];
            }
        }
    }
    free(Jacc); free(Kacc); free(T);
    return 0;
}

/* J_s = J(D_s), K_s = K(D_s) for dense D [nd][n][n]; J or K may be NULL. */
int jko_build_dense(int n, int naux, const double *L, int nd, const double *D,
                    double *J, double *K)
{
    return dense_maps(n, naux, L, nd, D, D, J, K, 0);
}

/* G_s = dE/dD_s = K(W_s) + J(V_s) [nd][n][n]; W or V may be NULL (zero). */
int jko_density_grad(int n, int naux, const double *L, int nd, const double *W,
                     const double *V, double *G)
{
    if (!G) return 1;
    return dense_maps(n, naux, L, nd, V, W, G, NULL, 1);
}

/* ------------------------------------------------------------------------
 * O5: scalar bra-ket pairings of many left and right weight densities, the
 * contraction of Eq. 4 (Sec. II.C) with plain (non-derivative) CD integrals,
 * i.e. the J and K terms Eq. 5 (Sec. II.D) combines:
 *   Jp[a][b] = sum_{mu nu lam sig} WL_a^{mu nu} (mu nu|lam sig) WR_b^{lam sig}
 *            = sum_P <L^P, WL_a> <L^P, WR_b>
 *   Kp[a][b] = sum_{mu nu lam sig} WL_a^{mu nu} (mu lam|nu sig) WR_b^{lam sig}
 *            = sum_P <WL_a, L^P WR_b (L^P)^T>
 * with factored WL_a = A_a B_a^T ([n][kl_a] blocks concatenated in a order)
 * and WR_b = X_b Y_b^T ([n][kr_b] blocks).  Per P: the two metric dots, then
 * M_b = L^P WR_b (L^P)^T and its Frobenius product with every WL_a.  Jp, Kp
 * are [nl][nr]; either may be NULL.
 * ---------------------------------------------------------------------- */
int jko_pairs(int n, int naux, const double *L, int nl, const int *kl,
              const double *A, const double *B, int nr, const int *kr,
              const double *X, const double *Y, double *Jp, double *Kp)
{
    if (n < 1 || naux < 0 || nl < 1 || nr < 1) return 1;
    size_t n2 = (size_t)n * n;
    ld *WL = (ld *)malloc((size_t)nl * n2 * sizeof(ld));
    ld *WR = (ld *)malloc((size_t)nr * n2 * sizeof(ld));
    ld *T = (ld *)malloc(n2 * sizeof(ld));
    ld *M = (ld *)malloc(n2 * sizeof(ld));
    ld *gl = (ld *)malloc((size_t)nl * sizeof(ld));
    ld *gr = (ld *)malloc((size_t)nr * sizeof(ld));
    ld *Jacc = (ld *)calloc((size_t)nl * nr, sizeof(ld));
    ld *Kacc = (ld *)calloc((size_t)nl * nr, sizeof(ld));
    int rc = 0;
    if (!WL || !WR || !T || !M || !gl || !gr || !Jacc || !Kacc) { rc = 2; goto out; }
    {
        size_t off = 0;
        for (int a = 0; a < nl; a++) {
            if (kl[a] < 1) { rc = 1; goto out; }
            dense_density(n, kl[a], A + off, B + off, WL + (size_t)a * n2);
            off += (size_t)n * kl[a];
        }
        off = 0;
        for (int b = 0; b < nr; b++) {
            if (kr[b] < 1) { rc = 1; goto out; }
            dense_density(n, kr[b], X + off, Y + off, WR + (size_t)b * n2);
            off += (size_t)n * kr[b];
        }
    }
    for (int P = 0; P < naux; P++) {
        const double *LP = L + (size_t)P * n2;
        for (int a = 0; a < nl; a++) gl[a] = frob_dl(n, LP, WL + (size_t)a * n2);
        for (int b = 0; b < nr; b++) gr[b] = frob_dl(n, LP, WR + (size_t)b * n2);
        for (int b = 0; b < nr; b++) {
            const ld *Wb = WR + (size_t)b * n2;
            #pragma omp parallel for schedule(static)
            for (int mu = 0; mu < n; mu++)
                for (int sig = 0; sig < n; sig++) {
                    ld t = 0.0L;
                    for (int lam = 0; lam < n; lam++)
                        t += (ld)LP[IDX2(mu, lam, n)] * Wb[IDX2(lam, sig, n)];
                    T[IDX2(mu, sig, n)] = t;
                }
            #pragma omp parallel for schedule(static)
            for (int mu = 0; mu < n; mu++)
                for (int nu = 0; nu < n; nu++) {
                    ld m = 0.0L;
                    for (int sig = 0; sig < n; sig++)
                        m += T[IDX2(mu, sig, n)] * (ld)LP[IDX2(nu, sig, n)];
                    M[IDX2(mu, nu, n)] = m;
                }
            for (int a = 0; a < nl; a++) {
                const ld *Wa = WL + (size_t)a * n2;
                ld s = 0.0L;
                for (size_t e = 0; e < n2; e++) s += Wa[e] * M[e];
                Kacc[(size_t)a * nr + b] += s;
                Jacc[(size_t)a * nr + b] += gl[a] * gr[b];
            }
        }
    }
    for (size_t e = 0; e < (size_t)nl * nr; e++) {
        if (Jp) Jp[e] = (double)Jacc[e];
        if (Kp) Kp[e] = (double)Kacc[e];
    }
out:
    free(WL); free(WR); free(T); free(M); free(gl); free(gr); free(Jacc); free(Kacc);
    return rc;
}
