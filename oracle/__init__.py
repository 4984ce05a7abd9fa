"""CPU oracle for the Cholesky J/K engine -- TEST INFRASTRUCTURE ONLY.

A slow, obviously correct FP64-in / long-double-accumulate implementation of
the paper's J/K build (Eq. 4, Sec. II.C) and its adjoint (Eq. 1, Sec. II.A),
written in plain C (``jk_oracle.c``) and called here through ctypes.  Only
``tests/``, ``__graft_entry__.smoke()`` and the cpu_baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path.

Parity pins (tests/test_oracle.py): brute force through the explicit
four-index tensor, closed forms (rank-1 factor, identity factor, elementary
symmetric factor, D = I), the identities of the J/K maps (J depends only on
D + D^T, K(D^T) = K(D)^T, symmetry, linearity, bra-ket invariance,
self-adjointness, positivity of <D, J(D)>) and central finite differences
of E for the adjoint.  The dense-density maps, the density gradient and the
pairings (tests/test_oracle_dense.py) are pinned the same way: brute force,
closed forms, exact differences of E in D, the chain rule to the factored
adjoint, and the bra-ket symmetry of the pairing scalars.
"""
from __future__ import annotations

import ctypes as ct

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ct.CDLL(path)
        dp = ct.POINTER(ct.c_double)
        ip = ct.POINTER(ct.c_int)
        L.jko_brute.argtypes = [ct.c_int, ct.c_int, dp, dp, dp, dp]
        L.jko_build.argtypes = [ct.c_int, ct.c_int, dp, ct.c_int, ip, dp, dp, dp, dp]
        L.jko_sample.argtypes = [ct.c_int, ct.c_int, dp, ct.c_int, ip, dp, dp,
                                 ct.c_int, ip, ip, ip, dp, dp]
        L.jko_adjoint.argtypes = [ct.c_int, ct.c_int, dp, ct.c_int, ip, dp, dp,
                                  dp, dp, dp, dp, dp]
        L.jko_adjoint_sample.argtypes = [ct.c_int, ct.c_int, dp, ct.c_int, ip, dp, dp, dp, dp,
                                         ct.c_int, ip, ip, ip, dp, dp, ct.c_int, ip, ip, ip, dp]
        L.jko_energy.argtypes = [ct.c_int, ct.c_int, dp, ct.c_int, ip, dp, dp,
                                 dp, dp, ct.POINTER(ct.c_longdouble)]
        L.jko_build_dense.argtypes = [ct.c_int, ct.c_int, dp, ct.c_int, dp, dp, dp]
        L.jko_density_grad.argtypes = [ct.c_int, ct.c_int, dp, ct.c_int, dp, dp, dp]
        L.jko_pairs.argtypes = [ct.c_int, ct.c_int, dp, ct.c_int, ip, dp, dp, ct.c_int, ip, dp, dp, dp, dp]
        for f in (L.jko_brute, L.jko_build, L.jko_sample, L.jko_adjoint, L.jko_adjoint_sample,
                  L.jko_energy, L.jko_build_dense, L.jko_density_grad, L.jko_pairs):
            f.restype = ct.c_int
        _lib = L
    return _lib


def _d(a):
    if a is None:
        return ct.POINTER(ct.c_double)()
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ct.POINTER(ct.c_double))


def _i(a):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.int32))
    return a, a.ctypes.data_as(ct.POINTER(ct.c_int))


def _cat(blocks):
    return np.ascontiguousarray(np.concatenate([np.asarray(b, np.float64).ravel() for b in blocks]))


def _check(rc, name):
    if rc != 0:
        raise RuntimeError(f"oracle {name} failed with code {rc}")


def brute(L: np.ndarray, D: np.ndarray):
    """O1: (J, K) for one dense density through the explicit 4-index tensor."""
    L = np.ascontiguousarray(L, np.float64)
    D = np.ascontiguousarray(D, np.float64)
    naux, n, _ = L.shape
    J = np.empty((n, n)); K = np.empty((n, n))
    _check(lib().jko_brute(n, naux, _d(L), _d(D), _d(J), _d(K)), "brute")
    return J, K


def build(L: np.ndarray, X: list, Y: list, want_j=True, want_k=True):
    """O2: (J, K) as [nd][n][n] arrays for factored densities D_s = X_s Y_s^T."""
    L = np.ascontiguousarray(L, np.float64)
    naux, n, _ = L.shape
    nd = len(X)
    ks, kp = _i([x.shape[1] for x in X])
    Xc, Yc = _cat(X), _cat(Y)
    J = np.empty((nd, n, n)) if want_j else None
    K = np.empty((nd, n, n)) if want_k else None
    _check(lib().jko_build(n, naux, _d(L), nd, kp, _d(Xc), _d(Yc), _d(J), _d(K)), "build")
    return J, K


def sample(L: np.ndarray, X: list, Y: list, s, mu, nu):
    """O2 at single entries: (J_s[mu,nu], K_s[mu,nu]) for index arrays s, mu, nu."""
    L = np.ascontiguousarray(L, np.float64)
    naux, n, _ = L.shape
    nd = len(X)
    ks, kp = _i([x.shape[1] for x in X])
    Xc, Yc = _cat(X), _cat(Y)
    sa, sp = _i(s); ma, mp = _i(mu); na, np_ = _i(nu)
    Jo = np.empty(sa.size); Ko = np.empty(sa.size)
    _check(lib().jko_sample(n, naux, _d(L), nd, kp, _d(Xc), _d(Yc), sa.size, sp, mp, np_,
                            _d(Jo), _d(Ko)), "sample")
    return Jo, Ko


def adjoint(L: np.ndarray, X: list, Y: list, W=None, V=None, want_dl=True):
    """O3: (dX list, dY list, dL [naux][n][n] or None) for
    E = sum_s <W_s, K_s> + <V_s, J_s>."""
    L = np.ascontiguousarray(L, np.float64)
    naux, n, _ = L.shape
    nd = len(X)
    ks, kp = _i([x.shape[1] for x in X])
    Xc, Yc = _cat(X), _cat(Y)
    Wc = _cat(W) if W is not None else None
    Vc = _cat(V) if V is not None else None
    dX = np.empty(Xc.size); dY = np.empty(Yc.size)
    dL = np.empty((naux, n, n)) if want_dl else None
    _check(lib().jko_adjoint(n, naux, _d(L), nd, kp, _d(Xc), _d(Yc), _d(Wc), _d(Vc),
                             _d(dX), _d(dY), _d(dL)), "adjoint")
    outX, outY, off = [], [], 0
    for k in ks:
        outX.append(dX[off:off + n * k].reshape(n, k))
        outY.append(dY[off:off + n * k].reshape(n, k))
        off += n * k
    return outX, outY, dL


def adjoint_sample(L: np.ndarray, X: list, Y: list, W=None, V=None, xsamp=None, lsamp=None):
    """O3 at single entries.  ``xsamp`` = (s, mu, i) index arrays for dX_s[mu,i]
    and dY_s[mu,i]; ``lsamp`` = (P, mu, nu) for dL^P[mu,nu].  Returns
    (dX values, dY values, dL values)."""
    L = np.ascontiguousarray(L, np.float64)
    naux, n, _ = L.shape
    nd = len(X)
    ks, kp = _i([x.shape[1] for x in X])
    Xc, Yc = _cat(X), _cat(Y)
    Wc = _cat(W) if W is not None else None
    Vc = _cat(V) if V is not None else None
    xs, xmu, xi = xsamp if xsamp is not None else ([], [], [])
    lP, lmu, lnu = lsamp if lsamp is not None else ([], [], [])
    (xa, xp), (ma, mp), (ia, ip_) = _i(xs), _i(xmu), _i(xi)
    (pa, pp), (la, lp), (na, np_) = _i(lP), _i(lmu), _i(lnu)
    dX = np.empty(max(xa.size, 1)); dY = np.empty(max(xa.size, 1)); dL = np.empty(max(pa.size, 1))
    _check(lib().jko_adjoint_sample(n, naux, _d(L), nd, kp, _d(Xc), _d(Yc), _d(Wc), _d(Vc),
                                    xa.size, xp, mp, ip_, _d(dX), _d(dY), pa.size, pp, lp, np_,
                                    _d(dL)), "adjoint_sample")
    return dX[:xa.size], dY[:xa.size], dL[:pa.size]


def energy(L: np.ndarray, X: list, Y: list, W=None, V=None) -> float:
    """E = sum_s <W_s, K_s> + <V_s, J_s> from the O2 build."""
    L = np.ascontiguousarray(L, np.float64)
    naux, n, _ = L.shape
    nd = len(X)
    ks, kp = _i([x.shape[1] for x in X])
    Xc, Yc = _cat(X), _cat(Y)
    Wc = _cat(W) if W is not None else None
    Vc = _cat(V) if V is not None else None
    E = ct.c_longdouble(0)
    _check(lib().jko_energy(n, naux, _d(L), nd, kp, _d(Xc), _d(Yc), _d(Wc), _d(Vc),
                            ct.byref(E)), "energy")
    return float(E.value)


def build_dense(L: np.ndarray, D, want_j=True, want_k=True):
    """O4: (J, K) as [nd][n][n] for dense, general densities D [nd][n][n]."""
    L = np.ascontiguousarray(L, np.float64)
    naux, n, _ = L.shape
    Dc = np.ascontiguousarray(np.asarray(D, np.float64).reshape(-1, n, n))
    nd = Dc.shape[0]
    J = np.empty((nd, n, n)) if want_j else None
    K = np.empty((nd, n, n)) if want_k else None
    _check(lib().jko_build_dense(n, naux, _d(L), nd, _d(Dc), _d(J), _d(K)), "build_dense")
    return J, K


def density_grad(L: np.ndarray, W=None, V=None, nd=None):
    """O4: G_s = dE/dD_s = K(W_s) + J(V_s), [nd][n][n], for
    E = sum_s <W_s, K(D_s)> + <V_s, J(D_s)>; W or V may be None (zero)."""
    L = np.ascontiguousarray(L, np.float64)
    naux, n, _ = L.shape
    Wc = None if W is None else np.ascontiguousarray(np.asarray(W, np.float64).reshape(-1, n, n))
    Vc = None if V is None else np.ascontiguousarray(np.asarray(V, np.float64).reshape(-1, n, n))
    if nd is None:
        nd = (Wc if Wc is not None else Vc).shape[0]
    G = np.empty((nd, n, n))
    _check(lib().jko_density_grad(n, naux, _d(L), nd, _d(Wc), _d(Vc), _d(G)), "density_grad")
    return G


def pairs(L: np.ndarray, A: list, B: list, X: list, Y: list, want_j=True, want_k=True):
    """O5: (Jp, Kp), each [nl][nr], Jp[a][b] = <WL_a, J(WR_b)> and
    Kp[a][b] = <WL_a, K(WR_b)> for WL_a = A_a B_a^T, WR_b = X_b Y_b^T."""
    L = np.ascontiguousarray(L, np.float64)
    naux, n, _ = L.shape
    nl, nr = len(A), len(X)
    kla, klp = _i([a.shape[1] for a in A])
    kra, krp = _i([x.shape[1] for x in X])
    Ac, Bc, Xc, Yc = _cat(A), _cat(B), _cat(X), _cat(Y)
    Jp = np.empty((nl, nr)) if want_j else None
    Kp = np.empty((nl, nr)) if want_k else None
    _check(lib().jko_pairs(n, naux, _d(L), nl, klp, _d(Ac), _d(Bc), nr, krp, _d(Xc), _d(Yc),
                           _d(Jp), _d(Kp)), "pairs")
    return Jp, Kp


def laplace_factors(CX, epsX, sx, CY, epsY, sy, alpha, w=None):
    """Energy-scaled coefficients of the Laplace (LT-AO) representation
    (Eq. 3, Sec. II.B): for quadrature point k,
    X_k[mu][p] = CX[mu][p] exp(sx alpha_k epsX[p] / 2) (times w_k when weights
    are given) and Y_k[mu][p] = CY[mu][p] exp(sy alpha_k epsY[p] / 2), so that
    D_k = X_k Y_k^T carries exp(alpha_k (sx epsX_p + sy epsY_p) / 2) per column
    pair p.  Returns the lists (X_k), (Y_k)."""
    CX, CY = np.asarray(CX, np.float64), np.asarray(CY, np.float64)
    epsX, epsY = np.asarray(epsX, np.float64), np.asarray(epsY, np.float64)
    X, Y = [], []
    for k, a in enumerate(alpha):
        xs = CX * np.exp(sx * a * epsX / 2.0)[None, :]
        if w is not None:
            xs = xs * w[k]
        X.append(np.ascontiguousarray(xs))
        Y.append(np.ascontiguousarray(CY * np.exp(sy * a * epsY / 2.0)[None, :]))
    return X, Y


def laplace(L: np.ndarray, CX, epsX, sx, CY, epsY, sy, alpha, w=None):
    """O6: the n_L builds of the Laplace representation (Eq. 3, Sec. II.B):
    J_k = J(X_k Y_k^T), K_k = K(X_k Y_k^T) on the energy-scaled coefficients
    (laplace_factors), each through O2.  Without weights: [nq][n][n] arrays;
    with weights w: the single sums sum_k w_k J_k, sum_k w_k K_k ([n][n], the
    weight folded into X_k, the sum over k in long double)."""
    X, Y = laplace_factors(CX, epsX, sx, CY, epsY, sy, alpha, w)
    J, K = build(L, X, Y)
    if w is None:
        return J, K
    return (np.sum(J.astype(np.longdouble), axis=0).astype(np.float64),
            np.sum(K.astype(np.longdouble), axis=0).astype(np.float64))
