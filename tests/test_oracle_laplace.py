"""Pins of the oracle's Laplace (LT-AO) builds (O6, Eq. 3): reduction to
brute force at alpha = 0, the closed form for one column pair, and the
Laplace identity itself: with a Gauss-Laguerre quadrature of
int_0^inf exp(-t y) dt = 1/y, the weighted sum over the quadrature points of
the energy-scaled builds approaches sum_p J(c_p c'_p^T) / y_p, where y_p is
half the gap of column pair p.  The paper prints no (alpha, w) tables, so the
quadrature here is this synthetic one.  CPU only."""
import numpy as np

import oracle


def _gl(nq):
    """(alpha, w) with sum_k w_k exp(-alpha_k y) ~ 1/y, from Gauss-Laguerre
    nodes t_k and weights u_k of int_0^inf exp(-t) f(t) dt:
    1/y = int exp(-t) exp(-t (y - 1)) dt ~ sum u_k exp(t_k) exp(-t_k y)."""
    t, u = np.polynomial.laguerre.laggauss(nq)
    return t, u * np.exp(t)


def _setup(n=7, naux=6, m=3, seed=0):
    rng = np.random.default_rng(seed)
    L = rng.standard_normal((naux, n, n))
    L = L + L.transpose(0, 2, 1)
    CX = rng.standard_normal((n, m))
    CY = rng.standard_normal((n, m))
    return L, CX, CY


def test_alpha_zero_is_plain_build():
    L, CX, CY = _setup()
    eps = np.array([-1.0, -0.5, -0.2])
    J, K = oracle.laplace(L, CX, eps, +1, CY, -eps, -1, alpha=[0.0, 0.0])
    Jb, Kb = oracle.brute(L, CX @ CY.T)
    for k in range(2):
        assert np.abs(J[k] - Jb).max() <= 1e-13 * np.abs(Jb).max()
        assert np.abs(K[k] - Kb).max() <= 1e-13 * np.abs(Kb).max()


def test_one_column_pair_closed_form():
    """m = 1: D_k = exp(alpha_k (sx ex + sy ey) / 2) c c'^T, so J_k and K_k
    are that factor times the brute-force maps of c c'^T."""
    L, CX, CY = _setup(m=1)
    ex, ey = -0.8, 0.3
    alpha = [0.0, 0.7, 2.5]
    J, K = oracle.laplace(L, CX, [ex], +1, CY, [ey], -1, alpha)
    Jb, Kb = oracle.brute(L, CX @ CY.T)
    for k, a in enumerate(alpha):
        f = np.exp(a * (ex - ey) / 2)
        assert np.abs(J[k] - f * Jb).max() <= 1e-13 * np.abs(f * Jb).max()
        assert np.abs(K[k] - f * Kb).max() <= 1e-13 * np.abs(f * Kb).max()


def test_weighted_sum_is_the_laplace_denominator():
    """Occupied columns (sx = +1, eps_i < 0) against virtual columns
    (sy = -1, eps_a > 0): column pair p carries exp(-alpha y_p) with
    y_p = (eps_a - eps_i) / 2, so the weighted sum tends to
    sum_p J(c_p c'_p^T) / y_p within the quadrature's own error."""
    L, CX, CY = _setup(m=3)
    ei = np.array([-1.2, -0.9, -0.7])
    ea = np.array([0.8, 1.1, 2.0])
    y = (ea - ei) / 2
    alpha, w = _gl(40)
    qerr = np.abs(np.array([np.sum(w * np.exp(-alpha * yp)) for yp in y]) - 1 / y)
    assert qerr.max() < 1e-6          # the quadrature is accurate on these gaps
    J, K = oracle.laplace(L, CX, ei, +1, CY, ea, -1, alpha, w)
    Jr = np.zeros_like(J); Kr = np.zeros_like(K); bound_j = bound_k = 0.0
    for p in range(3):
        Jb, Kb = oracle.brute(L, np.outer(CX[:, p], CY[:, p]))
        Jr += Jb / y[p]; Kr += Kb / y[p]
        bound_j += qerr[p] * np.abs(Jb).max(); bound_k += qerr[p] * np.abs(Kb).max()
    assert np.abs(J - Jr).max() <= bound_j + 1e-12 * np.abs(Jr).max()
    assert np.abs(K - Kr).max() <= bound_k + 1e-12 * np.abs(Kr).max()
    # a sign slip (exp(+alpha y)) or unweighted points would be far off
    assert np.abs(J - Jr).max() < 1e-4 * np.abs(Jr).max()


def test_weights_fold_into_the_left_factor():
    L, CX, CY = _setup()
    eps = np.array([-1.0, -0.5, -0.2])
    alpha, w = [0.3, 1.1, 2.0], np.array([0.5, -0.25, 2.0])
    J, K = oracle.laplace(L, CX, eps, +1, CX, eps, +1, alpha)
    Jw, Kw = oracle.laplace(L, CX, eps, +1, CX, eps, +1, alpha, w)
    assert np.abs(Jw - np.tensordot(w, J, 1)).max() <= 1e-13 * np.abs(Jw).max()
    assert np.abs(Kw - np.tensordot(w, K, 1)).max() <= 1e-13 * np.abs(Kw).max()
    # the occupied pseudo-density exp(alpha eps) weighted C C^T is symmetric,
    # and so are its J and K
    assert np.abs(K - K.transpose(0, 2, 1)).max() <= 1e-13 * np.abs(K).max()


def test_factors_recipe():
    CX = np.arange(6.0).reshape(3, 2)
    X, Y = oracle.laplace_factors(CX, [1.0, -2.0], -1, CX, [0.5, 0.5], +1, [2.0], [3.0])
    np.testing.assert_allclose(X[0], 3.0 * CX * np.exp(-np.array([1.0, -2.0]))[None, :], rtol=1e-15)
    np.testing.assert_allclose(Y[0], CX * np.exp(np.array([0.5, 0.5]))[None, :], rtol=1e-15)
