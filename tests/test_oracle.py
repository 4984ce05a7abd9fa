"""Pins for the CPU oracle, against things other than the oracle itself.

Each check is chosen so that a plausible slip in the oracle (a dropped term,
a wrong sign or index, a transposed operand) fails at least one of them:

* brute force through the explicit four-index tensor (Eq. 4, Sec. II.C);
* a hand-derived two-function example (tests/golden/jk_n2_hand.txt);
* closed forms: rank-1 factor, identity factor, elementary symmetric factor,
  D = I (reduces to a library matrix product);
* identities of the maps: J depends only on D + D^T (Sec. II.C), K(D^T) =
  K(D)^T, symmetry, linearity, bra-ket invariance, self-adjointness under
  <A,B> = Tr A^T B (Eq. 1, Sec. II.A), <D, J(D)> >= 0;
* the adjoint: exact directional derivatives (E is linear in X, in Y, and
  quadratic in L, so a central difference is exact up to rounding) and
  central finite differences at h = 1e-5.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2608_06536_b300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def rand_sym_factor(rng, naux, n):
    A = rng.standard_normal((naux, n, n))
    return np.ascontiguousarray(A + A.transpose(0, 2, 1))


# ----------------------------------------------------------------- golden

def load_golden():
    vals = {}
    with open(os.path.join(HERE, "golden", "jk_n2_hand.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *nums = line.split()
            vals[key] = [float(x) for x in nums]
    n, naux, k = (int(x) for x in vals["dims"])
    L = np.array([vals[f"L{p}"] for p in range(naux)]).reshape(naux, n, n)
    X = np.array(vals["X"]).reshape(n, k)
    Y = np.array(vals["Y"]).reshape(n, k)
    return L, X, Y, np.array(vals["J"]).reshape(n, n), np.array(vals["K"]).reshape(n, n)


def test_golden_hand_example():
    L, X, Y, Jg, Kg = load_golden()
    J, K = oracle.build(L, [X], [Y])
    np.testing.assert_array_equal(J[0], Jg)
    np.testing.assert_array_equal(K[0], Kg)
    Jb, Kb = oracle.brute(L, X @ Y.T)
    np.testing.assert_array_equal(Jb, Jg)
    np.testing.assert_array_equal(Kb, Kg)


# ------------------------------------------------------------ brute force

@pytest.mark.parametrize("n,naux,ks", [(7, 5, [3]), (5, 9, [1, 4]), (11, 3, [6, 2, 11])])
def test_factored_matches_brute_force(n, naux, ks):
    rng = np.random.default_rng(n * 100 + naux)
    L = rand_sym_factor(rng, naux, n)
    X = [rng.standard_normal((n, k)) for k in ks]
    Y = [rng.standard_normal((n, k)) for k in ks]
    J, K = oracle.build(L, X, Y)
    for s in range(len(ks)):
        Jb, Kb = oracle.brute(L, X[s] @ Y[s].T)
        assert rel(J[s], Jb) < 1e-13
        assert rel(K[s], Kb) < 1e-13


def test_sampled_matches_full():
    m = inputs.custom(13, 17, 5.0, [3, 5], [False, True])
    J, K = oracle.build(m.L, m.X, m.Y)
    rng = np.random.default_rng(1)
    s = rng.integers(0, 2, 40); mu = rng.integers(0, 13, 40); nu = rng.integers(0, 13, 40)
    Js, Ks = oracle.sample(m.L, m.X, m.Y, s, mu, nu)
    assert rel(Js, J[s, mu, nu]) < 1e-14
    assert rel(Ks, K[s, mu, nu]) < 1e-14


@pytest.mark.parametrize("withW,withV", [(True, True), (True, False), (False, True)])
def test_sampled_adjoint_matches_full(withW, withV):
    """The entry-by-entry adjoint evaluates the same formulas as the full one
    in a different order (right to left per entry); the full adjoint is pinned
    by finite differences below."""
    n, naux = 11, 7
    m = inputs.custom(n, naux, 3.0, [3, 4], [False, True])
    rng = np.random.default_rng(9)
    W = [rng.standard_normal((n, n)) for _ in range(2)] if withW else None
    V = [rng.standard_normal((n, n)) for _ in range(2)] if withV else None
    dX, dY, dL = oracle.adjoint(m.L, m.X, m.Y, W, V)
    s = rng.integers(0, 2, 30); mu = rng.integers(0, n, 30); i = rng.integers(0, 3, 30)
    P = rng.integers(0, naux, 30); a = rng.integers(0, n, 30); b = rng.integers(0, n, 30)
    sx, sy, sl = oracle.adjoint_sample(m.L, m.X, m.Y, W, V, (s, mu, i), (P, a, b))
    ex = np.array([dX[q][mu_, i_] for q, mu_, i_ in zip(s, mu, i)])
    ey = np.array([dY[q][mu_, i_] for q, mu_, i_ in zip(s, mu, i)])
    assert rel(sx, ex) < 1e-14 and rel(sy, ey) < 1e-14
    assert rel(sl, dL[P, a, b]) < 1e-14


# ----------------------------------------------------------- closed forms

def test_rank_one_factor():
    rng = np.random.default_rng(2)
    n = 9
    v = rng.standard_normal(n)
    L = np.outer(v, v)[None].copy()
    X, Y = rng.standard_normal((n, 4)), rng.standard_normal((n, 4))
    D = X @ Y.T
    expect = (v @ D @ v) * np.outer(v, v)
    J, K = oracle.build(L, [X], [Y])
    assert rel(J[0], expect) < 1e-14
    assert rel(K[0], expect) < 1e-14


def test_identity_factor():
    rng = np.random.default_rng(3)
    n, naux = 8, 6
    L = np.broadcast_to(np.eye(n), (naux, n, n)).copy()
    X, Y = rng.standard_normal((n, 3)), rng.standard_normal((n, 3))
    D = X @ Y.T
    J, K = oracle.build(L, [X], [Y])
    assert rel(J[0], naux * np.trace(D) * np.eye(n)) < 1e-14
    assert rel(K[0], naux * D) < 1e-14


@pytest.mark.parametrize("i,j", [(0, 3), (4, 1)])
def test_elementary_symmetric_factor(i, j):
    """L = E_ij + E_ji: K swaps and transposes the (i,j) block of D,
    J = (D_ij + D_ji) L."""
    rng = np.random.default_rng(4)
    n = 6
    L = np.zeros((1, n, n)); L[0, i, j] = L[0, j, i] = 1.0
    X, Y = rng.standard_normal((n, 2)), rng.standard_normal((n, 2))
    D = X @ Y.T
    Kx = np.zeros((n, n))
    Kx[i, j] = D[j, i]; Kx[j, i] = D[i, j]; Kx[i, i] = D[j, j]; Kx[j, j] = D[i, i]
    J, K = oracle.build(L, [X], [Y])
    assert rel(K[0], Kx) < 1e-15
    assert rel(J[0], (D[i, j] + D[j, i]) * L[0]) < 1e-15


def test_unit_density():
    """X = Y = I: K = sum_P (L^P)^2 and J = sum_P tr(L^P) L^P."""
    rng = np.random.default_rng(5)
    n, naux = 10, 7
    L = rand_sym_factor(rng, naux, n)
    I = np.eye(n)
    J, K = oracle.build(L, [I], [I])
    assert rel(K[0], np.einsum("pij,pjk->ik", L, L)) < 1e-14
    assert rel(J[0], np.einsum("p,pij->ij", np.einsum("pii->p", L), L)) < 1e-14


# ------------------------------------------------------------- identities

@pytest.fixture(scope="module")
def small():
    rng = np.random.default_rng(6)
    n, naux = 9, 11
    L = rand_sym_factor(rng, naux, n)
    X = [rng.standard_normal((n, 3)) for _ in range(3)]
    Y = [rng.standard_normal((n, 3)) for _ in range(3)]
    return L, X, Y


def test_j_depends_only_on_symmetric_part(small):
    L, X, Y = small
    J1, _ = oracle.build(L, X, Y)
    J2, _ = oracle.build(L, Y, X)          # D -> D^T
    assert rel(J1, J2) < 1e-14
    for s in range(3):
        assert rel(J1[s], J1[s].T) < 1e-15


def test_k_transpose(small):
    L, X, Y = small
    _, K1 = oracle.build(L, X, Y)
    _, K2 = oracle.build(L, Y, X)
    for s in range(3):
        assert rel(K2[s], K1[s].T) < 1e-14
        assert rel(K1[s], K1[s].T) > 1e-3   # non-symmetric D gives non-symmetric K
    _, Ks = oracle.build(L, X, X)
    for s in range(3):
        assert rel(Ks[s], Ks[s].T) < 1e-14


def test_linearity(small):
    L, X, Y = small
    J, K = oracle.build(L, X, Y)
    Jc, Kc = oracle.build(L, [np.hstack(X)], [np.hstack(Y)])   # D = sum_s X_s Y_s^T
    assert rel(Jc[0], J.sum(0)) < 1e-13
    assert rel(Kc[0], K.sum(0)) < 1e-13
    J2, K2 = oracle.build(L, [2.5 * x for x in X], Y)
    assert rel(J2, 2.5 * J) < 1e-14 and rel(K2, 2.5 * K) < 1e-14


def test_bra_ket_and_self_adjointness(small):
    L, X, Y = small
    n = L.shape[1]
    D = [X[s] @ Y[s].T for s in range(3)]
    J, K = oracle.build(L, X, Y)
    # <D0, J(D1)> = <D1, J(D0)>  and  tr(D0 K(D1)) = tr(D1 K(D0))
    assert abs(np.sum(D[0] * J[1]) - np.sum(D[1] * J[0])) < 1e-12 * abs(np.sum(D[0] * J[1]))
    t01, t10 = np.trace(D[0] @ K[1]), np.trace(D[1] @ K[0])
    assert abs(t01 - t10) < 1e-12 * abs(t01)
    # <W, K(D)> = <K(W), D> with a dense non-symmetric W = W I^T
    rng = np.random.default_rng(7)
    W = rng.standard_normal((n, n))
    _, KW = oracle.build(L, [W], [np.eye(n)])
    JW, _ = oracle.build(L, [W], [np.eye(n)])
    for s in range(3):
        a, b = np.sum(W * K[s]), np.sum(KW[0] * D[s])
        assert abs(a - b) < 1e-12 * abs(a)
        a, b = np.sum(W * J[s]), np.sum(JW[0] * D[s])
        assert abs(a - b) < 1e-12 * abs(a)


def test_coulomb_energy_nonnegative(small):
    L, X, Y = small
    J, _ = oracle.build(L, X, Y)
    for s in range(3):
        D = X[s] @ Y[s].T
        e = np.sum(D * J[s])
        gam = np.einsum("pij,ij->p", L, D)
        assert e >= 0
        assert abs(e - np.sum(gam ** 2)) < 1e-12 * e


# ---------------------------------------------------------------- adjoint

@pytest.fixture(scope="module")
def adj_case():
    rng = np.random.default_rng(8)
    n, naux, ks = 7, 6, [2, 3]
    L = rand_sym_factor(rng, naux, n)
    X = [rng.standard_normal((n, k)) for k in ks]
    Y = [rng.standard_normal((n, k)) for k in ks]
    W = [rng.standard_normal((n, n)) for _ in ks]
    V = [rng.standard_normal((n, n)) for _ in ks]
    return L, X, Y, W, V


def test_adjoint_exact_directional(adj_case):
    """E is linear in X (and in Y): <dE/dX, dX> = E(X -> dX) exactly."""
    L, X, Y, W, V = adj_case
    dX, dY, dL = oracle.adjoint(L, X, Y, W, V)
    rng = np.random.default_rng(9)
    for _ in range(4):
        hX = [rng.standard_normal(x.shape) for x in X]
        hY = [rng.standard_normal(y.shape) for y in Y]
        # E is bilinear in (X, Y) per density: E(hX, Y) = <dX, hX>
        lhs = sum(np.sum(a * b) for a, b in zip(dX, hX))
        rhs = oracle.energy(L, hX, Y, W, V)
        assert abs(lhs - rhs) < 1e-12 * max(abs(rhs), 1.0)
        lhs = sum(np.sum(a * b) for a, b in zip(dY, hY))
        rhs = oracle.energy(L, X, hY, W, V)
        assert abs(lhs - rhs) < 1e-12 * max(abs(rhs), 1.0)


def test_adjoint_factor_direction(adj_case):
    """E is quadratic in L: a central difference with any step is exact up to
    rounding; symmetric directions only (dE/dL is the symmetric gradient)."""
    L, X, Y, W, V = adj_case
    _, _, dL = oracle.adjoint(L, X, Y, W, V)
    assert rel(dL, dL.transpose(0, 2, 1)) < 1e-15
    rng = np.random.default_rng(10)
    for h in (1.0, 1e-3):
        H = rand_sym_factor(rng, *L.shape[:2])
        ep = oracle.energy(L + h * H, X, Y, W, V)
        em = oracle.energy(L - h * H, X, Y, W, V)
        fd = (ep - em) / (2 * h)
        an = np.sum(dL * H)
        assert abs(fd - an) < 1e-9 * max(abs(an), 1.0)


def test_adjoint_central_fd(adj_case):
    """Central finite differences at h = 1e-5 on random directions in (X, Y, L)."""
    L, X, Y, W, V = adj_case
    dX, dY, dL = oracle.adjoint(L, X, Y, W, V)
    rng = np.random.default_rng(11)
    h = 1e-5
    for _ in range(6):
        hX = [rng.standard_normal(x.shape) for x in X]
        hY = [rng.standard_normal(y.shape) for y in Y]
        H = rand_sym_factor(rng, *L.shape[:2])
        f = lambda t: oracle.energy(L + t * H, [x + t * a for x, a in zip(X, hX)],
                                    [y + t * b for y, b in zip(Y, hY)], W, V)
        fd = (f(h) - f(-h)) / (2 * h)
        an = (sum(np.sum(a * b) for a, b in zip(dX, hX)) +
              sum(np.sum(a * b) for a, b in zip(dY, hY)) + np.sum(dL * H))
        assert abs(fd - an) < 1e-6 * max(abs(an), 1.0)


def test_adjoint_separates_w_and_v(adj_case):
    """Seeds enter linearly: adjoint(W, V) = adjoint(W, 0) + adjoint(0, V)."""
    L, X, Y, W, V = adj_case
    a = oracle.adjoint(L, X, Y, W, V)
    b = oracle.adjoint(L, X, Y, W, None)
    c = oracle.adjoint(L, X, Y, None, V)
    for s in range(2):
        assert rel(a[0][s], b[0][s] + c[0][s]) < 1e-13
        assert rel(a[1][s], b[1][s] + c[1][s]) < 1e-13
    assert rel(a[2], b[2] + c[2]) < 1e-13


def test_generators_are_deterministic():
    a = inputs.custom(10, 4, 3.0, [2])
    b = inputs.custom(10, 4, 3.0, [2])
    np.testing.assert_array_equal(a.L, b.L)
    np.testing.assert_array_equal(a.X[0], b.X[0])
    assert np.array_equal(a.L, a.L.transpose(0, 2, 1))
    assert abs(a.L[3, 0, 0]) < 10 * np.exp(-1.0)
    q, _ = inputs.ground_density(30, 5, 0)
    np.testing.assert_allclose(q.T @ q, np.eye(5), atol=1e-14)
