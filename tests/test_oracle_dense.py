"""Pins of the oracle's dense-density maps (O4), the density gradient
dE/dD = K(W) + J(V) and the bra-ket pairings (O5), against things other than
themselves: brute force through the explicit four-index tensor (O1, and a
numpy einsum of the literal Eq. 4 sums), closed forms, exact central
differences of E (E is linear in D), the chain rule down to the factored
adjoint (O3, itself pinned by differences), and the bra-ket symmetry of the
pairing scalars.  CPU only."""
import numpy as np
import pytest

import oracle


def _factor(rng, n, naux, symmetric=True):
    L = rng.standard_normal((naux, n, n))
    if symmetric:
        L = L + L.transpose(0, 2, 1)
    return L


def _eri(L):
    """(mu nu|lam sig) = sum_P L^P_{mu nu} L^P_{lam sig}, by einsum."""
    return np.einsum("pab,pcd->abcd", L, L)


@pytest.mark.parametrize("symmetric", [True, False])
def test_dense_build_is_brute_force(symmetric):
    """O4 = O1 for general (non-symmetric) D; a non-symmetric L as well, so a
    transposed factor on either side of D cannot pass."""
    rng = np.random.default_rng(1)
    n, naux = 7, 5
    L = _factor(rng, n, naux, symmetric)
    D = rng.standard_normal((3, n, n))
    J, K = oracle.build_dense(L, D)
    for s in range(3):
        Jb, Kb = oracle.brute(L, D[s])
        assert np.abs(J[s] - Jb).max() <= 1e-13 * np.abs(Jb).max()
        assert np.abs(K[s] - Kb).max() <= 1e-13 * np.abs(Kb).max()
    # and the literal four-index sums, written independently of the C code
    eri = _eri(L)
    assert np.allclose(J[0], np.einsum("abcd,cd->ab", eri, D[0]), rtol=0, atol=1e-12 * np.abs(J[0]).max())
    assert np.allclose(K[0], np.einsum("acbd,cd->ab", eri, D[0]), rtol=0, atol=1e-12 * np.abs(K[0]).max())


def test_dense_build_equals_factored_build():
    """For D = X Y^T the dense maps agree with the factored build (O2)."""
    rng = np.random.default_rng(2)
    n, naux, k = 11, 9, 4
    L = _factor(rng, n, naux)
    X = [rng.standard_normal((n, k)) for _ in range(2)]
    Y = [rng.standard_normal((n, k)) for _ in range(2)]
    D = np.stack([x @ y.T for x, y in zip(X, Y)])
    J, K = oracle.build_dense(L, D)
    Jf, Kf = oracle.build(L, X, Y)
    assert np.abs(J - Jf).max() <= 1e-13 * np.abs(Jf).max()
    assert np.abs(K - Kf).max() <= 1e-13 * np.abs(Kf).max()


def test_dense_closed_forms():
    rng = np.random.default_rng(3)
    n = 6
    D = rng.standard_normal((1, n, n))
    # identity factor: J = naux tr(D) I, K = naux D
    naux = 4
    L = np.stack([np.eye(n)] * naux)
    J, K = oracle.build_dense(L, D)
    assert np.allclose(J[0], naux * np.trace(D[0]) * np.eye(n), rtol=0, atol=1e-13)
    assert np.allclose(K[0], naux * D[0], rtol=0, atol=1e-13)
    # rank-1 factor L = v v^T: J = K = (v^T D v) v v^T
    v = rng.standard_normal(n)
    J, K = oracle.build_dense(np.outer(v, v)[None], D)
    ref = (v @ D[0] @ v) * np.outer(v, v)
    assert np.allclose(J[0], ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    assert np.allclose(K[0], ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    # elementary symmetric factor E_ij + E_ji: K swaps rows/columns i <-> j
    i, j = 1, 4
    E = np.zeros((n, n)); E[i, j] = E[j, i] = 1.0
    _, K = oracle.build_dense(E[None], D)
    ref = np.zeros((n, n))
    ref[i, i], ref[i, j], ref[j, i], ref[j, j] = D[0, j, j], D[0, j, i], D[0, i, j], D[0, i, i]
    assert np.array_equal(K[0], ref)


def test_dense_identities():
    """J sees only the symmetric part of D; K(D^T) = K(D)^T; both linear."""
    rng = np.random.default_rng(4)
    n, naux = 8, 6
    L = _factor(rng, n, naux)
    D1, D2 = rng.standard_normal((2, n, n))
    J1, K1 = oracle.build_dense(L, D1[None])
    J1t, K1t = oracle.build_dense(L, D1.T.copy()[None])
    scale = np.abs(K1).max()
    assert np.abs(J1 - J1t).max() <= 1e-13 * np.abs(J1).max()
    assert np.abs(K1t[0] - K1[0].T).max() <= 1e-13 * scale
    a, b = 0.7, -1.9
    J2, K2 = oracle.build_dense(L, D2[None])
    J12, K12 = oracle.build_dense(L, (a * D1 + b * D2)[None])
    assert np.abs(J12 - (a * J1 + b * J2)).max() <= 1e-12 * np.abs(J12).max()
    assert np.abs(K12 - (a * K1 + b * K2)).max() <= 1e-12 * np.abs(K12).max()
    # J or K alone gives the same values
    Jo, Ko = oracle.build_dense(L, D1[None], want_k=False)
    assert Ko is None and np.array_equal(Jo, J1)
    Jo, Ko = oracle.build_dense(L, D1[None], want_j=False)
    assert Jo is None and np.array_equal(Ko, K1)


def _energy_brute(L, D, W, V):
    """E = sum_s <W_s, K(D_s)> + <V_s, J(D_s)> through O1."""
    e = 0.0
    for s in range(D.shape[0]):
        Jb, Kb = oracle.brute(L, D[s])
        e += np.sum(W[s] * Kb) + np.sum(V[s] * Jb)
    return e


def test_density_gradient_brute_and_exact_differences():
    rng = np.random.default_rng(5)
    n, naux, nd = 6, 5, 2
    L = _factor(rng, n, naux)
    D = rng.standard_normal((nd, n, n))
    W = rng.standard_normal((nd, n, n))
    V = rng.standard_normal((nd, n, n))
    G = oracle.density_grad(L, W, V)
    for s in range(nd):
        _, KW = oracle.brute(L, W[s])
        JV, _ = oracle.brute(L, V[s])
        assert np.abs(G[s] - (KW + JV)).max() <= 1e-13 * np.abs(G[s]).max()
    # E is linear in D: a central difference is exact up to rounding
    for _ in range(4):
        dD = rng.standard_normal((nd, n, n))
        h = 1e-2
        fd = (_energy_brute(L, D + h * dD, W, V) - _energy_brute(L, D - h * dD, W, V)) / (2 * h)
        assert abs(fd - np.sum(G * dD)) <= 1e-10 * abs(fd)
    # missing seeds are zero
    assert np.abs(oracle.density_grad(L, W, None) - oracle.build_dense(L, W, want_j=False)[1]).max() == 0.0
    assert np.abs(oracle.density_grad(L, None, V) - oracle.build_dense(L, V, want_k=False)[0]).max() == 0.0


def test_density_gradient_chain_rule_to_factored_adjoint():
    """dX_s = G_s Y_s and dY_s = G_s^T X_s for D_s = X_s Y_s^T: the factored
    adjoint (O3, pinned by differences of E) follows from G."""
    rng = np.random.default_rng(6)
    n, naux, ks = 9, 7, [3, 5]
    L = _factor(rng, n, naux)
    X = [rng.standard_normal((n, k)) for k in ks]
    Y = [rng.standard_normal((n, k)) for k in ks]
    W = [rng.standard_normal((n, n)) for _ in ks]
    V = [rng.standard_normal((n, n)) for _ in ks]
    dX, dY, _ = oracle.adjoint(L, X, Y, W, V, want_dl=False)
    G = oracle.density_grad(L, np.stack(W), np.stack(V))
    for s in range(len(ks)):
        assert np.abs(dX[s] - G[s] @ Y[s]).max() <= 1e-12 * np.abs(dX[s]).max()
        assert np.abs(dY[s] - G[s].T @ X[s]).max() <= 1e-12 * np.abs(dY[s]).max()


def _sets(rng, n, ks):
    return [rng.standard_normal((n, k)) for k in ks], [rng.standard_normal((n, k)) for k in ks]


@pytest.mark.parametrize("symmetric", [True, False])
def test_pairs_are_the_four_index_sums(symmetric):
    """Jp[a][b] = sum WL^{mu nu} (mu nu|lam sig) WR^{lam sig} and
    Kp[a][b] = sum WL^{mu nu} (mu lam|nu sig) WR^{lam sig}, by einsum, also for
    a non-symmetric L (so a transposed factor cannot pass)."""
    rng = np.random.default_rng(7)
    n, naux = 6, 4
    L = _factor(rng, n, naux, symmetric)
    A, B = _sets(rng, n, [2, 3])
    X, Y = _sets(rng, n, [1, 4, 2])
    Jp, Kp = oracle.pairs(L, A, B, X, Y)
    eri = _eri(L)
    for a in range(2):
        WL = A[a] @ B[a].T
        for b in range(3):
            WR = X[b] @ Y[b].T
            jr = np.einsum("ab,abcd,cd->", WL, eri, WR)
            kr = np.einsum("ab,acbd,cd->", WL, eri, WR)
            assert abs(Jp[a, b] - jr) <= 1e-12 * max(abs(jr), 1.0)
            assert abs(Kp[a, b] - kr) <= 1e-12 * max(abs(kr), 1.0)
            # and through O1's matrices
            Jb, Kb = oracle.brute(L, WR)
            assert abs(Jp[a, b] - np.sum(WL * Jb)) <= 1e-13 * max(abs(jr), 1.0)
            assert abs(Kp[a, b] - np.sum(WL * Kb)) <= 1e-13 * max(abs(kr), 1.0)


def test_pairs_bra_ket_symmetry_and_positivity():
    """The pairing scalars are invariant under WL <-> WR; the J pairing sees
    only symmetric parts; <W, J(W)> = sum_P gamma_P^2 >= 0."""
    rng = np.random.default_rng(8)
    n, naux = 10, 8
    L = _factor(rng, n, naux)
    A, B = _sets(rng, n, [3, 2])
    X, Y = _sets(rng, n, [4, 1, 2])
    Jp, Kp = oracle.pairs(L, A, B, X, Y)
    Jq, Kq = oracle.pairs(L, X, Y, A, B)
    sj, sk = np.abs(Jp).max(), np.abs(Kp).max()
    assert np.abs(Jp - Jq.T).max() <= 1e-13 * sj
    assert np.abs(Kp - Kq.T).max() <= 1e-13 * sk
    # transposing a left density (swap its factors) leaves J pairings unchanged
    Jt, Kt = oracle.pairs(L, B, A, X, Y)
    assert np.abs(Jt - Jp).max() <= 1e-13 * sj
    assert np.abs(Kt - Kp).max() > 1e-3 * sk     # K does see the antisymmetric part
    # <W, J(W)> on the diagonal of a set paired with itself
    Jd, _ = oracle.pairs(L, A, B, A, B)
    for a in range(2):
        W = A[a] @ B[a].T
        g = np.einsum("pab,ab->p", L, W)
        assert Jd[a, a] >= 0 and abs(Jd[a, a] - np.sum(g * g)) <= 1e-13 * np.sum(g * g)
