"""Dense (general, non-symmetric) densities on the GPU against the oracle:
J(D), K(D) (jk_build_dense) and the density gradient K(W) + J(V)
(jk_density_grad), in both precisions, on ragged sizes, several aux chunks
(so chunk results accumulate, through int64 split-K partials and through a
plain FP64 sum) and the single-map forms.  Dense inputs come from the seeded
recipe (N(0, 1/nbf^2) entries)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2608_06536_b300 import inputs
from tests._util import FP64_REL, SPLIT_ABS, abs_err, rel_err, to_np

pytestmark = pytest.mark.gpu

CASES = [(7, 5, 1, 0), (37, 53, 3, 0), (37, 53, 3, 17), (130, 70, 2, 0), (130, 70, 2, 30)]


@pytest.fixture(scope="module")
def eng():
    from paper_2608_06536_b300 import jk
    e = jk.Engine("cuda:0")
    yield e
    e.close()


def _case(n, naux, nd, seed=0):
    L = inputs.factor(n, naux, max(naux / 4, 1.0), seed)
    mats = [inputs.dense_densities(n, nd, seed=10 * seed + j) for j in range(3)]
    return L, mats


def _ok(prec, got, ref):
    return rel_err(got, ref) < FP64_REL if prec == "fp64" else abs_err(got, ref) < SPLIT_ABS


@pytest.mark.parametrize("prec", ["fp64", "split"])
@pytest.mark.parametrize("n,naux,nd,chunk", CASES)
def test_build_dense_vs_oracle(eng, prec, n, naux, nd, chunk):
    L, (D, _, _) = _case(n, naux, nd)
    Jo, Ko = oracle.build_dense(L, D)
    eng.set_option("aux_chunk", chunk)
    try:
        J, K = eng.build_dense(torch.from_numpy(L).cuda(), torch.from_numpy(D).cuda(), prec)
        eng.sync_status()
    finally:
        eng.set_option("aux_chunk", -1)
    assert _ok(prec, to_np(J), Jo) and _ok(prec, to_np(K), Ko)


@pytest.mark.parametrize("prec", ["fp64", "split"])
def test_build_dense_single_maps(eng, prec):
    L, (D, _, _) = _case(37, 53, 2, seed=1)
    Jo, Ko = oracle.build_dense(L, D)
    Ld, Dd = torch.from_numpy(L).cuda(), torch.from_numpy(D).cuda()
    J, K = eng.build_dense(Ld, Dd, prec, want_k=False)
    assert K is None and _ok(prec, to_np(J), Jo)
    J, K = eng.build_dense(Ld, Dd, prec, want_j=False)
    assert J is None and _ok(prec, to_np(K), Ko)
    eng.sync_status()


@pytest.mark.parametrize("prec", ["fp64", "split"])
@pytest.mark.parametrize("n,naux,nd,chunk", [CASES[1], CASES[2], CASES[4]])
def test_density_grad_vs_oracle(eng, prec, n, naux, nd, chunk):
    L, (_, W, V) = _case(n, naux, nd, seed=2)
    Ld, Wd, Vd = torch.from_numpy(L).cuda(), torch.from_numpy(W).cuda(), torch.from_numpy(V).cuda()
    eng.set_option("aux_chunk", chunk)
    try:
        for w, v, wd, vd in [(W, V, Wd, Vd), (W, None, Wd, None), (None, V, None, Vd)]:
            Go = oracle.density_grad(L, w, v, nd=nd)
            G = eng.density_grad(Ld, wd, vd, prec)
            eng.sync_status()
            assert _ok(prec, to_np(G), Go)
    finally:
        eng.set_option("aux_chunk", -1)


def test_density_grad_carries_to_factored_adjoint(eng):
    """jk_adjoint's dX_s, dY_s equal G_s Y_s and G_s^T X_s (FP64, on the GPU)."""
    m = inputs.custom(40, 60, 15.0, [5, 6], [False, False], seed=3)
    rng = np.random.default_rng(7)
    W = torch.tensor(rng.standard_normal((2, 40, 40))).cuda()
    V = torch.tensor(rng.standard_normal((2, 40, 40))).cuda()
    L = torch.from_numpy(m.L).cuda()
    X = [torch.from_numpy(x).cuda() for x in m.X]
    Y = [torch.from_numpy(y).cuda() for y in m.Y]
    dX, dY, _ = eng.adjoint(L, X, Y, m.sym, W, V, want_dl=False, precision="fp64")
    G = eng.density_grad(L, W, V, "fp64")
    eng.sync_status()
    for s in range(2):
        assert rel_err(to_np(dX[s]), to_np(G[s] @ Y[s])) < 1e-12
        assert rel_err(to_np(dY[s]), to_np(G[s].T @ X[s])) < 1e-12


def test_autograd_dense_gradient_is_the_density_gradient(eng):
    """jk_dense's backward gives d/dD of sum <A, J(D)> + <B, K(D)>, which is
    J(A) + K(B); checked against the oracle and against central differences of
    the forward (exact up to rounding: E is linear in D)."""
    from paper_2608_06536_b300.autograd import jk_dense
    L, (D, A, B) = _case(37, 53, 2, seed=4)
    Ld = torch.from_numpy(L).cuda()
    Dd = torch.from_numpy(D).cuda().requires_grad_(True)
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    J, K = jk_dense(Ld, Dd, "fp64", engine=eng)
    ((Ad * J).sum() + (Bd * K).sum()).backward()
    Go = oracle.density_grad(L, B, A, nd=2)
    assert rel_err(to_np(Dd.grad), Go) < FP64_REL
    rng = np.random.default_rng(8)
    dD = torch.from_numpy(rng.standard_normal(D.shape)).cuda()
    h = 1e-3
    with torch.no_grad():
        Jp, Kp = eng.build_dense(Ld, Dd + h * dD, "fp64")
        Jm, Km = eng.build_dense(Ld, Dd - h * dD, "fp64")
        fd = float(((Ad * (Jp - Jm)).sum() + (Bd * (Kp - Km)).sum()) / (2 * h))
    assert abs(fd - float((Dd.grad * dD).sum())) <= 1e-9 * abs(fd)
