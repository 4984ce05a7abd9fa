"""Laplace (LT-AO) builds on the GPU (jk_build_laplace) against the oracle
(O6): per-point J_k, K_k and the weighted sums, a non-symmetric
occupied-virtual pair of coefficient sets and a symmetric occupied one, both
precisions.  Quadrature: Gauss-Laguerre for 1/y (synthetic)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2608_06536_b300 import inputs
from tests._util import FP64_REL, SPLIT_ABS, abs_err, rel_err, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    from paper_2608_06536_b300 import jk
    e = jk.Engine("cuda:0")
    yield e
    e.close()


def _quad(nq):
    t, u = np.polynomial.laguerre.laggauss(nq)
    return t, u * np.exp(t)


def _ok(prec, got, ref):
    return rel_err(got, ref) < FP64_REL if prec == "fp64" else abs_err(got, ref) < SPLIT_ABS


@pytest.mark.parametrize("prec", ["fp64", "split"])
@pytest.mark.parametrize("n,naux,m,nq", [(37, 53, 5, 4), (130, 70, 9, 3)])
def test_laplace_vs_oracle(eng, prec, n, naux, m, nq):
    mol = inputs.custom(n, naux, max(naux / 4, 1.0), [m], [False], seed=4)
    CX, CY = mol.X[0], mol.Y[0]
    rng = np.random.default_rng(9)
    ei = -np.sort(rng.uniform(0.3, 1.5, m))
    ea = np.sort(rng.uniform(0.2, 2.0, m))
    alpha, w = _quad(nq)
    L = torch.from_numpy(mol.L).cuda()
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    # occupied against virtual, per point and weighted
    Jo, Ko = oracle.laplace(mol.L, CX, ei, +1, CY, ea, -1, alpha)
    J, K = eng.build_laplace(L, d(CX), d(ei), +1, alpha, None, d(CY), d(ea), -1, prec)
    assert J.shape == (nq, n, n) and _ok(prec, to_np(J), Jo) and _ok(prec, to_np(K), Ko)
    Jo, Ko = oracle.laplace(mol.L, CX, ei, +1, CY, ea, -1, alpha, w)
    J, K = eng.build_laplace(L, d(CX), d(ei), +1, alpha, w, d(CY), d(ea), -1, prec)
    assert J.shape == (n, n) and _ok(prec, to_np(J), Jo) and _ok(prec, to_np(K), Ko)
    # symmetric occupied pseudo-densities, K only
    Jo, Ko = oracle.laplace(mol.L, CX, ei, +1, CX, ei, +1, alpha, w)
    J, K = eng.build_laplace(L, d(CX), d(ei), +1, alpha, w, precision=prec, want_j=False)
    assert J is None and _ok(prec, to_np(K), Ko)
    eng.sync_status()
