"""Bra-ket pairings on the GPU (jk_pair) against the oracle: Jp[a][b] =
<W_L^a, J(W_R^b)>, Kp[a][b] = <W_L^a, K(W_R^b)> for factored left and right
densities (symmetric and non-symmetric on either side), both precisions, the
single-pairing forms, and the bra-ket symmetry pairs(R, L) = pairs(L, R)^T."""
import numpy as np
import pytest
import torch

import oracle
from paper_2608_06536_b300 import inputs
from tests._util import FP64_REL, SPLIT_ABS, abs_err, rel_err, to_np

pytestmark = pytest.mark.gpu

CASES = [
    (40, 60, [3, 5], [False, True], [4, 6, 2], [False, False, True]),
    (130, 70, [9, 3], [False, False], [12, 5], [True, False]),
]


@pytest.fixture(scope="module")
def eng():
    from paper_2608_06536_b300 import jk
    e = jk.Engine("cuda:0")
    yield e
    e.close()


def _sides(n, naux, kl, sl, kr, sr):
    mL = inputs.custom(n, naux, max(naux / 4, 1.0), kl, sl, seed=1)
    mR = inputs.custom(n, naux, max(naux / 4, 1.0), kr, sr, seed=2)
    return mL, mR


def _dev(m):
    return [torch.from_numpy(x).cuda() for x in m.X], [torch.from_numpy(y).cuda() for y in m.Y]


def _ok(prec, got, ref):
    return rel_err(got, ref) < FP64_REL if prec == "fp64" else abs_err(got, ref) < SPLIT_ABS


@pytest.mark.parametrize("prec", ["fp64", "split"])
@pytest.mark.parametrize("case", CASES)
def test_pairs_vs_oracle(eng, prec, case):
    n, naux, kl, sl, kr, sr = case
    mL, mR = _sides(n, naux, kl, sl, kr, sr)
    Jo, Ko = oracle.pairs(mL.L, mL.X, mL.Y, mR.X, mR.Y)
    L = torch.from_numpy(mL.L).cuda()
    (XL, YL), (XR, YR) = _dev(mL), _dev(mR)
    Jp, Kp = eng.pairs(L, XL, YL, sl, XR, YR, sr, prec)
    eng.sync_status()
    assert Jp.shape == (len(kl), len(kr)) and _ok(prec, to_np(Jp), Jo) and _ok(prec, to_np(Kp), Ko)
    Jp, Kp = eng.pairs(L, XL, YL, sl, XR, YR, sr, prec, want_k=False)
    assert Kp is None and _ok(prec, to_np(Jp), Jo)
    Jp, Kp = eng.pairs(L, XL, YL, sl, XR, YR, sr, prec, want_j=False)
    assert Jp is None and _ok(prec, to_np(Kp), Ko)
    eng.sync_status()


def test_pairs_bra_ket_symmetry(eng):
    n, naux, kl, sl, kr, sr = CASES[0]
    mL, mR = _sides(n, naux, kl, sl, kr, sr)
    L = torch.from_numpy(mL.L).cuda()
    (XL, YL), (XR, YR) = _dev(mL), _dev(mR)
    Jp, Kp = eng.pairs(L, XL, YL, sl, XR, YR, sr, "split")
    Jq, Kq = eng.pairs(L, XR, YR, sr, XL, YL, sl, "split")
    eng.sync_status()
    assert abs_err(to_np(Jp), to_np(Jq).T) < 2 * SPLIT_ABS
    assert abs_err(to_np(Kp), to_np(Kq).T) < 2 * SPLIT_ABS
