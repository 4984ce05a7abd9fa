"""Batched builds (grouped persistent launches), CUDA-graph replay and
aux-index chunk independence."""
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
    return jk.Engine("cuda:0")


def _gpu(m):
    L = torch.from_numpy(m.L).cuda()
    X = [torch.from_numpy(x).cuda() for x in m.X]
    Y = [torch.from_numpy(y).cuda() for y in m.Y]
    return L, X, Y


def _mols(shapes, seed0=0):
    out = []
    for i, (n, naux, ks, sym) in enumerate(shapes):
        m = inputs.custom(n, naux, max(naux / 5.0, 1.0), ks, sym, seed=seed0 + i)
        out.append(m)
    return out


SHAPES = [(40, 90, [4, 4], [False, True]), (75, 150, [7], [False]), (24, 60, [3, 2, 5], [False, False, False]),
          (130, 260, [13, 13], [False, False])]


@pytest.mark.parametrize("chunk", [0, 37])
def test_fp64_chunk_independence(eng, chunk):
    """Aux-index blocking is a pure memory knob (paper, Table 'precision'):
    FP64 results agree to summation-order level."""
    m = inputs.custom(64, 200, 40.0, [6, 5], [False, True])
    L, X, Y = _gpu(m)
    eng.set_aux_chunk(0)
    J0, K0 = eng.build(L, X, Y, m.sym, "fp64")
    eng.set_aux_chunk(chunk or 1)
    J1, K1 = eng.build(L, X, Y, m.sym, "fp64")
    eng.set_aux_chunk(0)
    assert rel_err(to_np(J1), to_np(J0)) < 1e-13
    assert rel_err(to_np(K1), to_np(K0)) < 1e-13


@pytest.mark.parametrize("chunk", [13, 50])
def test_split_chunk_independence(eng, chunk):
    m = inputs.custom(64, 200, 40.0, [6, 5], [False, True])
    Jo, Ko = oracle.build(m.L, m.X, m.Y)
    L, X, Y = _gpu(m)
    eng.set_aux_chunk(chunk)
    J, K = eng.build(L, X, Y, m.sym, "split")
    eng.sync_status()
    eng.set_aux_chunk(0)
    assert abs_err(to_np(J), Jo) < SPLIT_ABS and abs_err(to_np(K), Ko) < SPLIT_ABS


def test_split_adjoint_multi_chunk(eng):
    n = 40
    m = inputs.custom(n, 120, 30.0, [4, 6], [False, True])
    rng = np.random.default_rng(8)
    W = [rng.standard_normal((n, n)) for _ in range(2)]
    V = [rng.standard_normal((n, n)) for _ in range(2)]
    dXo, dYo, dLo = oracle.adjoint(m.L, m.X, m.Y, W, V)
    L, X, Y = _gpu(m)
    eng.set_aux_chunk(23)
    dX, dY, dL = eng.adjoint(L, X, Y, m.sym, torch.tensor(np.array(W)).cuda(),
                             torch.tensor(np.array(V)).cuda(), precision="split")
    eng.sync_status()
    eng.set_aux_chunk(0)
    assert abs_err(to_np(dL), dLo) < SPLIT_ABS
    assert abs_err(to_np(dX[0]), dXo[0]) < SPLIT_ABS and abs_err(to_np(dY[0]), dYo[0]) < SPLIT_ABS
    assert abs_err(to_np(dX[1]), dXo[1] + dYo[1]) < SPLIT_ABS


@pytest.mark.parametrize("chunk", [0, 45])
def test_split_batched_matches_oracle(eng, chunk):
    mols = _mols(SHAPES)
    args = [(*_gpu(m), m.sym) for m in mols]
    eng.set_aux_chunk(chunk)
    outs = eng.build_batched(args, "split")
    eng.sync_status()
    eng.set_aux_chunk(0)
    for m, (J, K) in zip(mols, outs):
        Jo, Ko = oracle.build(m.L, m.X, m.Y)
        assert abs_err(to_np(J), Jo) < SPLIT_ABS
        assert abs_err(to_np(K), Ko) < SPLIT_ABS


def test_split_batched_uses_grouped_launches(eng):
    """All panels of a wave go into one persistent launch, all rank updates
    into another (up to 32 problems per launch)."""
    mols = _mols(SHAPES)
    args = [(*_gpu(m), m.sym) for m in mols]
    eng.build_batched(args, "split")          # sizes the arena
    eng.profile(True)
    eng.profile_reset()
    eng.build_batched(args, "split")
    prof = eng.profile_read()
    eng.profile(False)
    nprob = len(mols) + sum(m.nd for m in mols)
    assert prof["ozgemm_tcgen05"][1] <= 2 + nprob // 32


def test_split_batched_graph_replay(eng):
    """A batched split build captured once in a CUDA graph and replayed gives
    the eager result; replay after changing the inputs in place follows them."""
    mols = _mols(SHAPES[:3], seed0=20)
    args = [(*_gpu(m), m.sym) for m in mols]
    eager = eng.build_batched(args, "split")
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            outs = eng.build_batched(args, "split", stream=s)
    torch.cuda.current_stream().wait_stream(s)
    g.replay()
    torch.cuda.synchronize()
    for (Je, Ke), (J, K) in zip(eager, outs):
        assert torch.equal(J, Je) and torch.equal(K, Ke)
    for L, X, Y, sym in args:          # X -> 2X, Y -> 2Y: every D, hence J and K, scales by 4
        for s_, (x, y) in enumerate(zip(X, Y)):
            x.mul_(2.0)
            if not sym[s_]:
                y.mul_(2.0)
    g.replay()
    torch.cuda.synchronize()
    for (Je, Ke), (J, K) in zip(eager, outs):
        assert abs_err(to_np(J), 4 * to_np(Je)) < 8 * SPLIT_ABS
        assert abs_err(to_np(K), 4 * to_np(Ke)) < 8 * SPLIT_ABS


def test_fp64_batched_uneven_vs_oracle(eng):
    mols = _mols(SHAPES[:3], seed0=40)
    args = [(*_gpu(m), m.sym) for m in mols]
    outs = eng.build_batched(args, "fp64")
    for m, (J, K) in zip(mols, outs):
        Jo, Ko = oracle.build(m.L, m.X, m.Y)
        assert rel_err(to_np(J), Jo) < FP64_REL and rel_err(to_np(K), Ko) < FP64_REL


@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_outputs_at_odd_offsets(eng, precision):
    """Outputs need only double alignment: odd nbf makes every other density's
    J_s, K_s start 8 bytes off a 16-byte boundary (batched), and a single
    build may write into a view that starts one double into a buffer."""
    mols = _mols([(37, 80, [3, 4, 2], [False, True, False]), (21, 40, [2, 2], [False, False])], seed0=60)
    args = [(*_gpu(m), m.sym) for m in mols]
    outs = eng.build_batched(args, precision)
    eng.sync_status()
    tol = (lambda a, b: rel_err(a, b) < FP64_REL) if precision == "fp64" else (lambda a, b: abs_err(a, b) < SPLIT_ABS)
    for m, (J, K) in zip(mols, outs):
        Jo, Ko = oracle.build(m.L, m.X, m.Y)
        assert tol(to_np(J), Jo) and tol(to_np(K), Ko)
    m = mols[0]
    L, X, Y = _gpu(m)
    buf = torch.full((2 * m.nd * m.n * m.n + 1,), float("nan"), dtype=torch.float64, device="cuda")
    J = buf[1:1 + m.nd * m.n * m.n].view(m.nd, m.n, m.n)
    K = buf[1 + m.nd * m.n * m.n:].view(m.nd, m.n, m.n)
    eng.build(L, X, Y, m.sym, precision, J=J, K=K)
    eng.sync_status()
    Jo, Ko = oracle.build(m.L, m.X, m.Y)
    assert tol(to_np(J), Jo) and tol(to_np(K), Ko)
    assert torch.isnan(buf[0])
