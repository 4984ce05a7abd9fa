"""The split builds' J on the tensor cores (JK_OPT_J_PATH = 1: the factor's aux
chunks sliced transposed over the upper triangle, gamma sliced, one sliced
GEMM per chunk, the product added onto both triangles in chunk order) against
the oracle, on ragged shapes, several chunks, chunks longer than one
super-chunk, the grouped schedule, J-only builds, a packed factor and batched
builds; and against the FP64 form of J (JK_OPT_J_PATH = 0) on the same
inputs.  The automatic choice takes the tensor cores only for large builds
(the headline and batch workloads, covered at full size elsewhere)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2608_06536_b300 import inputs, jk
from tests._util import SPLIT_ABS, abs_err, to_np

pytestmark = pytest.mark.gpu


def _gpu(m, packed=False):
    L = jk.pack_factor(m.L) if packed else torch.from_numpy(m.L)
    return (L.cuda(), [torch.from_numpy(x).cuda() for x in m.X], [torch.from_numpy(y).cuda() for y in m.Y])


def _engine(opts):
    eng = jk.Engine("cuda:0")
    for k, v in opts.items():
        eng.set_option(k, v)
    return eng


@pytest.mark.parametrize("n,naux,ks,sym,opts", [
    (7, 5, [3], [False], {}),
    (37, 53, [5, 1, 13], [False, True, False], {}),
    (130, 70, [9, 3, 20], [False, True, False], {"aux_chunk": 17}),
    (130, 70, [64, 3, 9], [False, False, True], {"schedule": 1, "aux_chunk": 30}),
    (20, 2100, [3, 2], [False, True], {}),
    (257, 90, [11, 5], [True, False], {"schedule": 1}),
])
def test_tensor_j_vs_oracle(n, naux, ks, sym, opts):
    m = inputs.custom(n, naux, max(naux / 4, 1.0), ks, sym)
    Jo, Ko = oracle.build(m.L, m.X, m.Y)
    eng = _engine({"j_path": 1, **opts})
    L, X, Y = _gpu(m)
    J, K = eng.build(L, X, Y, sym, "split")
    eng.sync_status()
    assert abs_err(to_np(J), Jo) < SPLIT_ABS
    assert abs_err(to_np(K), Ko) < SPLIT_ABS


def test_tensor_j_matches_fp64_form():
    """Both forms of J on the same inputs: K bit for bit (untouched by the
    choice), J within the split engine's error of each other."""
    m = inputs.custom(96, 300, 60.0, [8, 5, 12], [False, True, False])
    L, X, Y = _gpu(m)
    out = {}
    for path in (0, 1):
        eng = _engine({"j_path": path, "aux_chunk": 70})
        out[path] = [to_np(t) for t in eng.build(L, X, Y, m.sym, "split")]
        eng.sync_status()
    np.testing.assert_array_equal(out[0][1], out[1][1])
    assert abs_err(out[1][0], out[0][0]) < SPLIT_ABS
    assert np.array_equal(out[1][0], np.swapaxes(out[1][0], 1, 2))   # both triangles written alike


def test_tensor_j_only_and_packed_factor():
    m = inputs.custom(130, 70, 17.0, [9, 3, 20], [False, True, False])
    Jo, _ = oracle.build(m.L, m.X, m.Y)
    eng = _engine({"j_path": 1, "aux_chunk": 30})
    L, X, Y = _gpu(m)
    J, _ = eng.build(L, X, Y, m.sym, "split", want_k=False)
    eng.sync_status()
    assert abs_err(to_np(J), Jo) < SPLIT_ABS
    engp = _engine({"j_path": 1, "aux_chunk": 30, "packed_factor": 1})
    Lp, Xp, Yp = _gpu(m, packed=True)
    Jp, _ = engp.build(Lp, Xp, Yp, m.sym, "split", want_k=False)
    engp.sync_status()
    np.testing.assert_array_equal(to_np(Jp), to_np(J))      # the packed factor's J: the same bits


@pytest.mark.parametrize("chunk", [0, 45])
def test_tensor_j_batched(chunk):
    shapes = [(40, 90, [4, 4], [False, True]), (75, 150, [7], [False]), (24, 60, [3, 2, 5], [False, False, False]),
              (130, 260, [13, 13], [False, False])]
    mols = [inputs.custom(n, naux, max(naux / 5.0, 1.0), ks, sym, seed=i)
            for i, (n, naux, ks, sym) in enumerate(shapes)]
    eng = _engine({"j_path": 1, "aux_chunk": chunk})
    outs = eng.build_batched([(*_gpu(m), m.sym) for m in mols], "split")
    eng.sync_status()
    for m, (J, K) in zip(mols, outs):
        Jo, Ko = oracle.build(m.L, m.X, m.Y)
        assert abs_err(to_np(J), Jo) < SPLIT_ABS
        assert abs_err(to_np(K), Ko) < SPLIT_ABS
