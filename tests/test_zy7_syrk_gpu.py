"""The blocked symmetric rank update (JK_OPT_SYRK = 1, both engines) on
the GPU: for symmetric densities only the row blocks from the diagonal on are
formed (row views of the sliced T_X) and the rest is mirrored.  The mirrored
entries must equal their transposes exactly, and K must match the full rank update (option 0) within the split
tolerance and the oracle within the 1e-10 gate, through single- and
multi-chunk builds (FP64 chunk sums and int64 split-K partials), both launch
schedules, ragged nbf, and batched builds."""
import numpy as np
import pytest
import torch

import oracle
from paper_2608_06536_b300 import inputs
from tests._util import SPLIT_ABS, abs_err, to_np

pytestmark = pytest.mark.gpu


def _check_mirrored(Ks):
    """Entries left of their row's 128-row diagonal block are copies of their
    transposes (exactly); inside the diagonal blocks both halves are formed by
    the GEMM, equal to rounding."""
    n = Ks.shape[0]
    r, c = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    outside = c < 128 * (r // 128)
    np.testing.assert_array_equal(Ks[outside], Ks.T[outside])
    assert abs_err(Ks, Ks.T) < SPLIT_ABS


def _dev(m):
    L = torch.from_numpy(m.L).cuda()
    X = [torch.from_numpy(x).cuda() for x in m.X]
    Y = [torch.from_numpy(y).cuda() for y in m.Y]
    return L, X, Y


@pytest.mark.parametrize("n,naux,ks,sym,opts", [
    (300, 70, [20, 9, 33], [True, False, True], {"aux_chunk": 30, "precision": "fp64"}),  # FP64 engine
    (300, 70, [20, 9, 33], [True, False, True], {"schedule": 0, "aux_chunk": 30}),      # chunk sums
    (300, 120, [40, 7], [True, True], {"schedule": 0, "aux_chunk": 70}),                # split-K partials
    (257, 90, [64, 5, 11], [True, True, False], {"schedule": 1, "aux_chunk": 40}),      # grouped, ragged
    (100, 30, [7, 4], [True, False], {"schedule": 1, "raster": 1}),                     # one block, m-tile raster
    (400, 240, [40, 40], [True, False], {"schedule": 1}),                               # the multi-state shape
])
def test_blocked_symmetric_rank_update(n, naux, ks, sym, opts):
    from paper_2608_06536_b300 import jk
    opts = dict(opts)
    prec = opts.pop("precision", "split")
    m = inputs.custom(n, naux, max(naux / 4, 1.0), ks, sym)
    Jo, Ko = oracle.build(m.L, m.X, m.Y)
    L, X, Y = _dev(m)
    eng = jk.Engine("cuda:0")
    for k, v in opts.items():
        eng.set_option(k, v)
    J0, K0 = eng.build(L, X, Y, m.sym, prec)
    eng.set_option("syrk", 1)
    J1, K1 = eng.build(L, X, Y, m.sym, prec)
    eng.sync_status()
    J0, K0, J1, K1 = to_np(J0), to_np(K0), to_np(J1), to_np(K1)
    eng.close()
    np.testing.assert_array_equal(J1, J0)                      # J does not depend on the option
    assert abs_err(J1, Jo) < SPLIT_ABS and abs_err(K1, Ko) < SPLIT_ABS
    for s, sy in enumerate(m.sym):
        if sy:
            _check_mirrored(K1[s])
            assert abs_err(K1[s], K0[s]) < SPLIT_ABS
        else:
            np.testing.assert_array_equal(K1[s], K0[s])        # non-symmetric densities: same launches


def test_batched_blocked_symmetric_rank_update():
    from paper_2608_06536_b300 import jk
    shapes = [(60, 150, [6, 6]), (140, 222, [11]), (33, 99, [3, 3, 3])]
    mols, refs = [], []
    for i, (n, naux, ks) in enumerate(shapes):
        sym = [s % 2 == 0 for s in range(len(ks))]
        m = inputs.custom(n, naux, max(naux / 4, 1.0), ks, sym, seed=i)
        refs.append(oracle.build(m.L, m.X, m.Y))
        L, X, Y = _dev(m)
        mols.append((L, X, Y, m.sym))
    eng = jk.Engine("cuda:0")
    eng.set_option("syrk", 1)
    out = eng.build_batched(mols, "split")
    eng.sync_status()
    for (J, K), (Jo, Ko), mol in zip(out, refs, mols):
        assert abs_err(to_np(J), Jo) < SPLIT_ABS and abs_err(to_np(K), Ko) < SPLIT_ABS
        for s, sy in enumerate(mol[3]):
            if sy:
                _check_mirrored(to_np(K[s]))
    eng.close()
