"""Autotuner on the GPU: every configuration it can pick gives the oracle's
result, jk_autotune caches the fastest and later builds use it."""
import numpy as np
import pytest
import torch

import oracle
from paper_2608_06536_b300 import inputs
from tests._util import FP64_REL, SPLIT_ABS, abs_err, rel_err, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture()
def eng():
    from paper_2608_06536_b300 import jk
    jk.tune_clear()
    e = jk.Engine("cuda:0")
    yield e
    e.close()
    jk.tune_clear()


def _gpu(m):
    return (torch.from_numpy(m.L).cuda(), [torch.from_numpy(x).cuda() for x in m.X],
            [torch.from_numpy(y).cuda() for y in m.Y])


@pytest.mark.parametrize("chunk,schedule,raster", [
    (0, 0, 1), (0, 1, 0), (0, 1, 1), (37, 1, 1), (37, 0, 1), (300, 1, 0), (0, 0, 0), (300, 0, 0)])
def test_every_split_configuration_matches_oracle(eng, chunk, schedule, raster):
    m = inputs.custom(150, 300, 60.0, [12, 9, 20], [False, True, False], seed=3)
    Jo, Ko = oracle.build(m.L, m.X, m.Y)
    L, X, Y = _gpu(m)
    eng.set_option("aux_chunk", chunk)
    eng.set_option("schedule", schedule)
    eng.set_option("raster", raster)
    J, K = eng.build(L, X, Y, m.sym, "split")
    eng.sync_status()
    assert abs_err(to_np(J), Jo) < SPLIT_ABS and abs_err(to_np(K), Ko) < SPLIT_ABS


def test_autotune_split_caches_and_is_used(eng):
    from paper_2608_06536_b300 import jk
    m = inputs.custom(200, 500, 100.0, [16] * 4, [False, False, True, False], seed=4)
    Jo, Ko = oracle.build(m.L, m.X, m.Y)
    L, X, Y = _gpu(m)
    cfg, ms = eng.autotune(L, X, Y, m.sym, "split", reps=2)
    assert ms > 0 and cfg["schedule"] in (0, 1) and cfg["raster"] in (0, 1) and cfg["aux_chunk"] >= 0
    text = jk.tune_export()
    assert len(text.splitlines()) == 1
    fields = text.split()
    assert [int(v) for v in fields[10:14]] == [cfg["aux_chunk"], cfg["schedule"], cfg["raster"], cfg["tile"]]
    # the tuned configuration is applied to the next build: same launch count
    # as forcing it explicitly, and the oracle's result
    eng.profile(True)
    eng.profile_reset()
    n0 = eng.launch_count()
    J, K = eng.build(L, X, Y, m.sym, "split")
    tuned_launches = eng.launch_count() - n0
    eng.sync_status()
    assert abs_err(to_np(J), Jo) < SPLIT_ABS and abs_err(to_np(K), Ko) < SPLIT_ABS
    for name, v in cfg.items():
        eng.set_option(name, v)
    eng.set_option("use_tuned", 0)
    n0 = eng.launch_count()
    eng.build(L, X, Y, m.sym, "split")
    assert eng.launch_count() - n0 == tuned_launches
    eng.profile(False)


def test_autotune_fp64(eng):
    m = inputs.custom(64, 400, 80.0, [6, 5], [False, True], seed=5)
    Jo, Ko = oracle.build(m.L, m.X, m.Y)
    L, X, Y = _gpu(m)
    cfg, ms = eng.autotune(L, X, Y, m.sym, "fp64", reps=1)
    assert ms > 0 and cfg["schedule"] == 0 and cfg["raster"] == 0
    J, K = eng.build(L, X, Y, m.sym, "fp64")
    assert rel_err(to_np(J), Jo) < FP64_REL and rel_err(to_np(K), Ko) < FP64_REL


def test_autotune_batched(eng):
    from paper_2608_06536_b300 import jk
    mols = [inputs.custom(n, naux, naux / 5.0, ks, None, seed=10 + i)
            for i, (n, naux, ks) in enumerate([(60, 150, [6, 6]), (111, 222, [11]), (33, 99, [3, 3, 3])])]
    args = [(*_gpu(m), m.sym) for m in mols]
    cfg, ms = eng.autotune_batched(args, "split", reps=1)
    assert ms > 0 and cfg["schedule"] == 1
    assert len(jk.tune_export().splitlines()) == 1
    outs = eng.build_batched(args, "split")
    eng.sync_status()
    for m, (J, K) in zip(mols, outs):
        Jo, Ko = oracle.build(m.L, m.X, m.Y)
        assert abs_err(to_np(J), Jo) < SPLIT_ABS and abs_err(to_np(K), Ko) < SPLIT_ABS


def test_autotune_rejects_bad_arguments(eng):
    from paper_2608_06536_b300 import jk
    m = inputs.custom(20, 30, 10.0, [2], [False])
    L, X, Y = _gpu(m)
    with pytest.raises(jk.JKError):
        eng.autotune(L, X, Y, m.sym, "split", reps=0)
    assert jk.tune_export() == ""
