"""jk_build_host: host-resident inputs streamed to the device chunk by chunk,
against the oracle and against the device-resident build."""
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


def _host(m, pinned):
    def t(a):
        x = torch.from_numpy(np.ascontiguousarray(a))
        return x.pin_memory() if pinned else x
    return t(m.L), [t(x) for x in m.X], [t(y) for y in m.Y]


@pytest.mark.parametrize("precision", ["split", "fp64"])
@pytest.mark.parametrize("chunk,pinned", [(16, True), (0, True), (37, False)])
def test_host_build_matches_oracle(eng, precision, chunk, pinned):
    m = inputs.custom(70, 150, 40.0, [5, 7, 4], [False, True, False], seed=7)
    Jo, Ko = oracle.build(m.L, m.X, m.Y)
    L, X, Y = _host(m, pinned)
    eng.set_option("host_chunk", chunk)
    J, K = eng.build_host(L, X, Y, m.sym, precision)
    eng.set_option("host_chunk", 0)
    assert J.device.type == "cpu" and K.device.type == "cpu"
    if precision == "split":
        assert abs_err(J.numpy(), Jo) < SPLIT_ABS and abs_err(K.numpy(), Ko) < SPLIT_ABS
    else:
        assert rel_err(J.numpy(), Jo) < FP64_REL and rel_err(K.numpy(), Ko) < FP64_REL


def test_host_build_j_or_k_only(eng):
    m = inputs.custom(40, 90, 20.0, [4, 3], [False, False], seed=8)
    Jo, Ko = oracle.build(m.L, m.X, m.Y)
    L, X, Y = _host(m, True)
    eng.set_option("host_chunk", 20)
    J, K = eng.build_host(L, X, Y, m.sym, "split", want_k=False)
    assert K is None and abs_err(J.numpy(), Jo) < SPLIT_ABS
    J, K = eng.build_host(L, X, Y, m.sym, "split", want_j=False)
    assert J is None and abs_err(K.numpy(), Ko) < SPLIT_ABS
    eng.set_option("host_chunk", 0)


@pytest.mark.slow
def test_host_build_multi_state_matches_device_build(eng):
    """The 400/2400/8-density workload: streamed in chunks vs resident in HBM
    (they differ only by the order of the FP64 sums over aux chunks)."""
    m = inputs.multi_state()
    L, X, Y = _host(m, True)
    Jh, Kh = eng.build_host(L, X, Y, m.sym, "split")
    Jd, Kd = eng.build(L.cuda(), [x.cuda() for x in X], [y.cuda() for y in Y], m.sym, "split")
    eng.sync_status()
    assert abs_err(Jh.numpy(), to_np(Jd)) < SPLIT_ABS and abs_err(Kh.numpy(), to_np(Kd)) < SPLIT_ABS
    rng = np.random.default_rng(9)
    s, mu, nu = rng.integers(0, m.nd, 24), rng.integers(0, m.n, 24), rng.integers(0, m.n, 24)
    Jo, Ko = oracle.sample(m.L, m.X, m.Y, s, mu, nu)
    assert np.abs(Jh.numpy()[s, mu, nu] - Jo).max() < SPLIT_ABS
    assert np.abs(Kh.numpy()[s, mu, nu] - Ko).max() < SPLIT_ABS
