"""jk_build_host_packed on the GPU: the factor uploaded as packed upper
triangles and expanded on the device gives jk_build_host's result bit for bit,
and the oracle's within the precision's tolerance."""
import pytest
import torch

import oracle
from paper_2608_06536_b300 import inputs
from tests._util import FP64_REL, SPLIT_ABS, abs_err, rel_err

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["split", "fp64"])
def test_packed_host_build_matches(precision):
    from paper_2608_06536_b300 import jk
    m = inputs.custom(64, 200, 50.0, [8, 5, 3], [False, True, False], seed=6)
    Jo, Ko = oracle.build(m.L, m.X, m.Y)
    L = torch.from_numpy(m.L)
    X = [torch.from_numpy(x) for x in m.X]
    Y = [torch.from_numpy(y) for y in m.Y]
    eng = jk.Engine("cuda:0")
    eng.set_option("host_chunk", 37)
    Jf, Kf = eng.build_host(L, X, Y, m.sym, precision)
    Jp, Kp = eng.build_host(jk.pack_factor(L), X, Y, m.sym, precision, packed=True)
    eng.sync_status()
    assert torch.equal(Jp, Jf) and torch.equal(Kp, Kf)
    ok = (lambda a, b: rel_err(a, b) < FP64_REL) if precision == "fp64" else (lambda a, b: abs_err(a, b) < SPLIT_ABS)
    assert ok(Jp.numpy(), Jo) and ok(Kp.numpy(), Ko)
    eng.close()
