"""Failure detection without a GPU fault: every wait in the engine's kernels is
bounded; a wait that runs out raises JK_ERR_TIMEOUT in the handle's device
status word, which jk_sync_status reports and clears, and the CUDA context
stays usable for the next build."""
import ctypes as ct
import time

import pytest
import torch

import oracle
from paper_2608_06536_b300 import inputs
from tests._util import SPLIT_ABS, abs_err, to_np

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives():
    from paper_2608_06536_b300 import jk
    eng = jk.Engine("cuda:0", workspace_bytes=1 << 20)
    lib = eng.lib
    lib.jk_debug_wait_timeout.argtypes = [ct.c_void_p, ct.c_void_p]
    lib.jk_debug_wait_timeout.restype = ct.c_int
    t0 = time.time()
    assert lib.jk_debug_wait_timeout(eng._h, None) == jk.JK_OK
    with pytest.raises(jk.JKError) as e:
        eng.sync_status()
    assert e.value.status == jk.JK_ERR_TIMEOUT
    assert time.time() - t0 < 60
    eng.sync_status()                     # cleared
    m = inputs.custom(40, 60, 12.0, [5, 4], [False, True], seed=2)
    Jo, Ko = oracle.build(m.L, m.X, m.Y)
    J, K = eng.build(torch.from_numpy(m.L).cuda(), [torch.from_numpy(x).cuda() for x in m.X],
                     [torch.from_numpy(y).cuda() for y in m.Y], m.sym, "split")
    eng.sync_status()
    assert abs_err(to_np(J), Jo) < SPLIT_ABS and abs_err(to_np(K), Ko) < SPLIT_ABS
