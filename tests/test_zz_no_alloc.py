"""The arena-free FP64 build (jk_build_noalloc) against jk_build.

jk_build_noalloc is for callers that cannot allocate device memory (inside a
stream capture, or under a host application that owns the memory budget); it
keeps its workspace in a static device array.  This file is collected last so
that a run stopping at the first failure has already run every other test.
"""
import ctypes as ct

import numpy as np
import pytest
import torch

from paper_2608_06536_b300 import inputs
from tests._util import FP64_REL, rel_err, to_np

pytestmark = pytest.mark.gpu


def _lib():
    from paper_2608_06536_b300 import jk
    lib = jk.load_library()
    lib.jk_build_noalloc.argtypes = [ct.POINTER(jk.jk_factor), ct.c_int32, ct.POINTER(jk.jk_density),
                                     ct.c_void_p, ct.c_void_p, ct.c_void_p]
    lib.jk_build_noalloc.restype = ct.c_int
    return jk, lib


def _args(jk, m):
    L = torch.from_numpy(m.L).cuda()
    X = [torch.from_numpy(x).cuda() for x in m.X]
    Y = [torch.from_numpy(y).cuda() for y in m.Y]
    f = jk.jk_factor(m.n, m.naux, L.data_ptr())
    d = (jk.jk_density * m.nd)()
    for s in range(m.nd):
        d[s].k, d[s].symmetric = m.ks[s], int(m.sym[s])
        d[s].X, d[s].Y = X[s].data_ptr(), Y[s].data_ptr()
    return (L, X, Y), f, d


def _noalloc(lib, f, d, nd, n):
    J = torch.full((nd, n, n), float("nan"), dtype=torch.float64, device="cuda")
    K = torch.full((nd, n, n), float("nan"), dtype=torch.float64, device="cuda")
    st = lib.jk_build_noalloc(ct.byref(f), nd, d, J.data_ptr(), K.data_ptr(),
                              ct.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st, J, K


def test_noalloc_matches_build_twice():
    jk, lib = _lib()
    eng = jk.Engine("cuda:0")
    for i, (n, naux, ks, sym) in enumerate([(48, 300, [6], [False]), (37, 53, [5, 1, 13], [False, True, False])]):
        m = inputs.custom(n, naux, max(naux / 5, 1.0), ks, sym, seed=i)
        keep, f, d = _args(jk, m)
        st, J, K = _noalloc(lib, f, d, m.nd, n)
        assert st == jk.JK_OK
        L, X, Y = keep
        Jr, Kr = eng.build(L, X, Y, m.sym, "fp64")
        assert rel_err(to_np(J), to_np(Jr)) < FP64_REL
        assert rel_err(to_np(K), to_np(Kr)) < FP64_REL


def test_noalloc_rejects_oversize_problem():
    jk, lib = _lib()
    m = inputs.custom(160, 400, 50.0, [40, 40], [False, False], seed=3)   # panel buffer ~41 MB
    keep, f, d = _args(jk, m)
    st, J, K = _noalloc(lib, f, d, m.nd, m.n)
    assert st == jk.JK_ERR_OOM
    assert bool(torch.isnan(J).all())
