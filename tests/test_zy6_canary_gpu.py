"""Canary-guarded workspace and outputs on the GPU: every entry point runs in
an arena of exactly the queried size with pattern-filled guard regions on
both sides, and writes outputs that also sit between guards; afterwards
every guard byte must still hold the pattern (no device write strays outside
the memory a call is given)."""
import ctypes as ct

import pytest
import torch

from paper_2608_06536_b300 import inputs

pytestmark = pytest.mark.gpu

GUARD = 1 << 20
PATTERN = 0xA5
FP64, SPLIT = 0, 1


class Guarded:
    """`nbytes` usable device bytes at a 256-byte aligned offset inside a
    larger allocation whose remaining bytes hold PATTERN."""

    def __init__(self, nbytes):
        self.nbytes = int(nbytes)
        self.raw = torch.full((self.nbytes + 2 * GUARD,), PATTERN, dtype=torch.uint8, device="cuda")
        self.ptr = self.raw.data_ptr() + GUARD

    def intact(self):
        head = self.raw[:GUARD]
        tail = self.raw[GUARD + self.nbytes:]
        return bool((head == PATTERN).all()) and bool((tail == PATTERN).all())


@pytest.fixture(scope="module")
def lib():
    from paper_2608_06536_b300 import jk
    return jk.load_library()


def _mol(n, naux, ks, sym, seed=0):
    m = inputs.custom(n, naux, max(naux / 4, 1.0), ks, sym, seed=seed)
    L = torch.from_numpy(m.L).cuda()
    X = [torch.from_numpy(x).cuda() for x in m.X]
    Y = [torch.from_numpy(y).cuda() for y in m.Y]
    return m, L, X, Y


def _dens(jk, m, X, Y):
    d = (jk.jk_density * m.nd)()
    for s in range(m.nd):
        d[s].k, d[s].symmetric = m.ks[s], int(m.sym[s])
        d[s].X, d[s].Y = X[s].data_ptr(), None if m.sym[s] else Y[s].data_ptr()
    return d


def _run(lib, jk, op, f, d, nd, p, call, nmol=1, ndm=None):
    nb = ct.c_size_t()
    fa = f if isinstance(f, ct.Array) else (jk.jk_factor * 1)(f)
    ndm_c = (ct.c_int32 * len(ndm))(*ndm) if ndm else None
    assert lib.jk_workspace_query(op, nmol, fa, ndm_c, nd, d, p, ct.byref(nb)) == 0
    arena = Guarded(nb.value)
    h = ct.c_void_p()
    assert lib.jk_create(ct.byref(h), ct.c_void_p(arena.ptr), ct.c_size_t(arena.nbytes)) == 0
    try:
        st = call(h)
        assert st == 0, lib.jk_last_error(h)
        assert lib.jk_sync_status(h, None) == 0, lib.jk_last_error(h)
        torch.cuda.synchronize()
        assert arena.intact(), "a write landed outside the arena"
    finally:
        lib.jk_destroy(h)


@pytest.mark.parametrize("p", [FP64, SPLIT])
def test_build(lib, p):
    from paper_2608_06536_b300 import jk
    m, L, X, Y = _mol(37, 53, [5, 1, 13], [False, True, False])
    f, d = jk.jk_factor(m.n, m.naux, L.data_ptr()), _dens(jk, m, X, Y)
    J, K = Guarded(m.nd * m.n * m.n * 8), Guarded(m.nd * m.n * m.n * 8)
    _run(lib, jk, jk.JK_OP_BUILD, f, d, m.nd, p,
         lambda h: lib.jk_build(h, ct.byref(f), m.nd, d, ct.c_void_p(J.ptr), ct.c_void_p(K.ptr), p, None))
    assert J.intact() and K.intact()


def test_batched_and_adjoint(lib):
    from paper_2608_06536_b300 import jk
    m1, L1, X1, Y1 = _mol(60, 150, [6, 6], [False, False], seed=1)
    m2, L2, X2, Y2 = _mol(33, 99, [3], [False], seed=2)
    fa = (jk.jk_factor * 2)(jk.jk_factor(m1.n, m1.naux, L1.data_ptr()), jk.jk_factor(m2.n, m2.naux, L2.data_ptr()))
    da = (jk.jk_density * 3)(*_dens(jk, m1, X1, Y1), *_dens(jk, m2, X2, Y2))
    outs = [Guarded(60 * 60 * 8), Guarded(60 * 60 * 8), Guarded(33 * 33 * 8)]
    outk = [Guarded(60 * 60 * 8), Guarded(60 * 60 * 8), Guarded(33 * 33 * 8)]
    Jp = (ct.c_void_p * 3)(*[o.ptr for o in outs])
    Kp = (ct.c_void_p * 3)(*[o.ptr for o in outk])
    ndm = (ct.c_int32 * 2)(2, 1)
    _run(lib, jk, jk.JK_OP_BATCHED, fa, da, 3, SPLIT,
         lambda h: lib.jk_build_batched(h, 2, fa, ndm, da, Jp, Kp, SPLIT, None), nmol=2, ndm=[2, 1])
    assert all(o.intact() for o in outs + outk)
    # adjoint with dL
    m, L, X, Y = m1, L1, X1, Y1
    f, d = jk.jk_factor(m.n, m.naux, L.data_ptr()), _dens(jk, m, X, Y)
    W = torch.randn(2, 60, 60, dtype=torch.float64, device="cuda")
    tot = 60 * 12
    dX, dY, dL = Guarded(tot * 8), Guarded(tot * 8), Guarded(150 * 60 * 60 * 8)
    _run(lib, jk, jk.JK_OP_ADJOINT, f, d, 2, SPLIT,
         lambda h: lib.jk_adjoint(h, ct.byref(f), 2, d, ct.c_void_p(W.data_ptr()), ct.c_void_p(W.data_ptr()),
                                  ct.c_void_p(dX.ptr), ct.c_void_p(dY.ptr), ct.c_void_p(dL.ptr), SPLIT, None))
    assert dX.intact() and dY.intact() and dL.intact()


def test_dense_pairs_laplace(lib):
    from paper_2608_06536_b300 import jk
    m, L, X, Y = _mol(37, 53, [5, 3], [False, False])
    f = jk.jk_factor(m.n, m.naux, L.data_ptr())
    n, nd = m.n, 2
    D = torch.from_numpy(inputs.dense_densities(n, nd, seed=3)).cuda()
    O1, O2 = Guarded(nd * n * n * 8), Guarded(nd * n * n * 8)
    _run(lib, jk, jk.JK_OP_BUILD_DENSE, f, None, nd, SPLIT,
         lambda h: lib.jk_build_dense(h, ct.byref(f), nd, ct.c_void_p(D.data_ptr()), ct.c_void_p(O1.ptr),
                                      ct.c_void_p(O2.ptr), SPLIT, None))
    _run(lib, jk, jk.JK_OP_DENSITY_GRAD, f, None, nd, SPLIT,
         lambda h: lib.jk_density_grad(h, ct.byref(f), nd, ct.c_void_p(D.data_ptr()), ct.c_void_p(D.data_ptr()),
                                       ct.c_void_p(O1.ptr), SPLIT, None))
    assert O1.intact() and O2.intact()
    d = _dens(jk, m, X, Y)
    both = (jk.jk_density * 4)(*d, *d)
    Jp, Kp = Guarded(4 * 8), Guarded(4 * 8)
    _run(lib, jk, jk.JK_OP_PAIR, (jk.jk_factor * 2)(f, f), both, 4, SPLIT,
         lambda h: lib.jk_pair(h, ct.byref(f), 2, d, 2, d, ct.c_void_p(Jp.ptr), ct.c_void_p(Kp.ptr), SPLIT, None),
         nmol=2, ndm=[2, 2])
    assert Jp.intact() and Kp.intact()
    lp = (jk.jk_density * 1)()
    lp[0].k, lp[0].symmetric = 5, 0
    ei = torch.tensor([-1.0, -0.8, -0.6, -0.4, -0.3], dtype=torch.float64, device="cuda")
    ea = -ei
    alpha = (ct.c_double * 3)(0.3, 1.0, 2.5)
    w = (ct.c_double * 3)(0.5, 0.3, 0.2)
    JL, KL = Guarded(n * n * 8), Guarded(n * n * 8)
    _run(lib, jk, jk.JK_OP_LAPLACE, f, lp, 3, SPLIT,
         lambda h: lib.jk_build_laplace(h, ct.byref(f), 3, alpha, w, 5, ct.c_void_p(X[0].data_ptr()),
                                        ct.c_void_p(ei.data_ptr()), 1, ct.c_void_p(Y[0].data_ptr()),
                                        ct.c_void_p(ea.data_ptr()), -1, ct.c_void_p(JL.ptr),
                                        ct.c_void_p(KL.ptr), SPLIT, None))
    assert JL.intact() and KL.intact()
