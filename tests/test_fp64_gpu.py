"""Parity of the plain FP64 GPU engine against the CPU oracle (through the C ABI)."""
import ctypes as ct

import numpy as np
import pytest
import torch

import oracle
from paper_2608_06536_b300 import inputs
from tests._util import FP64_REL, rel_err, to_np

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


@pytest.mark.parametrize("n,naux,ks,sym", [
    (1, 1, [1], [False]),
    (7, 5, [3], [False]),
    (37, 53, [5, 1, 13], [False, True, False]),
    (65, 130, [16, 17], [True, False]),
    (130, 70, [64, 3, 9], [False, False, True]),
])
def test_build_ragged_vs_oracle(eng, n, naux, ks, sym):
    m = inputs.custom(n, naux, max(naux / 4, 1.0), ks, sym)
    Jo, Ko = oracle.build(m.L, m.X, m.Y)
    L, X, Y = _gpu(m)
    J, K = eng.build(L, X, Y, sym, "fp64")
    torch.cuda.synchronize()
    for s in range(len(ks)):
        assert rel_err(to_np(J[s]), Jo[s]) < FP64_REL
        assert rel_err(to_np(K[s]), Ko[s]) < FP64_REL


def test_build_one_molecule_small(eng):
    m = inputs.one_molecule_small()
    Jo, Ko = oracle.build(m.L, m.X, m.Y)
    L, X, Y = _gpu(m)
    J, K = eng.build(L, X, Y, m.sym, "fp64")
    assert rel_err(to_np(J), Jo) < FP64_REL
    assert rel_err(to_np(K), Ko) < FP64_REL


def test_build_multi_state_sampled(eng):
    """The 400/2400/8-density workload, full size, on sampled entries."""
    m = inputs.multi_state()
    L, X, Y = _gpu(m)
    J, K = eng.build(L, X, Y, m.sym, "fp64")
    rng = np.random.default_rng(0)
    ns = 96
    s = rng.integers(0, m.nd, ns); mu = rng.integers(0, m.n, ns); nu = rng.integers(0, m.n, ns)
    s[:2] = [0, 7]; mu[:2] = [0, m.n - 1]; nu[:2] = [m.n - 1, 0]
    Jo, Ko = oracle.sample(m.L, m.X, m.Y, s, mu, nu)
    Jg, Kg = to_np(J)[s, mu, nu], to_np(K)[s, mu, nu]
    scaleJ, scaleK = np.abs(to_np(J)).max(), np.abs(to_np(K)).max()
    assert np.abs(Jg - Jo).max() / scaleJ < FP64_REL
    assert np.abs(Kg - Ko).max() / scaleK < FP64_REL
    # properties at full size: J symmetric, K of the symmetric density symmetric
    Jn, Kn = to_np(J), to_np(K)
    assert rel_err(Jn, Jn.transpose(0, 2, 1)) < 1e-13
    assert rel_err(Kn[0], Kn[0].T) < 1e-13


def test_j_only_and_k_only(eng):
    m = inputs.custom(50, 40, 10.0, [4, 6], [False, True])
    L, X, Y = _gpu(m)
    J, K = eng.build(L, X, Y, m.sym, "fp64")
    J1, K1 = eng.build(L, X, Y, m.sym, "fp64", want_k=False)
    J2, K2 = eng.build(L, X, Y, m.sym, "fp64", want_j=False)
    assert K1 is None and J2 is None
    assert rel_err(to_np(J1), to_np(J)) < 1e-14
    assert torch.equal(K2, K)


def test_bitwise_deterministic(eng):
    m = inputs.custom(96, 200, 50.0, [8, 8], [False, False])
    L, X, Y = _gpu(m)
    J1, K1 = eng.build(L, X, Y, m.sym, "fp64")
    J2, K2 = eng.build(L, X, Y, m.sym, "fp64")
    assert torch.equal(J1, J2) and torch.equal(K1, K2)


def test_batched_matches_single(eng):
    mols = [inputs.custom(n, na, 8.0, ks, seed=i) for i, (n, na, ks) in
            enumerate([(20, 30, [2, 3]), (33, 17, [5]), (64, 80, [1, 7, 4])])]
    args = []
    for m in mols:
        L, X, Y = _gpu(m)
        args.append((L, X, Y, m.sym))
    outs = eng.build_batched(args, "fp64")
    for (L, X, Y, sym), (Jb, Kb) in zip(args, outs):
        J, K = eng.build(L, X, Y, sym, "fp64")
        assert torch.equal(J, Jb) and torch.equal(K, Kb)


@pytest.mark.parametrize("n,naux,ks,sym", [
    (9, 6, [2, 3], [False, False]),
    (33, 41, [4, 5], [True, False]),
])
def test_adjoint_vs_oracle(eng, n, naux, ks, sym):
    m = inputs.custom(n, naux, 7.0, ks, sym)
    rng = np.random.default_rng(3)
    W = [rng.standard_normal((n, n)) for _ in ks]
    V = [rng.standard_normal((n, n)) for _ in ks]
    dXo, dYo, dLo = oracle.adjoint(m.L, m.X, m.Y, W, V)
    L, X, Y = _gpu(m)
    dX, dY, dL = eng.adjoint(L, X, Y, m.sym, torch.tensor(np.array(W)).cuda(),
                             torch.tensor(np.array(V)).cuda(), precision="fp64")
    assert rel_err(to_np(dL), dLo) < FP64_REL
    for s in range(len(ks)):
        if sym[s]:
            # D = X X^T: both slots fold into dX; the oracle gives them apart
            assert rel_err(to_np(dX[s]), dXo[s] + dYo[s]) < FP64_REL
            assert np.all(to_np(dY[s]) == 0)
        else:
            assert rel_err(to_np(dX[s]), dXo[s]) < FP64_REL
            assert rel_err(to_np(dY[s]), dYo[s]) < FP64_REL


def test_adjoint_partial_seeds(eng):
    m = inputs.custom(21, 13, 5.0, [3], [False])
    rng = np.random.default_rng(4)
    W = [rng.standard_normal((21, 21))]
    L, X, Y = _gpu(m)
    Wt = torch.tensor(np.array(W)).cuda()
    dXo, dYo, dLo = oracle.adjoint(m.L, m.X, m.Y, W, None)
    dX, dY, dL = eng.adjoint(L, X, Y, m.sym, Wt, None, precision="fp64")
    assert rel_err(to_np(dX[0]), dXo[0]) < FP64_REL and rel_err(to_np(dL), dLo) < FP64_REL
    dXo, dYo, dLo = oracle.adjoint(m.L, m.X, m.Y, None, W)
    dX, dY, dL = eng.adjoint(L, X, Y, m.sym, None, Wt, want_dl=True, precision="fp64")
    assert rel_err(to_np(dY[0]), dYo[0]) < FP64_REL and rel_err(to_np(dL), dLo) < FP64_REL


def test_adjoint_central_fd_on_gpu(eng):
    """Central differences (h = 1e-5) of E computed by the GPU forward, on 32
    random directions, against the GPU adjoint."""
    n, naux, ks = 40, 60, [5, 6]
    m = inputs.custom(n, naux, 15.0, ks, [False, False])
    rng = np.random.default_rng(5)
    L, X, Y = _gpu(m)
    W = torch.tensor(rng.standard_normal((2, n, n))).cuda()
    V = torch.tensor(rng.standard_normal((2, n, n))).cuda()
    dX, dY, dL = eng.adjoint(L, X, Y, m.sym, W, V, precision="fp64")

    def E(Lp, Xp, Yp):
        J, K = eng.build(Lp, Xp, Yp, m.sym, "fp64")
        return float((W * K).sum() + (V * J).sum())

    h = 1e-5
    for _ in range(32):
        hX = [torch.tensor(rng.standard_normal(x.shape)).cuda() for x in X]
        hY = [torch.tensor(rng.standard_normal(y.shape)).cuda() for y in Y]
        H = torch.tensor(rng.standard_normal((naux, n, n))).cuda()
        H = H + H.transpose(1, 2)
        fp = E(L + h * H, [x + h * a for x, a in zip(X, hX)], [y + h * b for y, b in zip(Y, hY)])
        fm = E(L - h * H, [x - h * a for x, a in zip(X, hX)], [y - h * b for y, b in zip(Y, hY)])
        fd = (fp - fm) / (2 * h)
        an = float(sum((a * b).sum() for a, b in zip(dX, hX)) + sum((a * b).sum() for a, b in zip(dY, hY))
                   + (dL * H).sum())
        assert abs(fd - an) < 1e-6 * max(abs(an), 1.0)


def test_autograd_wrapper(eng):
    from paper_2608_06536_b300.autograd import jk as jk_fn
    n, naux = 12, 9
    m = inputs.custom(n, naux, 4.0, [2, 3], [False, True])
    L = torch.tensor(m.L, device="cuda", requires_grad=True)
    X = [torch.tensor(x, device="cuda", requires_grad=True) for x in m.X]
    Y = [torch.tensor(m.Y[0], device="cuda", requires_grad=True), None]
    J, K = jk_fn(L, X, Y, precision="fp64", engine=eng)
    rng = np.random.default_rng(6)
    W = torch.tensor(rng.standard_normal((2, n, n)), device="cuda")
    V = torch.tensor(rng.standard_normal((2, n, n)), device="cuda")
    E = (W * K).sum() + (V * J).sum()
    gL, gX0, gX1, gY0 = torch.autograd.grad(E, [L, X[0], X[1], Y[0]])
    dXo, dYo, dLo = oracle.adjoint(m.L, m.X, m.Y, list(to_np(W)), list(to_np(V)))
    assert rel_err(to_np(gL), dLo) < FP64_REL
    assert rel_err(to_np(gX0), dXo[0]) < FP64_REL
    assert rel_err(to_np(gY0), dYo[0]) < FP64_REL
    assert rel_err(to_np(gX1), dXo[1] + dYo[1]) < FP64_REL


def test_errors_are_reported_before_launch(eng):
    from paper_2608_06536_b300 import jk
    lib = jk.load_library()
    ws = torch.empty(4096, dtype=torch.uint8, device="cuda")
    h = ct.c_void_p()
    assert lib.jk_create(ct.byref(h), ct.c_void_p(ws.data_ptr()), 4096) == jk.JK_OK
    m = inputs.custom(30, 20, 5.0, [3])
    L, X, Y = _gpu(m)
    J = torch.full((1, 30, 30), 7.0, dtype=torch.float64, device="cuda")
    f = jk.jk_factor(30, 20, L.data_ptr())
    d = (jk.jk_density * 1)()
    d[0].k, d[0].symmetric, d[0].X, d[0].Y = 3, 0, X[0].data_ptr(), Y[0].data_ptr()
    # arena too small -> OOM, outputs untouched
    st = lib.jk_build(h, ct.byref(f), 1, d, ct.c_void_p(J.data_ptr()), None, jk.JK_FP64, None)
    assert st == jk.JK_ERR_OOM and b"arena" in lib.jk_last_error(h)
    # output not aligned to a double; input not aligned to 16 bytes
    st = lib.jk_build(h, ct.byref(f), 1, d, ct.c_void_p(J.data_ptr() + 4), None, jk.JK_FP64, None)
    assert st == jk.JK_ERR_ARG and b"aligned" in lib.jk_last_error(h)
    f8 = jk.jk_factor(30, 20, L.data_ptr() + 8)
    st = lib.jk_build(h, ct.byref(f8), 1, d, ct.c_void_p(J.data_ptr()), None, jk.JK_FP64, None)
    assert st == jk.JK_ERR_ARG and b"aligned" in lib.jk_last_error(h)
    # host pointer as factor
    hostL = np.zeros(30 * 30 * 20)
    f2 = jk.jk_factor(30, 20, hostL.ctypes.data)
    st = lib.jk_build(h, ct.byref(f2), 1, d, ct.c_void_p(J.data_ptr()), None, jk.JK_FP64, None)
    assert st == jk.JK_ERR_ARG and b"device" in lib.jk_last_error(h)
    # zero-width density
    d[0].k = 0
    assert lib.jk_build(h, ct.byref(f), 1, d, ct.c_void_p(J.data_ptr()), None, jk.JK_FP64, None) == jk.JK_ERR_SHAPE
    # bad precision enum
    d[0].k = 3
    assert lib.jk_build(h, ct.byref(f), 1, d, ct.c_void_p(J.data_ptr()), None, 9, None) == jk.JK_ERR_ARG
    assert lib.jk_sync_status(h, None) == jk.JK_OK
    torch.cuda.synchronize()
    assert bool((J == 7.0).all())
    lib.jk_destroy(h)
