"""Host-side checks of the Python binding (no GPU needed): shapes and
caller-supplied outputs are validated before any device work, since the C ABI
takes bare pointers and sizes."""
import numpy as np
import pytest
import torch

from paper_2608_06536_b300 import build as pkg_build
from paper_2608_06536_b300 import jk


@pytest.fixture(scope="module")
def eng():
    pkg_build.build()
    return jk.Engine("cuda:0")      # no device work until a call passes its checks


def _mol(n=6, naux=4, ks=(2, 3)):
    rng = np.random.default_rng(0)
    L = rng.standard_normal((naux, n, n))
    X = [rng.standard_normal((n, k)) for k in ks]
    Y = [rng.standard_normal((n, k)) for k in ks]
    return L, X, Y


def test_valid_shapes_pass():
    L, X, Y = _mol()
    assert jk._check_problem(L, X, Y, [False, True]) == (6, 4, 2)
    assert jk._check_problem(L, X, None, None) == (6, 4, 2)
    # a symmetric density's Y is not used, so its shape is not checked
    assert jk._check_problem(L, X, [Y[0], np.zeros(3)], [False, True]) == (6, 4, 2)


@pytest.mark.parametrize("case", ["L2d", "Lrect", "Lempty", "Xrows", "X1d", "Xk0", "Yshape", "nosym", "noY",
                                  "none"])
def test_bad_shapes_rejected_before_device_work(eng, case):
    L, X, Y = _mol()
    sym = [False, False]
    if case == "L2d":
        L = L[0]
    elif case == "Lrect":
        L = L[:, :, :5]
    elif case == "Lempty":
        L = L[:0]
    elif case == "Xrows":
        X[1] = X[1][:5]
    elif case == "X1d":
        X[0] = X[0][:, 0]
    elif case == "Xk0":
        X[0], Y[0] = X[0][:, :0], Y[0][:, :0]
    elif case == "Yshape":
        Y[1] = Y[1][:, :2]
    elif case == "nosym":
        sym = [False]
    elif case == "noY":
        Y = Y[:1]
    elif case == "none":
        X, Y, sym = [], [], []
    for call in (lambda: eng.build(L, X, Y, sym, "split"),
                 lambda: eng.build_host(L, X, Y, sym, "split"),
                 lambda: eng.adjoint(L, X, Y, sym, precision="split"),
                 lambda: eng.autotune(L, X, Y, sym, "split"),
                 lambda: eng.build_batched([(L, X, Y, sym)], "split")):
        with pytest.raises(ValueError):
            call()


def test_outputs_checked(eng):
    L, X, Y = _mol()
    sym = [False, False]
    good = torch.empty((2, 6, 6), dtype=torch.float64)
    jk._check_output(good, "J", (2, 6, 6), torch.device("cpu"))
    jk._check_output(None, "J", (2, 6, 6), torch.device("cpu"))
    bad = [torch.empty((2, 6, 6), dtype=torch.float32),          # dtype
           torch.empty((1, 6, 6), dtype=torch.float64),          # too few densities
           torch.empty((2, 6, 7), dtype=torch.float64)[:, :, :6]]  # not contiguous
    for t in bad:
        with pytest.raises(ValueError):
            jk._check_output(t, "J", (2, 6, 6), torch.device("cpu"))
        with pytest.raises(ValueError):
            eng.build_host(L, X, Y, sym, "split", J=t)
        with pytest.raises(ValueError):
            eng.build_host(L, X, Y, sym, "split", K=t)
    # a host tensor passed where the device build writes
    with pytest.raises(ValueError):
        eng.build(L, X, Y, sym, "split", J=good)


def test_adjoint_seed_sizes_checked(eng):
    L, X, Y = _mol()
    for W in (np.zeros((2, 6, 5)), np.zeros((1, 6, 6)), np.zeros((3, 6, 6))):
        with pytest.raises(ValueError):
            eng.adjoint(L, X, Y, [False, False], W=W, precision="split")
        with pytest.raises(ValueError):
            eng.adjoint(L, X, Y, [False, False], V=W, precision="split")


def test_batched_names_the_bad_molecule(eng):
    good = _mol()
    L, X, Y = _mol(n=7)
    X[0] = X[0][:6]
    with pytest.raises(ValueError, match="molecule 1"):
        eng.build_batched([(*good, None), (L, X, Y, None)], "split")
    with pytest.raises(ValueError):
        eng.build_batched([], "split")


@pytest.mark.parametrize("case", ["L2d", "Lrect", "Dshape", "Dnd0", "WVmismatch", "none"])
def test_dense_shapes_rejected_before_device_work(eng, case):
    rng = np.random.default_rng(1)
    n, naux = 6, 4
    L = rng.standard_normal((naux, n, n))
    D = rng.standard_normal((2, n, n))
    W, V = D, D
    if case == "L2d":
        L = L[0]
    elif case == "Lrect":
        L = L[:, :, :5]
    elif case == "Dshape":
        D = D[:, :, :5]
        W = V = D
    elif case == "Dnd0":
        D = D[:0]
        W = V = D
    elif case == "WVmismatch":
        V = D[:1]
    elif case == "none":
        D = W = V = None
    if case != "WVmismatch":
        with pytest.raises(ValueError):
            eng.build_dense(L, D, "split")
    with pytest.raises(ValueError):
        eng.density_grad(L, W, V, "split")


def test_dense_shape_helper():
    L = np.zeros((3, 5, 5))
    assert jk._check_dense(L, [("D", np.zeros((5, 5)))]) == (5, 3, 1)
    assert jk._check_dense(L, [("W", np.zeros((4, 5, 5))), ("V", None)]) == (5, 3, 4)
    assert jk._check_dense(L, [("W", None), ("V", np.zeros((2, 5, 5)))]) == (5, 3, 2)


def test_pairs_shapes_rejected_before_device_work(eng):
    L, X, Y = _mol()
    with pytest.raises(ValueError):
        eng.pairs(L, X, Y, None, None)                       # no right densities
    with pytest.raises(ValueError):
        eng.pairs(L, X, Y, None, [X[0][:5]], [Y[0][:5]])      # right rows != nbf
    with pytest.raises(ValueError):
        eng.pairs(L, [X[0][:, :0]], None, None, X, Y)         # zero-width left density
    with pytest.raises(ValueError):
        eng.pairs(L[0], X, Y, None, X, Y)                     # factor not [naux][nbf][nbf]


def test_laplace_shapes_rejected_before_device_work(eng):
    rng = np.random.default_rng(2)
    n, naux, m = 6, 4, 3
    L = rng.standard_normal((naux, n, n))
    C = rng.standard_normal((n, m))
    e = np.array([-1.0, -0.5, -0.2])
    bad = [dict(CX=C[:5]), dict(epsX=e[:2]), dict(CY=C), dict(CY=C[:, :2], epsY=e[:2]), dict(w=[1.0])]
    for kw in bad:
        args = dict(CX=C, epsX=e, sx=1, alpha=[0.5, 1.0])
        args.update(kw)
        with pytest.raises(ValueError):
            eng.build_laplace(L, **args)
    with pytest.raises(ValueError):
        eng.build_laplace(L[0], C, e, 1, [0.5])


class _RecordingLib:
    """The real library for host-only calls (the workspace query); compute
    entry points are recorded instead of called (no device here)."""
    COMPUTE = ("jk_build", "jk_adjoint", "jk_build_batched", "jk_build_dense", "jk_density_grad", "jk_pair",
               "jk_build_laplace", "jk_set_option", "jk_build_host", "jk_build_host_packed")

    def __init__(self, real):
        self.real, self.calls, self.queries = real, [], []

    def __getattr__(self, name):
        if name == "jk_workspace_query_handle":
            def query(h, op, nmol, f, ndm, nd, d, p, nb):
                st = self.real.jk_workspace_query(op, nmol, f, ndm, nd, d, p, nb)
                self.queries.append((op, nmol, nd, st, nb._obj.value))
                return st
            return query
        if name in self.COMPUTE:
            def record(*args):
                self.calls.append((name, args))
                return 0
            return record
        return getattr(self.real, name)


@pytest.fixture()
def rec():
    """An Engine on host tensors whose compute calls are recorded: the
    marshalling and the workspace query run for real."""
    import ctypes as ct
    import types
    pkg_build.build()
    e = object.__new__(jk.Engine)
    e.lib = _RecordingLib(jk.load_library())
    e.device = torch.device("cpu")
    e._ws, e._h, e._opts = None, ct.c_void_p(1), {}
    e.sized = []
    e._ensure = lambda nbytes: e.sized.append(nbytes)
    e.stream = types.SimpleNamespace(cuda_stream=0)
    yield e
    e._h = ct.c_void_p()      # the stand-in handle must never reach jk_destroy


def test_binding_queries_succeed_for_every_entry_point(rec):
    """Each binding method builds query arguments the library accepts and
    passes the compute entry point what its header declares."""
    rng = np.random.default_rng(3)
    n, naux = 8, 5
    L = rng.standard_normal((naux, n, n))
    X = [rng.standard_normal((n, k)) for k in (2, 3)]
    Y = [rng.standard_normal((n, k)) for k in (2, 3)]
    D = rng.standard_normal((2, n, n))
    st = rec.stream
    rec.build(L, X, Y, [False, True], "split", stream=st)
    rec.adjoint(L, X, Y, [False, False], D, D, precision="split", stream=st)
    rec.build_batched([(L, X, Y, None), (L[:, :6, :6], [x[:6] for x in X], None, [True, True])], "split",
                      stream=st)
    rec.build_dense(L, D, "split", stream=st)
    rec.density_grad(L, D, None, "split", stream=st)
    Jp, Kp = rec.pairs(L, X, Y, None, X[:1], Y[:1], None, "split", stream=st)
    assert Jp.shape == (2, 1) and Kp.shape == (2, 1)
    J, K = rec.build_laplace(L, X[0], np.array([-1.0, -0.5]), +1, [0.3, 1.2], [0.5, 2.0], Y[0],
                             np.array([0.4, 0.8]), -1, "split", stream=st)
    assert J.shape == (n, n) and K.shape == (n, n)
    J, K = rec.build_laplace(L, X[0], np.array([-1.0, -0.5]), +1, [0.3, 1.2, 2.0], stream=st)
    assert J.shape == (3, n, n)
    Jh, Kh = torch.empty((2, n, n), dtype=torch.float64), torch.empty((2, n, n), dtype=torch.float64)
    rec.build_host(L, X, Y, None, "split", J=Jh, K=Kh, stream=st, sync=False)
    rec.build_host(jk.pack_factor(L), X, Y, None, "split", J=Jh, K=Kh, stream=st, sync=False, packed=True)
    with pytest.raises(ValueError):
        rec.build_host(jk.pack_factor(L)[:, 1:], X, Y, None, "split", J=Jh, K=Kh, stream=st, packed=True)
    ops = [q[0] for q in rec.lib.queries]
    assert ops == [jk.JK_OP_BUILD, jk.JK_OP_ADJOINT, jk.JK_OP_BATCHED, jk.JK_OP_BUILD_DENSE,
                   jk.JK_OP_DENSITY_GRAD, jk.JK_OP_PAIR, jk.JK_OP_LAPLACE, jk.JK_OP_LAPLACE,
                   jk.JK_OP_BUILD_HOST, jk.JK_OP_BUILD_HOST_PACKED]
    assert all(q[3] == jk.JK_OK and q[4] > 0 for q in rec.lib.queries), rec.lib.queries
    assert rec.sized == [q[4] for q in rec.lib.queries]
    names = [c[0] for c in rec.lib.calls]
    assert names == ["jk_build", "jk_adjoint", "jk_build_batched", "jk_build_dense", "jk_density_grad", "jk_pair",
                     "jk_build_laplace", "jk_build_laplace", "jk_build_host", "jk_build_host_packed"]
    pair_args = rec.lib.calls[5][1]
    assert pair_args[2] == 2 and pair_args[4] == 1          # nl, nr
    lap_args = rec.lib.calls[6][1]
    assert lap_args[2] == 2 and lap_args[5] == 2 and lap_args[4] is not None   # nq, m, weights


def test_pack_factor_layout():
    rng = np.random.default_rng(4)
    L = rng.standard_normal((3, 6, 6))
    L = L + L.transpose(0, 2, 1)
    P = jk.pack_factor(L).numpy()
    assert P.shape == (3, 21)
    for p in range(3):
        t = 0
        for mu in range(6):
            for nu in range(mu, 6):
                assert P[p, t] == L[p, mu, nu]
                t += 1


def test_module_level_functions_dispatch_to_the_engine(rec, monkeypatch):
    """jk_build_dense, jk_density_grad, jk_pair and jk_build_laplace pass their
    arguments to the default engine's methods."""
    monkeypatch.setattr(jk, "default_engine", lambda device=None: rec)
    rng = np.random.default_rng(5)
    n, naux = 6, 4
    L = rng.standard_normal((naux, n, n))
    D = rng.standard_normal((2, n, n))
    X = [rng.standard_normal((n, 2))]
    st = rec.stream
    J, K = jk.jk_build_dense(L, D, "split", stream=st)
    assert J.shape == (2, n, n) and K.shape == (2, n, n)
    assert jk.jk_density_grad(L, D, None, "split", stream=st).shape == (2, n, n)
    Jp, Kp = jk.jk_pair(L, X, X, None, X, X, None, "split", stream=st)
    assert Jp.shape == (1, 1)
    J, K = jk.jk_build_laplace(L, X[0], np.array([-1.0, -0.5]), +1, [0.5], stream=st)
    assert J.shape == (1, n, n)
    assert [c[0] for c in rec.lib.calls] == ["jk_build_dense", "jk_density_grad", "jk_pair", "jk_build_laplace"]


def test_packed_factor_through_the_binding(rec):
    """With the packed_factor option the binding takes pack_factor(L)
    ([naux][n(n+1)/2]) for the ordinary builds, derives nbf from the
    densities (or CX), passes the library the factor's true nbf and naux, and
    rejects a dense or mis-sized factor before any device work."""
    rng = np.random.default_rng(6)
    n, naux = 8, 5
    L = rng.standard_normal((naux, n, n))
    L = L + L.transpose(0, 2, 1)
    P = jk.pack_factor(L)
    X = [rng.standard_normal((n, k)) for k in (2, 3)]
    Y = [rng.standard_normal((n, k)) for k in (2, 3)]
    st = rec.stream
    rec.set_option("packed_factor", 1)
    rec.build(P, X, Y, [False, True], "split", stream=st)
    rec.build_batched([(P, X, Y, None), (jk.pack_factor(L[:, :6, :6]), [x[:6] for x in X], None, [True, True])],
                      "split", stream=st)
    rec.pairs(P, X, Y, None, X[:1], Y[:1], None, "split", stream=st)
    J, K = rec.build_laplace(P, X[0], np.array([-1.0, -0.5]), +1, [0.3, 1.2], stream=st)
    assert J.shape == (2, n, n)
    for bad in (L, P[:, 1:], P[0]):
        with pytest.raises(ValueError):
            rec.build(bad, X, Y, None, "split")
        with pytest.raises(ValueError):
            rec.build_laplace(bad, X[0], np.array([-1.0, -0.5]), +1, [0.3])
    calls = [c for c in rec.lib.calls if c[0] != "jk_set_option"]
    assert [c[0] for c in calls] == ["jk_build", "jk_build_batched", "jk_pair", "jk_build_laplace"]
    f = calls[0][1][1]._obj
    assert (f.nbf, f.naux) == (n, naux)
    fac = calls[1][1][2]
    assert [(fac[m].nbf, fac[m].naux) for m in range(2)] == [(n, naux), (6, naux)]
    assert calls[3][1][1]._obj.nbf == n
    opt = [c for c in rec.lib.calls if c[0] == "jk_set_option"]
    assert opt and opt[0][1][1:] == (jk.OPTIONS["packed_factor"], 1)


def test_packed_factor_gradient_fold():
    """The packed factor's gradient is the dense one pulled back through the
    unpacking map p -> L (L_ij = L_ji = p_k): autograd through an explicit
    unpacking of random packed entries gives the fold, diagonal entries once."""
    from paper_2608_06536_b300.autograd import fold_packed_grad
    rng = np.random.default_rng(3)
    naux, n = 3, 7
    G = torch.tensor(rng.standard_normal((naux, n, n)))
    p = torch.tensor(rng.standard_normal((naux, n * (n + 1) // 2)), requires_grad=True)
    pos = {}
    k = 0
    for i in range(n):
        for j in range(i, n):
            pos[i, j] = pos[j, i] = k
            k += 1
    idx = torch.tensor([[pos[i, j] for j in range(n)] for i in range(n)])
    L = p[:, idx.reshape(-1)].reshape(naux, n, n)
    assert torch.equal(L, L.transpose(1, 2))
    (gp,) = torch.autograd.grad((G * L).sum(), [p])
    assert torch.equal(fold_packed_grad(G), gp)
    # by hand for one off-diagonal and one diagonal entry of aux index 1
    assert fold_packed_grad(G)[1, pos[2, 5]] == G[1, 2, 5] + G[1, 5, 2]
    assert fold_packed_grad(G)[1, pos[4, 4]] == G[1, 4, 4]
