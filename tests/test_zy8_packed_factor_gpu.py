"""A packed device factor (JK_OPT_PACKED_FACTOR = 1) on the GPU: the factor
lives on the device as packed upper triangles ([naux][n(n+1)/2], half the
memory); each aux chunk is expanded in the workspace before its products and
the FP64 J back-contraction reads the packed form.  With the same aux chunk the
results must equal the dense factor's bit for bit (the expansion is exact and
everything downstream is unchanged), and match the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2608_06536_b300 import inputs, jk
from tests._util import FP64_REL, SPLIT_ABS, abs_err, rel_err, to_np

pytestmark = pytest.mark.gpu


def _both(m, precision, opts, want_k=True):
    L = torch.from_numpy(m.L).cuda()
    P = jk.pack_factor(m.L).cuda()
    X = [torch.from_numpy(x).cuda() for x in m.X]
    Y = [torch.from_numpy(y).cuda() for y in m.Y]
    out = []
    for packed, fac in ((0, L), (1, P)):
        eng = jk.Engine("cuda:0")
        for k, v in opts.items():
            eng.set_option(k, v)
        eng.set_option("packed_factor", packed)
        J, K = eng.build(fac, X, Y, m.sym, precision, want_k=want_k)
        eng.sync_status()
        out.append((to_np(J), None if K is None else to_np(K)))
        eng.close()
    return out


@pytest.mark.parametrize("precision,n,naux,ks,sym,opts", [
    ("split", 130, 70, [9, 3, 20], [False, True, False], {"aux_chunk": 30, "schedule": 0}),
    ("split", 257, 90, [64, 5], [True, False], {"aux_chunk": 40, "schedule": 1, "syrk": 1}),
    ("split", 400, 600, [40] * 4, [True, False, False, False], {"aux_chunk": 600, "schedule": 1}),
    ("fp64", 37, 53, [5, 1, 13], [False, True, False], {"aux_chunk": 17}),
])
def test_packed_factor_equals_dense(precision, n, naux, ks, sym, opts):
    m = inputs.custom(n, naux, max(naux / 4, 1.0), ks, sym)
    (Jd, Kd), (Jp, Kp) = _both(m, precision, opts)
    np.testing.assert_array_equal(Jp, Jd)
    np.testing.assert_array_equal(Kp, Kd)
    Jo, Ko = oracle.build(m.L, m.X, m.Y)
    if precision == "split":
        assert abs_err(Jp, Jo) < SPLIT_ABS and abs_err(Kp, Ko) < SPLIT_ABS
    else:
        assert rel_err(Jp, Jo) < FP64_REL and rel_err(Kp, Ko) < FP64_REL


@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_packed_factor_j_only(precision):
    m = inputs.custom(37, 53, 13.0, [5, 13], [False, True])
    (Jd, _), (Jp, _) = _both(m, precision, {"aux_chunk": 17}, want_k=False)
    np.testing.assert_array_equal(Jp, Jd)
    Jo, _ = oracle.build(m.L, m.X, m.Y)
    if precision == "split":
        assert abs_err(Jp, Jo) < SPLIT_ABS
    else:
        assert rel_err(Jp, Jo) < FP64_REL


def test_packed_factor_batched():
    shapes = [(60, 150, [6, 6]), (140, 222, [11]), (33, 99, [3, 3, 3])]
    mols = [inputs.custom(n, naux, max(naux / 4, 1.0), ks, [s % 2 == 0 for s in range(len(ks))], seed=i)
            for i, (n, naux, ks) in enumerate(shapes)]
    outs = []
    for packed in (0, 1):
        eng = jk.Engine("cuda:0")
        eng.set_option("aux_chunk", 50)
        eng.set_option("packed_factor", packed)
        args = []
        for m in mols:
            fac = jk.pack_factor(m.L) if packed else torch.from_numpy(m.L)
            args.append((fac.cuda(), [torch.from_numpy(x).cuda() for x in m.X],
                         [torch.from_numpy(y).cuda() for y in m.Y], m.sym))
        res = eng.build_batched(args, "split")
        eng.sync_status()
        outs.append([(to_np(J), to_np(K)) for J, K in res])
        eng.close()
    for (Jd, Kd), (Jp, Kp), m in zip(outs[0], outs[1], mols):
        np.testing.assert_array_equal(Jp, Jd)
        np.testing.assert_array_equal(Kp, Kd)
        Jo, Ko = oracle.build(m.L, m.X, m.Y)
        assert abs_err(Jp, Jo) < SPLIT_ABS and abs_err(Kp, Ko) < SPLIT_ABS


def test_only_the_host_builds_refuse_a_packed_factor():
    """Every device-factor call takes the packed factor; the host builds,
    whose factor lives in host memory, refuse the option before any device
    work (JK_ERR_UNSUPPORTED).  A dense-shaped L under the option is a shape
    error the binding reports before the library is reached."""
    m = inputs.custom(20, 30, 8.0, [3], [False])
    eng = jk.Engine("cuda:0")
    eng.set_option("packed_factor", 1)
    P = jk.pack_factor(m.L)
    Xh = [torch.from_numpy(x) for x in m.X]
    Yh = [torch.from_numpy(y) for y in m.Y]
    for packed_link, fac in ((False, torch.from_numpy(m.L)), (True, P)):
        with pytest.raises(jk.JKError) as e:
            eng.build_host(fac, Xh, Yh, m.sym, "split", packed=packed_link)
        assert e.value.status == jk.JK_ERR_UNSUPPORTED
    L = torch.from_numpy(m.L).cuda()
    W = torch.zeros((1, 20, 20), dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        eng.build_dense(L, W, "split")
    with pytest.raises(ValueError):
        eng.build(L, [x.cuda() for x in Xh], [y.cuda() for y in Yh], m.sym, "split")
    # the device calls run on the packed factor
    J, K = eng.build_dense(P.cuda(), W, "split")
    eng.sync_status()
    assert float(torch.abs(J).max()) == 0.0 and float(torch.abs(K).max()) == 0.0
    eng.close()


def test_pack_factor_on_the_device():
    """jk_pack_factor writes exactly the host packing, and builds run on it."""
    m = inputs.custom(70, 45, 12.0, [5, 3], [False, True])
    L = torch.from_numpy(m.L).cuda()
    eng = jk.Engine("cuda:0")
    P = eng.pack_factor(L)
    eng.sync_status()
    np.testing.assert_array_equal(to_np(P), jk.pack_factor(m.L).numpy())
    np.testing.assert_array_equal(to_np(jk.pack_factor(L)), to_np(P))      # module-level, device input
    eng.set_option("packed_factor", 1)
    J, K = eng.build(P, [torch.from_numpy(x).cuda() for x in m.X], [torch.from_numpy(y).cuda() for y in m.Y],
                     m.sym, "split")
    eng.sync_status()
    Jo, Ko = oracle.build(m.L, m.X, m.Y)
    assert abs_err(to_np(J), Jo) < SPLIT_ABS and abs_err(to_np(K), Ko) < SPLIT_ABS
    eng.close()


@pytest.mark.parametrize("precision", ["split", "fp64"])
def test_packed_factor_dense_and_gradient(precision):
    """jk_build_dense and jk_density_grad on a packed factor: K equals the
    dense factor's bit for bit at the same chunk (the chunks are expanded);
    J's metric dots are summed over the packed triangles, so J agrees to
    rounding; both match the oracle."""
    m = inputs.custom(70, 45, 12.0, [1], [False])
    n = 70
    D = torch.from_numpy(inputs.dense_densities(n, 2, seed=3)).cuda()
    W = torch.from_numpy(inputs.dense_densities(n, 2, seed=4)).cuda()
    res = []
    for packed in (0, 1):
        eng = jk.Engine("cuda:0")
        eng.set_option("aux_chunk", 20)
        eng.set_option("packed_factor", packed)
        fac = jk.pack_factor(m.L).cuda() if packed else torch.from_numpy(m.L).cuda()
        J, K = eng.build_dense(fac, D, precision)
        G = eng.density_grad(fac, W, D, precision)
        eng.sync_status()
        res.append((to_np(J), to_np(K), to_np(G)))
        eng.close()
    (Jd, Kd, Gd), (Jp, Kp, Gp) = res
    np.testing.assert_array_equal(Kp, Kd)
    err, tol = (abs_err, SPLIT_ABS) if precision == "split" else (rel_err, FP64_REL)
    assert err(Jp, Jd) < tol and err(Gp, Gd) < tol
    Jo, Ko = oracle.build_dense(m.L, inputs.dense_densities(n, 2, seed=3))
    Go = oracle.density_grad(m.L, inputs.dense_densities(n, 2, seed=4), inputs.dense_densities(n, 2, seed=3), nd=2)
    assert err(Jp, Jo) < tol and err(Kp, Ko) < tol and err(Gp, Go) < tol


@pytest.mark.parametrize("precision", ["split", "fp64"])
def test_packed_factor_adjoint(precision):
    """jk_adjoint on a packed factor: the chunks are expanded for the products
    and the J terms' metric dots are summed over the triangles, so dX, dY and
    dL agree with the dense factor's to rounding and match the oracle."""
    m = inputs.custom(70, 45, 12.0, [5, 3], [False, True])
    rng = np.random.default_rng(9)
    W = [rng.standard_normal((70, 70)) for _ in range(2)]
    V = [rng.standard_normal((70, 70)) for _ in range(2)]
    dXo, dYo, dLo = oracle.adjoint(m.L, m.X, m.Y, W, V)
    Wd, Vd = torch.tensor(np.array(W)).cuda(), torch.tensor(np.array(V)).cuda()
    X = [torch.from_numpy(x).cuda() for x in m.X]
    Y = [torch.from_numpy(y).cuda() for y in m.Y]
    res = []
    for packed in (0, 1):
        eng = jk.Engine("cuda:0")
        eng.set_option("aux_chunk", 20)
        eng.set_option("packed_factor", packed)
        fac = jk.pack_factor(m.L).cuda() if packed else torch.from_numpy(m.L).cuda()
        dX, dY, dL = eng.adjoint(fac, X, Y, m.sym, Wd, Vd, precision=precision)
        eng.sync_status()
        res.append(([to_np(t) for t in dX], [to_np(t) for t in dY], to_np(dL)))
        eng.close()
    (dXd, dYd, dLd), (dXp, dYp, dLp) = res
    if precision == "split":
        err = abs_err
        tol = SPLIT_ABS
    else:
        err = rel_err
        tol = FP64_REL
    # density 0 is non-symmetric; density 1 is symmetric (D = X X^T), whose
    # two gradient slots the library folds into dX (dY zero) while the oracle
    # gives them apart
    assert err(dXp[0], dXd[0]) < tol and err(dXp[0], dXo[0]) < tol
    assert err(dYp[0], dYd[0]) < tol and err(dYp[0], dYo[0]) < tol
    assert err(dXp[1], dXd[1]) < tol and err(dXp[1], dXo[1] + dYo[1]) < tol
    assert np.all(dYp[1] == 0) and np.all(dYd[1] == 0)
    assert err(dLp, dLd) < tol and err(dLp, dLo) < tol


@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_packed_factor_autograd(precision):
    """Through the autograd wrapper a packed factor gets its gradient in its
    own layout: the dense factor's dL folded onto the upper triangles."""
    from paper_2608_06536_b300.autograd import fold_packed_grad, jk as jk_fn
    m = inputs.custom(40, 30, 9.0, [4, 3], [False, True])
    rng = np.random.default_rng(11)
    W = torch.tensor(rng.standard_normal((2, 40, 40))).cuda()
    V = torch.tensor(rng.standard_normal((2, 40, 40))).cuda()
    grads = []
    for packed in (0, 1):
        eng = jk.Engine("cuda:0")
        eng.set_option("packed_factor", packed)
        fac = jk.pack_factor(m.L) if packed else torch.from_numpy(m.L)
        L = fac.cuda().requires_grad_(True)
        X = [torch.from_numpy(x).cuda().requires_grad_(True) for x in m.X]
        Y = [torch.from_numpy(m.Y[0]).cuda().requires_grad_(True), None]
        J, K = jk_fn(L, X, Y, precision=precision, engine=eng)
        E = (W * K).sum() + (V * J).sum()
        g = torch.autograd.grad(E, [L, X[0], X[1], Y[0]])
        eng.sync_status()
        grads.append(g)
        eng.close()
    (gLd, *gd), (gLp, *gp) = grads
    assert tuple(gLp.shape) == (30, 40 * 41 // 2)
    err, tol = (abs_err, SPLIT_ABS) if precision == "split" else (rel_err, FP64_REL)
    assert err(to_np(gLp), to_np(fold_packed_grad(gLd))) < tol
    for a, b in zip(gp, gd):
        assert err(to_np(a), to_np(b)) < tol
    _, _, dLo = oracle.adjoint(m.L, m.X, m.Y, list(to_np(W)), list(to_np(V)))
    assert err(to_np(gLp), to_np(fold_packed_grad(torch.from_numpy(dLo)))) < tol
