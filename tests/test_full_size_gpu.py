"""The five workload shapes at full size.

* multi-state (nbf 400, naux 2400, 8 densities): split and FP64 builds against
  the oracle on sampled entries;
* large single molecule (nbf 1000, naux 5000, 16 densities of width 100,
  40 GB factor): split against the oracle on sampled entries, and against the
  FP64 engine element by element on two densities;
* adjoint case (nbf 600, naux 3600, 8 densities of width 60): split adjoint
  through the autograd wrapper and FP64 adjoint against the oracle's sampled
  adjoint, and both against central differences (h = 1e-5) on 32 random
  directions;
* uneven batch (64 molecules, nbf in [100, 600], 208 GB of factors): one
  batched split build, captured in a CUDA graph and replayed, against the
  oracle on sampled entries of three molecules and the FP64 engine on the six
  smallest.

Tolerance for the split path: 1e-10 absolute in output units for J, K, dX,
dY and dL, or the FP64 engine's own error on the same entries where that is
larger.  The adjoint's dX, dY at the 600/3600 size are sums of n * naux =
2.2e6 products and reach |dX| ~ 5e4; the split adjoint forms them from 56-bit
(seven-slice) operands, which keeps them inside that gate, and both engines'
errors are printed.
"""
import gc
import json

import numpy as np
import pytest
import torch

import oracle
from paper_2608_06536_b300 import inputs
from tests._util import FP64_REL, SPLIT_ABS, abs_err, to_np

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _release():
    gc.collect()
    torch.cuda.empty_cache()


@pytest.fixture(scope="module")
def eng():
    from paper_2608_06536_b300 import jk
    e = jk.Engine("cuda:0")
    yield e
    e.close()
    _release()


def _report(case, **kw):
    print("\n" + json.dumps({"case": case, **{k: (float(v) if isinstance(v, (np.floating, float)) else v)
                                            for k, v in kw.items()}}), flush=True)


def _dev(arrs):
    return [torch.from_numpy(a).cuda() for a in arrs]


def _samples(rng, nd, n, count):
    s = rng.integers(0, nd, count)
    mu = rng.integers(0, n, count)
    nu = rng.integers(0, n, count)
    s[:2] = [0, nd - 1]
    mu[:2] = [0, n - 1]
    nu[:2] = [n - 1, 0]
    return s, mu, nu


def _gate(fp64_err):
    return max(SPLIT_ABS, fp64_err)


def test_multi_state_full(eng):
    m = inputs.multi_state()
    L = torch.from_numpy(m.L).cuda()
    X, Y = _dev(m.X), _dev(m.Y)
    J, K = eng.build(L, X, Y, m.sym, "split")
    eng.sync_status()
    Jf, Kf = eng.build(L, X, Y, m.sym, "fp64")
    s, mu, nu = _samples(np.random.default_rng(1), m.nd, m.n, 128)
    Jo, Ko = oracle.sample(m.L, m.X, m.Y, s, mu, nu)
    Jn, Kn, Jfn, Kfn = to_np(J), to_np(K), to_np(Jf), to_np(Kf)
    eJ, eK = np.abs(Jn[s, mu, nu] - Jo).max(), np.abs(Kn[s, mu, nu] - Ko).max()
    fJ, fK = np.abs(Jfn[s, mu, nu] - Jo).max(), np.abs(Kfn[s, mu, nu] - Ko).max()
    _report("multi_state", split_J=eJ, split_K=eK, fp64_J=fJ, fp64_K=fK,
            split_vs_fp64_J=abs_err(Jn, Jfn), split_vs_fp64_K=abs_err(Kn, Kfn),
            max_J=np.abs(Jfn).max(), max_K=np.abs(Kfn).max())
    assert eJ <= SPLIT_ABS and eK <= SPLIT_ABS
    assert fJ <= FP64_REL * np.abs(Jfn).max() and fK <= FP64_REL * np.abs(Kfn).max()
    assert abs_err(Jn, Jfn) < 2 * SPLIT_ABS and abs_err(Kn, Kfn) < 2 * SPLIT_ABS
    # the configuration bench.py times on this workload (its autotuner's pick):
    # all aux indices in one chunk, grouped launches, n-tile raster
    for name, v in (("aux_chunk", 3834), ("schedule", 1), ("raster", 0)):
        eng.set_option(name, v)
    Jt, Kt = eng.build(L, X, Y, m.sym, "split")
    eng.sync_status()
    for name in ("aux_chunk", "schedule", "raster"):
        eng.set_option(name, -1)
    Jtn, Ktn = to_np(Jt), to_np(Kt)
    tJ, tK = np.abs(Jtn[s, mu, nu] - Jo).max(), np.abs(Ktn[s, mu, nu] - Ko).max()
    _report("multi_state_bench_config", split_J=tJ, split_K=tK, vs_default_J=abs_err(Jtn, Jn),
            vs_default_K=abs_err(Ktn, Kn))
    assert tJ <= SPLIT_ABS and tK <= SPLIT_ABS
    assert abs_err(Jtn, Jfn) < 2 * SPLIT_ABS and abs_err(Ktn, Kfn) < 2 * SPLIT_ABS


def test_large_single_full(eng):
    m = inputs.large_single()
    L = inputs.factor_device(m.n, m.naux, m.tau, m.seed)
    X, Y = _dev(m.X), _dev(m.Y)
    J, K = eng.build(L, X, Y, m.sym, "split")
    eng.sync_status()
    sel = [0, m.nd - 1]
    Jf, Kf = eng.build(L, [X[i] for i in sel], [Y[i] for i in sel], [False] * len(sel), "fp64")
    Jn, Kn, Jfn, Kfn = to_np(J), to_np(K), to_np(Jf), to_np(Kf)
    dJ = max(abs_err(Jn[i], Jfn[j]) for j, i in enumerate(sel))
    dK = max(abs_err(Kn[i], Kfn[j]) for j, i in enumerate(sel))
    Lh = L.cpu().numpy()
    del L
    _release()
    rng = np.random.default_rng(2)
    s, mu, nu = _samples(rng, m.nd, m.n, 48)
    Jo, Ko = oracle.sample(Lh, m.X, m.Y, s, mu, nu)
    eJ, eK = np.abs(Jn[s, mu, nu] - Jo).max(), np.abs(Kn[s, mu, nu] - Ko).max()
    on_sel = np.isin(s, sel)
    pos = np.array([sel.index(q) if q in sel else 0 for q in s])
    fJ = np.abs(Jfn[pos, mu, nu] - Jo)[on_sel].max()
    fK = np.abs(Kfn[pos, mu, nu] - Ko)[on_sel].max()
    _report("large_single", split_J=eJ, split_K=eK, fp64_J=fJ, fp64_K=fK, split_vs_fp64_J=dJ,
            split_vs_fp64_K=dK, max_J=np.abs(Jfn).max(), max_K=np.abs(Kfn).max())
    del Lh
    assert fJ <= FP64_REL * np.abs(Jfn).max() and fK <= FP64_REL * np.abs(Kfn).max()
    assert eJ <= _gate(fJ) and eK <= _gate(fK)


def test_adjoint_full(eng):
    from paper_2608_06536_b300.autograd import jk as jk_fn
    m, W, V = inputs.adjoint_case(with_factor=False)
    n, naux, nd = m.n, m.naux, m.nd
    L = inputs.factor_device(n, naux, m.tau, m.seed)
    Wd = torch.tensor(np.array(W)).cuda()
    Vd = torch.tensor(np.array(V)).cuda()
    X, Y = _dev(m.X), _dev(m.Y)

    # split precision through the autograd wrapper
    Lg = L.detach().requires_grad_(True)
    Xg = [x.detach().requires_grad_(True) for x in X]
    Yg = [y.detach().requires_grad_(True) for y in Y]
    Jt, Kt = jk_fn(Lg, Xg, Yg, precision="split", engine=eng)
    E = (Wd * Kt).sum() + (Vd * Jt).sum()
    grads = torch.autograd.grad(E, [Lg] + Xg + Yg)
    gL, gX, gY = grads[0], grads[1:1 + nd], grads[1 + nd:]
    del Jt, Kt, E, Lg
    # FP64 adjoint through the C-ABI directly
    dXf, dYf, dLf = eng.adjoint(L, X, Y, m.sym, Wd, Vd, precision="fp64")

    # oracle at sampled entries
    Lh = L.cpu().numpy()
    rng = np.random.default_rng(3)
    xs = (rng.integers(0, nd, 16), rng.integers(0, n, 16), rng.integers(0, m.ks[0], 16))
    ls = (rng.integers(0, naux, 16), rng.integers(0, n, 16), rng.integers(0, n, 16))
    ls[0][:2] = [0, naux - 1]
    ox, oy, ol = oracle.adjoint_sample(Lh, m.X, m.Y, W, V, xs, ls)
    del Lh

    def at(lst, idx):
        return np.array([float(lst[q][a, b]) for q, a, b in zip(*idx)])
    sx, sy, sl = at(gX, xs), at(gY, xs), to_np(gL)[ls]
    fx, fy, fl = at(dXf, xs), at(dYf, xs), to_np(dLf)[ls]
    err = {"split_dX": np.abs(sx - ox).max(), "split_dY": np.abs(sy - oy).max(),
           "split_dL": np.abs(sl - ol).max(), "fp64_dX": np.abs(fx - ox).max(),
           "fp64_dY": np.abs(fy - oy).max(), "fp64_dL": np.abs(fl - ol).max(),
           "max_dX": np.abs(ox).max(), "max_dL": np.abs(ol).max(),
           "split_vs_fp64_dL": abs_err(to_np(gL), to_np(dLf))}

    # central differences of E along 32 random directions (split forward)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    h = 1e-5

    def energy(Lp, Xp, Yp):
        J, K = eng.build(Lp, Xp, Yp, m.sym, "split")
        return float((Wd * K).sum() + (Vd * J).sum())

    # E(t) along a direction is a polynomial of degree 4 in t (quadratic in L,
    # linear in X and in Y): the central difference carries an h^2 truncation
    # term, the five-point stencil (8[E(h) - E(-h)] - [E(2h) - E(-2h)]) / 12h
    # none, so it checks the adjoint down to the forward's rounding.
    worst = {"central_split": 0.0, "central_fp64": 0.0, "stencil_split": 0.0, "stencil_fp64": 0.0}
    for _ in range(32):
        H = torch.randn((naux, n, n), dtype=torch.float64, device="cuda", generator=gen)
        H = 0.5 * (H + H.transpose(1, 2))
        hX = [torch.randn(x.shape, dtype=torch.float64, device="cuda", generator=gen) for x in X]
        hY = [torch.randn(y.shape, dtype=torch.float64, device="cuda", generator=gen) for y in Y]
        ev = {}
        Lp = torch.empty_like(L)
        for t in (1, -1, 2, -2):
            torch.add(L, H, alpha=t * h, out=Lp)
            ev[t] = energy(Lp, [x + t * h * a for x, a in zip(X, hX)], [y + t * h * b for y, b in zip(Y, hY)])
        del Lp
        central = (ev[1] - ev[-1]) / (2 * h)
        stencil = (8 * (ev[1] - ev[-1]) - (ev[2] - ev[-2])) / (12 * h)
        for tag, (ax, ay, al) in (("split", (gX, gY, gL)), ("fp64", (dXf, dYf, dLf))):
            an = float(sum((a * b).sum() for a, b in zip(ax, hX)) + sum((a * b).sum() for a, b in zip(ay, hY))
                       + (al * H).sum())
            scale = max(abs(an), 1.0)
            worst["central_" + tag] = max(worst["central_" + tag], abs(central - an) / scale)
            worst["stencil_" + tag] = max(worst["stencil_" + tag], abs(stencil - an) / scale)
        del H
    max_dx = max(float(t.abs().max()) for t in list(dXf) + list(dYf))
    _report("adjoint", max_dX_full=max_dx, **worst, **err)
    # central differences: h^2 truncation only (the same for both adjoints)
    assert worst["central_split"] < 5e-7 and worst["central_fp64"] < 5e-7
    assert worst["stencil_split"] < 1e-8 and worst["stencil_fp64"] < 1e-8
    assert err["fp64_dX"] <= FP64_REL * max_dx and err["fp64_dY"] <= FP64_REL * max_dx
    assert err["fp64_dL"] <= FP64_REL * err["max_dL"]
    assert err["split_dX"] <= _gate(err["fp64_dX"]) and err["split_dY"] <= _gate(err["fp64_dY"])
    assert err["split_dL"] <= SPLIT_ABS
    del gL, dLf, L
    _release()


def test_uneven_batch_full(eng):
    _release()
    mols = inputs.uneven_batch(with_factor=False)
    args = [(inputs.factor_device(m.n, m.naux, m.tau, m.seed), _dev(m.X), _dev(m.Y), m.sym) for m in mols]
    eager = eng.build_batched(args, "split")
    eng.sync_status()
    torch.cuda.synchronize()

    g = torch.cuda.CUDAGraph()
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(st):
        with torch.cuda.graph(g, stream=st):
            outs = eng.build_batched(args, "split", stream=st)
    torch.cuda.current_stream().wait_stream(st)
    g.replay()
    torch.cuda.synchronize()
    eng.sync_status()
    for (Je, Ke), (J, K) in zip(eager, outs):
        assert torch.equal(J, Je) and torch.equal(K, Ke)
    del g, outs

    # oracle: smallest, a middle and the largest molecule, 12 entries each
    order = sorted(range(len(mols)), key=lambda i: mols[i].n)
    worst = {"J": 0.0, "K": 0.0}
    rng = np.random.default_rng(4)
    for mi in (order[0], order[len(order) // 2], order[-1]):
        m = mols[mi]
        Lh = args[mi][0].cpu().numpy()
        s, mu, nu = _samples(rng, m.nd, m.n, 12)
        Jo, Ko = oracle.sample(Lh, m.X, m.Y, s, mu, nu)
        Jn, Kn = to_np(eager[mi][0]), to_np(eager[mi][1])
        worst["J"] = max(worst["J"], np.abs(Jn[s, mu, nu] - Jo).max())
        worst["K"] = max(worst["K"], np.abs(Kn[s, mu, nu] - Ko).max())
        del Lh

    # the FP64 engine, batched, on the six smallest molecules
    small = order[:6]
    f64 = eng.build_batched([args[i] for i in small], "fp64")
    d = {"J": 0.0, "K": 0.0}
    for i, (Jf, Kf) in zip(small, f64):
        d["J"] = max(d["J"], abs_err(to_np(eager[i][0]), to_np(Jf)))
        d["K"] = max(d["K"], abs_err(to_np(eager[i][1]), to_np(Kf)))
    _report("uneven_batch", split_J=worst["J"], split_K=worst["K"], split_vs_fp64_small_J=d["J"],
            split_vs_fp64_small_K=d["K"], molecules=len(mols), densities=sum(m.nd for m in mols))
    del args, eager, f64
    _release()
    assert worst["J"] <= SPLIT_ABS and worst["K"] <= SPLIT_ABS
    assert d["J"] < 2 * SPLIT_ABS and d["K"] < 2 * SPLIT_ABS
