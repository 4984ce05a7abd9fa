"""torch.autograd wrapper: J, K forward and the hand-written adjoint backward.

Forward calls ``jk_build``; backward calls ``jk_adjoint`` with V = dE/dJ and
W = dE/dK, so for E = sum_s <W_s, K_s> + <V_s, J_s> autograd returns exactly
the library's adjoint (the self-adjoint form of Eq. 1, Sec. II.A).  The
panels L^P X, L^P Y are recomputed in the backward pass, never stored.
"""
from __future__ import annotations

import torch

from . import jk as _jk


class _JKFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, engine, precision, sym, L, *xy):
        nd = len(sym)
        X = [xy[2 * s] for s in range(nd)]
        Y = [xy[2 * s + 1] for s in range(nd)]
        J, K = engine.build(L, X, Y, sym, precision)
        ctx.engine, ctx.precision, ctx.sym = engine, precision, sym
        ctx.save_for_backward(L, *xy)
        return J, K

    @staticmethod
    def backward(ctx, gJ, gK):
        L, *xy = ctx.saved_tensors
        nd = len(ctx.sym)
        X = [xy[2 * s] for s in range(nd)]
        Y = [xy[2 * s + 1] for s in range(nd)]
        want_dl = ctx.needs_input_grad[3]
        dX, dY, dL = ctx.engine.adjoint(L, X, Y, ctx.sym, W=gK, V=gJ, want_dl=want_dl,
                                        precision=ctx.precision)
        grads = []
        for s in range(nd):
            if ctx.sym[s]:
                # D = X X^T: the library folds both slots into dX.
                grads += [dX[s], torch.zeros_like(dY[s])]
            else:
                grads += [dX[s], dY[s]]
        if want_dl and L.dim() == 2:
            dL = fold_packed_grad(dL)
        return (None, None, None, dL if want_dl else None, *grads)


def fold_packed_grad(dL):
    """The gradient with respect to a packed factor ([naux][n(n+1)/2], the
    row-major upper triangles of the symmetric L^P) from the dense one
    ([naux][n][n]): an off-diagonal packed entry stands for both L^P_ij and
    L^P_ji, so it collects dL_ij + dL_ji; a diagonal entry collects dL_ii once."""
    n = int(dL.shape[-1])
    iu = torch.triu_indices(n, n, device=dL.device)
    off = (iu[0] != iu[1]).to(dL.dtype)
    return (dL[:, iu[0], iu[1]] + off * dL[:, iu[1], iu[0]]).contiguous()


def jk(L, X, Y=None, sym=None, precision="fp64", engine=None):
    """Differentiable (J, K), each [nd][n][n], for D_s = X_s Y_s^T.

    L is the dense factor [naux][n][n], or the packed one [naux][n(n+1)/2]
    when the engine runs with the packed_factor option; its gradient has L's
    own layout (folded onto the upper triangles for a packed factor).

    For a symmetric density pass Y_s = None (or sym[s] = True); its gradient
    then arrives entirely on X_s.
    """
    nd = len(X)
    sym = tuple(bool(sym[s]) if sym is not None else (Y is None or Y[s] is None) for s in range(nd))
    Y = [X[s] if (sym[s] or Y is None or Y[s] is None) else Y[s] for s in range(nd)]
    engine = engine if engine is not None else _jk.default_engine(L.device)
    xy = []
    for s in range(nd):
        xy += [X[s], Y[s]]
    return _JKFunction.apply(engine, precision, sym, L, *xy)


class _JKDenseFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, engine, precision, L, D):
        J, K = engine.build_dense(L, D, precision)
        ctx.engine, ctx.precision = engine, precision
        ctx.save_for_backward(L)
        return J, K

    @staticmethod
    def backward(ctx, gJ, gK):
        (L,) = ctx.saved_tensors
        if ctx.needs_input_grad[2]:
            raise NotImplementedError("jk_dense differentiates with respect to D only")
        # dE/dD = K(dE/dK) + J(dE/dJ): K and J are self-adjoint (Eq. 1, Sec. II.A)
        G = ctx.engine.density_grad(L, W=gK.contiguous(), V=gJ.contiguous(), precision=ctx.precision)
        return None, None, None, G


def jk_dense(L, D, precision="fp64", engine=None):
    """Differentiable (J, K), each [nd][n][n], for dense general densities D
    ([nd][n][n]); the gradient with respect to D is the density gradient
    K(dE/dK) + J(dE/dJ) (jk_density_grad).  L is not differentiated."""
    engine = engine if engine is not None else _jk.default_engine(L.device)
    return _JKDenseFunction.apply(engine, precision, L, D)
