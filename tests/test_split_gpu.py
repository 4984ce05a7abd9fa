"""Split-precision (BF16 slices on tcgen05) path: the sliced GEMM building block
and the J/K build, against exact references and the CPU oracle."""
import ctypes as ct

import numpy as np
import pytest
import torch

import oracle
from paper_2608_06536_b300 import inputs
from tests._util import SPLIT_ABS, abs_err, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dbg():
    from paper_2608_06536_b300 import jk
    lib = jk.load_library()
    lib.jk_debug_sliced_gemm.argtypes = [ct.c_void_p, ct.c_int32, ct.c_int32, ct.c_int32,
                                         ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p]
    lib.jk_debug_sliced_gemm.restype = ct.c_int
    lib.jk_debug_sliced_gemm_workspace.argtypes = [ct.c_int32, ct.c_int32, ct.c_int32]
    lib.jk_debug_sliced_gemm_workspace.restype = ct.c_size_t
    lib.jk_set_option.argtypes = [ct.c_void_p, ct.c_int, ct.c_int64]
    lib.jk_debug_sliced_gemm_slices.argtypes = [ct.c_void_p, ct.c_int32, ct.c_int32, ct.c_int32, ct.c_void_p,
                                                ct.c_void_p, ct.c_void_p, ct.c_int32, ct.c_void_p]
    lib.jk_debug_sliced_gemm_slices.restype = ct.c_int
    lib.jk_debug_sliced_gemm_workspace_slices.argtypes = [ct.c_int32, ct.c_int32, ct.c_int32, ct.c_int32]
    lib.jk_debug_sliced_gemm_workspace_slices.restype = ct.c_size_t
    return lib


def sliced_gemm(lib, A, B, raster=-1, slices=6, tile=-1):
    M, K = A.shape
    N = B.shape[0]
    ws = torch.empty(lib.jk_debug_sliced_gemm_workspace_slices(M, N, K, slices), dtype=torch.uint8, device="cuda")
    h = ct.c_void_p()
    assert lib.jk_create(ct.byref(h), ct.c_void_p(ws.data_ptr()), ws.numel()) == 0
    assert lib.jk_set_option(h, 2, raster) == 0 and lib.jk_set_option(h, 9, tile) == 0
    Ad = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    Bd = torch.from_numpy(np.ascontiguousarray(B)).cuda()
    C = torch.full((M, N), float("nan"), dtype=torch.float64, device="cuda")
    if slices == 6 and tile == -1:
        st = lib.jk_debug_sliced_gemm(h, M, N, K, Ad.data_ptr(), Bd.data_ptr(), C.data_ptr(), None)
    else:
        st = lib.jk_debug_sliced_gemm_slices(h, M, N, K, Ad.data_ptr(), Bd.data_ptr(), C.data_ptr(), slices, None)
    assert st == 0, lib.jk_last_error(h)
    assert lib.jk_sync_status(h, None) == 0, lib.jk_last_error(h)
    lib.jk_destroy(h)
    return to_np(C)


def exact_product(A, B):
    return (A.astype(np.longdouble) @ B.T.astype(np.longdouble))


@pytest.mark.parametrize("raster", [0, 1])
@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (128, 128, 128), (300, 200, 500), (129, 257, 2047), (700, 90, 64),
                                   (130, 500, 100)])
def test_sliced_gemm_random(dbg, M, N, K, raster):
    """Odd and even tile counts along M and N, ragged tails in every
    dimension, both tile orders."""
    rng = np.random.default_rng(M + N + K)
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((N, K))
    C = sliced_gemm(dbg, A, B, raster=raster)
    ref = exact_product(A, B)
    assert np.all(np.isfinite(C))
    # error budget: 2^-48 of each row's scale per operand, summed over K
    scale = np.abs(A).max(1)[:, None] * np.abs(B).max(1)[None, :] * np.sqrt(K)
    assert float(np.max(np.abs(C - ref) / scale)) < 2.0 ** -44


@pytest.mark.parametrize("raster", [0, 1])
def test_sliced_gemm_split_k(dbg, raster):
    """K > 2048: int64 partials summed in 128-bit integers (the padding rows
    of a ragged row tile must not land in the next super-chunk's rows)."""
    rng = np.random.default_rng(11)
    M, N, K = 140, 130, 5000
    A = rng.standard_normal((M, K)) * np.exp(-np.arange(K) / 2000.0)
    B = rng.standard_normal((N, K))
    C = sliced_gemm(dbg, A, B, raster=raster)
    ref = exact_product(A, B)
    scale = np.abs(A).max(1)[:, None] * np.abs(B).max(1)[None, :] * np.sqrt(K)
    assert float(np.max(np.abs(C - ref) / scale)) < 2.0 ** -44


def test_sliced_gemm_integers_exact(dbg):
    """Integer operands: every slice is exact, every accumulation window must
    be exact in the tensor core's FP32 accumulator, so C equals the exact
    product bit for bit (including a large accumulator next to small terms)."""
    rng = np.random.default_rng(12)
    M, N, K = 256, 128, 1024
    A = rng.integers(-1000, 1001, (M, K)).astype(np.float64)
    B = rng.integers(-1000, 1001, (N, K)).astype(np.float64)
    A[:, :64] = 1000.0
    B[:, :64] = 1000.0
    A[:, 64:128] = 1.0
    for raster in (0, 1):
        C = sliced_gemm(dbg, A, B, raster=raster)
        np.testing.assert_array_equal(C, (A.astype(np.int64) @ B.T.astype(np.int64)).astype(np.float64))
    C = sliced_gemm(dbg, A, B)
    ref = (A.astype(np.int64) @ B.T.astype(np.int64)).astype(np.float64)
    np.testing.assert_array_equal(C, ref)


# Seven slices (56-bit operands, 28 slice pairs, exact windows on diagonals
# 0-4) and six slices on 64-column tiles: the configurations of the split
# adjoint and of the tile-width tuning candidate.
@pytest.mark.parametrize("slices,tile,bound", [(7, -1, 2.0 ** -50), (6, 1, 2.0 ** -44)])
@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (129, 257, 2047), (300, 65, 500), (140, 130, 5000)])
def test_sliced_gemm_configurations(dbg, M, N, K, slices, tile, bound):
    rng = np.random.default_rng(M * 7 + N + K)
    A = rng.standard_normal((M, K)) * np.exp(-np.arange(K) / 3000.0)
    B = rng.standard_normal((N, K))
    C = sliced_gemm(dbg, A, B, slices=slices, tile=tile)
    ref = exact_product(A, B)
    assert np.all(np.isfinite(C))
    scale = np.abs(A).max(1)[:, None] * np.abs(B).max(1)[None, :] * np.sqrt(K)
    assert float(np.max(np.abs(C - ref) / scale)) < bound


@pytest.mark.parametrize("slices,tile", [(7, -1), (6, 1)])
def test_sliced_gemm_configurations_integers_exact(dbg, slices, tile):
    """Integer operands are exact in both configurations (every exact window,
    diagonal 4 of the seven-slice split included, stays exact in FP32)."""
    rng = np.random.default_rng(13)
    M, N, K = 256, 130, 1024
    A = rng.integers(-1000, 1001, (M, K)).astype(np.float64)
    B = rng.integers(-1000, 1001, (N, K)).astype(np.float64)
    A[:, :64] = 1000.0
    B[:, :64] = 1000.0
    for raster in (0, 1):
        C = sliced_gemm(dbg, A, B, raster=raster, slices=slices, tile=tile)
        np.testing.assert_array_equal(C, (A.astype(np.int64) @ B.T.astype(np.int64)).astype(np.float64))


def test_seven_slices_are_more_accurate(dbg):
    """On the same random product the 56-bit operands leave at least 16x less
    error than the 48-bit ones (the reason the split adjoint uses them)."""
    rng = np.random.default_rng(21)
    A = rng.standard_normal((200, 3000))
    B = rng.standard_normal((150, 3000))
    ref = exact_product(A, B)
    e6 = float(np.max(np.abs(sliced_gemm(dbg, A, B, slices=6) - ref)))
    e7 = float(np.max(np.abs(sliced_gemm(dbg, A, B, slices=7) - ref)))
    assert e7 * 16 < e6, (e6, e7)


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
    (7, 5, [3], [False]),
    (37, 53, [5, 1, 13], [False, True, False]),
    (130, 70, [64, 3, 9], [False, False, True]),
])
def test_split_build_ragged_vs_oracle(eng, n, naux, ks, sym):
    m = inputs.custom(n, naux, max(naux / 4, 1.0), ks, sym)
    Jo, Ko = oracle.build(m.L, m.X, m.Y)
    L, X, Y = _gpu(m)
    J, K = eng.build(L, X, Y, sym, "split")
    eng.sync_status()
    for s in range(len(ks)):
        assert abs_err(to_np(J[s]), Jo[s]) < SPLIT_ABS
        assert abs_err(to_np(K[s]), Ko[s]) < SPLIT_ABS


def test_split_build_one_molecule_small(eng):
    m = inputs.one_molecule_small()
    Jo, Ko = oracle.build(m.L, m.X, m.Y)
    L, X, Y = _gpu(m)
    J, K = eng.build(L, X, Y, m.sym, "split")
    eng.sync_status()
    assert abs_err(to_np(J), Jo) < SPLIT_ABS
    assert abs_err(to_np(K), Ko) < SPLIT_ABS


def test_split_build_deterministic(eng):
    m = inputs.custom(96, 200, 50.0, [8, 8], [False, True])
    L, X, Y = _gpu(m)
    J1, K1 = eng.build(L, X, Y, m.sym, "split")
    J2, K2 = eng.build(L, X, Y, m.sym, "split")
    assert torch.equal(J1, J2) and torch.equal(K1, K2)


# ------------------------------------------------------------------ adjoint

@pytest.mark.parametrize("n,naux,ks,sym", [
    (9, 6, [2, 3], [False, False]),
    (33, 41, [4, 5], [True, False]),
    (70, 150, [8, 16, 3], [False, False, True]),
])
def test_split_adjoint_vs_oracle(eng, n, naux, ks, sym):
    m = inputs.custom(n, naux, max(naux / 5, 1.0), ks, sym)
    rng = np.random.default_rng(3)
    W = [rng.standard_normal((n, n)) for _ in ks]
    V = [rng.standard_normal((n, n)) for _ in ks]
    dXo, dYo, dLo = oracle.adjoint(m.L, m.X, m.Y, W, V)
    L, X, Y = _gpu(m)
    dX, dY, dL = eng.adjoint(L, X, Y, m.sym, torch.tensor(np.array(W)).cuda(),
                             torch.tensor(np.array(V)).cuda(), precision="split")
    eng.sync_status()
    assert abs_err(to_np(dL), dLo) < SPLIT_ABS
    for s in range(len(ks)):
        if sym[s]:
            assert abs_err(to_np(dX[s]), dXo[s] + dYo[s]) < SPLIT_ABS
            assert np.all(to_np(dY[s]) == 0)
        else:
            assert abs_err(to_np(dX[s]), dXo[s]) < SPLIT_ABS
            assert abs_err(to_np(dY[s]), dYo[s]) < SPLIT_ABS


def test_split_adjoint_partial_seeds(eng):
    n = 21
    m = inputs.custom(n, 13, 5.0, [3], [False])
    rng = np.random.default_rng(4)
    W = [rng.standard_normal((n, n))]
    L, X, Y = _gpu(m)
    Wt = torch.tensor(np.array(W)).cuda()
    dXo, dYo, dLo = oracle.adjoint(m.L, m.X, m.Y, W, None)
    dX, dY, dL = eng.adjoint(L, X, Y, m.sym, Wt, None, precision="split")
    assert abs_err(to_np(dX[0]), dXo[0]) < SPLIT_ABS and abs_err(to_np(dL), dLo) < SPLIT_ABS
    dXo, dYo, dLo = oracle.adjoint(m.L, m.X, m.Y, None, W)
    dX, dY, dL = eng.adjoint(L, X, Y, m.sym, None, Wt, precision="split")
    assert abs_err(to_np(dY[0]), dYo[0]) < SPLIT_ABS and abs_err(to_np(dL), dLo) < SPLIT_ABS
    dX, dY, dL = eng.adjoint(L, X, Y, m.sym, Wt, Wt, want_dl=False, precision="split")
    assert dL is None


def test_split_autograd_matches_fp64(eng):
    from paper_2608_06536_b300.autograd import jk as jk_fn
    n, naux = 40, 60
    m = inputs.custom(n, naux, 12.0, [5, 4], [False, True])
    rng = np.random.default_rng(6)
    Wn = rng.standard_normal((2, n, n)); Vn = rng.standard_normal((2, n, n))
    grads = {}
    for prec in ("fp64", "split"):
        L = torch.tensor(m.L, device="cuda", requires_grad=True)
        X = [torch.tensor(x, device="cuda", requires_grad=True) for x in m.X]
        Y = [torch.tensor(m.Y[0], device="cuda", requires_grad=True), None]
        J, K = jk_fn(L, X, Y, precision=prec, engine=eng)
        E = (torch.tensor(Wn, device="cuda") * K).sum() + (torch.tensor(Vn, device="cuda") * J).sum()
        grads[prec] = [to_np(g) for g in torch.autograd.grad(E, [L, X[0], X[1], Y[0]])]
    for a, b in zip(grads["fp64"], grads["split"]):
        assert abs_err(b, a) < SPLIT_ABS
