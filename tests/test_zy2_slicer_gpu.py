"""The FP32-digit vector slicer (JK_OPT_SLICER = 1) on the GPU: the sliced
GEMM on integer operands stays exact bit for bit, random products stay within
the split's error bound, and builds match the oracle (and the default
integer-digit slicer) within the split tolerance."""
import ctypes as ct

import numpy as np
import pytest
import torch

import oracle
from paper_2608_06536_b300 import inputs
from tests._util import SPLIT_ABS, abs_err, to_np

pytestmark = pytest.mark.gpu

OPT_SLICER = 6


@pytest.fixture(scope="module")
def lib():
    from paper_2608_06536_b300 import jk
    L = jk.load_library()
    L.jk_debug_sliced_gemm.argtypes = [ct.c_void_p, ct.c_int32, ct.c_int32, ct.c_int32,
                                       ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p]
    L.jk_debug_sliced_gemm.restype = ct.c_int
    L.jk_debug_sliced_gemm_workspace.argtypes = [ct.c_int32, ct.c_int32, ct.c_int32]
    L.jk_debug_sliced_gemm_workspace.restype = ct.c_size_t
    L.jk_set_option.argtypes = [ct.c_void_p, ct.c_int, ct.c_int64]
    return L


def _gemm(lib, A, B, slicer):
    M, K = A.shape
    N = B.shape[0]
    ws = torch.empty(lib.jk_debug_sliced_gemm_workspace(M, N, K), dtype=torch.uint8, device="cuda")
    h = ct.c_void_p()
    assert lib.jk_create(ct.byref(h), ct.c_void_p(ws.data_ptr()), ws.numel()) == 0
    assert lib.jk_set_option(h, OPT_SLICER, slicer) == 0
    Ad = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    Bd = torch.from_numpy(np.ascontiguousarray(B)).cuda()
    C = torch.full((M, N), float("nan"), dtype=torch.float64, device="cuda")
    st = lib.jk_debug_sliced_gemm(h, M, N, K, Ad.data_ptr(), Bd.data_ptr(), C.data_ptr(), None)
    assert st == 0, lib.jk_last_error(h)
    assert lib.jk_sync_status(h, None) == 0, lib.jk_last_error(h)
    lib.jk_destroy(h)
    return to_np(C)


def test_integer_operands_stay_exact(lib):
    rng = np.random.default_rng(12)
    M, N, K = 256, 128, 1024
    A = rng.integers(-1000, 1001, (M, K)).astype(np.float64)
    B = rng.integers(-1000, 1001, (N, K)).astype(np.float64)
    A[:, :64] = 1000.0
    B[:, :64] = 1000.0
    A[:, 64:128] = 1.0
    C = _gemm(lib, A, B, 1)
    np.testing.assert_array_equal(C, (A.astype(np.int64) @ B.T.astype(np.int64)).astype(np.float64))


@pytest.mark.parametrize("M,N,K", [(300, 200, 500), (129, 257, 2048), (130, 90, 4096)])
def test_random_products_within_bound(lib, M, N, K):
    rng = np.random.default_rng(M + N + K)
    A = rng.standard_normal((M, K)) * np.exp(rng.uniform(-8, 8, (M, 1)))
    B = rng.standard_normal((N, K))
    C = _gemm(lib, A, B, 1)
    ref = A.astype(np.longdouble) @ B.T.astype(np.longdouble)
    scale = np.abs(A).max(1)[:, None] * np.abs(B).max(1)[None, :] * np.sqrt(K)
    assert float(np.max(np.abs(C - ref) / scale)) < 2.0 ** -44


@pytest.mark.parametrize("n,naux,ks,sym", [(40, 53, [5, 12, 7], [False, True, False]),
                                           (132, 70, [64, 3, 9], [False, False, True])])
def test_build_matches_oracle(n, naux, ks, sym):
    from paper_2608_06536_b300 import jk
    m = inputs.custom(n, naux, max(naux / 4, 1.0), ks, sym)
    Jo, Ko = oracle.build(m.L, m.X, m.Y)
    L = torch.from_numpy(m.L).cuda()
    X = [torch.from_numpy(x).cuda() for x in m.X]
    Y = [torch.from_numpy(y).cuda() for y in m.Y]
    eng = jk.Engine("cuda:0")
    J0, K0 = eng.build(L, X, Y, m.sym, "split")
    eng.set_option("slicer", 1)
    J1, K1 = eng.build(L, X, Y, m.sym, "split")
    eng.sync_status()
    assert abs_err(to_np(J1), Jo) < SPLIT_ABS and abs_err(to_np(K1), Ko) < SPLIT_ABS
    assert abs_err(to_np(K1), to_np(K0)) < SPLIT_ABS
    eng.close()
