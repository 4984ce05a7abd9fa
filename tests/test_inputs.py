"""The seeded input recipe (paper_2608_06536_b300/inputs.py) against its own
statement: symmetric factors drawn as upper triangles in row-major order and
scaled by exp(-P/tau), each P from its own stream; orthonormal ground
coefficients; N(0, 1/nbf) transition factors; the workload shapes (the
multi-state, large, adjoint and uneven-batch configurations, with the factor
sizes quoted for them); determinism; and no J/K arithmetic in the module."""
import math
import os

import numpy as np
import pytest

from paper_2608_06536_b300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))


def test_factor_slices_follow_the_recipe():
    n, tau = 9, 7.0
    for P in (0, 3, 11):
        M = inputs.factor_slice(n, P, tau, seed=5)
        np.testing.assert_array_equal(M, M.T)
        draws = np.random.default_rng([5, 1, P]).standard_normal(n * (n + 1) // 2)
        iu = np.triu_indices(n)                         # row-major upper triangle
        np.testing.assert_allclose(M[iu], draws * math.exp(-P / tau), rtol=0, atol=0)
    L = inputs.factor(n, 6, tau, seed=5, P0=2)
    for j in range(6):
        np.testing.assert_array_equal(L[j], inputs.factor_slice(n, 2 + j, tau, seed=5))


def test_densities_follow_the_recipe():
    n = 300
    X, Y = inputs.transition_density(n, 50, 2, seed=1)
    assert X.shape == Y.shape == (n, 50) and not np.array_equal(X, Y)
    for A in (X, Y):
        assert abs(A.std() * math.sqrt(n) - 1.0) < 0.02
    C, C2 = inputs.ground_density(n, 40, 0, seed=1)
    assert C is C2
    np.testing.assert_allclose(C.T @ C, np.eye(40), atol=1e-13)
    D = inputs.dense_density(n, 3, seed=1)
    assert D.shape == (n, n) and abs(D.std() * n - 1.0) < 0.01
    W, V = inputs.adjoint_seeds(50, 1, seed=1)
    assert abs(W.std() - 1.0) < 0.05 and abs(V.std() - 1.0) < 0.05


def test_workload_shapes():
    m = inputs.multi_state(with_factor=False)
    assert (m.n, m.naux, m.tau, m.ks, m.sym) == (400, 2400, 400.0, [40] * 8, [True] + [False] * 7)
    assert m.n * m.n * m.naux * 8 == pytest.approx(3.07e9, rel=0.01)
    big = inputs.large_single()
    assert (big.n, big.naux, big.ks) == (1000, 5000, [100] * 16) and big.L is None
    assert big.n ** 2 * big.naux * 8 == pytest.approx(40e9, rel=0.01)
    small = inputs.one_molecule_small(with_factor=False)
    assert (small.n, small.naux, small.ks, small.sym) == (48, 300, [6], [False])
    shapes = inputs.uneven_batch_shapes()
    assert len(shapes) == 64 and all(100 <= n <= 600 and 1 <= nd <= 16 for n, nd in shapes)
    assert shapes == inputs.uneven_batch_shapes()
    assert sum(nd for _, nd in shapes) == 560
    assert sum(6 * n * n * n * 8 for n, _ in shapes) == pytest.approx(208e9, rel=0.01)
    mols = inputs.uneven_batch(with_factor=False)
    assert all(mm.naux == 6 * mm.n and mm.tau == mm.n and mm.ks == [mm.n // 10] * len(mm.ks)
               and not any(mm.sym) for mm in mols)


def test_determinism_and_seeds():
    a = inputs.custom(20, 7, 3.0, [3, 2], [False, True], seed=4)
    b = inputs.custom(20, 7, 3.0, [3, 2], [False, True], seed=4)
    c = inputs.custom(20, 7, 3.0, [3, 2], [False, True], seed=5)
    np.testing.assert_array_equal(a.L, b.L)
    for u, v in zip(a.X + a.Y, b.X + b.Y):
        np.testing.assert_array_equal(u, v)
    assert not np.array_equal(a.L, c.L) and not np.array_equal(a.X[0], c.X[0])


def test_module_holds_no_jk_arithmetic():
    """It imports only number generation (numpy, torch's device generator) and
    the standard library: neither the oracle nor the library."""
    import ast
    tree = ast.parse(open(os.path.join(HERE, "..", "paper_2608_06536_b300", "inputs.py")).read())
    mods = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            mods |= {a.name.split(".")[0] for a in node.names}
        elif isinstance(node, ast.ImportFrom):
            mods.add("." if node.level else node.module.split(".")[0])
    assert mods <= {"__future__", "math", "dataclasses", "numpy", "torch"}, mods
