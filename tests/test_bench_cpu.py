"""Host-side pieces of bench.py and of the input recipe (no GPU needed): the
algorithmic flop model of the metric, the peaks it divides by, and the
device-side factor generator's properties (run on the CPU)."""
import json
import math
import os

import numpy as np
import pytest
import torch

import bench
from paper_2608_06536_b300 import inputs


def test_build_flops_model():
    # per density: panels 2n^2k naux per half-transform (one for a symmetric
    # density), rank update 2n^2k naux (half of it when symmetric), J 2n^2 naux,
    # gamma 2nk naux
    n, A = 400, 2400
    ks, sym = [40] * 8, [True] + [False] * 7
    expect = sum((2 + 1 if s else 4 + 2) * n * n * k * A + 2 * n * n * A + 2 * n * k * A for k, s in zip(ks, sym))
    assert bench.build_flops(n, A, ks, sym) == pytest.approx(expect, rel=1e-15)
    assert bench.build_flops(n, A, ks, sym) == pytest.approx(6.98e11, rel=2e-3)
    assert bench.panel_rank_flops(n, A, ks, sym) == pytest.approx(45 * n * n * 40 * A, rel=1e-15)


def test_adjoint_flops_model():
    n, A, k = 600, 3600, 60
    one = 12 * n * n * k * A + 4 * n * n * k * A + 4 * n * n * A
    assert bench.adjoint_flops(n, A, [k] * 8, [False] * 8) == pytest.approx(8 * one, rel=1e-15)


def test_peaks_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    d, src = bench.load_peaks()
    assert src == "fallback" and d["bf16_tflops_sustained"] == 1400.0 and d["hbm_gbs"] == 6400.0
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"bf16_tflops_sustained": 1371.7}))
    d, src = bench.load_peaks()
    assert src == "measured" and d["bf16_tflops_sustained"] == 1371.7


def test_factor_device_recipe_on_cpu():
    n, naux, tau = 9, 40, 7.0
    L = inputs.factor_device(n, naux, tau, seed=3, device="cpu")
    assert L.shape == (naux, n, n) and L.dtype == torch.float64
    assert torch.equal(L, L.transpose(1, 2))                       # symmetric
    assert torch.equal(L, inputs.factor_device(n, naux, tau, seed=3, device="cpu"))   # deterministic
    assert not torch.equal(L, inputs.factor_device(n, naux, tau, seed=4, device="cpu"))
    # undo the exp(-P/tau) scale: the upper triangles are then N(0,1) draws
    unscaled = L * torch.exp(torch.arange(naux, dtype=torch.float64) / tau)[:, None, None]
    iu = torch.triu_indices(n, n)
    v = unscaled[:, iu[0], iu[1]].flatten().numpy()
    assert abs(v.mean()) < 5 / math.sqrt(v.size) and abs(v.std() - 1.0) < 0.05


def test_host_recipe_matches_its_statement():
    L = inputs.factor(6, 3, 2.0, seed=1)
    for P in range(3):
        M = inputs.factor_slice(6, P, 2.0, seed=1)
        np.testing.assert_array_equal(L[P], M)
        assert np.array_equal(M, M.T)
        rng = np.random.default_rng([1, 1, P])
        iu = np.triu_indices(6)
        np.testing.assert_allclose(M[iu], rng.standard_normal(iu[0].size) * math.exp(-P / 2.0), rtol=0, atol=0)


def test_dense_flops_model():
    # per dense density: K = panels L^P D (2 n^3 per P) + reduction against
    # L^P (2 n^3 per P); J = metric dot (2 n^2 per P) + back-contraction
    # (2 n^2 per P)
    n, A, nd = 400, 2400, 8
    assert bench.dense_flops(n, A, nd) == pytest.approx(nd * A * (2 * n**3 + 2 * n**3 + 2 * n * n + 2 * n * n),
                                                        rel=1e-15)


def test_dense_density_recipe():
    D = inputs.dense_density(50, 2, seed=3)
    assert D.shape == (50, 50) and not np.array_equal(D, D.T)
    rng = np.random.default_rng([3, 4, 2])
    np.testing.assert_array_equal(D, rng.standard_normal((50, 50)) / 50)
    S = inputs.dense_densities(50, 3, seed=3)
    np.testing.assert_array_equal(S[2], D)


def test_pair_flops_model():
    # right build + per map and right density: U_b = M_b Z_L and the pair dots
    n, A = 400, 2400
    kl, kr = [40] * 8, [40] * 8
    ctot_l = 8 * 80
    expect = bench.build_flops(n, A, kr, [False] * 8) + 2 * 8 * (2 * n * n * ctot_l + 8 * 2 * n * 40)
    assert bench.pair_flops(n, A, kl, [False] * 8, kr, [False] * 8) == pytest.approx(expect, rel=1e-15)
    # a symmetric left density contributes one column block
    assert bench.pair_flops(n, A, [40], [True], [40], [False]) < bench.pair_flops(n, A, [40], [False], [40], [False])


def test_custom_densities_recipe():
    X, Y = inputs.custom_densities(30, [3, 4], seed=2)
    for s, k in enumerate([3, 4]):
        x, y = inputs.transition_density(30, k, s, seed=2)
        np.testing.assert_array_equal(X[s], x)
        np.testing.assert_array_equal(Y[s], y)


def test_jstream_model():
    # the upper triangle of each L^P read once, J written once; one FMA per
    # upper-triangle entry, aux index and density
    n, A, nd = 1000, 5000, 16
    by, fl = bench.jstream_bytes_flops(n, A, nd)
    tri = n * (n + 1) // 2
    assert by == 8 * tri * A + 8 * nd * n * n and fl == 2 * tri * A * nd


def test_kernel_source_hash_tracks_the_sources(tmp_path, monkeypatch):
    """ncu figures are reported only for the kernel sources they were taken
    on: the hash changes with any byte of those sources."""
    import shutil
    src = tmp_path / "paper_2608_06536_b300" / "csrc"
    src.mkdir(parents=True)
    for name in bench.KERNEL_SOURCES:
        shutil.copy(os.path.join(bench.ROOT, "paper_2608_06536_b300", "csrc", name), src / name)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash()
    with open(src / "tc.cuh", "a") as f:
        f.write("\n")
    assert bench.kernel_source_hash() != h0


def test_headline_sample_entries_cover_the_corners():
    s, mu, nu = bench.sample_entries(np.random.default_rng(0), 16, 1000, 24)
    assert (s[0], mu[0], nu[0]) == (0, 0, 999) and (s[1], mu[1], nu[1]) == (15, 999, 0)
    assert s.max() < 16 and mu.max() < 1000 and nu.max() < 1000


def test_cpu_sample_is_a_named_exact_subset():
    for case, (nds, na) in bench.CPU_SAMPLE.items():
        m = bench.cpu_sample_molecule(case)
        assert 1 <= nds <= m.nd and 1 <= na <= m.naux
