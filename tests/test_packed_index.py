"""The packed upper-triangle layout (csrc/packed.cuh), compiled as host C++:
positions run 0, 1, ... in row-major order of the upper triangle, and the
inverse used by the symmetric J back-contraction (a square-root closed form
plus correction steps) returns the right (row, column) at every position for
n <= 300 and at every row start, its neighbours and random positions for n up
to the library's limit of 65535.  The binding's pack_factor uses the same
layout."""
import os
import subprocess

import pytest
import torch

from paper_2608_06536_b300 import jk

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    out = tmp_path_factory.mktemp("packed") / "check_packed"
    subprocess.run(["g++", "-O2", "-std=c++17", "-Wall", "-Wextra", "-Werror", "-o", str(out),
                    os.path.join(HERE, "digits", "check_packed.cpp")], check=True)
    return str(out)


def test_layout_and_inverse(exe):
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.startswith("ok ") and int(out.stdout.split()[1]) > 2_000_000


@pytest.mark.parametrize("n", [1, 2, 7, 33])
def test_pack_factor_uses_the_kernel_layout(exe, n):
    pos = [int(v) for v in subprocess.run([exe, "dump", str(n)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    L = torch.randn(2, n, n, dtype=torch.float64, generator=torch.Generator().manual_seed(n))
    L = L + L.transpose(1, 2)
    P = jk.pack_factor(L)
    assert P.shape == (2, n * (n + 1) // 2)
    k = 0
    for a in range(n):
        for b in range(a, n):
            assert P[1, pos[k]] == L[1, a, b] and P[1, pos[k]] == L[1, b, a]
            k += 1
