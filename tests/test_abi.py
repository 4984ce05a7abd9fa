"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every entry point include/jk.h declares, and validates arguments before any
device work."""
import ctypes as ct
import os
import re

import pytest

from paper_2608_06536_b300 import build as pkg_build
from paper_2608_06536_b300 import jk

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(jk_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    pkg_build.build()
    return jk.load_library()


def test_exports_every_declared_symbol(lib):
    names = declared_symbols()
    assert "jk_build" in names and "jk_build_batched" in names and "jk_adjoint" in names
    raw = ct.CDLL(jk.LIB_PATH)
    missing = [n for n in names if not hasattr(raw, n)]
    assert not missing, missing


def test_status_strings_and_version(lib):
    assert lib.jk_status_string(jk.JK_OK) == b"ok"
    assert lib.jk_status_string(jk.JK_ERR_OOM) == b"workspace arena too small"
    assert lib.jk_version().startswith(b"jk-b300")


def _one(n=10, naux=7, k=3, sym=0):
    f = jk.jk_factor(n, naux, 0x1000)
    d = (jk.jk_density * 1)()
    d[0].k, d[0].symmetric, d[0].X, d[0].Y = k, sym, 0x2000, 0x3000
    return f, d


def test_workspace_query_host_only(lib):
    f, d = _one()
    nb = ct.c_size_t()
    fa = (jk.jk_factor * 1)(f)
    assert lib.jk_workspace_query(jk.JK_OP_BUILD, 1, fa, None, 1, d, jk.JK_FP64, ct.byref(nb)) == jk.JK_OK
    small = nb.value
    assert small > 0
    f2, d2 = _one(n=100, naux=500, k=20)
    fa2 = (jk.jk_factor * 1)(f2)
    assert lib.jk_workspace_query(jk.JK_OP_BUILD, 1, fa2, None, 1, d2, jk.JK_FP64, ct.byref(nb)) == jk.JK_OK
    assert nb.value > small
    assert lib.jk_workspace_query(jk.JK_OP_ADJOINT, 1, fa2, None, 1, d2, jk.JK_FP64, ct.byref(nb)) == jk.JK_OK


@pytest.mark.parametrize("n,naux,k", [(0, 5, 1), (5, 0, 1), (5, 5, 0), (5, 5, 100), (65536, 1, 1),
                                      (46341, 1, 46341), (50000, 1, 60000)])
def test_workspace_query_rejects_bad_shapes(lib, n, naux, k):
    f, d = _one(n, naux, k)
    nb = ct.c_size_t()
    fa = (jk.jk_factor * 1)(f)
    assert lib.jk_workspace_query(jk.JK_OP_BUILD, 1, fa, None, 1, d, jk.JK_FP64, ct.byref(nb)) == jk.JK_ERR_SHAPE


def test_density_width_limit(lib):
    """nbf*k up to 2^31 - 1 is accepted, one more element is not (kernels index X_s with 32 bits)."""
    nb = ct.c_size_t()
    for n, k, want in [(46340, 46341, jk.JK_OK), (46341, 46341, jk.JK_ERR_SHAPE), (65535, 32768, jk.JK_OK),
                       (65535, 32769, jk.JK_ERR_SHAPE)]:
        f, d = _one(n, 1, k)
        fa = (jk.jk_factor * 1)(f)
        assert lib.jk_workspace_query(jk.JK_OP_BUILD, 1, fa, None, 1, d, jk.JK_FP64, ct.byref(nb)) == want, (n, k)


def test_workspace_query_rejects_bad_args(lib):
    f, d = _one()
    fa = (jk.jk_factor * 1)(f)
    nb = ct.c_size_t()
    assert lib.jk_workspace_query(jk.JK_OP_BUILD, 1, fa, None, 1, d, 7, ct.byref(nb)) == jk.JK_ERR_ARG
    assert lib.jk_workspace_query(jk.JK_OP_BUILD, 1, fa, None, 1, d, jk.JK_FP64, None) == jk.JK_ERR_ARG
    assert lib.jk_workspace_query(9, 1, fa, None, 1, d, jk.JK_FP64, ct.byref(nb)) == jk.JK_ERR_ARG
    # batched: nd must equal the sum of nd_per_mol
    ndm = (ct.c_int32 * 1)(1)
    assert lib.jk_workspace_query(jk.JK_OP_BATCHED, 1, fa, ndm, 2, d, jk.JK_FP64, ct.byref(nb)) == jk.JK_ERR_SHAPE


def test_batched_split_must_cover_nd_exactly(lib):
    """nd_per_mol must split the nd densities exactly, with no zero or negative
    count; a split that runs past nd is refused before d is read beyond it."""
    f, _ = _one()
    fa = (jk.jk_factor * 2)(f, f)
    d = (jk.jk_density * 2)()
    for s in range(2):
        d[s].k, d[s].symmetric, d[s].X, d[s].Y = 3, 0, 0x2000, 0x3000
    nb = ct.c_size_t()
    cfg = jk.jk_tune_config()
    for split, nd, want in [((1, 1), 2, jk.JK_OK), ((1, 2), 2, jk.JK_ERR_SHAPE), ((2, 1), 2, jk.JK_ERR_SHAPE),
                            ((1, 1), 1, jk.JK_ERR_SHAPE), ((0, 2), 2, jk.JK_ERR_SHAPE), ((-1, 3), 2, jk.JK_ERR_SHAPE),
                            ((1, 1), 3, jk.JK_ERR_SHAPE)]:
        ndm = (ct.c_int32 * 2)(*split)
        assert lib.jk_workspace_query(jk.JK_OP_BATCHED, 2, fa, ndm, nd, d, jk.JK_FP64, ct.byref(nb)) == want
        got = lib.jk_tune_lookup(jk.JK_OP_BATCHED, 2, fa, ndm, nd, d, jk.JK_FP64, 148, ct.byref(cfg))
        assert got == (jk.JK_ERR_UNSUPPORTED if want == jk.JK_OK else want)


def test_create_rejects_bad_arena(lib):
    h = ct.c_void_p()
    assert lib.jk_create(None, None, 0) == jk.JK_ERR_ARG
    assert lib.jk_create(ct.byref(h), None, 1 << 20) == jk.JK_ERR_ARG
    assert lib.jk_create(ct.byref(h), ct.c_void_p(0x1001), 1 << 20) == jk.JK_ERR_ARG
    assert not h.value


def test_calls_on_null_handle(lib):
    f, d = _one()
    assert lib.jk_build(None, ct.byref(f), 1, d, None, None, 0, None) == jk.JK_ERR_ARG
    assert lib.jk_adjoint(None, ct.byref(f), 1, d, None, None, None, None, None, 0, None) == jk.JK_ERR_ARG
    assert lib.jk_sync_status(None, None) == jk.JK_ERR_ARG
    assert lib.jk_last_error(None) == b""


def test_host_build_query_is_staging_plus_one_chunk(lib):
    """JK_OP_BUILD_HOST: two staging chunks of the factor and the device copies
    of densities and outputs, plus one chunk's build; less than the resident
    build for a factor much larger than its chunks, and growing with nbf."""
    nb_host, nb_dev = ct.c_size_t(), ct.c_size_t()
    f, d = _one(n=400, naux=2400, k=40)
    fa = (jk.jk_factor * 1)(f)
    for p in (jk.JK_FP64, jk.JK_SPLIT_BF16):
        assert lib.jk_workspace_query(jk.JK_OP_BUILD_HOST, 1, fa, None, 1, d, p, ct.byref(nb_host)) == jk.JK_OK
        assert lib.jk_workspace_query(jk.JK_OP_BUILD, 1, fa, None, 1, d, p, ct.byref(nb_dev)) == jk.JK_OK
        # at least the two staging buffers of ~naux/12 aux indices each
        assert nb_host.value >= 2 * (2400 // 12) * 400 * 400 * 8
        if p == jk.JK_SPLIT_BF16:
            assert nb_host.value < nb_dev.value + 2 * (2400 // 12 + 1) * 400 * 400 * 8
    f2, d2 = _one(n=200, naux=2400, k=40)
    fa2 = (jk.jk_factor * 1)(f2)
    assert lib.jk_workspace_query(jk.JK_OP_BUILD_HOST, 1, fa2, None, 1, d2, jk.JK_FP64, ct.byref(nb_dev)) == jk.JK_OK
    assert nb_dev.value < nb_host.value
    assert lib.jk_build_host(None, ct.byref(f), 1, d, None, None, 0, None) == jk.JK_ERR_ARG


def test_headers_are_c99_and_link(lib, tmp_path):
    """The ABI is plain C: a C99 program including both headers compiles with
    -pedantic -Werror, links against libjk.so and makes a host-only call."""
    import subprocess
    src = tmp_path / "t.c"
    src.write_text(
        '#include <stdio.h>\n#include "jk.h"\n#include "jk_debug.h"\n'
        "int main(void) {\n"
        "    jk_factor f = {10, 7, (const double *)0x1000};\n"
        "    jk_density d = {3, 0, (const double *)0x2000, (const double *)0x3000};\n"
        "    size_t b = 0;\n"
        "    jk_status s = jk_workspace_query(JK_OP_BUILD, 1, &f, NULL, 1, &d, JK_FP64, &b);\n"
        '    printf("%s\\n", jk_status_string(s));\n'
        "    return s == JK_OK && b > 0 ? 0 : 1;\n}\n")
    libdir = os.path.dirname(jk.LIB_PATH)
    exe = tmp_path / "t"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(src), "-L", libdir, "-ljk", f"-Wl,-rpath,{libdir}", "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "ok"


def test_noalloc_host_checks(lib):
    """jk_build_noalloc refuses bad arguments and oversize problems before any
    CUDA call, so these need no device (pointers are never dereferenced)."""
    lib.jk_build_noalloc.argtypes = [ct.POINTER(jk.jk_factor), ct.c_int32, ct.POINTER(jk.jk_density),
                                     ct.c_void_p, ct.c_void_p, ct.c_void_p]
    lib.jk_build_noalloc.restype = ct.c_int
    J, K = ct.c_void_p(0x10000), ct.c_void_p(0x20000)

    def call(n=10, naux=7, k=3, nd=1, L=0x1000, X=0x2000, J=J, K=K):
        f = jk.jk_factor(n, naux, L)
        d = (jk.jk_density * max(nd, 1))()
        for s in range(max(nd, 1)):
            d[s].k, d[s].symmetric, d[s].X, d[s].Y = k, 0, X, 0x3000
        return lib.jk_build_noalloc(ct.byref(f), nd, d, J, K, None)

    assert call(J=None, K=None) == jk.JK_OK                  # nothing to form
    assert lib.jk_build_noalloc(None, 1, None, J, K, None) == jk.JK_ERR_ARG
    for kw in [dict(n=0), dict(n=65536), dict(naux=0), dict(nd=0), dict(nd=65), dict(k=0), dict(k=41),
               dict(n=65535, k=32769)]:
        assert call(**kw) == jk.JK_ERR_SHAPE, kw
    for kw in [dict(L=0x1008), dict(X=0x2008), dict(J=ct.c_void_p(0x10008)), dict(K=ct.c_void_p(0x20008)),
               dict(L=0)]:
        assert call(**kw) == jk.JK_ERR_ARG, kw
    # panel buffer of naux * nbf * 2k doubles well above the static scratch
    assert call(n=160, naux=400, k=40) == jk.JK_ERR_OOM


def test_dense_query_host_only(lib):
    """JK_OP_BUILD_DENSE / JK_OP_DENSITY_GRAD: only f and nd are read (d may be
    NULL); the answer grows with nd and the gradient's covers J formed apart."""
    nb = ct.c_size_t()

    def q(op, n, naux, nd, p, f=None):
        fa = (jk.jk_factor * 1)(jk.jk_factor(n, naux, 0x1000)) if f is None else f
        st = lib.jk_workspace_query(op, 1, fa, None, nd, None, p, ct.byref(nb))
        return st, nb.value

    for p in (jk.JK_FP64, jk.JK_SPLIT_BF16):
        st1, b1 = q(jk.JK_OP_BUILD_DENSE, 100, 500, 1, p)
        st2, b2 = q(jk.JK_OP_BUILD_DENSE, 100, 500, 4, p)
        st3, b3 = q(jk.JK_OP_DENSITY_GRAD, 100, 500, 4, p)
        assert st1 == st2 == st3 == jk.JK_OK and 0 < b1 < b2 < b3
        # the gradient needs exactly one more [nd][n][n] block than the build
        assert b3 - b2 == 4 * 100 * 100 * 8
        for n, naux, nd in [(0, 5, 1), (5, 0, 1), (5, 5, 0), (5, 5, 65), (65536, 1, 1)]:
            assert q(jk.JK_OP_BUILD_DENSE, n, naux, nd, p)[0] == jk.JK_ERR_SHAPE
    assert lib.jk_workspace_query(jk.JK_OP_BUILD_DENSE, 1, None, None, 1, None, jk.JK_FP64, ct.byref(nb)) == jk.JK_ERR_ARG
    # the factored ops still need their densities
    fa = (jk.jk_factor * 1)(jk.jk_factor(10, 7, 0x1000))
    assert lib.jk_workspace_query(jk.JK_OP_BUILD, 1, fa, None, 1, None, jk.JK_FP64, ct.byref(nb)) == jk.JK_ERR_ARG


def test_dense_calls_on_null_handle(lib):
    f = jk.jk_factor(10, 7, 0x1000)
    D = ct.c_void_p(0x2000)
    assert lib.jk_build_dense(None, ct.byref(f), 1, D, D, D, 0, None) == jk.JK_ERR_ARG
    assert lib.jk_density_grad(None, ct.byref(f), 1, D, D, D, 0, None) == jk.JK_ERR_ARG


def test_pair_query_host_only(lib):
    """JK_OP_PAIR: nmol = 2, nd_per_mol = {nl, nr}, d = left then right, one
    factor; the answer grows with the right count (their J, K are built)."""
    nb = ct.c_size_t()
    fa = (jk.jk_factor * 1)(jk.jk_factor(100, 500, 0x1000))
    d = (jk.jk_density * 8)()
    for s in range(8):
        d[s].k, d[s].symmetric, d[s].X, d[s].Y = 10, s % 2, 0x2000, 0x3000

    def q(nmol, split, nd, p=jk.JK_FP64):
        ndm = (ct.c_int32 * len(split))(*split)
        return lib.jk_workspace_query(jk.JK_OP_PAIR, nmol, fa, ndm, nd, d, p, ct.byref(nb)), nb.value

    st1, b1 = q(2, (4, 2), 6)
    st2, b2 = q(2, (4, 4), 8)
    assert st1 == st2 == jk.JK_OK and 0 < b1 < b2
    assert q(2, (4, 4), 8, jk.JK_SPLIT_BF16)[0] == jk.JK_OK
    for nmol, split, nd in [(1, (4, 4), 8), (3, (4, 2, 2), 8), (2, (4, 4), 7), (2, (0, 4), 4), (2, (6, 4), 8)]:
        assert q(nmol, split, nd)[0] == jk.JK_ERR_SHAPE, (nmol, split, nd)


def test_pair_call_on_null_handle(lib):
    f = jk.jk_factor(10, 7, 0x1000)
    d = (jk.jk_density * 1)()
    d[0].k, d[0].symmetric, d[0].X, d[0].Y = 3, 0, 0x2000, 0x3000
    assert lib.jk_pair(None, ct.byref(f), 1, d, 1, d, None, None, 0, None) == jk.JK_ERR_ARG


def test_laplace_query_and_checks(lib):
    """JK_OP_LAPLACE: nd = nq points, d[0] gives m and symmetry; the
    non-symmetric form needs more (two scaled coefficient sets)."""
    nb = ct.c_size_t()
    fa = (jk.jk_factor * 1)(jk.jk_factor(100, 500, 0x1000))
    d = (jk.jk_density * 1)()
    d[0].k, d[0].symmetric = 10, 1
    assert lib.jk_workspace_query(jk.JK_OP_LAPLACE, 1, fa, None, 6, d, jk.JK_FP64, ct.byref(nb)) == jk.JK_OK
    b_sym = nb.value
    d[0].symmetric = 0
    assert lib.jk_workspace_query(jk.JK_OP_LAPLACE, 1, fa, None, 6, d, jk.JK_FP64, ct.byref(nb)) == jk.JK_OK
    assert nb.value > b_sym
    for nq, k in [(0, 10), (65, 10), (6, 0), (6, 401)]:
        d[0].k = k
        assert lib.jk_workspace_query(jk.JK_OP_LAPLACE, 1, fa, None, nq, d, jk.JK_FP64, ct.byref(nb)) == jk.JK_ERR_SHAPE
    f = jk.jk_factor(10, 7, 0x1000)
    a = (ct.c_double * 2)(0.5, 1.0)
    assert lib.jk_build_laplace(None, ct.byref(f), 2, a, None, 3, 0x2000, 0x3000, 1, None, None, 0,
                                0x4000, 0x5000, 0, None) == jk.JK_ERR_ARG


def test_packed_host_query(lib):
    """JK_OP_BUILD_HOST_PACKED adds the two packed staging chunks to the host
    build's workspace."""
    nb_full, nb_packed = ct.c_size_t(), ct.c_size_t()
    f, d = _one(n=100, naux=600, k=10)
    fa = (jk.jk_factor * 1)(f)
    for p in (jk.JK_FP64, jk.JK_SPLIT_BF16):
        assert lib.jk_workspace_query(jk.JK_OP_BUILD_HOST, 1, fa, None, 1, d, p, ct.byref(nb_full)) == jk.JK_OK
        assert lib.jk_workspace_query(jk.JK_OP_BUILD_HOST_PACKED, 1, fa, None, 1, d, p, ct.byref(nb_packed)) == jk.JK_OK
        chunk = (600 + 11) // 12
        assert nb_packed.value - nb_full.value >= 2 * chunk * (100 * 101 // 2) * 8
    assert lib.jk_build_host_packed(None, ct.byref(f), 1, d, None, None, 0, None) == jk.JK_ERR_ARG


def test_binding_constants_match_the_header():
    """The binding's option, operation, status and precision codes (and the host
    simulation's option table) are the values include/jk.h declares."""
    hdr = open(os.path.join(ROOT, "include", "jk.h")).read()
    enum = {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(JK_[A-Z0-9_]+)\s*=\s*(\d+)", hdr)}
    for name, code in jk.OPTIONS.items():
        assert enum["JK_OPT_" + name.upper()] == code, name
    assert {k for k in enum if k.startswith("JK_OPT_")} == {"JK_OPT_" + k.upper() for k in jk.OPTIONS}
    for name in ("JK_OK", "JK_ERR_ARG", "JK_ERR_SHAPE", "JK_ERR_OOM", "JK_ERR_CUDA", "JK_ERR_TIMEOUT",
                 "JK_ERR_UNSUPPORTED", "JK_FP64", "JK_SPLIT_BF16", "JK_OP_BUILD", "JK_OP_ADJOINT", "JK_OP_BATCHED",
                 "JK_OP_BUILD_HOST", "JK_OP_BUILD_DENSE", "JK_OP_DENSITY_GRAD", "JK_OP_PAIR", "JK_OP_LAPLACE",
                 "JK_OP_BUILD_HOST_PACKED"):
        assert getattr(jk, name) == enum[name], name
    sim = open(os.path.join(ROOT, "tests", "hostsim", "drive.py")).read()
    table = sim.split("OPT = {", 1)[1].split("}", 1)[0]
    assert {k: int(v) for k, v in re.findall(r'"(\w+)": (\d+)', table)} == jk.OPTIONS
