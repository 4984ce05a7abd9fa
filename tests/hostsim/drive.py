"""Child process of tests/test_hostsim.py (TEST INFRASTRUCTURE): drives every
entry point of libjk.so on host memory while the CUDA runtime is the
recording stand-in (cudart_shim.c, first on LD_LIBRARY_PATH), and prints one
JSON object per case: the status, the recorded launches and tensor maps, and
the memory ranges the call owns.  It must not import torch (torch would load
the real runtime first).  Kernels do not run; values are not checked."""
import ctypes as ct
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


class jk_factor(ct.Structure):
    _fields_ = [("nbf", ct.c_int32), ("naux", ct.c_int32), ("L", ct.c_void_p)]


class jk_density(ct.Structure):
    _fields_ = [("k", ct.c_int32), ("symmetric", ct.c_int32), ("X", ct.c_void_p), ("Y", ct.c_void_p)]


class jk_tune_config(ct.Structure):
    _fields_ = [("aux_chunk", ct.c_int32), ("schedule", ct.c_int32), ("raster", ct.c_int32), ("tile", ct.c_int32)]


_lib = ct.CDLL(os.path.join(ROOT, "paper_2608_06536_b300", "libjk.so"))
_lib.jk_last_error.restype = ct.c_char_p
ENTRIES = {"jk_build", "jk_build_batched", "jk_build_host", "jk_build_host_packed", "jk_adjoint", "jk_build_dense",
           "jk_density_grad", "jk_pair", "jk_build_laplace", "jk_build_noalloc", "jk_autotune", "jk_autotune_batched",
           "jk_debug_sliced_gemm"}
TWICE = [False]       # call each entry point twice on its handle and record only the second call
FAIL_AT = [-1]        # make this launch of the first call fail, then call again (--fail-launch=N)
FIRST = {}            # status and message of that failed first call


class _Lib:
    """The library; with TWICE set, an entry point runs once untraced (the
    eager call that does any one-time set-up) and then once traced."""

    def __getattr__(self, name):
        fn = getattr(_lib, name)
        if name not in ENTRIES:
            return fn

        def call(*args):
            if FAIL_AT[0] >= 0:
                shim.shim_fail_launch_at(FAIL_AT[0])
                st = fn(*args)
                shim.shim_fail_launch_at(-1)
                h = args[0] if name != "jk_build_noalloc" else None
                FIRST.update(status=st, error=_lib.jk_last_error(h).decode() if h else "")
                shim.shim_reset()
                violations.clear()
                decoded[0] = 0
            if TWICE[0]:
                st = fn(*args)
                if st != 0:
                    return st
                shim.shim_reset()
                violations.clear()
                decoded[0] = 0
            return fn(*args)
        return call


lib = _Lib()
shim = ct.CDLL("libcudart.so.13")
shim.shim_launch.restype = ct.c_char_p
assert hasattr(shim, "shim_reset"), "the stand-in runtime is not the one loaded"

OPT = {"aux_chunk": 0, "schedule": 1, "raster": 2, "use_tuned": 3, "host_chunk": 5, "slicer": 6,
       "syrk": 7, "packed_factor": 8, "tile": 9, "adjoint_slices": 10, "j_path": 11}

# ---- kernel arguments ----------------------------------------------------------
# Each decoder reads one kernel's arguments (layouts as in the CUDA sources)
# and returns the byte ranges [lo, hi) its pointer arguments can touch, from
# the kernel's own index bounds; every range must lie in memory the call owns.
VP, I32, I64, F64 = ct.c_void_p, ct.c_int32, ct.c_int64, ct.c_double
SUPER, MAXD = 2048, 64


def _slices_of(name):
    """Slices per operand of a slicer launch, from its template argument."""
    return 7 if "ILi7E" in name else 6


class Src(ct.Structure):
    _fields_ = [("p", VP), ("sr", I64), ("sko", I64), ("ski", I64), ("kin", I32), ("rin", I32), ("sri", I64)]


class SliceJob(ct.Structure):
    _fields_ = [("src", Src), ("e", VP), ("out", VP), ("sstride", I64), ("rows", I32), ("K", I32), ("Kpad", I32),
                ("rpe", I32), ("nsc", I32), ("vec", I32), ("flat", I32), ("eb0", I32), ("sb0", I32), ("nbx", I32),
                ("nby", I32)]


class SliceGroup(ct.Structure):
    _fields_ = [("j", SliceJob * 200), ("njob", I32)]


class PanelSeg(ct.Structure):
    _fields_ = [("e", VP), ("c0", I32), ("k", I32), ("nsc", I32), ("n", I32)]


class PanelItem(ct.Structure):
    _fields_ = [("T", VP), ("ldT", I64), ("n", I32), ("rows", I32), ("seg0", I32), ("nseg", I32), ("b0", I32),
                ("rpb", I32), ("lanes", I32)]


class PanelExpo(ct.Structure):
    _fields_ = [("nitem", I32), ("nseg", I32), ("it", PanelItem * 64), ("s", PanelSeg * 800)]


class ReduceJob(ct.Structure):
    _fields_ = [("P", VP), ("pz", I64), ("ldp", I64), ("eA", VP), ("eB", VP), ("out", VP), ("ldo", I64), ("e0", I64),
                ("nz", I32), ("M", I32), ("N", I32), ("arpe", I32), ("brpe", I32), ("accumulate", I32), ("frac", I32)]


class ReduceGroup(ct.Structure):
    _fields_ = [("j", ReduceJob * 240), ("njob", I32)]


class PackJob(ct.Structure):
    _fields_ = [("src", VP), ("Z", VP), ("e0", I64), ("n", I32), ("k", I32), ("ctot", I32), ("off", I32)]


class PackGroup(ct.Structure):
    _fields_ = [("j", PackJob * 600), ("njob", I32)]


class GOp(ct.Structure):
    _fields_ = [("p", VP), ("sb", I64), ("sr", I64), ("sko", I64), ("ski", I64), ("kin", I32)]


class DensTab(ct.Structure):
    _fields_ = [("Y", VP * MAXD), ("offX", I32 * MAXD), ("k", I32 * MAXD)]


class OutTab(ct.Structure):
    _fields_ = [("p", VP * 8)]


class JOut(ct.Structure):
    _fields_ = [("p", VP * 64)]


class GammaJob(ct.Structure):
    _fields_ = [("T", VP), ("gamma", VP), ("ldT", I64), ("n", I32), ("np", I32), ("nd", I32), ("P0", I32),
                ("ldg", I32), ("d0", I32), ("b0", I32)]


class GammaGroup(ct.Structure):
    _fields_ = [("j", GammaJob * 64), ("Y", VP * 1024), ("offX", I32 * 1024), ("k", I32 * 1024), ("njob", I32)]


class TriJob(ct.Structure):
    _fields_ = [("L", VP), ("pstride", I64), ("e", VP), ("out", VP), ("ss4", I64), ("n", I32), ("P0", I32),
                ("np", I32), ("Kpad", I32), ("nsc", I32), ("pk", I32), ("ebx", I32), ("sbx", I32), ("sby", I32),
                ("eb0", I32), ("sb0", I32)]


class TriGroup(ct.Structure):
    _fields_ = [("j", TriJob * 64), ("njob", I32)]


class JAddJob(ct.Structure):
    _fields_ = [("C", VP), ("ldc", I64), ("e0", I64), ("n", I32), ("nd", I32), ("acc", I32), ("p0", I32)]


class JAddGroup(ct.Structure):
    _fields_ = [("j", JAddJob * 64), ("ptr", VP * 1024), ("njob", I32)]


class PairTab(ct.Structure):
    _fields_ = [("offA", I32 * MAXD), ("offB", I32 * MAXD), ("k", I32 * MAXD)]


class OzArgs(ct.Structure):
    _fields_ = [("M", I32), ("N", I32), ("K", I32), ("nsuper", I32), ("eA", VP), ("a_rpe", I32), ("eB", VP),
                ("b_rpe", I32), ("C", VP), ("ldc", I64), ("P", VP), ("pz", I64), ("ldp", I64),
                ("use_tma_store", I32), ("err", VP)]


class OzTail(ct.Structure):
    _fields_ = [("tile0", I32), ("ntn", I32), ("ntm", I32), ("cfg", I32)]


# one problem of a grouped launch: three 128-byte tensor maps (A, B, C), its
# arguments, its tile counts; 64-byte aligned (the maps' alignment)
OZ_ARGS_OFF = 3 * 128
OZ_PROB_BYTES = (OZ_ARGS_OFF + ct.sizeof(OzArgs) + ct.sizeof(OzTail) + 63) // 64 * 64
OZ_BM = 128
# slice configurations of the sliced GEMM: id -> (slices, tile width, fraction bits)
OZ_CFG = {0: (6, 80, 48), 1: (6, 64, 48), 2: (7, 64, 51)}


def _a(args, i, t):
    return t.from_address(args[i])


def _v(args, i, t):
    return t.from_address(args[i]).value


def _lin_max(n, inner, s_out, s_in):
    """max over idx < n of (idx // inner) * s_out + (idx % inner) * s_in (strides >= 0)."""
    if n <= 0:
        return 0
    q, r = divmod(n - 1, inner)
    best = q * s_out + r * s_in
    if q > 0:
        best = max(best, (q - 1) * s_out + (inner - 1) * s_in)
    return best


def _src_range(src, rows, K, esize=8):
    assert min(src.sr, src.sko, src.ski, src.sri) >= 0, "negative stride"
    hi = _lin_max(rows, src.rin, src.sr, src.sri) + _lin_max(K, src.kin, src.sko, src.ski)
    return (src.p, src.p + (hi + 1) * esize, "src")


def _gop_range(g, batch, rows, K):
    assert min(g.sb, g.sr, g.sko, g.ski) >= 0, "negative stride"
    hi = (batch - 1) * g.sb + (rows - 1) * g.sr + _lin_max(K, g.kin, g.sko, g.ski)
    return (g.p, g.p + (hi + 1) * 8, "gop")


def dec_expo(grid, args):
    src, rows, K, rpe, e = _a(args, 0, Src), _v(args, 1, I32), _v(args, 2, I32), _v(args, 3, I32), _v(args, 4, VP)
    assert (grid[0] - 1) * rpe < rows <= grid[0] * rpe and grid[1] == (K + SUPER - 1) // SUPER, (grid, rows, K)
    return [_src_range(src, rows, K), (e, e + 4 * grid[0] * grid[1], "e")]


def dec_expo_flat(grid, args):
    p, ln, e = _v(args, 0, VP), _v(args, 1, I64), _v(args, 2, VP)
    assert ln >= 1 and p % 8 == 0
    return [(p, p + 8 * grid[0] * ln, "p"), (e, e + 4 * grid[0], "e")]


def _slice(grid, args, esize_out, per, nslice):
    src, rows, K, Kpad = _a(args, 0, Src), _v(args, 1, I32), _v(args, 2, I32), _v(args, 3, I32)
    e, rpe, nsc, out, ss = _v(args, 4, VP), _v(args, 5, I32), _v(args, 6, I32), _v(args, 7, VP), _v(args, 8, I64)
    assert grid[0] * 256 * per >= Kpad and Kpad % 16 == 0 and K <= Kpad
    ne = ((rows - 1) // rpe) * nsc + (K - 1) // SUPER + 1
    nout = (nslice - 1) * ss + (rows * Kpad) // per
    return [_src_range(src, rows, K), (e, e + 4 * ne, "e"), (out, out + esize_out * nout, "slices")]


def dec_slice(grid, args, name):
    return _slice(grid, args, 8, 4, _slices_of(name))


def dec_slice4(grid, args, name):
    src = _a(args, 0, Src)
    assert src.ski == 1 and src.kin % 4 == 0 and _v(args, 2, I32) % 4 == 0 and src.p % 16 == 0
    return _slice(grid, args, 8, 4, _slices_of(name))


def _group_jobs(g, key, blocks_of):
    """The jobs of a grouped launch, checked to tile the launch's blocks in order."""
    assert 1 <= g.njob <= len(g.j), g.njob
    b = 0
    for i in range(g.njob):
        jb = g.j[i]
        assert getattr(jb, key) == b, (i, getattr(jb, key), b)
        b += blocks_of(jb)
    return [g.j[i] for i in range(g.njob)], b


def _expo_blocks(jb):
    groups = (jb.rows - 1) // jb.rpe + 1
    return groups if jb.flat else groups * jb.nsc


def dec_expo_group(grid, args):
    jobs, nb = _group_jobs(SliceGroup.from_address(args[0]), "eb0", _expo_blocks)
    assert grid[0] == nb, (grid, nb)
    res = []
    for jb in jobs:
        assert jb.nsc == (jb.K + SUPER - 1) // SUPER and jb.Kpad % 16 == 0 and jb.K <= jb.Kpad
        groups = (jb.rows - 1) // jb.rpe + 1
        if jb.flat:
            # contiguous runs of rpe * K doubles (any alignment and parity)
            assert jb.nsc == 1 and jb.src.p % 8 == 0 and jb.rows % jb.rpe == 0
            assert jb.src.rin == 1 and jb.src.ski == 1 and jb.src.kin == jb.K and jb.src.sr == jb.K
        res += [_src_range(jb.src, jb.rows, jb.K), (jb.e, jb.e + 4 * groups * jb.nsc, "e")]
    return res


def _panel_items(g):
    """The panels of a row-wise exponent launch, checked to tile its blocks and
    its segments in order."""
    assert 1 <= g.nitem <= 64 and 1 <= g.nseg <= 800, (g.nitem, g.nseg)
    b = seg = 0
    out = []
    for i in range(g.nitem):
        pi = g.it[i]
        assert pi.b0 == b and pi.seg0 == seg and pi.n >= 1 and pi.rows % pi.n == 0 and pi.nseg >= 1, (i, pi.b0, b)
        # rows per block, lane groups that tile a warp, the panel's operands
        # staged in the block's shared table
        assert 1 <= pi.rpb and pi.lanes in (4, 8, 16, 32) and pi.nseg <= 128, (pi.rpb, pi.lanes, pi.nseg)
        np_ = pi.rows // pi.n
        segs = [g.s[j] for j in range(pi.seg0, pi.seg0 + pi.nseg)]
        for sg in segs:
            assert sg.n == pi.n and 1 <= sg.k <= SUPER and sg.nsc == (np_ * sg.k + SUPER - 1) // SUPER
            assert sg.c0 >= 0 and sg.c0 + sg.k <= pi.ldT
        out.append((pi, segs))
        b += (pi.rows + pi.rpb - 1) // pi.rpb
        seg += pi.nseg
    assert seg == g.nseg
    return out, b


def dec_int_fill(grid, args):
    g = PanelExpo.from_address(args[0])
    items, _ = _panel_items(g)
    assert grid[1] == g.nseg
    return [(sg.e, sg.e + 4 * sg.n * sg.nsc, "e") for _, segs in items for sg in segs]


def dec_panel_colmax(grid, args):
    g = PanelExpo.from_address(args[0])
    items, nb = _panel_items(g)
    assert grid[0] == nb, (grid, nb)
    res = []
    for pi, segs in items:
        res.append((pi.T, pi.T + 8 * ((pi.rows - 1) * pi.ldT + max(sg.c0 + sg.k for sg in segs)), "T"))
        res += [(sg.e, sg.e + 4 * sg.n * sg.nsc, "e") for sg in segs]
    return res


def dec_slice_group(grid, args, name):
    jobs, nb = _group_jobs(SliceGroup.from_address(args[0]), "sb0", lambda jb: jb.nbx * jb.nby)
    assert grid[0] == nb, (grid, nb)
    nslice = _slices_of(name)
    res = []
    for jb in jobs:
        per, esize = 4, 8   # four BF16 values per 8-byte word
        if jb.vec:
            assert jb.src.ski == 1 and jb.src.kin % 4 == 0 and jb.K % 4 == 0 and jb.src.p % 16 == 0
        assert jb.nbx * 256 * per >= jb.Kpad and jb.nby >= 1 and jb.sstride * per == jb.rows * jb.Kpad
        ne = ((jb.rows - 1) // jb.rpe) * jb.nsc + (jb.K - 1) // SUPER + 1
        nout = (nslice - 1) * jb.sstride + (jb.rows * jb.Kpad) // per
        res += [_src_range(jb.src, jb.rows, jb.K), (jb.e, jb.e + 4 * ne, "e"), (jb.out, jb.out + esize * nout, "slices")]
    return res


def dec_reduce_group(grid, args):
    g = ReduceGroup.from_address(args[0])
    total = _v(args, 1, I64)
    jobs, nel = _group_jobs(g, "e0", lambda jb: jb.M * jb.N)
    assert nel == total and grid[0] * 256 >= total, (grid, total, nel)
    res = []
    for jb in jobs:
        assert jb.frac in (48, 51)
        res += [(jb.P, jb.P + 8 * ((jb.nz - 1) * jb.pz + (jb.M - 1) * jb.ldp + jb.N), "P"),
                (jb.eA, jb.eA + 4 * ((jb.M - 1) // jb.arpe + 1) * jb.nz, "eA"),
                (jb.eB, jb.eB + 4 * ((jb.N - 1) // jb.brpe + 1) * jb.nz, "eB"),
                (jb.out, jb.out + 8 * ((jb.M - 1) * jb.ldo + jb.N), "out")]
    return res


def dec_dgemm(grid, args):
    M, N, K = _v(args, 0, I32), _v(args, 1, I32), _v(args, 2, I32)
    A, B, C, ldc, scb = _a(args, 3, GOp), _a(args, 4, GOp), _v(args, 5, VP), _v(args, 6, I64), _v(args, 7, I64)
    nb = grid[2]
    assert grid[0] * 64 >= N and grid[1] * 64 >= M
    return [_gop_range(A, nb, M, K), _gop_range(B, nb, N, K),
            (C, C + 8 * ((nb - 1) * scb + (M - 1) * ldc + N), "C")]


def dec_pack_cols(grid, args):
    src, n, k, Z, ctot, off = (_v(args, 0, VP), _v(args, 1, I32), _v(args, 2, I32), _v(args, 3, VP),
                               _v(args, 4, I32), _v(args, 5, I32))
    assert off + k <= ctot
    return [(src, src + 8 * n * k, "src"), (Z, Z + 8 * ((n - 1) * ctot + off + k), "Z")]


def dec_pack_group(grid, args):
    total = _v(args, 1, I64)
    jobs, nel = _group_jobs(PackGroup.from_address(args[0]), "e0", lambda jb: jb.n * jb.k)
    assert nel == total and grid[0] * 256 >= total, (grid, total, nel)
    res = []
    for jb in jobs:
        assert jb.off + jb.k <= jb.ctot
        res += [(jb.src, jb.src + 8 * jb.n * jb.k, "src"), (jb.Z, jb.Z + 8 * ((jb.n - 1) * jb.ctot + jb.off + jb.k), "Z")]
    return res


def dec_frob(grid, args):
    L, n2, M, nd, g, ldg, P0 = (_v(args, 0, VP), _v(args, 1, I64), _v(args, 2, VP), _v(args, 3, I32),
                                _v(args, 4, VP), _v(args, 5, I32), _v(args, 6, I32))
    assert grid[1] == (nd + 3) // 4
    return [(L, L + 8 * (P0 + grid[0]) * n2, "L"), (M, M + 8 * nd * n2, "Mats"),
            (g, g + 8 * ((nd - 1) * ldg + P0 + grid[0]), "gamma")]


def dec_frob_packed(grid, args):
    L, n, M, nd, g, ldg, P0 = (_v(args, 0, VP), _v(args, 1, I32), _v(args, 2, VP), _v(args, 3, I32),
                               _v(args, 4, VP), _v(args, 5, I32), _v(args, 6, I32))
    assert grid[1] == (nd + 3) // 4
    return [(L, L + 8 * (P0 + grid[0]) * (n * (n + 1) // 2), "L"), (M, M + 8 * nd * n * n, "Mats"),
            (g, g + 8 * ((nd - 1) * ldg + P0 + grid[0]), "gamma")]


def dec_gamma_panel(grid, args):
    T, n, ctot, tab, g, ldg, P0 = (_v(args, 0, VP), _v(args, 1, I32), _v(args, 2, I64), _a(args, 3, DensTab),
                                   _v(args, 4, VP), _v(args, 5, I32), _v(args, 6, I32))
    np_, nd = grid[0], grid[1]
    out = [(g, g + 8 * ((nd - 1) * ldg + P0 + np_), "gamma")]
    for s in range(nd):
        k, off = tab.k[s], tab.offX[s]
        assert off + k <= ctot
        out.append((T, T + 8 * ((np_ - 1) * n * ctot + (n - 1) * ctot + off + k), "T"))
        out.append((tab.Y[s], tab.Y[s] + 8 * n * k, "Y"))
    return out


def dec_gamma_group(grid, args):
    g = GammaGroup.from_address(args[0])
    jobs, nb = _group_jobs(g, "b0", lambda jb: jb.np * jb.nd)
    assert grid[0] == nb, (grid, nb)
    out, d = [], 0
    for jb in jobs:
        assert jb.d0 == d and jb.nd >= 1 and jb.np >= 1 and d + jb.nd <= 1024, (jb.d0, d)
        out.append((jb.gamma, jb.gamma + 8 * ((jb.nd - 1) * jb.ldg + jb.P0 + jb.np), "gamma"))
        for s in range(jb.nd):
            k, off = g.k[d + s], g.offX[d + s]
            assert off + k <= jb.ldT
            out.append((jb.T, jb.T + 8 * ((jb.np - 1) * jb.n * jb.ldT + (jb.n - 1) * jb.ldT + off + k), "T"))
            out.append((g.Y[d + s], g.Y[d + s] + 8 * jb.n * k, "Y"))
        d += jb.nd
    return out


def _jstream_args(args):
    return (_v(args, 0, VP), _v(args, 1, I32), _v(args, 2, I32), _v(args, 3, I32), _v(args, 4, VP),
            _v(args, 5, I32), _v(args, 6, I32), _a(args, 7, OutTab))


def dec_jstream_sym(grid, args, name):
    ns = int(name.split("ILi")[1].split("E")[0])
    L, n, P0, np_, g, ldg, acc, o = _jstream_args(args)
    assert grid[0] * 64 >= n * (n + 1) // 2 and P0 >= 0 and np_ >= 1 and acc in (0, 1)
    per = n * (n + 1) // 2 if "Lb1E" in name else n * n          # packed factor: upper triangles
    out = [(L + 8 * P0 * per, L + 8 * (P0 + np_) * per, "L"), (g, g + 8 * ((ns - 1) * ldg + P0 + np_), "g")]
    out += [(o.p[j], o.p[j] + 8 * n * n, "J") for j in range(ns)]
    return out


def _tri_args(args, name):
    """(packed?, L, n, pstride, P0, np) of a transposed-factor slicing launch."""
    pk = "ILb1E" in name
    L, n, ps, P0, np_ = _v(args, 0, VP), _v(args, 1, I32), _v(args, 2, I64), _v(args, 3, I32), _v(args, 4, I32)
    ntri = n * (n + 1) // 2
    assert ps == (ntri if pk else n * n) and P0 >= 0 and np_ >= 1, (pk, ps, n, P0, np_)
    return pk, L, n, ps, P0, np_, ntri


def dec_expo_tri(grid, args, name):
    pk, L, n, ps, P0, np_, ntri = _tri_args(args, name)
    nsc, e = _v(args, 5, I32), _v(args, 6, VP)
    assert nsc == (np_ + SUPER - 1) // SUPER and grid[1] == nsc and grid[0] * 256 >= ntri, (grid, nsc, ntri)
    return [(L + 8 * P0 * ps, L + 8 * (P0 + np_) * ps, "L"), (e, e + 4 * ntri * nsc, "e")]


TRI_TT, TRI_TK = 128, 32  # the transposed slicer's tile (rows t, aux indices kk)


def dec_slice_tri(grid, args, name):
    pk, L, n, ps, P0, np_, ntri = _tri_args(args, name)
    Kpad, nsc, e, out, ss4 = _v(args, 5, I32), _v(args, 6, I32), _v(args, 7, VP), _v(args, 8, VP), _v(args, 9, I64)
    sby = _v(args, 10, I32)
    assert Kpad == (np_ + 15) // 16 * 16 and nsc == (np_ + SUPER - 1) // SUPER and ss4 * 4 == ntri * Kpad
    assert sby == -(-Kpad // TRI_TK) and grid[0] == -(-ntri // TRI_TT) * sby and grid[1] == 1 and out % 16 == 0, \
        (grid, ntri, Kpad, sby)
    return [(L + 8 * P0 * ps, L + 8 * (P0 + np_) * ps, "L"), (e, e + 4 * ntri * nsc, "e"),
            (out, out + 8 * 6 * ss4, "slices")]


def _tri_job_check(jb):
    ntri = jb.n * (jb.n + 1) // 2
    assert jb.pstride == (ntri if jb.pk else jb.n * jb.n) and jb.P0 >= 0 and jb.np >= 1, (jb.pk, jb.pstride)
    assert jb.Kpad == (jb.np + 15) // 16 * 16 and jb.nsc == (jb.np + SUPER - 1) // SUPER and jb.ss4 * 4 == ntri * jb.Kpad
    assert jb.ebx * 256 >= ntri and jb.sbx == -(-ntri // TRI_TT) and jb.sby == -(-jb.Kpad // TRI_TK) and jb.out % 16 == 0
    return ntri


def dec_expo_tri_group(grid, args):
    jobs, nb = _group_jobs(TriGroup.from_address(args[0]), "eb0", lambda jb: jb.ebx * jb.nsc)
    assert grid[0] == nb, (grid, nb)
    res = []
    for jb in jobs:
        ntri = _tri_job_check(jb)
        res += [(jb.L + 8 * jb.P0 * jb.pstride, jb.L + 8 * (jb.P0 + jb.np) * jb.pstride, "L"),
                (jb.e, jb.e + 4 * ntri * jb.nsc, "e")]
    return res


def dec_slice_tri_group(grid, args):
    jobs, nb = _group_jobs(TriGroup.from_address(args[0]), "sb0", lambda jb: jb.sbx * jb.sby)
    assert grid[0] == nb, (grid, nb)
    res = []
    for jb in jobs:
        ntri = _tri_job_check(jb)
        res += [(jb.L + 8 * jb.P0 * jb.pstride, jb.L + 8 * (jb.P0 + jb.np) * jb.pstride, "L"),
                (jb.e, jb.e + 4 * ntri * jb.nsc, "e"), (jb.out, jb.out + 8 * 6 * jb.ss4, "slices")]
    return res


def dec_j_tri_add_group(grid, args):
    g = JAddGroup.from_address(args[0])
    total = _v(args, 1, I64)
    jobs, nel = _group_jobs(g, "e0", lambda jb: jb.n * (jb.n + 1) // 2)
    assert nel == total and grid[0] * 256 >= total, (grid, total, nel)
    res, p = [], 0
    for jb in jobs:
        ntri = jb.n * (jb.n + 1) // 2
        assert jb.p0 == p and 1 <= jb.nd and jb.ldc >= jb.nd and jb.acc in (0, 1) and p + jb.nd <= 1024
        res.append((jb.C, jb.C + 8 * ((ntri - 1) * jb.ldc + jb.nd), "C"))
        res += [(g.ptr[p + s], g.ptr[p + s] + 8 * jb.n * jb.n, "J") for s in range(jb.nd)]
        p += jb.nd
    return res


def dec_j_tri_add(grid, args):
    C, ldc, n, nd, acc, jo = _v(args, 0, VP), _v(args, 1, I64), _v(args, 2, I32), _v(args, 3, I32), \
        _v(args, 4, I32), _a(args, 5, JOut)
    ntri = n * (n + 1) // 2
    assert 1 <= nd <= 64 and ldc >= nd and acc in (0, 1) and grid[0] * 256 >= ntri
    return [(C, C + 8 * ((ntri - 1) * ldc + nd), "C")] + [(jo.p[s], jo.p[s] + 8 * n * n, "J") for s in range(nd)]


def dec_axpy(grid, args):
    y, x, cnt = _v(args, 0, VP), _v(args, 1, VP), _v(args, 2, I64)
    return [(y, y + 8 * cnt, "y"), (x, x + 8 * cnt, "x")]


def dec_sum_parts_ld(grid, args):
    out, ldo, part, nb, M, N = (_v(args, 0, VP), _v(args, 1, I64), _v(args, 2, VP), _v(args, 3, I32),
                                _v(args, 4, I32), _v(args, 5, I32))
    assert grid[0] * 256 >= M * N and ldo >= N, (grid, M, N, ldo)
    return [(out, out + 8 * ((M - 1) * ldo + N), "out"), (part, part + 8 * nb * M * N, "part")]


def dec_pack_sym(grid, args):
    F, n, np_, P = _v(args, 0, VP), _v(args, 1, I32), _v(args, 2, I64), _v(args, 3, VP)
    tri = n * (n + 1) // 2
    assert grid[0] * 256 >= np_ * tri
    return [(F, F + 8 * np_ * n * n, "full"), (P, P + 8 * np_ * tri, "packed")]


def dec_mirror_blocks(grid, args):
    K, n, bm = _v(args, 0, VP), _v(args, 1, I32), _v(args, 2, I32)
    assert bm >= 1 and grid[0] * 256 >= n * n, (grid, n)
    return [(K, K + 8 * n * n, "K")]


def dec_sum_parts(grid, args):
    out, part, nb, cnt = _v(args, 0, VP), _v(args, 1, VP), _v(args, 2, I32), _v(args, 3, I64)
    return [(out, out + 8 * cnt, "out"), (part, part + 8 * nb * cnt, "part")]


def dec_reduce(grid, args):
    P, pz, ldp, nz, M, N = (_v(args, 0, VP), _v(args, 1, I64), _v(args, 2, I64), _v(args, 3, I32),
                            _v(args, 4, I32), _v(args, 5, I32))
    eA, arpe, eB, brpe, out, ldo = (_v(args, 6, VP), _v(args, 7, I32), _v(args, 8, VP), _v(args, 9, I32),
                                    _v(args, 10, VP), _v(args, 11, I64))
    return [(P, P + 8 * ((nz - 1) * pz + (M - 1) * ldp + N), "P"),
            (eA, eA + 4 * ((M - 1) // arpe + 1) * nz, "eA"), (eB, eB + 4 * ((N - 1) // brpe + 1) * nz, "eB"),
            (out, out + 8 * ((M - 1) * ldo + N), "out")]


def dec_pair_dot(grid, args):
    ZL, U, n, ctot, tab, out, nr = (_v(args, 0, VP), _v(args, 1, VP), _v(args, 2, I32), _v(args, 3, I32),
                                    _a(args, 4, PairTab), _v(args, 5, VP), _v(args, 6, I32))
    nl = grid[0]
    assert grid[1] == nr
    res = [(out, out + 8 * nl * nr, "out")]
    for a in range(nl):
        k = tab.k[a]
        assert tab.offA[a] + k <= ctot and tab.offB[a] + k <= ctot
        res.append((ZL, ZL + 8 * ((n - 1) * ctot + tab.offA[a] + k), "ZL"))
        res.append((U, U + 8 * ((nr - 1) * n * ctot + (n - 1) * ctot + tab.offB[a] + k), "U"))
    return res


def dec_laplace_scale(grid, args):
    C, eps, n, m, nq, out = (_v(args, 0, VP), _v(args, 1, VP), _v(args, 2, I32), _v(args, 3, I32),
                             _v(args, 6, I32), _v(args, 7, VP))
    assert grid[0] * 256 >= n * m * nq and 1 <= nq <= MAXD
    return [(C, C + 8 * n * m, "C"), (eps, eps + 8 * m, "eps"), (out, out + 8 * nq * n * m, "out")]


def dec_weighted_sum(grid, args):
    out, part, nq, cnt = _v(args, 0, VP), _v(args, 1, VP), _v(args, 3, I32), _v(args, 4, I64)
    assert 1 <= nq <= MAXD
    return [(out, out + 8 * cnt, "out"), (part, part + 8 * nq * cnt, "part")]


def dec_gterms(grid, args):
    G, n2, nd = _v(args, 0, VP), _v(args, 1, I64), _v(args, 3, I32)
    D, V, c, g, ldg, P0 = (_v(args, 4, VP), _v(args, 5, VP), _v(args, 6, VP), _v(args, 7, VP), _v(args, 8, I32),
                           _v(args, 9, I32))
    np_ = grid[1]
    res = [(G, G + 8 * np_ * n2, "G")]
    top = 8 * ((nd - 1) * ldg + P0 + np_)
    if D:
        res += [(D, D + 8 * nd * n2, "D"), (c, c + top, "c")]
    if V:
        res += [(V, V + 8 * nd * n2, "V"), (g, g + top, "g")]
    return res


def dec_symmetrize(grid, args):
    G, n, dL = _v(args, 0, VP), _v(args, 1, I32), _v(args, 2, VP)
    return [(G, G + 8 * grid[1] * n * n, "G"), (dL, dL + 8 * grid[1] * n * n, "dL")]


def dec_sym_dl(grid, args):
    G, GV, n, dL = _v(args, 0, VP), _v(args, 1, VP), _v(args, 2, I32), _v(args, 3, VP)
    nb = 8 * grid[1] * n * n
    res = [(G, G + nb, "G"), (dL, dL + nb, "dL")]
    if GV:
        res.append((GV, GV + nb, "GV"))
    return res


def dec_fold(grid, args):
    dX, dY, cnt = _v(args, 0, VP), _v(args, 1, VP), _v(args, 2, I64)
    return [(dX, dX + 8 * cnt, "dX"), (dY, dY + 8 * cnt, "dY")]


def dec_pack_ag(grid, args):
    AG, ldag, off, U, Vp, X, cps, P0, n, k, np_ = (
        _v(args, 0, VP), _v(args, 1, I64), _v(args, 2, I32), _v(args, 3, VP), _v(args, 4, VP), _v(args, 5, VP),
        _v(args, 6, VP), _v(args, 7, I32), _v(args, 8, I32), _v(args, 9, I32), _v(args, 10, I32))
    assert off + 3 * k <= ldag
    res = [(AG, AG + 8 * ((np_ * n - 1) * ldag + off + 3 * k), "AG")]
    for ptr_, what in ((U, "U"), (Vp, "Vp")):
        if ptr_:
            res.append((ptr_, ptr_ + 8 * n * np_ * k, what))
    if cps:
        res += [(cps, cps + 8 * (P0 + np_), "cps"), (X, X + 8 * n * k, "X")]
    return res


def dec_pack_bg(grid, args):
    BG, ldbg, off, X, Y, n, k = (_v(args, 0, VP), _v(args, 1, I64), _v(args, 2, I32), _v(args, 3, VP),
                                 _v(args, 4, VP), _v(args, 5, I32), _v(args, 6, I32))
    assert off + 3 * k <= ldbg
    return [(BG, BG + 8 * ((n - 1) * ldbg + off + 3 * k), "BG"), (X, X + 8 * n * k, "X"), (Y, Y + 8 * n * k, "Y")]


def dec_unpack_sym(grid, args):
    P, n, np_, F = _v(args, 0, VP), _v(args, 1, I32), _v(args, 2, I64), _v(args, 3, VP)
    assert grid[0] * 256 >= np_ * n * n
    return [(P, P + 8 * np_ * (n * (n + 1) // 2), "packed"), (F, F + 8 * np_ * n * n, "full")]


def dec_ozgemm(grid, args):
    base = args[0]
    nprob = I32.from_address(base + 32 * OZ_PROB_BYTES).value
    nunits = I32.from_address(base + 32 * OZ_PROB_BYTES + 4).value
    assert 1 <= nprob <= 32, nprob
    units, res = 0, []
    for i in range(nprob):
        pb = base + i * OZ_PROB_BYTES
        a = OzArgs.from_address(pb + OZ_ARGS_OFF)
        t = OzTail.from_address(pb + OZ_ARGS_OFF + ct.sizeof(OzArgs))
        assert t.tile0 == units, (t.tile0, units)
        units += t.ntn * t.ntm * a.nsuper
        assert a.M >= 1 and a.N >= 1 and a.K >= 1 and a.nsuper == (a.K + SUPER - 1) // SUPER
        assert t.cfg in OZ_CFG, t.cfg
        bn = OZ_CFG[t.cfg][1]
        assert t.ntm == (a.M + OZ_BM - 1) // OZ_BM and t.ntn == (a.N + bn - 1) // bn
        nsc = a.nsuper
        res.append((a.eA, a.eA + 4 * ((a.M - 1) // a.a_rpe + 1) * nsc, "eA"))
        res.append((a.eB, a.eB + 4 * ((a.N - 1) // a.b_rpe + 1) * nsc, "eB"))
        if not a.use_tma_store:
            res.append((a.C, a.C + 8 * ((a.M - 1) * a.ldc + a.N), "C"))
    assert units == nunits, (units, nunits)
    return res


# ---- FP64 kernels executed on the simulated device memory (--exec) -------------
# The arithmetic of each FP64-engine kernel, in numpy, run at launch time on the
# host buffers that stand in for device memory, so that FP64 calls produce
# values the oracle can check.  Split-engine kernels are not executed.
EXEC = [False]


def dv(ptr, count):
    """The `count` doubles at address ptr, as a writable numpy view."""
    return np.ctypeslib.as_array(ct.cast(ct.c_void_p(ptr), ct.POINTER(ct.c_double)), shape=(max(count, 1),))


def _gop_gather(g, b, rows, K):
    r = np.arange(rows)[:, None]
    kk = np.arange(K)[None, :]
    idx = b * g.sb + r * g.sr + (kk // g.kin) * g.sko + (kk % g.kin) * g.ski
    return dv(g.p, int(idx.max()) + 1)[idx]


def ex_dgemm(grid, args):
    M, N, K = _v(args, 0, I32), _v(args, 1, I32), _v(args, 2, I32)
    A, B, C, ldc, scb = _a(args, 3, GOp), _a(args, 4, GOp), _v(args, 5, VP), _v(args, 6, I64), _v(args, 7, I64)
    alpha, beta = _v(args, 8, F64), _v(args, 9, F64)
    for b in range(grid[2]):
        prod = _gop_gather(A, b, M, K) @ _gop_gather(B, b, N, K).T
        idx = b * scb + np.arange(M)[:, None] * ldc + np.arange(N)[None, :]
        Cv = dv(C, int(idx.max()) + 1)
        Cv[idx] = alpha * prod + (beta * Cv[idx] if beta != 0.0 else 0.0)


def ex_pack_cols(grid, args):
    src, n, k, Z, ctot, off = (_v(args, 0, VP), _v(args, 1, I32), _v(args, 2, I32), _v(args, 3, VP),
                               _v(args, 4, I32), _v(args, 5, I32))
    idx = np.arange(n)[:, None] * ctot + off + np.arange(k)[None, :]
    dv(Z, int(idx.max()) + 1)[idx] = dv(src, n * k).reshape(n, k)


def ex_pack_group(grid, args):
    g = PackGroup.from_address(args[0])
    for i in range(g.njob):
        jb = g.j[i]
        idx = np.arange(jb.n)[:, None] * jb.ctot + jb.off + np.arange(jb.k)[None, :]
        dv(jb.Z, int(idx.max()) + 1)[idx] = dv(jb.src, jb.n * jb.k).reshape(jb.n, jb.k)


def ex_frob(grid, args):
    L, n2, M, nd, g, ldg, P0 = (_v(args, 0, VP), _v(args, 1, I64), _v(args, 2, VP), _v(args, 3, I32),
                                _v(args, 4, VP), _v(args, 5, I32), _v(args, 6, I32))
    Lm = dv(L, (P0 + grid[0]) * n2).reshape(-1, n2)[P0:P0 + grid[0]]
    Mm = dv(M, nd * n2).reshape(nd, n2)
    gv = dv(g, (nd - 1) * ldg + P0 + grid[0])
    for s in range(nd):
        gv[s * ldg + P0:s * ldg + P0 + grid[0]] = Lm @ Mm[s]


def ex_frob_packed(grid, args):
    L, n, M, nd, g, ldg, P0 = (_v(args, 0, VP), _v(args, 1, I32), _v(args, 2, VP), _v(args, 3, I32),
                               _v(args, 4, VP), _v(args, 5, I32), _v(args, 6, I32))
    iu = np.triu_indices(n)
    tri = len(iu[0])
    P = dv(L, (P0 + grid[0]) * tri).reshape(-1, tri)[P0:P0 + grid[0]]
    full = np.zeros((grid[0], n, n))
    full[:, iu[0], iu[1]] = P
    full[:, iu[1], iu[0]] = P
    Mm = dv(M, nd * n * n).reshape(nd, n * n)
    gv = dv(g, (nd - 1) * ldg + P0 + grid[0])
    for s in range(nd):
        gv[s * ldg + P0:s * ldg + P0 + grid[0]] = full.reshape(grid[0], -1) @ Mm[s]


def ex_gamma_panel(grid, args):
    T, n, ctot, tab, g, ldg, P0 = (_v(args, 0, VP), _v(args, 1, I32), _v(args, 2, I64), _a(args, 3, DensTab),
                                   _v(args, 4, VP), _v(args, 5, I32), _v(args, 6, I32))
    np_, nd = grid[0], grid[1]
    Tm = dv(T, np_ * n * ctot).reshape(np_, n, ctot)
    gv = dv(g, (nd - 1) * ldg + P0 + np_)
    for s in range(nd):
        k, off = tab.k[s], tab.offX[s]
        Ys = dv(tab.Y[s], n * k).reshape(n, k)
        gv[s * ldg + P0:s * ldg + P0 + np_] = np.einsum("pik,ik->p", Tm[:, :, off:off + k], Ys)


def ex_gamma_group(grid, args):
    g = GammaGroup.from_address(args[0])
    for i in range(g.njob):
        jb = g.j[i]
        n, ctot, np_ = jb.n, jb.ldT, jb.np
        Tm = dv(jb.T, np_ * n * ctot).reshape(np_, n, ctot)
        gv = dv(jb.gamma, (jb.nd - 1) * jb.ldg + jb.P0 + np_)
        for s in range(jb.nd):
            k, off = g.k[jb.d0 + s], g.offX[jb.d0 + s]
            Ys = dv(g.Y[jb.d0 + s], n * k).reshape(n, k)
            gv[s * jb.ldg + jb.P0:s * jb.ldg + jb.P0 + np_] = np.einsum("pik,ik->p", Tm[:, :, off:off + k], Ys)


def ex_jstream_sym(grid, args, name):
    ns = int(name.split("ILi")[1].split("E")[0])
    L, n, P0, np_, g, ldg, acc, o = _jstream_args(args)
    naux = P0 + np_
    if "Lb1E" in name:                                            # packed upper triangles
        iu = np.triu_indices(n)
        P = dv(L, naux * len(iu[0])).reshape(naux, -1)[P0:]
        full = np.zeros((np_, n, n))
        full[:, iu[0], iu[1]] = P
        full[:, iu[1], iu[0]] = P
        Lm = full.reshape(np_, n * n)
    else:
        Lm = dv(L, naux * n * n).reshape(naux, n * n)[P0:]
    for j in range(ns):
        out = dv(g + 8 * j * ldg, naux)[P0:] @ Lm
        out = out.reshape(n, n)
        sym = np.triu(out).ravel() + np.triu(out, 1).T.ravel()   # upper triangle, mirrored
        if acc:
            dv(o.p[j], n * n)[:] += sym
        else:
            dv(o.p[j], n * n)[:] = sym


def _tri_columns(L, n, ps, P0, np_, pk):
    """A[t][kk] = L^{P0+kk}[mu][nu] over the upper-triangle positions t."""
    ntri = n * (n + 1) // 2
    F = dv(L, (P0 + np_) * ps).reshape(P0 + np_, ps)[P0:]
    if pk:
        return F.T.copy()
    iu = np.triu_indices(n)
    return F[:, iu[0] * n + iu[1]].T.copy()


def ex_expo_tri(grid, args, name):
    pk, L, n, ps, P0, np_, ntri = _tri_args(args, name)
    nsc, e = _v(args, 5, I32), _v(args, 6, VP)
    A = np.abs(_tri_columns(L, n, ps, P0, np_, pk))
    ev = uv(e, ntri * nsc, np.int32).reshape(ntri, nsc)
    for z in range(nsc):
        ev[:, z] = _expo_of(A[:, z * SUPER:(z + 1) * SUPER].max(axis=1))


def ex_slice_tri(grid, args, name):
    pk, L, n, ps, P0, np_, ntri = _tri_args(args, name)
    Kpad, nsc, e, out = _v(args, 5, I32), _v(args, 6, I32), _v(args, 7, VP), _v(args, 8, VP)
    A = _tri_columns(L, n, ps, P0, np_, pk)
    ev = uv(e, ntri * nsc, np.int32).reshape(ntri, nsc)
    E = ev[:, np.arange(np_) // SUPER]
    planes = _digits_bf16(A, E, 6)
    o = uv(out, 6 * ntri * Kpad, np.uint16).reshape(6, ntri, Kpad)
    o[:] = 0
    for j in range(6):
        o[j, :, :np_] = planes[j]


def _expo_tri_exec(L, n, ps, P0, np_, pk, nsc, e):
    ntri = n * (n + 1) // 2
    A = np.abs(_tri_columns(L, n, ps, P0, np_, pk))
    ev = uv(e, ntri * nsc, np.int32).reshape(ntri, nsc)
    for z in range(nsc):
        ev[:, z] = _expo_of(A[:, z * SUPER:(z + 1) * SUPER].max(axis=1))


def _slice_tri_exec(L, n, ps, P0, np_, pk, Kpad, nsc, e, out):
    ntri = n * (n + 1) // 2
    A = _tri_columns(L, n, ps, P0, np_, pk)
    ev = uv(e, ntri * nsc, np.int32).reshape(ntri, nsc)
    planes = _digits_bf16(A, ev[:, np.arange(np_) // SUPER], 6)
    o = uv(out, 6 * ntri * Kpad, np.uint16).reshape(6, ntri, Kpad)
    o[:] = 0
    for j in range(6):
        o[j, :, :np_] = planes[j]


def ex_expo_tri_group(grid, args):
    g = TriGroup.from_address(args[0])
    for i in range(g.njob):
        jb = g.j[i]
        _expo_tri_exec(jb.L, jb.n, jb.pstride, jb.P0, jb.np, jb.pk, jb.nsc, jb.e)


def ex_slice_tri_group(grid, args):
    g = TriGroup.from_address(args[0])
    for i in range(g.njob):
        jb = g.j[i]
        _slice_tri_exec(jb.L, jb.n, jb.pstride, jb.P0, jb.np, jb.pk, jb.Kpad, jb.nsc, jb.e, jb.out)


def _j_tri_add_exec(C, ldc, n, nd, acc, ptrs):
    ntri = n * (n + 1) // 2
    Cm = dv(C, ntri * ldc).reshape(ntri, ldc)
    iu = np.triu_indices(n)
    for s in range(nd):
        J = dv(ptrs[s], n * n).reshape(n, n)
        v = Cm[:, s] + (J[iu] if acc else 0.0)
        J[iu] = v
        J[iu[1], iu[0]] = v


def ex_j_tri_add_group(grid, args):
    g = JAddGroup.from_address(args[0])
    for i in range(g.njob):
        jb = g.j[i]
        _j_tri_add_exec(jb.C, jb.ldc, jb.n, jb.nd, jb.acc, [g.ptr[jb.p0 + s] for s in range(jb.nd)])


def ex_j_tri_add(grid, args):
    C, ldc, n, nd, acc, jo = _v(args, 0, VP), _v(args, 1, I64), _v(args, 2, I32), _v(args, 3, I32), \
        _v(args, 4, I32), _a(args, 5, JOut)
    ntri = n * (n + 1) // 2
    Cm = dv(C, ntri * ldc).reshape(ntri, ldc)
    iu = np.triu_indices(n)
    for s in range(nd):
        J = dv(jo.p[s], n * n).reshape(n, n)
        v = Cm[:, s] + (J[iu] if acc else 0.0)
        J[iu] = v
        J[iu[1], iu[0]] = v


def ex_axpy(grid, args):
    y, x, cnt = _v(args, 0, VP), _v(args, 1, VP), _v(args, 2, I64)
    dv(y, cnt)[:] += dv(x, cnt)


def ex_sum_parts_ld(grid, args):
    out, ldo, part, nb, M, N, acc = (_v(args, 0, VP), _v(args, 1, I64), _v(args, 2, VP), _v(args, 3, I32),
                                     _v(args, 4, I32), _v(args, 5, I32), _v(args, 6, I32))
    tot = dv(part, nb * M * N).reshape(nb, M, N).sum(axis=0)
    idx = np.arange(M)[:, None] * ldo + np.arange(N)[None, :]
    o = dv(out, (M - 1) * ldo + N)
    o[idx] = (o[idx] if acc else 0.0) + tot


def ex_pack_sym(grid, args):
    F, n, np_, P = _v(args, 0, VP), _v(args, 1, I32), _v(args, 2, I64), _v(args, 3, VP)
    iu = np.triu_indices(n)
    dv(P, np_ * len(iu[0])).reshape(np_, -1)[:] = dv(F, np_ * n * n).reshape(np_, n, n)[:, iu[0], iu[1]]


def ex_mirror_blocks(grid, args):
    K, n, bm = _v(args, 0, VP), _v(args, 1, I32), _v(args, 2, I32)
    M = dv(K, n * n).reshape(n, n)
    r, c = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    mask = c < bm * (r // bm)
    M[mask] = M.T.copy()[mask]


def ex_sum_parts(grid, args):
    out, part, nb, cnt, acc = _v(args, 0, VP), _v(args, 1, VP), _v(args, 2, I32), _v(args, 3, I64), _v(args, 4, I32)
    tot = dv(part, nb * cnt).reshape(nb, cnt).sum(axis=0)
    o = dv(out, cnt)
    o[:] = (o if acc else 0.0) + tot


def ex_pair_dot(grid, args):
    ZL, U, n, ctot, tab, out, nr = (_v(args, 0, VP), _v(args, 1, VP), _v(args, 2, I32), _v(args, 3, I32),
                                    _a(args, 4, PairTab), _v(args, 5, VP), _v(args, 6, I32))
    Zm = dv(ZL, n * ctot).reshape(n, ctot)
    Um = dv(U, nr * n * ctot).reshape(nr, n, ctot)
    ov = dv(out, grid[0] * nr)
    for a in range(grid[0]):
        k, oa, ob = tab.k[a], tab.offA[a], tab.offB[a]
        for b in range(nr):
            ov[a * nr + b] = np.sum(Zm[:, oa:oa + k] * Um[b, :, ob:ob + k])


def ex_laplace_scale(grid, args):
    C, eps, n, m, sgn = _v(args, 0, VP), _v(args, 1, VP), _v(args, 2, I32), _v(args, 3, I32), _v(args, 4, F64)
    al = (F64 * MAXD).from_address(args[5])
    nq, out = _v(args, 6, I32), _v(args, 7, VP)
    Cm, ev = dv(C, n * m).reshape(n, m), dv(eps, m)
    o = dv(out, nq * n * m).reshape(nq, n, m)
    for k in range(nq):
        o[k] = Cm * np.exp(sgn * al[k] * ev * 0.5)[None, :]


def ex_weighted_sum(grid, args):
    out, part = _v(args, 0, VP), _v(args, 1, VP)
    w = (F64 * MAXD).from_address(args[2])
    nq, cnt = _v(args, 3, I32), _v(args, 4, I64)
    dv(out, cnt)[:] = np.tensordot(np.array(w[:nq]), dv(part, nq * cnt).reshape(nq, cnt), 1)


def ex_unpack_sym(grid, args):
    P, n, np_, F = _v(args, 0, VP), _v(args, 1, I32), _v(args, 2, I64), _v(args, 3, VP)
    t = n * (n + 1) // 2
    iu = np.triu_indices(n)
    Pm = dv(P, np_ * t).reshape(np_, t)
    Fm = dv(F, np_ * n * n).reshape(np_, n, n)
    for p in range(np_):
        M = np.zeros((n, n))
        M[iu] = Pm[p]
        Fm[p] = M + np.triu(M, 1).T


def ex_gterms(grid, args):
    G, n2, nd = _v(args, 0, VP), _v(args, 1, I64), _v(args, 3, I32)
    D, V, c, g, ldg, P0 = (_v(args, 4, VP), _v(args, 5, VP), _v(args, 6, VP), _v(args, 7, VP), _v(args, 8, I32),
                           _v(args, 9, I32))
    np_ = grid[1]
    Gm = dv(G, np_ * n2).reshape(np_, n2)
    for p in range(np_):
        for s in range(nd):
            if D:
                Gm[p] += dv(c, s * ldg + P0 + p + 1)[s * ldg + P0 + p] * dv(D, nd * n2).reshape(nd, n2)[s]
            if V:
                Gm[p] += dv(g, s * ldg + P0 + p + 1)[s * ldg + P0 + p] * dv(V, nd * n2).reshape(nd, n2)[s]


def ex_symmetrize(grid, args):
    G, n, dL = _v(args, 0, VP), _v(args, 1, I32), _v(args, 2, VP)
    np_ = grid[1]
    Gm = dv(G, np_ * n * n).reshape(np_, n, n)
    dv(dL, np_ * n * n).reshape(np_, n, n)[:] = 0.5 * (Gm + Gm.transpose(0, 2, 1))


def ex_fold(grid, args):
    dX, dY, cnt = _v(args, 0, VP), _v(args, 1, VP), _v(args, 2, I64)
    dv(dX, cnt)[:] += dv(dY, cnt)
    dv(dY, cnt)[:] = 0.0


# ---- split engine, executed --------------------------------------------------
# Exponents and digit slices as the slicers define them; the sliced GEMM as
# the exact sum of the rebuilt 48-bit operands per 2048-element super-chunk
# (int64 partials in units of 2^-48, or FP64 output); the partial reduction
# in FP64.  This checks the orchestration of the split paths, not the
# tensor-core arithmetic (which tests/test_split_gpu.py covers on the GPU).

def uv(ptr, count, dtype):
    ctype = {np.uint16: ct.c_uint16, np.int32: ct.c_int32, np.int64: ct.c_int64}[dtype]
    return np.ctypeslib.as_array(ct.cast(ct.c_void_p(ptr), ct.POINTER(ctype)), shape=(max(count, 1),))


def _src_gather(src, rows, K):
    r = np.arange(rows)[:, None]
    kk = np.arange(K)[None, :]
    idx = (r // src.rin) * src.sr + (r % src.rin) * src.sri + (kk // src.kin) * src.sko + (kk % src.kin) * src.ski
    return dv(src.p, int(idx.max()) + 1)[idx]


def _expo_of(m):
    """e with max|x| < 2^e from the maximum magnitude (-1000 for zero)."""
    m = np.asarray(m, dtype=np.float64)
    e = np.frexp(m)[1].astype(np.int64)
    return np.where(m > 0, e, -1000)


def _expo_job(src, rows, K, rpe, e, ngroups, nsc):
    X = np.abs(_src_gather(src, rows, K))
    ev = uv(e, ngroups * nsc, np.int32)
    for g in range(ngroups):
        for z in range(nsc):
            blk = X[g * rpe:min(rows, g * rpe + rpe), z * SUPER:min(K, (z + 1) * SUPER)]
            ev[g * nsc + z] = _expo_of(blk.max() if blk.size else 0.0)


def ex_expo(grid, args):
    src, rows, K, rpe, e = _a(args, 0, Src), _v(args, 1, I32), _v(args, 2, I32), _v(args, 3, I32), _v(args, 4, VP)
    _expo_job(src, rows, K, rpe, e, grid[0], grid[1])


def ex_expo_group(grid, args):
    g = SliceGroup.from_address(args[0])
    for i in range(g.njob):
        jb = g.j[i]
        _expo_job(jb.src, jb.rows, jb.K, jb.rpe, jb.e, (jb.rows - 1) // jb.rpe + 1, jb.nsc)


def ex_int_fill(grid, args):
    g = PanelExpo.from_address(args[0])
    for i in range(g.nseg):
        uv(g.s[i].e, g.s[i].n * g.s[i].nsc, np.int32)[:] = -1000


def ex_panel_colmax(grid, args):
    """Each operand's exponent of (row mu, super-chunk z) from the panel rows
    (p, mu): the exponent of the maximum over that group of its columns."""
    g = PanelExpo.from_address(args[0])
    for i in range(g.nitem):
        pi = g.it[i]
        n, np_ = pi.n, pi.rows // pi.n
        T = np.abs(dv(pi.T, pi.rows * pi.ldT).reshape(pi.rows, pi.ldT))
        for j in range(pi.seg0, pi.seg0 + pi.nseg):
            sg = g.s[j]
            blk = T[:, sg.c0:sg.c0 + sg.k].reshape(np_, n, sg.k).transpose(1, 0, 2).reshape(n, np_ * sg.k)
            ev = uv(sg.e, n * sg.nsc, np.int32).reshape(n, sg.nsc)
            for z in range(sg.nsc):
                part = blk[:, z * SUPER:(z + 1) * SUPER]
                ev[:, z] = np.maximum(ev[:, z], _expo_of(part.max(axis=1)))


def ex_expo_flat(grid, args):
    p, ln, e = _v(args, 0, VP), _v(args, 1, I64), _v(args, 2, VP)
    X = np.abs(dv(p, grid[0] * ln).reshape(grid[0], ln))
    uv(e, grid[0], np.int32)[:] = _expo_of(X.max(axis=1))


def _digits_bf16(x, e, nslice=6):
    """The nslice BF16 slice words of x at exponent e (integer balanced
    digits of the 8 * nslice-bit fixed-point value)."""
    bits = 8 * nslice
    xs = np.abs(x) * np.exp2(bits - e.astype(np.float64))
    # the fixed-point value, rounded half away from zero; beyond 2^53 the
    # product is an exact integer already (a double's significand)
    F = np.where(xs < 2.0 ** 52, np.floor(xs + 0.5), xs)
    F = (np.sign(x) * F).astype(np.int64)
    q = [None] * nslice
    for j in range(nslice - 1, 0, -1):
        q[j] = ((F + 128) & 255) - 128
        F = (F - q[j]) >> 8
    q[0] = F
    return [((q[j].astype(np.float64) * 2.0 ** (-8 * (j + 1))).astype(np.float32).view(np.uint32) >> 16)
            .astype(np.uint16) for j in range(nslice)]


def ex_slice(grid, args, name):
    src, rows, K, Kpad = _a(args, 0, Src), _v(args, 1, I32), _v(args, 2, I32), _v(args, 3, I32)
    e, rpe, nsc, out = _v(args, 4, VP), _v(args, 5, I32), _v(args, 6, I32), _v(args, 7, VP)
    _slice_job(src, rows, K, Kpad, e, rpe, nsc, out, _slices_of(name))


def ex_slice_group(grid, args, name):
    g = SliceGroup.from_address(args[0])
    for i in range(g.njob):
        jb = g.j[i]
        _slice_job(jb.src, jb.rows, jb.K, jb.Kpad, jb.e, jb.rpe, jb.nsc, jb.out, _slices_of(name))


def _slice_job(src, rows, K, Kpad, e, rpe, nsc, out, nslice):
    X = _src_gather(src, rows, K)
    ev = uv(e, ((rows - 1) // rpe + 1) * nsc, np.int32)
    E = ev[(np.arange(rows)[:, None] // rpe) * nsc + np.arange(K)[None, :] // SUPER]
    planes = _digits_bf16(X, E, nslice)
    o = uv(out, nslice * rows * Kpad, np.uint16).reshape(nslice, rows, Kpad)
    o[:] = 0
    for j in range(nslice):
        o[j, :, :K] = planes[j]


def _tmap(ptr):
    w = (ct.c_uint64 * 16).from_address(ptr)
    assert w[0] == 0x6A6B73696D6D6170, "tensor map not encoded by the stand-in"
    return {"dtype": w[1] >> 32, "rank": w[1] & 0xFFFFFFFF, "base": w[2], "dims": [w[3], w[4], w[5]],
            "strides": [0, w[6], w[7]]}


def _operand(tm, e, rpe, rows, K, nsuper):
    """Rebuilt operand values in units of 2^(exponent): [rows][K] float64, and
    the exponents [rows][nsuper]."""
    Kpad, nrows = tm["dims"][0], tm["dims"][1]
    assert tm["strides"][1] == 2 * Kpad, tm
    nslice = tm["dims"][2]                       # one plane per slice
    pstride = tm["strides"][2] // 2              # elements between planes (a row view keeps its parent's)
    flat = uv(tm["base"], (nslice - 1) * pstride + nrows * Kpad, np.uint16)
    vals = np.zeros((rows, K))
    for j in range(nslice):
        plane = flat[j * pstride:j * pstride + nrows * Kpad].reshape(nrows, Kpad)[:rows, :K]
        vals += (plane.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    ev = uv(e, ((rows - 1) // rpe + 1) * nsuper, np.int32).reshape(-1, nsuper)[np.arange(rows) // rpe]
    return vals, ev


def ex_ozgemm(grid, args):
    base = args[0]
    nprob = I32.from_address(base + 32 * OZ_PROB_BYTES).value
    for i in range(nprob):
        pb = base + i * OZ_PROB_BYTES
        a = OzArgs.from_address(pb + OZ_ARGS_OFF)
        t = OzTail.from_address(pb + OZ_ARGS_OFF + ct.sizeof(OzArgs))
        frac = OZ_CFG[t.cfg][2]
        tA, tB = _tmap(pb), _tmap(pb + 128)
        assert tA["dims"][2] == tB["dims"][2] == OZ_CFG[t.cfg][0]
        A, eA = _operand(tA, a.eA, a.a_rpe, a.M, a.K, a.nsuper)
        B, eB = _operand(tB, a.eB, a.b_rpe, a.N, a.K, a.nsuper)
        for z in range(a.nsuper):
            S = A[:, z * SUPER:(z + 1) * SUPER] @ B[:, z * SUPER:(z + 1) * SUPER].T
            if a.nsuper == 1:
                idx = np.arange(a.M)[:, None] * a.ldc + np.arange(a.N)[None, :]
                dv(a.C, int(idx.max()) + 1)[idx] = np.ldexp(S, eA[:, z:z + 1] + eB[:, z][None, :])
            else:
                idx = z * a.pz + np.arange(a.M)[:, None] * a.ldp + np.arange(a.N)[None, :]
                uv(a.P, int(idx.max()) + 1, np.int64)[idx] = np.rint(S * 2.0 ** frac).astype(np.int64)


def ex_reduce(grid, args):
    P, pz, ldp, nz, M, N = (_v(args, 0, VP), _v(args, 1, I64), _v(args, 2, I64), _v(args, 3, I32),
                            _v(args, 4, I32), _v(args, 5, I32))
    eA, arpe, eB, brpe, out, ldo, acc, frac = (_v(args, 6, VP), _v(args, 7, I32), _v(args, 8, VP), _v(args, 9, I32),
                                               _v(args, 10, VP), _v(args, 11, I64), _v(args, 12, I32),
                                               _v(args, 13, I32))
    _reduce_job(P, pz, ldp, nz, M, N, eA, arpe, eB, brpe, out, ldo, acc, frac)


def ex_reduce_group(grid, args):
    g = ReduceGroup.from_address(args[0])
    for i in range(g.njob):
        jb = g.j[i]
        _reduce_job(jb.P, jb.pz, jb.ldp, jb.nz, jb.M, jb.N, jb.eA, jb.arpe, jb.eB, jb.brpe, jb.out, jb.ldo,
                    jb.accumulate, jb.frac)


def _reduce_job(P, pz, ldp, nz, M, N, eA, arpe, eB, brpe, out, ldo, acc, frac):
    ea = uv(eA, ((M - 1) // arpe + 1) * nz, np.int32).reshape(-1, nz)[np.arange(M) // arpe]
    eb = uv(eB, ((N - 1) // brpe + 1) * nz, np.int32).reshape(-1, nz)[np.arange(N) // brpe]
    tot = np.zeros((M, N))
    for z in range(nz):
        idx = z * pz + np.arange(M)[:, None] * ldp + np.arange(N)[None, :]
        Pz = uv(P, int(idx.max()) + 1, np.int64)[idx].astype(np.float64)
        tot += np.ldexp(Pz, ea[:, z:z + 1] + eb[:, z][None, :] - frac)
    oidx = np.arange(M)[:, None] * ldo + np.arange(N)[None, :]
    o = dv(out, int(oidx.max()) + 1)
    o[oidx] = (o[oidx] if acc else 0.0) + tot


def ex_pack_ag(grid, args):
    AG, ldag, off, U, Vp, X, cps, P0, n, k, np_ = (
        _v(args, 0, VP), _v(args, 1, I64), _v(args, 2, I32), _v(args, 3, VP), _v(args, 4, VP), _v(args, 5, VP),
        _v(args, 6, VP), _v(args, 7, I32), _v(args, 8, I32), _v(args, 9, I32), _v(args, 10, I32))
    pm = np.arange(np_ * n)
    mu, p = pm % n, pm // n
    rows = dv(AG, (np_ * n - 1) * ldag + off + 3 * k)
    for i in range(k):
        uo = mu * np_ * k + p * k + i
        rows[pm * ldag + off + i] = dv(U, n * np_ * k)[uo] if U else 0.0
        rows[pm * ldag + off + k + i] = dv(Vp, n * np_ * k)[uo] if Vp else 0.0
        rows[pm * ldag + off + 2 * k + i] = (dv(cps, P0 + np_)[P0 + p] * dv(X, n * k)[mu * k + i]) if cps else 0.0


def ex_pack_bg(grid, args):
    BG, ldbg, off, X, Y, n, k = (_v(args, 0, VP), _v(args, 1, I64), _v(args, 2, I32), _v(args, 3, VP),
                                 _v(args, 4, VP), _v(args, 5, I32), _v(args, 6, I32))
    Xm, Ym = dv(X, n * k).reshape(n, k), dv(Y, n * k).reshape(n, k)
    rows = dv(BG, (n - 1) * ldbg + off + 3 * k)
    for nu in range(n):
        b = nu * ldbg + off
        rows[b:b + k], rows[b + k:b + 2 * k], rows[b + 2 * k:b + 3 * k] = Xm[nu], Ym[nu], Ym[nu]


def ex_sym_dl(grid, args):
    G, GV, n, dL = _v(args, 0, VP), _v(args, 1, VP), _v(args, 2, I32), _v(args, 3, VP)
    np_ = grid[1]
    Gm = dv(G, np_ * n * n).reshape(np_, n, n)
    v = 0.5 * (Gm + Gm.transpose(0, 2, 1))
    if GV:
        Vm = dv(GV, np_ * n * n).reshape(np_, n, n)
        v = v + 0.5 * (Vm + Vm.transpose(0, 2, 1))
    dv(dL, np_ * n * n).reshape(np_, n, n)[:] = v


EXECUTORS = [
    ("dgemm_nt_kernel", ex_dgemm), ("pack_cols_kernel", ex_pack_cols), ("frob_stream_kernel", ex_frob),
    ("gamma_panel_kernel", ex_gamma_panel), ("jstream_sym_kernel", ex_jstream_sym), ("axpy_kernel", ex_axpy),
    ("expo_tri_kernel", ex_expo_tri), ("slice_tri_kernel", ex_slice_tri), ("j_tri_add_kernel", ex_j_tri_add),
    ("expo_tri_group_kernel", ex_expo_tri_group), ("slice_tri_group_kernel", ex_slice_tri_group),
    ("j_tri_add_group_kernel", ex_j_tri_add_group), ("gamma_group_kernel", ex_gamma_group),
    ("sum_parts_kernel", ex_sum_parts), ("pair_dot_kernel", ex_pair_dot), ("laplace_scale_kernel", ex_laplace_scale),
    ("weighted_sum_kernel", ex_weighted_sum), ("unpack_sym_kernel", ex_unpack_sym), ("gterms_kernel", ex_gterms),
    ("symmetrize_kernel", ex_symmetrize), ("fold_sym_split_kernel", ex_fold), ("fold_sym_kernel", ex_fold),
    ("pack_group_kernel", ex_pack_group), ("int_fill_kernel", ex_int_fill), ("panel_colmax_kernel", ex_panel_colmax),
    ("expo_group_kernel", ex_expo_group), ("slice_group_kernel", ex_slice_group),
    ("reduce_group_kernel", ex_reduce_group),
    ("expo_flat_kernel", ex_expo_flat), ("expo_kernel", ex_expo), ("slice4f_kernel", ex_slice),
    ("slice4_kernel", ex_slice), ("slice_kernel", ex_slice), ("ozgemm_kernel", ex_ozgemm),
    ("reduce_partials_kernel", ex_reduce), ("pack_ag_kernel", ex_pack_ag), ("pack_bg_kernel", ex_pack_bg),
    ("sym_dl_kernel", ex_sym_dl), ("mirror_blocks_kernel", ex_mirror_blocks), ("sum_parts_ld_kernel", ex_sum_parts_ld),
    ("pack_sym_kernel", ex_pack_sym), ("frob_packed_kernel", ex_frob_packed),
]

DECODERS = [
    ("expo_tri_kernel", dec_expo_tri), ("slice_tri_kernel", dec_slice_tri), ("j_tri_add_kernel", dec_j_tri_add),
    ("expo_tri_group_kernel", dec_expo_tri_group), ("slice_tri_group_kernel", dec_slice_tri_group),
    ("j_tri_add_group_kernel", dec_j_tri_add_group), ("gamma_group_kernel", dec_gamma_group),
    ("pack_group_kernel", dec_pack_group), ("int_fill_kernel", dec_int_fill), ("panel_colmax_kernel", dec_panel_colmax),
    ("expo_group_kernel", dec_expo_group), ("slice_group_kernel", dec_slice_group),
    ("reduce_group_kernel", dec_reduce_group),
    ("expo_flat_kernel", dec_expo_flat), ("expo_kernel", dec_expo), ("slice4_kernel", dec_slice4),
    ("slice_kernel", dec_slice), ("dgemm_nt_kernel", dec_dgemm), ("pack_cols_kernel", dec_pack_cols),
    ("frob_stream_kernel", dec_frob), ("gamma_panel_kernel", dec_gamma_panel), ("axpy_kernel", dec_axpy),
    ("sum_parts_kernel", dec_sum_parts), ("reduce_partials_kernel", dec_reduce), ("pair_dot_kernel", dec_pair_dot),
    ("laplace_scale_kernel", dec_laplace_scale), ("weighted_sum_kernel", dec_weighted_sum),
    ("ozgemm_kernel", dec_ozgemm), ("jstream_sym_kernel", dec_jstream_sym), ("gterms_kernel", dec_gterms),
    ("slice4f_kernel", dec_slice4), ("unpack_sym_kernel", dec_unpack_sym),
    ("symmetrize_kernel", dec_symmetrize), ("sym_dl_kernel", dec_sym_dl), ("fold_sym_split_kernel", dec_fold),
    ("fold_sym_kernel", dec_fold), ("pack_ag_kernel", dec_pack_ag), ("pack_bg_kernel", dec_pack_bg),
    ("mirror_blocks_kernel", dec_mirror_blocks), ("sum_parts_ld_kernel", dec_sum_parts_ld),
    ("pack_sym_kernel", dec_pack_sym), ("frob_packed_kernel", dec_frob_packed),
]
violations, decoded, undecoded = [], [0], set()


def _inside(lo, hi):
    if hi <= lo:
        return True
    for base, nbytes, _label, *_ in owned + statics():
        if base <= lo and hi <= base + nbytes:
            return True
    return False


def statics():
    out, i = [], 0
    p, sz = ct.c_void_p(), ct.c_size_t()
    while shim.shim_var(i, ct.byref(p), ct.byref(sz)):
        if p.value:
            out.append((p.value, sz.value, "static"))
        i += 1
    return out


@ct.CFUNCTYPE(None, ct.c_char_p, ct.POINTER(ct.c_uint), ct.POINTER(ct.c_uint), ct.POINTER(ct.c_void_p))
def on_launch(name, grid, block, args):
    name = name.decode()
    g = (grid[0], grid[1], grid[2])
    for key, fn in DECODERS:
        if key in name:
            try:
                ranges = (fn(g, args, name) if fn in (dec_jstream_sym, dec_slice, dec_slice4, dec_slice_group,
                                                      dec_expo_tri, dec_slice_tri)
                          else fn(g, args))
            except AssertionError as e:
                violations.append(f"{key}: inconsistent arguments {e}")
                return
            decoded[0] += 1
            bad = False
            for lo, hi, what in ranges:
                if not _inside(lo, hi):
                    bad = True
                    violations.append(f"{key}: {what} [{lo:#x}, {hi:#x}) outside the call's memory")
            if EXEC[0] and not bad:
                for ekey, ex in EXECUTORS:
                    if ekey in name:
                        ex(g, args, name) if ex in (ex_jstream_sym, ex_slice, ex_slice_group, ex_expo_tri,
                                                    ex_slice_tri) else ex(g, args)
                        break
            return
    undecoded.add(name)


shim.shim_set_hook(on_launch)
rng = np.random.default_rng(0)
owned = []      # (base, nbytes, label) of every buffer a case hands to the library


BIG = [False]     # full-size cases: inputs left as untouched zero pages
PACKED_MODE = [False]   # factors handed over as packed upper triangles (JK_OPT_PACKED_FACTOR)
ARENA_SCALE = [1.0]   # the arena handed to each call, as a fraction of the queried size


def buf(shape, label, fill=True):
    """A 256-byte aligned float64 array the library may address."""
    n = int(np.prod(shape))
    raw = np.zeros(n * 8 + 256, np.uint8)
    off = (-raw.ctypes.data) % 256
    a = raw[off:off + n * 8].view(np.float64).reshape(shape)
    if fill and not BIG[0]:
        a[...] = rng.standard_normal(shape) / max(shape[-1], 1)
    owned.append((a.ctypes.data, a.nbytes, label, raw))
    return a


def ptr(a):
    return None if a is None else ct.c_void_p(a.ctypes.data)


def factor_of(L, n, naux, tag):
    """The jk_factor of L: L itself, or (PACKED_MODE) a packed copy of its upper
    triangles, the only factor memory the library then sees."""
    if not PACKED_MODE[0]:
        return jk_factor(n, naux, L.ctypes.data)
    iu = np.triu_indices(n)
    LP = buf((naux, n * (n + 1) // 2), f"{tag}.Lpacked", fill=False)
    if not BIG[0]:
        LP[...] = L[:, iu[0], iu[1]]
    owned[:] = [o for o in owned if o[0] != L.ctypes.data]     # the dense copy is the test's alone
    return jk_factor(n, naux, LP.ctypes.data)


def packed(case):
    """The same case with every factor passed as packed upper triangles."""
    def fn():
        PACKED_MODE[0] = True
        try:
            return case()
        finally:
            PACKED_MODE[0] = False
    return fn


def mol(n, naux, ks, sym, tag="m"):
    L = buf((naux, n, n), f"{tag}.L")
    if not BIG[0]:
        L[...] = L + L.transpose(0, 2, 1)      # L^P symmetric, as the engine assumes
    X = [buf((n, k), f"{tag}.X{s}") for s, k in enumerate(ks)]
    Y = [buf((n, k), f"{tag}.Y{s}") for s, k in enumerate(ks)]
    d = (jk_density * len(ks))()
    for s, k in enumerate(ks):
        d[s].k, d[s].symmetric, d[s].X = k, int(sym[s]), X[s].ctypes.data
        d[s].Y = None if sym[s] else Y[s].ctypes.data
    return factor_of(L, n, naux, tag), d, L, X, Y


def handle(nbytes, opts, scaled=True):
    if scaled:
        nbytes = max(int(nbytes * ARENA_SCALE[0]), 1 << 16)
    ws = buf((nbytes // 8 + 1,), "arena", fill=False)
    h = ct.c_void_p()
    st = lib.jk_create(ct.byref(h), ct.c_void_p(ws.ctypes.data), ct.c_size_t(nbytes))
    assert st == 0, st
    for name, v in opts.items():
        assert lib.jk_set_option(h, OPT[name], ct.c_int64(v)) == 0
    return h


def query(op, f, d, nd, p, nmol=1, ndm=None, h=None):
    nb = ct.c_size_t()
    fa = f if isinstance(f, ct.Array) else (jk_factor * 1)(f)
    ndm_c = (ct.c_int32 * len(ndm))(*ndm) if ndm else None
    if h is None:
        st = lib.jk_workspace_query(op, nmol, fa, ndm_c, nd, d, p, ct.byref(nb))
    else:
        st = lib.jk_workspace_query_handle(h, op, nmol, fa, ndm_c, nd, d, p, ct.byref(nb))
    assert st == 0, (op, st)
    return nb.value


CHECKS = []   # (label, computed, oracle reference) of the current case, with --exec


def oracle_mod():
    sys.path.insert(0, ROOT)
    import oracle
    return oracle


def check(label, got, ref):
    CHECKS.append((label, np.array(got, dtype=np.float64), np.array(ref, dtype=np.float64)))


def _ylist(X, Y, sym):
    return [X[s] if sym[s] else Y[s] for s in range(len(X))]


def record(name, status, h):
    launches = []
    g, b, c = (ct.c_uint * 3)(), (ct.c_uint * 3)(), (ct.c_uint * 3)()
    sm = ct.c_size_t()
    for i in range(shim.shim_launch_count()):
        kname = shim.shim_launch(i, g, b, c, ct.byref(sm)).decode()
        launches.append([kname, list(g), list(b), list(c), sm.value])
    tmaps = []
    drs = (ct.c_int * 3)()
    base = ct.c_ulonglong()
    dims, strides = (ct.c_ulonglong * 5)(), (ct.c_ulonglong * 5)()
    box = (ct.c_uint * 5)()
    for i in range(shim.shim_tmap_count()):
        shim.shim_tmap(i, drs, ct.byref(base), dims, strides, box)
        r = drs[1]
        tmaps.append({"dtype": drs[0], "rank": r, "swizzle": drs[2], "base": base.value, "dims": list(dims)[:r],
                      "strides": list(strides)[:r], "box": list(box)[:r]})
    err = lib.jk_last_error(h).decode() if h else ""
    print(json.dumps({"case": name, "status": status, "error": err, "launches": launches, "tmaps": tmaps,
                      "copies": shim.shim_copy_count(), "syncs": shim.shim_sync_count(), "first": dict(FIRST),
                      "setups": shim.shim_setup_count(),
                      "owned": [[o[0], o[1], o[2]] for o in owned + statics()], "violations": list(violations),
                      "checks": [[lab, float(np.abs(g - r).max() / max(np.abs(r).max(), 1e-300))]
                                 for lab, g, r in CHECKS],
                      "decoded": decoded[0], "undecoded": sorted(undecoded)}), flush=True)


def run(name, fn):
    owned.clear()
    violations.clear()
    undecoded.clear()
    CHECKS.clear()
    FIRST.clear()
    decoded[0] = 0
    shim.shim_reset()
    try:
        status, h = fn()
    except AssertionError as e:         # a query or set-up step refused the case
        status, h = -1, None
        violations.append(f"driver: {e!r}")
    record(name, status, h)
    if h:
        lib.jk_destroy(h)


# ---- the cases ----------------------------------------------------------------

def build_case(n, naux, ks, sym, p, opts, want="JK"):
    def fn():
        f, d, L, X, Y = mol(n, naux, ks, sym)
        h = handle(1 << 20, opts, scaled=False)
        nb = query(0, f, d, len(ks), p, h=h)
        lib.jk_destroy(h)
        h = handle(nb, opts)
        J = buf((len(ks), n, n), "J", False) if "J" in want else None
        K = buf((len(ks), n, n), "K", False) if "K" in want else None
        st = lib.jk_build(h, ct.byref(f), len(ks), d, ptr(J), ptr(K), p, None)
        if EXEC[0] and st == 0:
            Jo, Ko = oracle_mod().build(L, X, _ylist(X, Y, sym))
            if J is not None:
                check("J", J, Jo)
            if K is not None:
                check("K", K, Ko)
        return st, h
    return fn


def sliced_gemm_case(M, N, K, opts):
    def fn():
        A, B, C = buf((M, K), "A"), buf((N, K), "B"), buf((M, N), "C", False)
        lib.jk_debug_sliced_gemm_workspace.restype = ct.c_size_t
        nb = lib.jk_debug_sliced_gemm_workspace(M, N, K)
        h = handle(nb, opts)
        st = lib.jk_debug_sliced_gemm(h, M, N, K, ptr(A), ptr(B), ptr(C), None)
        if EXEC[0] and st == 0:
            check("C", C, A.astype(np.longdouble) @ B.T.astype(np.longdouble))
        return st, h
    return fn


def autotune_batched_case(shapes, p):
    def fn():
        fs, ds, outs = [], [], []
        for m, (n, naux, ks) in enumerate(shapes):
            f, d, *_ = mol(n, naux, ks, [False] * len(ks), tag=f"m{m}")
            fs.append(f)
            ds += list(d)
            outs += [(buf((n, n), f"J{m}.{s}", False), buf((n, n), f"K{m}.{s}", False)) for s in range(len(ks))]
        fa = (jk_factor * len(fs))(*fs)
        da = (jk_density * len(ds))(*ds)
        ndm = [len(s[2]) for s in shapes]
        nb = query(2, fa, da, len(ds), p, nmol=len(fs), ndm=ndm)
        h = handle(4 * nb, {})
        Jp = (ct.c_void_p * len(outs))(*[o[0].ctypes.data for o in outs])
        Kp = (ct.c_void_p * len(outs))(*[o[1].ctypes.data for o in outs])
        cfg, ms = jk_tune_config(), ct.c_double()
        st = lib.jk_autotune_batched(h, len(fs), fa, (ct.c_int32 * len(ndm))(*ndm), da, Jp, Kp, p, None, 1,
                                     ct.byref(cfg), ct.byref(ms))
        lib.jk_tune_clear()
        return st, h
    return fn


def batched_case(shapes, p, opts, sym=False):
    def fn():
        fs, ds, outs, mols = [], [], [], []
        for m, (n, naux, ks) in enumerate(shapes):
            sy = [sym and s % 2 == 0 for s in range(len(ks))]     # every other density symmetric
            f, d, L, X, Y = mol(n, naux, ks, sy, tag=f"m{m}")
            fs.append(f)
            ds += list(d)
            mols.append((L, X, _ylist(X, Y, sy)))
            outs += [(buf((n, n), f"J{m}.{s}", False), buf((n, n), f"K{m}.{s}", False)) for s in range(len(ks))]
        fa = (jk_factor * len(fs))(*fs)
        da = (jk_density * len(ds))(*ds)
        ndm = [len(s[2]) for s in shapes]
        h = handle(1 << 20, opts, scaled=False)
        nb = query(2, fa, da, len(ds), p, nmol=len(fs), ndm=ndm, h=h)
        lib.jk_destroy(h)
        h = handle(nb, opts)
        Jp = (ct.c_void_p * len(outs))(*[o[0].ctypes.data for o in outs])
        Kp = (ct.c_void_p * len(outs))(*[o[1].ctypes.data for o in outs])
        st = lib.jk_build_batched(h, len(fs), fa, (ct.c_int32 * len(ndm))(*ndm), da, Jp, Kp, p, None)
        if EXEC[0] and st == 0:
            i = 0
            for m, (L, X, Y) in enumerate(mols):
                Jo, Ko = oracle_mod().build(L, X, Y)
                for s_ in range(len(X)):
                    check(f"J{m}.{s_}", outs[i][0], Jo[s_])
                    check(f"K{m}.{s_}", outs[i][1], Ko[s_])
                    i += 1
        return st, h
    return fn


def host_case(n, naux, ks, p, opts, packed=False):
    def fn():
        f, d, L, X, Y = mol(n, naux, ks, [False] * len(ks))
        if packed:
            Lp = buf((naux, n * (n + 1) // 2), "Lpacked", fill=False)
            if not BIG[0]:
                iu = np.triu_indices(n)
                Lp[...] = L[:, iu[0], iu[1]]
            f = jk_factor(n, naux, Lp.ctypes.data)
        h = handle(1 << 20, opts, scaled=False)
        nb = query(8 if packed else 3, f, d, len(ks), p, h=h)
        lib.jk_destroy(h)
        h = handle(nb, opts)
        J, K = buf((len(ks), n, n), "J", False), buf((len(ks), n, n), "K", False)
        call = lib.jk_build_host_packed if packed else lib.jk_build_host
        st = call(h, ct.byref(f), len(ks), d, ptr(J), ptr(K), p, None)
        if EXEC[0] and st == 0:
            Jo, Ko = oracle_mod().build(L, X, Y)
            check("J", J, Jo)
            check("K", K, Ko)
        return st, h
    return fn


def adjoint_case(n, naux, ks, sym, p, opts, want_dl=True):
    def fn():
        f, d, L, X, Y = mol(n, naux, ks, sym)
        nd, tot = len(ks), n * sum(ks)
        W, V = buf((nd, n, n), "W"), buf((nd, n, n), "V")
        dX, dY = buf((tot,), "dX", False), buf((tot,), "dY", False)
        dL = buf((naux, n, n), "dL", False) if want_dl else None
        h = handle(1 << 20, opts, scaled=False)
        nb = query(1, f, d, nd, p, h=h)
        lib.jk_destroy(h)
        h = handle(nb, opts)
        st = lib.jk_adjoint(h, ct.byref(f), nd, d, ptr(W), ptr(V), ptr(dX), ptr(dY), ptr(dL), p, None)
        if EXEC[0] and st == 0:
            dXo, dYo, dLo = oracle_mod().adjoint(L, X, _ylist(X, Y, sym), list(W), list(V), want_dl=want_dl)
            off = 0
            for s_, k in enumerate(ks):
                gx, gy = dX[off:off + n * k].reshape(n, k), dY[off:off + n * k].reshape(n, k)
                check(f"dX{s_}", gx, dXo[s_] + dYo[s_] if sym[s_] else dXo[s_])
                if not sym[s_]:
                    check(f"dY{s_}", gy, dYo[s_])
                off += n * k
            if want_dl:
                check("dL", dL, dLo)
        return st, h
    return fn


def dense_case(n, naux, nd, p, opts, grad=None):
    def fn():
        L = buf((naux, n, n), "L")
        if not BIG[0]:
            L[...] = L + L.transpose(0, 2, 1)
        f = factor_of(L, n, naux, "m")
        A, B = buf((nd, n, n), "A"), buf((nd, n, n), "B")
        O1, O2 = buf((nd, n, n), "O1", False), buf((nd, n, n), "O2", False)
        h = handle(1 << 20, opts, scaled=False)
        nb = query(5 if grad else 4, f, None, nd, p, h=h)
        lib.jk_destroy(h)
        h = handle(nb, opts)
        if grad is None:
            st = lib.jk_build_dense(h, ct.byref(f), nd, ptr(A), ptr(O1), ptr(O2), p, None)
            if EXEC[0] and st == 0:
                Jo, Ko = oracle_mod().build_dense(L, A)
                check("J", O1, Jo)
                check("K", O2, Ko)
            return st, h
        W = A if "W" in grad else None
        V = B if "V" in grad else None
        st = lib.jk_density_grad(h, ct.byref(f), nd, ptr(W), ptr(V), ptr(O1), p, None)
        if EXEC[0] and st == 0:
            check("G", O1, oracle_mod().density_grad(L, W, V, nd=nd))
        return st, h
    return fn


def pair_case(n, naux, kl, sl, kr, sr, p, opts):
    def fn():
        f, dl, L, XL, YL = mol(n, naux, kl, sl, tag="left")
        XR = [buf((n, k), f"right.X{s}") for s, k in enumerate(kr)]
        YR = [buf((n, k), f"right.Y{s}") for s, k in enumerate(kr)]
        dr = (jk_density * len(kr))()
        for s, k in enumerate(kr):
            dr[s].k, dr[s].symmetric, dr[s].X = k, int(sr[s]), XR[s].ctypes.data
            dr[s].Y = None if sr[s] else YR[s].ctypes.data
        both = (jk_density * (len(kl) + len(kr)))(*dl, *dr)
        h = handle(1 << 20, opts, scaled=False)
        nb = query(6, (jk_factor * 2)(f, f), both, len(kl) + len(kr), p, nmol=2, ndm=[len(kl), len(kr)], h=h)
        lib.jk_destroy(h)
        h = handle(nb, opts)
        Jp, Kp = buf((len(kl), len(kr)), "Jp", False), buf((len(kl), len(kr)), "Kp", False)
        st = lib.jk_pair(h, ct.byref(f), len(kl), dl, len(kr), dr, ptr(Jp), ptr(Kp), p, None)
        if EXEC[0] and st == 0:
            Jo, Ko = oracle_mod().pairs(L, XL, _ylist(XL, YL, sl), XR, _ylist(XR, YR, sr))
            check("Jp", Jp, Jo)
            check("Kp", Kp, Ko)
        return st, h
    return fn


def laplace_case(n, naux, m, nq, sym, weighted, p, opts):
    def fn():
        L = buf((naux, n, n), "L")
        if not BIG[0]:
            L[...] = L + L.transpose(0, 2, 1)
        f = factor_of(L, n, naux, "m")
        CX, CY = buf((n, m), "CX"), buf((n, m), "CY")
        eX, eY = buf((m,), "epsX"), buf((m,), "epsY")
        d = (jk_density * 1)()
        d[0].k, d[0].symmetric = m, int(sym)
        h = handle(1 << 20, opts, scaled=False)
        nb = query(7, f, d, nq, p, h=h)
        lib.jk_destroy(h)
        h = handle(nb, opts)
        shape = (n, n) if weighted else (nq, n, n)
        J, K = buf(shape, "J", False), buf(shape, "K", False)
        alpha = (ct.c_double * nq)(*[0.2 * (k + 1) for k in range(nq)])
        w = (ct.c_double * nq)(*[1.0 / (k + 1) for k in range(nq)]) if weighted else None
        lib.jk_build_laplace.argtypes = [ct.c_void_p, ct.POINTER(jk_factor), ct.c_int32, ct.POINTER(ct.c_double),
                                         ct.POINTER(ct.c_double), ct.c_int32, ct.c_void_p, ct.c_void_p, ct.c_int32,
                                         ct.c_void_p, ct.c_void_p, ct.c_int32, ct.c_void_p, ct.c_void_p, ct.c_int,
                                         ct.c_void_p]
        st = lib.jk_build_laplace(h, ct.byref(f), nq, alpha, w, m, ptr(CX), ptr(eX), 1,
                                  None if sym else ptr(CY), None if sym else ptr(eY), 0 if sym else -1,
                                  ptr(J), ptr(K), p, None)
        if EXEC[0] and st == 0:
            Jo, Ko = oracle_mod().laplace(L, CX, eX, 1, CX if sym else CY, eX if sym else eY, 1 if sym else -1,
                                          np.array(alpha[:]), np.array(w[:]) if weighted else None)
            check("J", J, Jo)
            check("K", K, Ko)
        return st, h
    return fn


def pack_factor_case(n, naux):
    """jk_pack_factor, then a build on the packed factor it wrote."""
    def fn():
        f, d, L, X, Y = mol(n, naux, [5, 3], [False, True])
        h = handle(1 << 20, {}, scaled=False)
        P = buf((naux, n * (n + 1) // 2), "P", False)
        lib.jk_pack_factor.argtypes = [ct.c_void_p, ct.c_int32, ct.c_int32, ct.c_void_p, ct.c_void_p, ct.c_void_p]
        st = lib.jk_pack_factor(h, n, naux, ptr(L), ptr(P), None)
        if st != 0:
            return st, h
        bad = [lib.jk_pack_factor(h, 0, naux, ptr(L), ptr(P), None), lib.jk_pack_factor(h, n, 0, ptr(L), ptr(P), None),
               lib.jk_pack_factor(h, n, naux, None, ptr(P), None),
               lib.jk_pack_factor(h, n, naux, ptr(L), ct.c_void_p(L.ctypes.data + 8), None)]
        assert bad == [2, 2, 1, 1], bad
        if EXEC[0]:
            iu = np.triu_indices(n)
            check("P", P, L[:, iu[0], iu[1]])
        lib.jk_destroy(h)
        opts = {"packed_factor": 1}
        h = handle(1 << 20, opts, scaled=False)
        fp = jk_factor(n, naux, P.ctypes.data)
        nb = query(0, fp, d, 2, SPLIT, h=h)
        lib.jk_destroy(h)
        h = handle(nb, opts)
        J, K = buf((2, n, n), "J", False), buf((2, n, n), "K", False)
        st = lib.jk_build(h, ct.byref(fp), 2, d, ptr(J), ptr(K), SPLIT, None)
        if EXEC[0] and st == 0:
            Jo, Ko = oracle_mod().build(L, X, _ylist(X, Y, [False, True]))
            check("J", J, Jo)
            check("K", K, Ko)
        return st, h
    return fn


def packed_refused_case():
    """With JK_OPT_PACKED_FACTOR set, the host builds (their factor is in host
    memory) refuse the call before any device work."""
    def fn():
        n, naux, ks = 20, 30, [3, 4]
        f, d, L, X, Y = mol(n, naux, ks, [False, False])
        nd = len(ks)
        h = handle(1 << 24, {"packed_factor": 1}, scaled=False)
        O = buf((nd, n, n), "O", False)
        got = {
            "host": lib.jk_build_host(h, ct.byref(f), nd, d, ptr(O), None, SPLIT, None),
            "host_packed": lib.jk_build_host_packed(h, ct.byref(f), nd, d, ptr(O), None, SPLIT, None),
        }
        nb = ct.c_size_t()
        for op in (3, 8):
            got[f"query{op}"] = lib.jk_workspace_query_handle(h, op, 1, (jk_factor * 1)(f), None, nd, d, SPLIT,
                                                               ct.byref(nb))
        bad = {k: v for k, v in got.items() if v != 6}
        assert not bad, bad
        return 0, h
    return fn


def j_path_threshold_case():
    """The workspace queries follow the split builds' J path: the automatic
    choice equals the tensor-core form's size above 4e9 multiply-adds of J's
    FP64 work (the headline workload) and the FP64 form's below it (the
    multi-state workload), and the two forms' sizes differ (the tensor-core
    form takes the transposed chunk's slices, and its aux chunk is smaller
    where the workspace budget bounds it).  Only sizes are queried: the factor
    is never touched."""
    def fn():
        got = {}
        for label, n, naux, ks in (("headline", 1000, 5000, [100] * 16), ("multi_state", 400, 2400, [40] * 8)):
            f = jk_factor(n, naux, ct.c_void_p(1 << 20))
            d = (jk_density * len(ks))()
            for s_, k in enumerate(ks):
                d[s_].k, d[s_].symmetric, d[s_].X, d[s_].Y = k, 0, 1 << 20, 1 << 20
            q = {"auto": query(0, f, d, len(ks), SPLIT)}
            for jp in (-1, 0, 1):
                h = handle(1 << 20, {"j_path": jp}, scaled=False)
                q[jp] = query(0, f, d, len(ks), SPLIT, h=h)
                lib.jk_destroy(h)
            got[label] = q
        hd, ms = got["headline"], got["multi_state"]
        assert hd["auto"] == hd[-1] == hd[1] != hd[0], hd
        assert ms["auto"] == ms[-1] == ms[0] != ms[1], ms
        return 0, None
    return fn


def noalloc_case(n, naux, ks):
    def fn():
        f, d, L, X, Y = mol(n, naux, ks, [False] * len(ks))
        J, K = buf((len(ks), n, n), "J", False), buf((len(ks), n, n), "K", False)
        st = lib.jk_build_noalloc(ct.byref(f), len(ks), d, ptr(J), ptr(K), None)
        if EXEC[0] and st == 0:
            Jo, Ko = oracle_mod().build(L, X, Y)
            check("J", J, Jo)
            check("K", K, Ko)
        return st, None
    return fn


def autotune_case(n, naux, ks, p):
    def fn():
        f, d, *_ = mol(n, naux, ks, [False] * len(ks))
        nb = query(0, f, d, len(ks), p)
        h = handle(4 * nb, {})
        J, K = buf((len(ks), n, n), "J", False), buf((len(ks), n, n), "K", False)
        cfg, ms = jk_tune_config(), ct.c_double()
        st = lib.jk_autotune(h, ct.byref(f), len(ks), d, ptr(J), ptr(K), p, None, 1, ct.byref(cfg), ct.byref(ms))
        lib.jk_tune_clear()
        return st, h
    return fn


FP64, SPLIT = 0, 1
CASES = {
    "build_fp64": build_case(37, 53, [5, 1, 13], [False, True, False], FP64, {}),
    "build_fp64_chunks": build_case(37, 53, [5, 1, 13], [False, True, False], FP64, {"aux_chunk": 17}),
    "build_split": build_case(37, 53, [5, 1, 13], [False, True, False], SPLIT, {}),
    "build_split_grouped_raster1": build_case(130, 70, [64, 3, 9], [False, False, True], SPLIT,
                                              {"schedule": 1, "raster": 1, "aux_chunk": 17}),
    "build_split_raster1_chunks": build_case(130, 70, [64, 3, 9], [False, False, True], SPLIT,
                                             {"schedule": 0, "raster": 1, "aux_chunk": 30}),
    "build_split_nbf_above_superchunk": build_case(2100, 3, [2], [False], SPLIT, {}),
    "build_split_fp32_digits": build_case(400, 60, [40, 40], [True, False], SPLIT, {"slicer": 1, "schedule": 1}),
    "build_split_j_only": build_case(37, 53, [5, 13], [False, True], SPLIT, {}, want="J"),
    "build_split_j_tensor": build_case(37, 53, [5, 1, 13], [False, True, False], SPLIT, {"j_path": 1}),
    "build_split_j_tensor_chunks": build_case(130, 70, [9, 3, 20], [False, True, False], SPLIT,
                                              {"j_path": 1, "aux_chunk": 17}),
    "build_split_j_tensor_grouped": build_case(130, 70, [9, 3, 20], [False, True, False], SPLIT,
                                               {"j_path": 1, "schedule": 1, "aux_chunk": 30}),
    "build_split_j_tensor_superchunks": build_case(20, 2100, [3, 2], [False, True], SPLIT, {"j_path": 1}),
    "build_split_j_tensor_j_only": build_case(37, 53, [5, 13], [False, True], SPLIT, {"j_path": 1}, want="J"),
    "build_split_j_tensor_packed": packed(build_case(130, 70, [9, 3, 20], [False, True, False], SPLIT,
                                                     {"j_path": 1, "packed_factor": 1, "aux_chunk": 30})),
    "batched_split_j_tensor": batched_case([(60, 150, [6, 6]), (111, 222, [11]), (33, 99, [3, 3, 3])], SPLIT,
                                           {"j_path": 1}),
    "batched_split_j_tensor_packed": packed(batched_case([(60, 150, [6, 6]), (140, 222, [11])], SPLIT,
                                                         {"j_path": 1, "packed_factor": 1}, sym=True)),
    "build_split_syrk": build_case(300, 70, [20, 9, 33], [True, False, True], SPLIT,
                                   {"syrk": 1, "schedule": 0, "aux_chunk": 30}),
    "build_split_syrk_partials": build_case(300, 120, [40, 7], [True, True], SPLIT,
                                            {"syrk": 1, "schedule": 0, "aux_chunk": 70}),
    "build_split_syrk_grouped": build_case(257, 90, [64, 5, 11], [True, True, False], SPLIT,
                                           {"syrk": 1, "schedule": 1, "aux_chunk": 40}),
    "build_fp64_syrk": build_case(300, 70, [20, 9, 33], [True, False, True], FP64, {"syrk": 1, "aux_chunk": 30}),
    "build_fp64_syrk_packed": packed(build_case(257, 40, [12, 5], [True, True], FP64,
                                                {"syrk": 1, "packed_factor": 1})),
    "build_split_syrk_small_raster1": build_case(100, 30, [7, 4], [True, False], SPLIT,
                                                 {"syrk": 1, "schedule": 1, "raster": 1}),
    "batched_split_syrk": batched_case([(60, 150, [6, 6]), (140, 222, [11]), (33, 99, [3, 3, 3])], SPLIT,
                                       {"syrk": 1}, sym=True),
    "build_split_k_only_grouped": build_case(37, 53, [5, 13], [False, True], SPLIT, {"schedule": 1}, want="K"),
    "build_fp64_j_only": build_case(37, 53, [5, 13], [False, True], FP64, {}, want="J"),
    "sliced_gemm": sliced_gemm_case(129, 257, 2047, {}),
    "sliced_gemm_split_k_raster1": sliced_gemm_case(140, 130, 5000, {"raster": 1}),
    "autotune_batched_split": autotune_batched_case([(60, 150, [6, 6]), (111, 222, [11]), (33, 99, [3, 3])], SPLIT),
    "batched_split": batched_case([(60, 150, [6, 6]), (111, 222, [11]), (33, 99, [3, 3, 3])], SPLIT, {}),
    "batched_fp64": batched_case([(60, 150, [6, 6]), (33, 99, [3])], FP64, {}),
    "host_split": host_case(64, 200, [8, 5], SPLIT, {"host_chunk": 37}),
    "host_fp64": host_case(64, 200, [8, 5], FP64, {}),
    "host_packed_split": host_case(64, 200, [8, 5], SPLIT, {"host_chunk": 37}, packed=True),
    "host_packed_fp64": host_case(33, 90, [4], FP64, {}, packed=True),
    "adjoint_fp64": adjoint_case(33, 41, [4, 5], [True, False], FP64, {}),
    "adjoint_split": adjoint_case(70, 150, [8, 16, 3], [False, False, True], SPLIT, {}),
    "adjoint_split_no_dl_chunks": adjoint_case(70, 150, [8, 3], [False, False], SPLIT, {"aux_chunk": 40}, False),
    "dense_fp64": dense_case(37, 53, 3, FP64, {}),
    "dense_fp64_chunks": dense_case(37, 53, 3, FP64, {"aux_chunk": 17}),
    "dense_split": dense_case(130, 70, 2, SPLIT, {}),
    "dense_split_chunks": dense_case(130, 70, 2, SPLIT, {"aux_chunk": 30}),
    "dense_split_raster1": dense_case(37, 53, 3, SPLIT, {"aux_chunk": 17, "raster": 1}),
    "dense_split_nbf_above_superchunk": dense_case(2100, 2, 1, SPLIT, {}),
    "grad_split_WV": dense_case(37, 53, 3, SPLIT, {"aux_chunk": 17}, grad="WV"),
    "grad_split_W": dense_case(37, 53, 3, SPLIT, {}, grad="W"),
    "grad_fp64_V": dense_case(37, 53, 3, FP64, {}, grad="V"),
    "pairs_fp64": pair_case(40, 60, [3, 5], [False, True], [4, 6, 2], [False, False, True], FP64, {}),
    "pairs_split": pair_case(130, 70, [9, 3], [False, False], [12, 5], [True, False], SPLIT, {}),
    "pairs_split_grouped": pair_case(40, 60, [3, 5], [False, True], [4, 6, 2], [False, False, True], SPLIT,
                                     {"schedule": 1}),
    "laplace_split": laplace_case(37, 53, 5, 4, False, False, SPLIT, {}),
    "laplace_split_weighted_sym": laplace_case(130, 70, 9, 3, True, True, SPLIT, {}),
    "laplace_fp64_weighted": laplace_case(37, 53, 5, 4, False, True, FP64, {}),
    "noalloc": noalloc_case(37, 53, [5, 1, 13]),
    "build_split_packed": packed(build_case(130, 70, [9, 3, 20], [False, True, False], SPLIT,
                                            {"packed_factor": 1, "aux_chunk": 30})),
    "build_split_packed_grouped_syrk": packed(build_case(
        257, 90, [64, 5], [True, False], SPLIT, {"packed_factor": 1, "schedule": 1, "aux_chunk": 40, "syrk": 1})),
    "build_split_packed_j_only": packed(build_case(37, 53, [5, 13], [False, True], SPLIT,
                                                   {"packed_factor": 1, "aux_chunk": 17}, want="J")),
    "build_fp64_packed": packed(build_case(37, 53, [5, 1, 13], [False, True, False], FP64,
                                           {"packed_factor": 1, "aux_chunk": 17})),
    "build_fp64_packed_j_only": packed(build_case(37, 53, [5, 13], [False, True], FP64,
                                                  {"packed_factor": 1, "aux_chunk": 17}, want="J")),
    "batched_split_packed": packed(batched_case([(60, 150, [6, 6]), (140, 222, [11]), (33, 99, [3, 3, 3])], SPLIT,
                                                {"packed_factor": 1}, sym=True)),
    "batched_fp64_packed": packed(batched_case([(60, 150, [6, 6]), (33, 99, [3])], FP64, {"packed_factor": 1})),
    "pairs_split_packed": packed(pair_case(40, 60, [3, 5], [False, True], [4, 6, 2], [False, False, True], SPLIT,
                                           {"packed_factor": 1})),
    "laplace_split_packed": packed(laplace_case(37, 53, 5, 4, False, True, SPLIT, {"packed_factor": 1})),
    "pack_factor_then_build": pack_factor_case(70, 45),
    "dense_split_packed": packed(dense_case(130, 70, 2, SPLIT, {"packed_factor": 1, "aux_chunk": 30})),
    "dense_fp64_packed": packed(dense_case(37, 53, 3, FP64, {"packed_factor": 1, "aux_chunk": 17})),
    "grad_split_WV_packed": packed(dense_case(37, 53, 3, SPLIT, {"packed_factor": 1}, grad="WV")),
    "grad_fp64_V_packed": packed(dense_case(40, 33, 2, FP64, {"packed_factor": 1}, grad="V")),
    "adjoint_split_packed": packed(adjoint_case(70, 150, [8, 16, 3], [False, False, True], SPLIT,
                                                {"packed_factor": 1, "aux_chunk": 40})),
    "adjoint_fp64_packed": packed(adjoint_case(33, 41, [4, 5], [True, False], FP64,
                                               {"packed_factor": 1, "aux_chunk": 10})),
    "autotune_split": autotune_case(37, 53, [5, 13], SPLIT),
}

# Full sizes of the measured workloads (bench.py): only the host path runs, so
# the factors are never touched and cost no memory beyond their page tables.
FULL_CASES = {
    "full_multi_state_tuned": build_case(400, 2400, [40] * 8, [True] + [False] * 7, SPLIT,
                                         {"aux_chunk": 3834, "schedule": 1, "raster": 0}),
    "full_multi_state_default": build_case(400, 2400, [40] * 8, [True] + [False] * 7, SPLIT, {}),
    "full_multi_state_syrk": build_case(400, 2400, [40] * 8, [True] + [False] * 7, SPLIT,
                                        {"aux_chunk": 3834, "schedule": 1, "raster": 0, "syrk": 1}),
    "full_multi_state_raster1": build_case(400, 2400, [40] * 8, [True] + [False] * 7, SPLIT,
                                           {"schedule": 1, "raster": 1}),
    "full_dense": dense_case(400, 2400, 8, SPLIT, {}),
    "full_density_grad": dense_case(400, 2400, 8, SPLIT, {}, grad="WV"),
    "full_pairs": pair_case(400, 2400, [40] * 8, [False] * 8, [40] * 8, [False] * 8, SPLIT, {}),
    "full_laplace": laplace_case(400, 2400, 40, 8, False, True, SPLIT, {}),
    "full_adjoint": adjoint_case(600, 3600, [60] * 8, [False] * 8, SPLIT, {}),
    "full_host": host_case(400, 2400, [40] * 8, SPLIT, {}),
    "full_host_packed": host_case(400, 2400, [40] * 8, SPLIT, {}, packed=True),
    "full_multi_state_packed": packed(build_case(400, 2400, [40] * 8, [True] + [False] * 7, SPLIT,
                                                 {"packed_factor": 1, "schedule": 1})),
}

# Calls that must be refused before any device work, and query-only checks
# (run by name only).
REFUSE_CASES = {
    "packed_refused": packed_refused_case(),
    "j_path_threshold": j_path_threshold_case(),
}

# ---- random cases ----------------------------------------------------------------
EDGE_N = [1, 2, 3, 4, 7, 8, 15, 16, 17, 31, 33, 63, 64, 65, 79, 80, 81, 127, 128, 129, 160, 255, 256, 257]


def fuzz_cases(count, seed):
    """Random entry points, shapes (edges of the 128 x 80 tiles, the 16-element
    K-steps and odd sizes) and options; sizes kept small enough for host memory."""
    g = np.random.default_rng(seed)
    out = {}
    for i in range(count):
        n = int(g.choice(EDGE_N)) if g.random() < 0.6 else int(g.integers(1, 300))
        naux = int(g.integers(1, max(2, min(400, 6_000_000 // (n * n)))))
        nd = int(g.integers(1, 5)) if g.random() < 0.8 else int(g.integers(5, 65))
        ks = [int(g.integers(1, min(4 * n, 80) + 1)) for _ in range(nd)]
        sym = [bool(g.random() < 0.3) for _ in range(nd)]
        p = int(g.integers(0, 2))
        opts = {}
        if g.random() < 0.5:
            opts["aux_chunk"] = int(g.integers(1, naux + 3))
        for name in ("schedule", "raster", "slicer", "syrk", "j_path"):
            if g.random() < 0.5:
                opts[name] = int(g.integers(0, 2))
        kind = g.choice(["build", "adjoint", "dense", "grad", "pairs", "laplace", "batched", "host"])
        pk = kind != "host" and g.random() < 0.3   # packed device factor
        if pk:
            opts["packed_factor"] = 1
        label = f"fuzz{i}_{kind}_n{n}_a{naux}_p{p}" + ("_packed" if pk else "")
        if kind == "build":
            out[label] = build_case(n, naux, ks, sym, p, opts, want=str(g.choice(["JK", "JK", "J", "K"])))
        elif kind == "adjoint":
            out[label] = adjoint_case(n, naux, ks[:4], sym[:4], p, opts, want_dl=bool(g.random() < 0.5))
        elif kind == "dense":
            out[label] = dense_case(n, naux, min(nd, 8), p, opts)
        elif kind == "grad":
            out[label] = dense_case(n, naux, min(nd, 8), p, opts, grad=str(g.choice(["W", "V", "WV"])))
        elif kind == "pairs":
            nr = int(g.integers(1, 5))
            out[label] = pair_case(n, naux, ks[:4], sym[:4], ks[:nr], [False] * nr, p, opts)
        elif kind == "laplace":
            out[label] = laplace_case(n, naux, ks[0], int(g.integers(1, 9)), bool(g.random() < 0.5),
                                      bool(g.random() < 0.5), p, opts)
        elif kind == "batched":
            shapes = []
            for _ in range(int(g.integers(1, 5))):
                nm = int(g.integers(1, 120))
                shapes.append((nm, int(g.integers(1, 150)),
                               [int(g.integers(1, min(20, 4 * nm) + 1)) for _ in range(int(g.integers(1, 4)))]))
            out[label] = batched_case(shapes, p, {k: v for k, v in opts.items() if k != "schedule"})
        else:
            opts.pop("schedule", None)
            if g.random() < 0.5:
                opts["host_chunk"] = int(g.integers(1, naux + 3))
            out[label] = host_case(n, naux, ks[:4], p, opts)
        if pk:
            out[label] = packed(out[label])
    return out


if __name__ == "__main__":
    args = sys.argv[1:]
    for a in [a for a in args if a.startswith("--fuzz=")]:
        count, seed = (int(v) for v in a.split("=", 1)[1].split(","))
        CASES.clear()
        CASES.update(fuzz_cases(count, seed))
        args.remove(a)
    for a in [a for a in args if a.startswith("--arena-scale=")]:
        ARENA_SCALE[0] = float(a.split("=", 1)[1])
        args.remove(a)
    if "--twice" in args:
        TWICE[0] = True
        args.remove("--twice")
    if "--exec" in args:
        EXEC[0] = True
        args.remove("--exec")
    for a in [a for a in args if a.startswith("--fail-launch=")]:
        FAIL_AT[0] = int(a.split("=", 1)[1])
        args.remove(a)
    names = args or list(CASES)
    for name in names:
        BIG[0] = name in FULL_CASES
        run(name, CASES.get(name) or FULL_CASES.get(name) or REFUSE_CASES[name])
