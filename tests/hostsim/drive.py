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
    _fields_ = [("aux_chunk", ct.c_int32), ("schedule", ct.c_int32), ("raster", ct.c_int32), ("cluster", ct.c_int32)]


lib = ct.CDLL(os.path.join(ROOT, "paper_2608_06536_b300", "libjk.so"))
lib.jk_last_error.restype = ct.c_char_p
shim = ct.CDLL("libcudart.so.13")
shim.shim_launch.restype = ct.c_char_p
assert hasattr(shim, "shim_reset"), "the stand-in runtime is not the one loaded"

OPT = {"aux_chunk": 0, "schedule": 1, "raster": 2, "use_tuned": 3, "cluster": 4, "host_chunk": 5}
rng = np.random.default_rng(0)
owned = []      # (base, nbytes, label) of every buffer a case hands to the library


def buf(shape, label, fill=True):
    """A 256-byte aligned float64 array the library may address."""
    n = int(np.prod(shape))
    raw = np.zeros(n * 8 + 256, np.uint8)
    off = (-raw.ctypes.data) % 256
    a = raw[off:off + n * 8].view(np.float64).reshape(shape)
    if fill:
        a[...] = rng.standard_normal(shape) / max(shape[-1], 1)
    owned.append((a.ctypes.data, a.nbytes, label, raw))
    return a


def ptr(a):
    return None if a is None else ct.c_void_p(a.ctypes.data)


def mol(n, naux, ks, sym, tag="m"):
    L = buf((naux, n, n), f"{tag}.L")
    X = [buf((n, k), f"{tag}.X{s}") for s, k in enumerate(ks)]
    Y = [buf((n, k), f"{tag}.Y{s}") for s, k in enumerate(ks)]
    d = (jk_density * len(ks))()
    for s, k in enumerate(ks):
        d[s].k, d[s].symmetric, d[s].X = k, int(sym[s]), X[s].ctypes.data
        d[s].Y = None if sym[s] else Y[s].ctypes.data
    return jk_factor(n, naux, L.ctypes.data), d, L, X, Y


def handle(nbytes, opts):
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
                      "owned": [[o[0], o[1], o[2]] for o in owned]}), flush=True)


def run(name, fn):
    owned.clear()
    shim.shim_reset()
    status, h = fn()
    record(name, status, h)
    if h:
        lib.jk_destroy(h)


# ---- the cases ----------------------------------------------------------------

def build_case(n, naux, ks, sym, p, opts):
    def fn():
        f, d, *_ = mol(n, naux, ks, sym)
        h = handle(1 << 20, opts)
        nb = query(0, f, d, len(ks), p, h=h)
        lib.jk_destroy(h)
        h = handle(nb, opts)
        J, K = buf((len(ks), n, n), "J", False), buf((len(ks), n, n), "K", False)
        return lib.jk_build(h, ct.byref(f), len(ks), d, ptr(J), ptr(K), p, None), h
    return fn


def batched_case(shapes, p, opts):
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
        h = handle(1 << 20, opts)
        nb = query(2, fa, da, len(ds), p, nmol=len(fs), ndm=ndm, h=h)
        lib.jk_destroy(h)
        h = handle(nb, opts)
        Jp = (ct.c_void_p * len(outs))(*[o[0].ctypes.data for o in outs])
        Kp = (ct.c_void_p * len(outs))(*[o[1].ctypes.data for o in outs])
        return lib.jk_build_batched(h, len(fs), fa, (ct.c_int32 * len(ndm))(*ndm), da, Jp, Kp, p, None), h
    return fn


def host_case(n, naux, ks, p, opts):
    def fn():
        f, d, *_ = mol(n, naux, ks, [False] * len(ks))
        h = handle(1 << 20, opts)
        nb = query(3, f, d, len(ks), p, h=h)
        lib.jk_destroy(h)
        h = handle(nb, opts)
        J, K = buf((len(ks), n, n), "J", False), buf((len(ks), n, n), "K", False)
        return lib.jk_build_host(h, ct.byref(f), len(ks), d, ptr(J), ptr(K), p, None), h
    return fn


def adjoint_case(n, naux, ks, sym, p, opts, want_dl=True):
    def fn():
        f, d, *_ = mol(n, naux, ks, sym)
        nd, tot = len(ks), n * sum(ks)
        W, V = buf((nd, n, n), "W"), buf((nd, n, n), "V")
        dX, dY = buf((tot,), "dX", False), buf((tot,), "dY", False)
        dL = buf((naux, n, n), "dL", False) if want_dl else None
        h = handle(1 << 20, opts)
        nb = query(1, f, d, nd, p, h=h)
        lib.jk_destroy(h)
        h = handle(nb, opts)
        return lib.jk_adjoint(h, ct.byref(f), nd, d, ptr(W), ptr(V), ptr(dX), ptr(dY), ptr(dL), p, None), h
    return fn


def dense_case(n, naux, nd, p, opts, grad=None):
    def fn():
        L = buf((naux, n, n), "L")
        f = jk_factor(n, naux, L.ctypes.data)
        A, B = buf((nd, n, n), "A"), buf((nd, n, n), "B")
        O1, O2 = buf((nd, n, n), "O1", False), buf((nd, n, n), "O2", False)
        h = handle(1 << 20, opts)
        nb = query(5 if grad else 4, f, None, nd, p, h=h)
        lib.jk_destroy(h)
        h = handle(nb, opts)
        if grad is None:
            return lib.jk_build_dense(h, ct.byref(f), nd, ptr(A), ptr(O1), ptr(O2), p, None), h
        W = A if "W" in grad else None
        V = B if "V" in grad else None
        return lib.jk_density_grad(h, ct.byref(f), nd, ptr(W), ptr(V), ptr(O1), p, None), h
    return fn


def pair_case(n, naux, kl, sl, kr, sr, p, opts):
    def fn():
        f, dl, L, *_ = mol(n, naux, kl, sl, tag="left")
        XR = [buf((n, k), f"right.X{s}") for s, k in enumerate(kr)]
        YR = [buf((n, k), f"right.Y{s}") for s, k in enumerate(kr)]
        dr = (jk_density * len(kr))()
        for s, k in enumerate(kr):
            dr[s].k, dr[s].symmetric, dr[s].X = k, int(sr[s]), XR[s].ctypes.data
            dr[s].Y = None if sr[s] else YR[s].ctypes.data
        both = (jk_density * (len(kl) + len(kr)))(*dl, *dr)
        h = handle(1 << 20, opts)
        nb = query(6, (jk_factor * 2)(f, f), both, len(kl) + len(kr), p, nmol=2, ndm=[len(kl), len(kr)], h=h)
        lib.jk_destroy(h)
        h = handle(nb, opts)
        Jp, Kp = buf((len(kl), len(kr)), "Jp", False), buf((len(kl), len(kr)), "Kp", False)
        return lib.jk_pair(h, ct.byref(f), len(kl), dl, len(kr), dr, ptr(Jp), ptr(Kp), p, None), h
    return fn


def laplace_case(n, naux, m, nq, sym, weighted, p, opts):
    def fn():
        L = buf((naux, n, n), "L")
        f = jk_factor(n, naux, L.ctypes.data)
        CX, CY = buf((n, m), "CX"), buf((n, m), "CY")
        eX, eY = buf((m,), "epsX"), buf((m,), "epsY")
        d = (jk_density * 1)()
        d[0].k, d[0].symmetric = m, int(sym)
        h = handle(1 << 20, opts)
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
        return st, h
    return fn


def noalloc_case(n, naux, ks):
    def fn():
        f, d, *_ = mol(n, naux, ks, [False] * len(ks))
        J, K = buf((len(ks), n, n), "J", False), buf((len(ks), n, n), "K", False)
        return lib.jk_build_noalloc(ct.byref(f), len(ks), d, ptr(J), ptr(K), None), None
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
    "build_split_grouped_clustered": build_case(130, 70, [64, 3, 9], [False, False, True], SPLIT,
                                                {"schedule": 1, "cluster": 1, "raster": 1, "aux_chunk": 17}),
    "build_split_clustered_chunks": build_case(130, 70, [64, 3, 9], [False, False, True], SPLIT,
                                               {"schedule": 0, "cluster": 1, "aux_chunk": 30}),
    "build_split_nbf_above_superchunk": build_case(2100, 3, [2], [False], SPLIT, {}),
    "batched_split": batched_case([(60, 150, [6, 6]), (111, 222, [11]), (33, 99, [3, 3, 3])], SPLIT, {}),
    "batched_fp64": batched_case([(60, 150, [6, 6]), (33, 99, [3])], FP64, {}),
    "host_split": host_case(64, 200, [8, 5], SPLIT, {"host_chunk": 37}),
    "host_fp64": host_case(64, 200, [8, 5], FP64, {}),
    "adjoint_fp64": adjoint_case(33, 41, [4, 5], [True, False], FP64, {}),
    "adjoint_split": adjoint_case(70, 150, [8, 16, 3], [False, False, True], SPLIT, {}),
    "adjoint_split_no_dl_chunks": adjoint_case(70, 150, [8, 3], [False, False], SPLIT, {"aux_chunk": 40}, False),
    "dense_fp64": dense_case(37, 53, 3, FP64, {}),
    "dense_fp64_chunks": dense_case(37, 53, 3, FP64, {"aux_chunk": 17}),
    "dense_split": dense_case(130, 70, 2, SPLIT, {}),
    "dense_split_chunks": dense_case(130, 70, 2, SPLIT, {"aux_chunk": 30}),
    "dense_split_clustered": dense_case(37, 53, 3, SPLIT, {"aux_chunk": 17, "cluster": 1}),
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
    "autotune_split": autotune_case(37, 53, [5, 13], SPLIT),
}

if __name__ == "__main__":
    names = sys.argv[1:] or list(CASES)
    for name in names:
        run(name, CASES[name])
