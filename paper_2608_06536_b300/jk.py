"""Thin ctypes binding of libjk.so (argument marshalling only).

Every step of the J/K path runs in the library's CUDA kernels; this module
only turns torch tensors into device pointers and sizes, owns the workspace
arena (a torch byte tensor) and raises on a non-OK status.  There is no CPU
fallback: without the compiled library the import of the engine fails.
"""
from __future__ import annotations

import ctypes as ct
import os
import threading

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libjk.so")

JK_OK, JK_ERR_ARG, JK_ERR_SHAPE, JK_ERR_OOM, JK_ERR_CUDA, JK_ERR_TIMEOUT, JK_ERR_UNSUPPORTED = range(7)
JK_FP64, JK_SPLIT_BF16 = 0, 1
(JK_OP_BUILD, JK_OP_ADJOINT, JK_OP_BATCHED, JK_OP_BUILD_HOST, JK_OP_BUILD_DENSE, JK_OP_DENSITY_GRAD,
 JK_OP_PAIR, JK_OP_LAPLACE, JK_OP_BUILD_HOST_PACKED) = range(9)

PRECISIONS = {"fp64": JK_FP64, "split": JK_SPLIT_BF16, "split_bf16": JK_SPLIT_BF16}


class jk_factor(ct.Structure):
    _fields_ = [("nbf", ct.c_int32), ("naux", ct.c_int32), ("L", ct.c_void_p)]


class jk_density(ct.Structure):
    _fields_ = [("k", ct.c_int32), ("symmetric", ct.c_int32),
                ("X", ct.c_void_p), ("Y", ct.c_void_p)]


class jk_tune_config(ct.Structure):
    _fields_ = [("aux_chunk", ct.c_int32), ("schedule", ct.c_int32), ("raster", ct.c_int32), ("tile", ct.c_int32)]

    def as_dict(self) -> dict:
        return {"aux_chunk": self.aux_chunk, "schedule": self.schedule, "raster": self.raster, "tile": self.tile}


OPTIONS = {"aux_chunk": 0, "schedule": 1, "raster": 2, "use_tuned": 3, "host_chunk": 5, "slicer": 6,
           "syrk": 7, "packed_factor": 8, "tile": 9, "adjoint_slices": 10, "j_path": 11}
# each option's value on a fresh handle (-1: not set, tuned or default configuration)
OPTION_DEFAULTS = {"aux_chunk": -1, "schedule": -1, "raster": -1, "use_tuned": 1, "host_chunk": 0,
                   "slicer": 0, "syrk": 0, "packed_factor": 0, "tile": -1, "adjoint_slices": 7, "j_path": -1}


class JKError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"jk status {status}: {msg}")
        self.status = status


_lib = None
_lib_lock = threading.Lock()


def load_library(path: str = LIB_PATH):
    """Load libjk.so and declare its C signatures (raises if it is missing)."""
    global _lib
    with _lib_lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise ImportError(f"libjk.so not built at {path}; run paper_2608_06536_b300/build.py")
        L = ct.CDLL(path)
        vp, sz = ct.c_void_p, ct.c_size_t
        L.jk_create.argtypes = [ct.POINTER(vp), vp, sz]
        L.jk_destroy.argtypes = [vp]
        L.jk_workspace_query.argtypes = [ct.c_int, ct.c_int32, ct.POINTER(jk_factor),
                                         ct.POINTER(ct.c_int32), ct.c_int32,
                                         ct.POINTER(jk_density), ct.c_int, ct.POINTER(sz)]
        L.jk_build.argtypes = [vp, ct.POINTER(jk_factor), ct.c_int32, ct.POINTER(jk_density),
                               vp, vp, ct.c_int, vp]
        L.jk_build_host.argtypes = [vp, ct.POINTER(jk_factor), ct.c_int32, ct.POINTER(jk_density),
                                    vp, vp, ct.c_int, vp]
        L.jk_build_host.restype = ct.c_int
        L.jk_build_host_packed.argtypes = L.jk_build_host.argtypes
        L.jk_build_host_packed.restype = ct.c_int
        L.jk_build_batched.argtypes = [vp, ct.c_int32, ct.POINTER(jk_factor),
                                       ct.POINTER(ct.c_int32), ct.POINTER(jk_density),
                                       ct.POINTER(vp), ct.POINTER(vp), ct.c_int, vp]
        L.jk_adjoint.argtypes = [vp, ct.POINTER(jk_factor), ct.c_int32, ct.POINTER(jk_density),
                                 vp, vp, vp, vp, vp, ct.c_int, vp]
        L.jk_workspace_query_handle.argtypes = [vp, ct.c_int, ct.c_int32, ct.POINTER(jk_factor),
                                                ct.POINTER(ct.c_int32), ct.c_int32,
                                                ct.POINTER(jk_density), ct.c_int, ct.POINTER(sz)]
        L.jk_autotune.argtypes = [vp, ct.POINTER(jk_factor), ct.c_int32, ct.POINTER(jk_density),
                                  vp, vp, ct.c_int, vp, ct.c_int32, ct.POINTER(jk_tune_config),
                                  ct.POINTER(ct.c_double)]
        L.jk_autotune_batched.argtypes = [vp, ct.c_int32, ct.POINTER(jk_factor), ct.POINTER(ct.c_int32),
                                          ct.POINTER(jk_density), ct.POINTER(vp), ct.POINTER(vp), ct.c_int,
                                          vp, ct.c_int32, ct.POINTER(jk_tune_config), ct.POINTER(ct.c_double)]
        L.jk_tune_lookup.argtypes = [ct.c_int, ct.c_int32, ct.POINTER(jk_factor), ct.POINTER(ct.c_int32),
                                     ct.c_int32, ct.POINTER(jk_density), ct.c_int, ct.c_int32,
                                     ct.POINTER(jk_tune_config)]
        L.jk_build_dense.argtypes = [vp, ct.POINTER(jk_factor), ct.c_int32, vp, vp, vp, ct.c_int, vp]
        L.jk_density_grad.argtypes = [vp, ct.POINTER(jk_factor), ct.c_int32, vp, vp, vp, ct.c_int, vp]
        L.jk_pair.argtypes = [vp, ct.POINTER(jk_factor), ct.c_int32, ct.POINTER(jk_density), ct.c_int32,
                              ct.POINTER(jk_density), vp, vp, ct.c_int, vp]
        L.jk_pair.restype = ct.c_int
        dpp = ct.POINTER(ct.c_double)
        L.jk_build_laplace.argtypes = [vp, ct.POINTER(jk_factor), ct.c_int32, dpp, dpp, ct.c_int32, vp, vp,
                                       ct.c_int32, vp, vp, ct.c_int32, vp, vp, ct.c_int, vp]
        L.jk_build_laplace.restype = ct.c_int
        L.jk_pack_factor.argtypes = [vp, ct.c_int32, ct.c_int32, vp, vp, vp]
        L.jk_pack_factor.restype = ct.c_int
        L.jk_build_dense.restype = ct.c_int
        L.jk_density_grad.restype = ct.c_int
        L.jk_tune_export.argtypes = [ct.c_char_p, sz, ct.POINTER(sz)]
        L.jk_tune_import.argtypes = [ct.c_char_p]
        for f in (L.jk_workspace_query_handle, L.jk_autotune, L.jk_autotune_batched, L.jk_tune_lookup,
                  L.jk_tune_export, L.jk_tune_import, L.jk_tune_clear):
            f.restype = ct.c_int
        L.jk_sync_status.argtypes = [vp, vp]
        L.jk_set_option.argtypes = [vp, ct.c_int, ct.c_int64]
        L.jk_set_option.restype = ct.c_int
        L.jk_status_string.argtypes = [ct.c_int]
        L.jk_status_string.restype = ct.c_char_p
        L.jk_last_error.argtypes = [vp]
        L.jk_last_error.restype = ct.c_char_p
        L.jk_version.restype = ct.c_char_p
        L.jk_launch_count.argtypes = [vp]
        L.jk_launch_count.restype = ct.c_int64
        L.jk_profile_enable.argtypes = [vp, ct.c_int32]
        L.jk_profile_reset.argtypes = [vp]
        L.jk_profile_kinds.restype = ct.c_int32
        L.jk_profile_kind_name.argtypes = [ct.c_int32]
        L.jk_profile_kind_name.restype = ct.c_char_p
        L.jk_profile_read.argtypes = [vp, ct.c_int32, ct.POINTER(ct.c_double), ct.POINTER(ct.c_int64)]
        L.jk_issued_tensor_flops.argtypes = [vp]
        L.jk_issued_tensor_flops.restype = ct.c_double
        for f in (L.jk_profile_enable, L.jk_profile_reset, L.jk_profile_read):
            f.restype = ct.c_int
        L.jk_debug_fp64_fma.argtypes = [vp, ct.c_int32, ct.c_int32, vp, ct.POINTER(ct.c_double), vp]
        L.jk_debug_fp64_fma.restype = ct.c_int
        for f in (L.jk_create, L.jk_destroy, L.jk_workspace_query, L.jk_build,
                  L.jk_build_batched, L.jk_adjoint, L.jk_sync_status):
            f.restype = ct.c_int
        _lib = L
        return L


def _ptr(t):
    return None if t is None else ct.c_void_p(t.data_ptr())


def _dev_f64(t, device):
    """Contiguous float64 tensor on `device` with a 16-byte aligned base."""
    t = torch.as_tensor(t, dtype=torch.float64, device=device)
    if not t.is_contiguous() or t.data_ptr() % 16:
        t = t.contiguous().clone()
    return t


def _host_f64(t):
    """Contiguous float64 CPU tensor (pinned inputs keep their pinning)."""
    t = torch.as_tensor(t, dtype=torch.float64)
    if t.device.type != "cpu":
        raise ValueError("build_host takes host (CPU) tensors")
    return t.contiguous()


def _shape(t):
    return tuple(int(v) for v in t.shape)


def _check_problem(L, X, Y=None, sym=None, packed=False):
    """Shapes of one molecule, checked before any device work: the C ABI takes
    pointers and sizes only, so a mismatch here would become an out-of-bounds
    access in the kernels.  L is [naux][nbf][nbf] (packed: [naux][nbf(nbf+1)/2],
    nbf taken from X); X_s (and Y_s of a non-symmetric density) is [nbf][k_s].
    Returns (nbf, naux, nd)."""
    if packed:
        Ls = _shape(L)
        n = _shape(X[0])[0] if len(X) and len(_shape(X[0])) == 2 else 0
        if len(Ls) != 2 or n < 1 or Ls[1] != n * (n + 1) // 2 or Ls[0] < 1:
            raise ValueError(f"packed L must be [naux][{n * (n + 1) // 2}] for nbf = {n}, got {Ls}")
        return _check_shapes((Ls[0], n, n), X, Y, sym)
    return _check_shapes(_shape(L), X, Y, sym)


def _check_shapes(Ls, X, Y=None, sym=None):
    """_check_problem with the factor given by its shape."""
    if len(Ls) != 3 or Ls[1] != Ls[2] or min(Ls) < 1:
        raise ValueError(f"L must be [naux][nbf][nbf] with naux, nbf >= 1, got {Ls}")
    naux, n = Ls[0], Ls[1]
    nd = len(X)
    if nd < 1:
        raise ValueError("at least one density is required")
    if sym is not None and len(sym) != nd:
        raise ValueError(f"sym has {len(sym)} entries for {nd} densities")
    if Y is not None and len(Y) != nd:
        raise ValueError(f"Y has {len(Y)} entries for {nd} densities")
    for s in range(nd):
        xs = _shape(X[s])
        if len(xs) != 2 or xs[0] != n or xs[1] < 1:
            raise ValueError(f"X[{s}] must be [{n}][k] with k >= 1, got {xs}")
        symmetric = (sym is not None and sym[s]) or Y is None or Y[s] is None
        if not symmetric and _shape(Y[s]) != xs:
            raise ValueError(f"Y[{s}] must have the shape of X[{s}] {xs}, got {_shape(Y[s])}")
    return n, naux, nd


def _check_dense(L, mats, packed=False):
    """Shapes of a dense call: L [naux][nbf][nbf] (packed: [naux][nbf(nbf+1)/2],
    nbf taken from the matrices) and each given matrix stack [nd][nbf][nbf] (a
    single [nbf][nbf] matrix counts as nd = 1), all with the same nd.  Returns
    (nbf, naux, nd)."""
    Ls = _shape(L)
    if packed:
        first = next((_shape(m) for _, m in mats if m is not None), ())
        n = first[-1] if len(first) >= 2 else 0
        if len(Ls) != 2 or n < 1 or Ls[1] != n * (n + 1) // 2 or Ls[0] < 1:
            raise ValueError(f"packed L must be [naux][{n * (n + 1) // 2}] for nbf = {n}, got {Ls}")
        Ls = (Ls[0], n, n)
    if len(Ls) != 3 or Ls[1] != Ls[2] or min(Ls) < 1:
        raise ValueError(f"L must be [naux][nbf][nbf] with naux, nbf >= 1, got {Ls}")
    naux, n = Ls[0], Ls[1]
    nd = None
    for name, m in mats:
        if m is None:
            continue
        ms = _shape(m)
        if len(ms) == 2:
            ms = (1,) + ms
        if len(ms) != 3 or ms[1:] != (n, n) or ms[0] < 1:
            raise ValueError(f"{name} must be [nd][{n}][{n}], got {_shape(m)}")
        if nd is not None and ms[0] != nd:
            raise ValueError(f"{name} holds {ms[0]} matrices, another input {nd}")
        nd = ms[0]
    if nd is None:
        raise ValueError("at least one input matrix is required")
    return n, naux, nd


def _check_output(t, name, shape, device):
    """A caller-supplied output: contiguous float64 of exactly `shape` on
    `device`, 8-byte aligned (the library writes shape's elements through
    the bare pointer)."""
    if t is None:
        return
    if (t.dtype != torch.float64 or t.device != device or _shape(t) != tuple(shape)
            or not t.is_contiguous() or t.data_ptr() % 8):
        raise ValueError(f"{name} must be a contiguous float64 tensor of shape {tuple(shape)} on {device}, "
                         f"got {t.dtype} {_shape(t)} on {t.device}")


def pack_factor(L):
    """[naux][n(n+1)/2]: the packed upper triangle (row-major, diagonal
    included) of each symmetric L^P of a [naux][n][n] tensor or array, on the
    input's device: the layout jk_build_host_packed uploads and the packed
    device factor (option packed_factor) holds.  A device tensor is packed by
    the library (jk_pack_factor); a host one (the host link's input) by an
    index gather on the host."""
    L = torch.as_tensor(L, dtype=torch.float64)
    if L.is_cuda:
        return default_engine(L.device).pack_factor(L)
    n = int(L.shape[-1])
    iu = torch.triu_indices(n, n)
    return L[:, iu[0], iu[1]].contiguous()


def _stream_ptr(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ct.c_void_p(s.cuda_stream)


class Densities:
    """Factored densities D_s = X_s Y_s^T marshalled for the C ABI."""

    def __init__(self, X, Y=None, sym=None, device=None):
        nd = len(X)
        sym = list(sym) if sym is not None else [False] * nd
        Y = list(Y) if Y is not None else [None] * nd
        self.X = [_dev_f64(x, device) for x in X]
        self.Y = [None if (sym[s] or Y[s] is None) else _dev_f64(Y[s], device) for s in range(nd)]
        self.sym = [bool(sym[s] or Y[s] is None) for s in range(nd)]
        self.k = [int(x.shape[1]) for x in self.X]
        self.n = int(self.X[0].shape[0])
        arr = (jk_density * nd)()
        for s in range(nd):
            arr[s].k = self.k[s]
            arr[s].symmetric = 1 if self.sym[s] else 0
            arr[s].X = self.X[s].data_ptr()
            arr[s].Y = self.Y[s].data_ptr() if self.Y[s] is not None else None
        self.c = arr

    def __len__(self):
        return len(self.X)


class Engine:
    """One handle over a device workspace arena (grown on demand)."""

    def __init__(self, device=None, workspace_bytes: int = 0):
        self.lib = load_library()
        dev = torch.device(device) if device is not None else torch.device("cuda")
        if dev.type != "cuda":
            raise ValueError("the J/K engine runs on a CUDA device only")
        if dev.index is None:
            dev = torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        self._ws = None
        self._h = ct.c_void_p()
        self._opts = {}
        if workspace_bytes:
            self._ensure(workspace_bytes)

    # -- arena ---------------------------------------------------------------
    def _ensure(self, nbytes: int):
        if self._ws is not None and self._ws.numel() >= nbytes:
            return
        self.close()
        nbytes = max(int(nbytes), 1 << 20)
        self._ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        h = ct.c_void_p()
        self._check(self.lib.jk_create(ct.byref(h), ct.c_void_p(self._ws.data_ptr()), nbytes), None)
        self._h = h
        if getattr(self, "_profile_on", False):
            self.lib.jk_profile_enable(self._h, 1)
        for code, value in self._opts.items():
            self._check(self.lib.jk_set_option(self._h, code, value), self._h)

    def close(self):
        if self._h:
            self.lib.jk_destroy(self._h)
            self._h = ct.c_void_p()
        self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def workspace_bytes(self) -> int:
        return 0 if self._ws is None else self._ws.numel()

    def _check(self, status, h):
        if status != JK_OK:
            msg = self.lib.jk_last_error(h).decode() if h else ""
            if not msg:
                msg = self.lib.jk_status_string(status).decode()
            raise JKError(status, msg)

    def sync_status(self, stream=None):
        self._check(self.lib.jk_sync_status(self._h, _stream_ptr(stream)), self._h)

    @property
    def _packed(self) -> bool:
        return self._opts.get(OPTIONS["packed_factor"], 0) == 1

    def _record(self, stream):
        """Work issued on a stream other than the current one keeps the arena
        from being reused (after a later growth) until that work is done."""
        if stream is not None and self._ws is not None and stream != torch.cuda.current_stream(self.device):
            self._ws.record_stream(stream)

    # -- options ---------------------------------------------------------------
    def set_option(self, name: str, value: int):
        """Handle option (JK_OPT_*): "aux_chunk" (>= 0, 0 = automatic, -1 =
        tuned/default), "schedule", "raster" and "tile" (-1 = tuned/default,
        0, 1), "use_tuned" (0 or 1), "host_chunk" (>= 0, 0 = automatic),
        "slicer" (0 integer digits, 1 FP32 digits), "syrk" (symmetric
        densities, both engines: 0 full rank update, 1 blocked symmetric rank
        update with the rest mirrored), "packed_factor" (1: the factor given
        to every device call (build, build_batched, adjoint, build_dense,
        density_grad, pairs, build_laplace, autotune*) is pack_factor(L),
        [naux][n(n+1)/2] on the device; half the memory), "tile" (0: sliced
        GEMM tiles of 128 x 80 outputs, 1: 128 x 64), "adjoint_slices" (6 or
        7, default 7: BF16 slices per operand of the split adjoint's products),
        "j_path" (split builds' J: -1 automatic, 0 FP64 pass on a second
        stream, 1 tensor cores).  Kept across arena growth."""
        code = OPTIONS[name]
        self._opts[code] = int(value)
        if self._h:
            self._check(self.lib.jk_set_option(self._h, code, int(value)), self._h)

    def set_aux_chunk(self, naux_per_chunk: int):
        """This many aux indices per internal chunk (0 = automatic)."""
        self.set_option("aux_chunk", naux_per_chunk)

    # -- instrumentation -----------------------------------------------------
    def launch_count(self) -> int:
        return int(self.lib.jk_launch_count(self._h)) if self._h else 0

    def issued_tensor_flops(self) -> float:
        return float(self.lib.jk_issued_tensor_flops(self._h)) if self._h else 0.0

    def profile(self, on: bool = True):
        if self._h:
            self._check(self.lib.jk_profile_enable(self._h, 1 if on else 0), self._h)
        self._profile_on = on

    def profile_reset(self):
        if self._h:
            self._check(self.lib.jk_profile_reset(self._h), self._h)

    def profile_read(self) -> dict:
        """{kind name: (total ms, launches)} since the last reset."""
        out = {}
        if not self._h:
            return out
        for kind in range(self.lib.jk_profile_kinds()):
            ms, cnt = ct.c_double(), ct.c_int64()
            self._check(self.lib.jk_profile_read(self._h, kind, ct.byref(ms), ct.byref(cnt)), self._h)
            if cnt.value:
                out[self.lib.jk_profile_kind_name(kind).decode()] = (ms.value, cnt.value)
        return out

    # -- queries -------------------------------------------------------------
    def fp64_fma_probe(self, blocks_per_sm: int = 8, iters: int = 1 << 16, stream=None) -> float:
        """Launch the library's FP64 FMA-rate kernel on `stream` (the current
        stream by default) and return the FP64 flops it performs; time it with
        CUDA events on that stream."""
        self._ensure(1 << 20)
        if getattr(self, "_sink", None) is None:
            self._sink = torch.zeros(1, dtype=torch.float64, device=self.device)
        flops = ct.c_double()
        st = self.lib.jk_debug_fp64_fma(self._h, int(blocks_per_sm), int(iters), ct.c_void_p(self._sink.data_ptr()),
                                        ct.byref(flops), _stream_ptr(stream))
        self._check(st, self._h)
        return flops.value

    def query(self, op, factors, dens_c, nd_per_mol, nd, precision) -> int:
        """Arena bytes for a call under this handle's options and tuned configs."""
        if not self._h:
            self._ensure(1 << 20)
        nbytes = ct.c_size_t()
        ndm = (ct.c_int32 * len(nd_per_mol))(*nd_per_mol) if nd_per_mol else None
        st = self.lib.jk_workspace_query_handle(self._h, op, len(factors), factors, ndm, nd, dens_c,
                                                precision, ct.byref(nbytes))
        self._check(st, None)
        return nbytes.value

    # -- entry points --------------------------------------------------------
    def build(self, L, X, Y=None, sym=None, precision="fp64", want_j=True, want_k=True,
              J=None, K=None, stream=None):
        """J_s, K_s ([nd][n][n] float64) for D_s = X_s Y_s^T over factor L."""
        p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        n, _, nd = _check_problem(L, X, Y, sym, self._packed)
        if want_j:
            _check_output(J, "J", (nd, n, n), self.device)
        if want_k:
            _check_output(K, "K", (nd, n, n), self.device)
        L = _dev_f64(L, self.device)
        dens = Densities(X, Y, sym, self.device)
        naux = int(L.shape[0])
        f = jk_factor(n, naux, L.data_ptr())
        self._ensure(self.query(JK_OP_BUILD, (jk_factor * 1)(f), dens.c, None, nd, p))
        if want_j and J is None:
            J = torch.empty((nd, n, n), dtype=torch.float64, device=self.device)
        if want_k and K is None:
            K = torch.empty((nd, n, n), dtype=torch.float64, device=self.device)
        st = self.lib.jk_build(self._h, ct.byref(f), nd, dens.c, _ptr(J if want_j else None),
                               _ptr(K if want_k else None), p, _stream_ptr(stream))
        self._check(st, self._h)
        self._record(stream)
        return (J if want_j else None), (K if want_k else None)

    def build_host(self, L, X, Y=None, sym=None, precision="split", want_j=True, want_k=True,
                   J=None, K=None, stream=None, sync=True, packed=False):
        """J, K for host-resident inputs (CPU float64 tensors, ideally pinned):
        the factor streams to the device chunk by chunk, overlapped with the
        build; J, K ([nd][n][n], CPU) are written at the end of the stream's
        work (sync=True waits for it).  With packed=True, L is given as
        pack_factor(L) ([naux][n(n+1)/2]): half the bytes are uploaded."""
        p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        n, _, nd = _check_problem(L, X, Y, sym, packed)
        if want_j:
            _check_output(J, "J", (nd, n, n), torch.device("cpu"))
        if want_k:
            _check_output(K, "K", (nd, n, n), torch.device("cpu"))
        L = _host_f64(L)
        X = [_host_f64(x) for x in X]
        sym = list(sym) if sym is not None else [False] * nd
        Y = list(Y) if Y is not None else [None] * nd
        Y = [None if (sym[s] or Y[s] is None) else _host_f64(Y[s]) for s in range(nd)]
        symf = [sym[s] or Y[s] is None for s in range(nd)]
        naux = int(L.shape[0])
        f = jk_factor(n, naux, L.data_ptr())
        op = JK_OP_BUILD_HOST_PACKED if packed else JK_OP_BUILD_HOST
        call = self.lib.jk_build_host_packed if packed else self.lib.jk_build_host
        dens = (jk_density * nd)()
        for s in range(nd):
            dens[s].k = int(X[s].shape[1])
            dens[s].symmetric = 1 if symf[s] else 0
            dens[s].X = X[s].data_ptr()
            dens[s].Y = Y[s].data_ptr() if Y[s] is not None else None
        self._ensure(self.query(op, (jk_factor * 1)(f), dens, None, nd, p))
        if want_j and J is None:
            J = torch.empty((nd, n, n), dtype=torch.float64).pin_memory()
        if want_k and K is None:
            K = torch.empty((nd, n, n), dtype=torch.float64).pin_memory()
        st = call(self._h, ct.byref(f), nd, dens, _ptr(J if want_j else None), _ptr(K if want_k else None), p,
                  _stream_ptr(stream))
        self._check(st, self._h)
        self._record(stream)
        if sync:
            self.sync_status(stream)
        return (J if want_j else None), (K if want_k else None)

    def build_dense(self, L, D, precision="fp64", want_j=True, want_k=True, J=None, K=None, stream=None):
        """J(D_s), K(D_s) ([nd][n][n] float64) for dense, general densities
        D ([nd][n][n] or [n][n])."""
        p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        n, naux, nd = _check_dense(L, [("D", D)], self._packed)
        if want_j:
            _check_output(J, "J", (nd, n, n), self.device)
        if want_k:
            _check_output(K, "K", (nd, n, n), self.device)
        L = _dev_f64(L, self.device)
        D = _dev_f64(D, self.device).reshape(nd, n, n)
        f = jk_factor(n, naux, L.data_ptr())
        self._ensure(self.query(JK_OP_BUILD_DENSE, (jk_factor * 1)(f), None, None, nd, p))
        if want_j and J is None:
            J = torch.empty((nd, n, n), dtype=torch.float64, device=self.device)
        if want_k and K is None:
            K = torch.empty((nd, n, n), dtype=torch.float64, device=self.device)
        st = self.lib.jk_build_dense(self._h, ct.byref(f), nd, _ptr(D), _ptr(J if want_j else None),
                                     _ptr(K if want_k else None), p, _stream_ptr(stream))
        self._check(st, self._h)
        self._record(stream)
        return (J if want_j else None), (K if want_k else None)

    def density_grad(self, L, W=None, V=None, precision="fp64", G=None, stream=None):
        """G_s = dE/dD_s = K(W_s) + J(V_s) ([nd][n][n] float64) for
        E = sum_s <W_s, K(D_s)> + <V_s, J(D_s)>; W or V may be None (zero)."""
        p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        n, naux, nd = _check_dense(L, [("W", W), ("V", V)], self._packed)
        _check_output(G, "G", (nd, n, n), self.device)
        L = _dev_f64(L, self.device)
        W = None if W is None else _dev_f64(W, self.device).reshape(nd, n, n)
        V = None if V is None else _dev_f64(V, self.device).reshape(nd, n, n)
        f = jk_factor(n, naux, L.data_ptr())
        self._ensure(self.query(JK_OP_DENSITY_GRAD, (jk_factor * 1)(f), None, None, nd, p))
        if G is None:
            G = torch.empty((nd, n, n), dtype=torch.float64, device=self.device)
        st = self.lib.jk_density_grad(self._h, ct.byref(f), nd, _ptr(W), _ptr(V), _ptr(G), p,
                                      _stream_ptr(stream))
        self._check(st, self._h)
        self._record(stream)
        return G

    def pairs(self, L, XL, YL=None, symL=None, XR=None, YR=None, symR=None, precision="fp64",
              want_j=True, want_k=True, stream=None):
        """(Jp, Kp), each [nl][nr] float64: Jp[a][b] = <W_L^a, J(W_R^b)> and
        Kp[a][b] = <W_L^a, K(W_R^b)> for left densities W_L^a = XL_a YL_a^T and
        right densities W_R^b = XR_b YR_b^T over one factor L."""
        p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        if XR is None:
            raise ValueError("right densities XR are required")
        n, naux, nl = _check_problem(L, XL, YL, symL, self._packed)
        _, _, nr = _check_problem(L, XR, YR, symR, self._packed)
        L = _dev_f64(L, self.device)
        left = Densities(XL, YL, symL, self.device)
        right = Densities(XR, YR, symR, self.device)
        f = jk_factor(n, naux, L.data_ptr())
        both = (jk_density * (nl + nr))(*left.c, *right.c)
        # the pair query takes two groups (left, right) over one factor
        self._ensure(self.query(JK_OP_PAIR, (jk_factor * 2)(f, f), both, [nl, nr], nl + nr, p))
        Jp = torch.empty((nl, nr), dtype=torch.float64, device=self.device) if want_j else None
        Kp = torch.empty((nl, nr), dtype=torch.float64, device=self.device) if want_k else None
        st = self.lib.jk_pair(self._h, ct.byref(f), nl, left.c, nr, right.c, _ptr(Jp), _ptr(Kp), p,
                              _stream_ptr(stream))
        self._check(st, self._h)
        self._record(stream)
        return Jp, Kp

    def build_laplace(self, L, CX, epsX, sx, alpha, w=None, CY=None, epsY=None, sy=None, precision="fp64",
                      want_j=True, want_k=True, stream=None):
        """The nq Laplace builds on energy-scaled coefficients
        X_k = CX diag(exp(sx alpha_k epsX / 2)), Y_k likewise from CY, epsY, sy
        (CY None: Y_k = X_k).  Returns (J, K): [nq][n][n] per point, or the
        weighted sums [n][n] when w is given."""
        p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        Ls = _shape(L)
        if self._packed:
            n = _shape(CX)[0] if len(_shape(CX)) == 2 else 0
            if len(Ls) != 2 or n < 1 or Ls[1] != n * (n + 1) // 2 or Ls[0] < 1:
                raise ValueError(f"packed L must be [naux][{n * (n + 1) // 2}] for nbf = {n}, got {Ls}")
            Ls = (Ls[0], n, n)
        if len(Ls) != 3 or Ls[1] != Ls[2] or min(Ls) < 1:
            raise ValueError(f"L must be [naux][nbf][nbf] with naux, nbf >= 1, got {Ls}")
        naux, n = Ls[0], Ls[1]
        sym = CY is None
        if sym != (epsY is None):
            raise ValueError("CY and epsY must both be given or both omitted")
        cs = _shape(CX)
        if len(cs) != 2 or cs[0] != n or cs[1] < 1:
            raise ValueError(f"CX must be [{n}][m], got {cs}")
        m = cs[1]
        if _shape(epsX) != (m,) or (not sym and (_shape(CY) != cs or _shape(epsY) != (m,))):
            raise ValueError(f"epsX (and CY, epsY) must match CX's m = {m}")
        alpha = [float(a) for a in alpha]
        nq = len(alpha)
        if w is not None and len(w) != nq:
            raise ValueError(f"w has {len(w)} entries for {nq} quadrature points")
        L = _dev_f64(L, self.device)
        CX, epsX = _dev_f64(CX, self.device), _dev_f64(epsX, self.device)
        if not sym:
            CY, epsY = _dev_f64(CY, self.device), _dev_f64(epsY, self.device)
        f = jk_factor(n, naux, L.data_ptr())
        d = (jk_density * 1)()
        d[0].k, d[0].symmetric = m, 1 if sym else 0
        self._ensure(self.query(JK_OP_LAPLACE, (jk_factor * 1)(f), d, None, nq, p))
        shape = (n, n) if w is not None else (nq, n, n)
        J = torch.empty(shape, dtype=torch.float64, device=self.device) if want_j else None
        K = torch.empty(shape, dtype=torch.float64, device=self.device) if want_k else None
        a_arr = (ct.c_double * nq)(*alpha)
        w_arr = (ct.c_double * nq)(*[float(x) for x in w]) if w is not None else None
        st = self.lib.jk_build_laplace(self._h, ct.byref(f), nq, a_arr, w_arr, m, _ptr(CX), _ptr(epsX), int(sx),
                                       _ptr(CY) if not sym else None, _ptr(epsY) if not sym else None,
                                       int(sy) if sy is not None else 0, _ptr(J), _ptr(K), p, _stream_ptr(stream))
        self._check(st, self._h)
        self._record(stream)
        return J, K

    def pack_factor(self, L, P=None, stream=None):
        """jk_pack_factor: [naux][n(n+1)/2] packed upper triangles of a device
        factor [naux][n][n] (into P if given)."""
        Ls = _shape(L)
        if len(Ls) != 3 or Ls[1] != Ls[2] or min(Ls) < 1:
            raise ValueError(f"L must be [naux][nbf][nbf] with naux, nbf >= 1, got {Ls}")
        naux, n = Ls[0], Ls[1]
        L = _dev_f64(L, self.device)
        _check_output(P, "P", (naux, n * (n + 1) // 2), self.device)
        if P is None:
            P = torch.empty((naux, n * (n + 1) // 2), dtype=torch.float64, device=self.device)
        if not self._h:
            self._ensure(1 << 20)
        self._check(self.lib.jk_pack_factor(self._h, n, naux, _ptr(L), _ptr(P), _stream_ptr(stream)), self._h)
        self._record(stream)
        return P

    def autotune(self, L, X, Y=None, sym=None, precision="split", reps: int = 3, stream=None):
        """Time the candidate configurations of this build and cache the
        fastest for its shape bucket; returns (config dict, ms per build)."""
        p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        n, naux, nd = _check_problem(L, X, Y, sym, self._packed)
        L = _dev_f64(L, self.device)
        dens = Densities(X, Y, sym, self.device)
        f = jk_factor(n, naux, L.data_ptr())
        self._ensure(self._tune_bytes(JK_OP_BUILD, (jk_factor * 1)(f), dens.c, None, nd, p))
        J = torch.empty((nd, n, n), dtype=torch.float64, device=self.device)
        K = torch.empty((nd, n, n), dtype=torch.float64, device=self.device)
        cfg, ms = jk_tune_config(), ct.c_double()
        st = self.lib.jk_autotune(self._h, ct.byref(f), nd, dens.c, _ptr(J), _ptr(K), p,
                                  _stream_ptr(stream), int(reps), ct.byref(cfg), ct.byref(ms))
        self._check(st, self._h)
        self._record(stream)
        return cfg.as_dict(), ms.value

    def autotune_batched(self, mols, precision="split", reps: int = 3, stream=None):
        """As autotune, for a batched build over `mols` (see build_batched)."""
        p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        fac, dall, nd_per, keep, outs = self._marshal_batched(mols)
        ndt = sum(nd_per)
        self._ensure(self._tune_bytes(JK_OP_BATCHED, fac, dall, nd_per, ndt, p))
        Jp, Kp, _ = self._batched_outputs(keep[1], True, True)
        ndm = (ct.c_int32 * len(mols))(*nd_per)
        cfg, ms = jk_tune_config(), ct.c_double()
        st = self.lib.jk_autotune_batched(self._h, len(mols), fac, ndm, dall, Jp, Kp, p, _stream_ptr(stream),
                                          int(reps), ct.byref(cfg), ct.byref(ms))
        self._check(st, self._h)
        self._record(stream)
        return cfg.as_dict(), ms.value

    def _tune_bytes(self, op, factors, dens_c, nd_per_mol, nd, p) -> int:
        """Arena for the largest candidate of an autotune: the automatic
        configuration at twice its aux chunk, and the grouped schedule."""
        saved = dict(self._opts)
        need = self.query(op, factors, dens_c, nd_per_mol, nd, p)
        try:
            for sched in ((0, 1) if op == JK_OP_BUILD else (1,)):
                self.set_option("schedule", sched)
                self.set_option("aux_chunk", 0)
                need = max(need, self.query(op, factors, dens_c, nd_per_mol, nd, p))
        finally:
            self._opts = saved
            if self._h:
                for name, code in OPTIONS.items():
                    self._check(self.lib.jk_set_option(self._h, code, saved.get(code, OPTION_DEFAULTS[name])),
                                self._h)
        return int(need * 2)

    def _marshal_batched(self, mols):
        nmol = len(mols)
        Ls, dens = [], []
        fac = (jk_factor * nmol)()
        nd_per = []
        if nmol < 1:
            raise ValueError("at least one molecule is required")
        shapes = []
        for m, (L, X, Y, sym) in enumerate(mols):
            try:
                shapes.append(_check_problem(L, X, Y, sym, self._packed))
            except ValueError as e:
                raise ValueError(f"molecule {m}: {e}") from None
        for m, (L, X, Y, sym) in enumerate(mols):
            L = _dev_f64(L, self.device)
            d = Densities(X, Y, sym, self.device)
            Ls.append(L); dens.append(d)
            fac[m] = jk_factor(shapes[m][0], shapes[m][1], L.data_ptr())
            nd_per.append(len(d))
        ndt = sum(nd_per)
        dall = (jk_density * ndt)()
        i = 0
        for d in dens:
            for s in range(len(d)):
                dall[i] = d.c[s]; i += 1
        return fac, dall, nd_per, (Ls, dens), None

    def _batched_outputs(self, dens, want_j, want_k):
        ndt = sum(len(d) for d in dens)
        Jp = (ct.c_void_p * ndt)(); Kp = (ct.c_void_p * ndt)()
        outs, i = [], 0
        for d in dens:
            n = d.n
            Jm = torch.empty((len(d), n, n), dtype=torch.float64, device=self.device) if want_j else None
            Km = torch.empty((len(d), n, n), dtype=torch.float64, device=self.device) if want_k else None
            outs.append((Jm, Km))
            for s in range(len(d)):
                if want_j:
                    Jp[i] = Jm[s].data_ptr()
                if want_k:
                    Kp[i] = Km[s].data_ptr()
                i += 1
        return Jp, Kp, outs

    def build_batched(self, mols, precision="fp64", want_j=True, want_k=True, stream=None):
        """mols: list of (L, X list, Y list or None, sym list or None).
        Returns per-molecule (J, K) lists of [nd_m][n_m][n_m] tensors."""
        p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        fac, dall, nd_per, keep, _ = self._marshal_batched(mols)
        ndt = sum(nd_per)
        self._ensure(self.query(JK_OP_BATCHED, fac, dall, nd_per, ndt, p))
        Jp, Kp, outs = self._batched_outputs(keep[1], want_j, want_k)
        ndm = (ct.c_int32 * len(mols))(*nd_per)
        st = self.lib.jk_build_batched(self._h, len(mols), fac, ndm, dall, Jp if want_j else None,
                                       Kp if want_k else None, p, _stream_ptr(stream))
        self._check(st, self._h)
        self._record(stream)
        return outs

    def adjoint(self, L, X, Y=None, sym=None, W=None, V=None, want_dl=True,
                precision="fp64", stream=None):
        """(dX list, dY list, dL or None) for E = sum_s <W_s,K_s> + <V_s,J_s>."""
        p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        n, naux, nd = _check_problem(L, X, Y, sym, self._packed)
        for name, t in (("W", W), ("V", V)):
            if t is not None and torch.as_tensor(t).numel() != nd * n * n:
                raise ValueError(f"{name} must hold [{nd}][{n}][{n}] values")
        L = _dev_f64(L, self.device)
        dens = Densities(X, Y, sym, self.device)
        f = jk_factor(n, naux, L.data_ptr())
        W = None if W is None else _dev_f64(W, self.device).reshape(nd, n, n)
        V = None if V is None else _dev_f64(V, self.device).reshape(nd, n, n)
        self._ensure(self.query(JK_OP_ADJOINT, (jk_factor * 1)(f), dens.c, None, nd, p))
        tot = sum(n * k for k in dens.k)
        dX = torch.empty(tot, dtype=torch.float64, device=self.device)
        dY = torch.empty(tot, dtype=torch.float64, device=self.device)
        dL = torch.empty((naux, n, n), dtype=torch.float64, device=self.device) if want_dl else None
        st = self.lib.jk_adjoint(self._h, ct.byref(f), nd, dens.c, _ptr(W), _ptr(V), _ptr(dX),
                                 _ptr(dY), _ptr(dL), p, _stream_ptr(stream))
        self._check(st, self._h)
        self._record(stream)
        outX, outY, off = [], [], 0
        for k in dens.k:
            outX.append(dX[off:off + n * k].view(n, k))
            outY.append(dY[off:off + n * k].view(n, k))
            off += n * k
        return outX, outY, dL


_default = {}


def default_engine(device=None) -> Engine:
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    key = (dev.type, dev.index)
    if key not in _default:
        _default[key] = Engine(dev)
    return _default[key]


def jk_build(L, X, Y=None, sym=None, precision="fp64", **kw):
    return default_engine(L.device if torch.is_tensor(L) and L.is_cuda else None).build(
        L, X, Y, sym, precision, **kw)


def jk_build_batched(mols, precision="fp64", **kw):
    return default_engine().build_batched(mols, precision, **kw)


def jk_adjoint(L, X, Y=None, sym=None, W=None, V=None, precision="fp64", **kw):
    return default_engine(L.device if torch.is_tensor(L) and L.is_cuda else None).adjoint(
        L, X, Y, sym, W, V, precision=precision, **kw)


def _engine_for(L):
    return default_engine(L.device if torch.is_tensor(L) and L.is_cuda else None)


def jk_build_dense(L, D, precision="fp64", **kw):
    """J(D_s), K(D_s) for dense densities D ([nd][n][n]) on the default engine."""
    return _engine_for(L).build_dense(L, D, precision, **kw)


def jk_density_grad(L, W=None, V=None, precision="fp64", **kw):
    """dE/dD_s = K(W_s) + J(V_s) on the default engine."""
    return _engine_for(L).density_grad(L, W, V, precision, **kw)


def jk_pair(L, XL, YL=None, symL=None, XR=None, YR=None, symR=None, precision="fp64", **kw):
    """Bra-ket pairings (Jp, Kp) on the default engine (see Engine.pairs)."""
    return _engine_for(L).pairs(L, XL, YL, symL, XR, YR, symR, precision, **kw)


def jk_build_laplace(L, CX, epsX, sx, alpha, w=None, CY=None, epsY=None, sy=None, precision="fp64", **kw):
    """Laplace (LT-AO) builds on the default engine (see Engine.build_laplace)."""
    return _engine_for(L).build_laplace(L, CX, epsX, sx, alpha, w, CY, epsY, sy, precision, **kw)


def tune_export() -> str:
    """The process-wide autotuner cache as text (one entry per line)."""
    lib = load_library()
    n = ct.c_size_t()
    lib.jk_tune_export(None, 0, ct.byref(n))
    buf = ct.create_string_buffer(n.value + 1)
    lib.jk_tune_export(buf, n.value + 1, ct.byref(n))
    return buf.value.decode()


def tune_import(text: str):
    """Merge cache entries produced by tune_export (raises on a bad line)."""
    st = load_library().jk_tune_import(text.encode())
    if st != JK_OK:
        raise JKError(st, "malformed autotuner cache text")


def tune_clear():
    load_library().jk_tune_clear()

