"""Shared helpers for the GPU parity tests (tolerances and comparisons)."""
import numpy as np

# Plain FP64 engine: max|gpu - oracle| / max|oracle| per output array.
FP64_REL = 1e-12
# Split-precision engine: absolute error in output units (Hartree-scaled).
SPLIT_ABS = 1e-10


def rel_err(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = max(float(np.abs(ref).max()), 1e-300)
    return float(np.abs(got - ref).max()) / scale


def abs_err(got, ref):
    return float(np.abs(np.asarray(got, np.float64) - np.asarray(ref, np.float64)).max())


def to_np(t):
    return t.detach().cpu().numpy()
