"""Seeded synthetic inputs for the Cholesky J/K engine.

This module only draws numbers; it holds none of the J/K arithmetic.  It is the
one module shared by the CPU oracle tests and the CUDA path (tests, bench,
smoke), so both sides always see bit-identical inputs.

Recipe (the paper's molecules and basis sets are not available; these synthetic
shapes stand in for them, with nbf spanning the paper's 236-472 AO range):

* Cholesky factor L^P (P = 0..naux-1, 0-based), symmetric nbf x nbf: the upper
  triangle including the diagonal is drawn N(0,1) in row-major order and
  mirrored, then scaled by exp(-P/tau).  Each L^P is drawn from its own stream
  ``default_rng([seed, 1, P])`` so any single P can be regenerated alone.
* Non-symmetric transition density D = X Y^T: X then Y, each nbf x k with
  N(0, 1/nbf) entries (std 1/sqrt(nbf)), stream ``default_rng([seed, 2, s])``.
* Symmetric ground density D = C_o C_o^T: C_o is the Q factor of the reduced QR
  of an nbf x k N(0,1) matrix (stream ``[seed, 2, s]``); X = Y = C_o.
* Adjoint seeds W_s, V_s: nbf x nbf N(0,1), stream ``[seed, 3, s]``.
* Dense (general, non-symmetric) density D_s: nbf x nbf with N(0, 1/nbf^2)
  entries, the scale of X Y^T with N(0, 1/nbf) factors of width about nbf;
  stream ``[seed, 4, s]``.
* Uneven batch: molecule sizes nbf ~ U{100..600}, densities per molecule
  ~ U{1..16} from stream ``[seed, 0]``; molecule m then uses seed
  ``seed * 1000 + m`` for its own factor and densities.
* Factors too large to draw on the host in reasonable time (the 40 GB
  single molecule, the 208 GB uneven batch, the 10 GB adjoint case) are drawn
  on the device by ``factor_device``: the same symmetric N(0,1) * exp(-P/tau)
  recipe, with torch's Philox generator seeded from ``[seed, 1]``.  Tests
  that check such a factor against the CPU code copy it back to the host.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def factor_slice(n: int, P: int, tau: float, seed: int = 0) -> np.ndarray:
    """L^P (nbf x nbf, float64, symmetric) for one aux index P."""
    rng = np.random.default_rng([seed, 1, P])
    iu = np.triu_indices(n)
    M = np.zeros((n, n), dtype=np.float64)
    M[iu] = rng.standard_normal(iu[0].size)
    M = M + np.triu(M, 1).T
    M *= math.exp(-P / tau)
    return M


def factor(n: int, naux: int, tau: float, seed: int = 0, P0: int = 0) -> np.ndarray:
    """L^P for P = P0 .. P0+naux-1 as one [naux][n][n] float64 array."""
    L = np.empty((naux, n, n), dtype=np.float64)
    for j in range(naux):
        L[j] = factor_slice(n, P0 + j, tau, seed)
    return L


def factor_device(n: int, naux: int, tau: float, seed: int = 0, device="cuda",
                  block: int = 64):
    """L^P for P = 0 .. naux-1 drawn on the device as [naux][n][n] float64:
    an n x n N(0,1) draw per P whose upper triangle (with the diagonal) is
    kept and mirrored, scaled by exp(-P/tau).  Deterministic for a given
    (n, naux, tau, seed) and block size."""
    import torch
    state = np.random.SeedSequence([seed, 1]).generate_state(2, dtype=np.uint32)
    g = torch.Generator(device=device)
    g.manual_seed(int(state[0]) << 32 | int(state[1]))
    L = torch.empty((naux, n, n), dtype=torch.float64, device=device)
    upper = torch.ones((n, n), dtype=torch.bool, device=device).triu_()
    for P0 in range(0, naux, block):
        b = min(block, naux - P0)
        R = torch.randn((b, n, n), dtype=torch.float64, device=device, generator=g)
        R = torch.where(upper, R, R.transpose(1, 2))
        scale = torch.exp(-torch.arange(P0, P0 + b, dtype=torch.float64, device=device) / tau)
        L[P0:P0 + b] = R * scale[:, None, None]
    return L


def transition_density(n: int, k: int, s: int, seed: int = 0):
    """(X, Y), each [n][k] float64 with N(0, 1/n) entries."""
    rng = np.random.default_rng([seed, 2, s])
    sd = 1.0 / math.sqrt(n)
    X = rng.standard_normal((n, k)) * sd
    Y = rng.standard_normal((n, k)) * sd
    return np.ascontiguousarray(X), np.ascontiguousarray(Y)


def ground_density(n: int, k: int, s: int, seed: int = 0):
    """(C_o, C_o) with orthonormal columns: the symmetric density C_o C_o^T."""
    rng = np.random.default_rng([seed, 2, s])
    Q, _ = np.linalg.qr(rng.standard_normal((n, k)), mode="reduced")
    Q = np.ascontiguousarray(Q)
    return Q, Q


def dense_density(n: int, s: int, seed: int = 0) -> np.ndarray:
    """D_s, [n][n] float64 with N(0, 1/n^2) entries (general, non-symmetric)."""
    rng = np.random.default_rng([seed, 4, s])
    return np.ascontiguousarray(rng.standard_normal((n, n)) / n)


def dense_densities(n: int, nd: int, seed: int = 0) -> np.ndarray:
    """[nd][n][n]: dense_density for s = 0 .. nd-1."""
    return np.stack([dense_density(n, s, seed) for s in range(nd)])


def adjoint_seeds(n: int, s: int, seed: int = 0):
    """(W_s, V_s), each [n][n] float64 N(0,1)."""
    rng = np.random.default_rng([seed, 3, s])
    W = rng.standard_normal((n, n))
    V = rng.standard_normal((n, n))
    return W, V


@dataclass
class Molecule:
    """One J/K problem: a factor and its list of factored densities."""
    n: int
    naux: int
    tau: float
    seed: int
    ks: list = field(default_factory=list)      # width of each density
    sym: list = field(default_factory=list)     # True -> D = X X^T
    X: list = field(default_factory=list)
    Y: list = field(default_factory=list)
    L: np.ndarray | None = None

    @property
    def nd(self) -> int:
        return len(self.ks)

    def materialize_factor(self) -> np.ndarray:
        if self.L is None:
            self.L = factor(self.n, self.naux, self.tau, self.seed)
        return self.L


def molecule(n: int, naux: int, tau: float, dens: list, seed: int = 0,
             with_factor: bool = True) -> Molecule:
    """Build a Molecule.  ``dens`` is a list of (k, symmetric) pairs."""
    m = Molecule(n=n, naux=naux, tau=tau, seed=seed)
    for s, (k, sym) in enumerate(dens):
        X, Y = ground_density(n, k, s, seed) if sym else transition_density(n, k, s, seed)
        m.ks.append(k)
        m.sym.append(bool(sym))
        m.X.append(X)
        m.Y.append(Y)
    if with_factor:
        m.materialize_factor()
    return m


# ---------------------------------------------------------------------------
# The workloads: sizes follow the five benchmark configurations of the engine.
# ---------------------------------------------------------------------------

def one_molecule_small(seed: int = 0, with_factor: bool = True) -> Molecule:
    """nbf=48, naux=300, tau=60, one non-symmetric density of width 6."""
    return molecule(48, 300, 60.0, [(6, False)], seed, with_factor)


def multi_state(seed: int = 0, with_factor: bool = True) -> Molecule:
    """nbf=400, naux=2400, tau=400: one symmetric ground density (k=40) plus
    seven non-symmetric transition densities (k=40)."""
    dens = [(40, True)] + [(40, False)] * 7
    return molecule(400, 2400, 400.0, dens, seed, with_factor)


def large_single(seed: int = 0, with_factor: bool = False) -> Molecule:
    """nbf=1000, naux=5000, tau=1000, 16 non-symmetric densities of width 100."""
    return molecule(1000, 5000, 1000.0, [(100, False)] * 16, seed, with_factor)


def adjoint_case(seed: int = 0, with_factor: bool = True):
    """nbf=600, naux=3600, tau=600, 8 non-symmetric densities (k=60) plus
    W_s, V_s seeds."""
    m = molecule(600, 3600, 600.0, [(60, False)] * 8, seed, with_factor)
    W, V = zip(*(adjoint_seeds(600, s, seed) for s in range(8)))
    return m, list(W), list(V)


def uneven_batch_shapes(nmol: int = 64, seed: int = 0):
    """[(nbf, nd)] for the uneven batch: nbf ~ U{100..600}, nd ~ U{1..16}."""
    rng = np.random.default_rng([seed, 0])
    nbf = rng.integers(100, 601, size=nmol)
    nd = rng.integers(1, 17, size=nmol)
    return [(int(a), int(b)) for a, b in zip(nbf, nd)]


def uneven_batch(nmol: int = 64, seed: int = 0, with_factor: bool = True,
                 shapes=None):
    """Molecules with naux = 6*nbf, tau = nbf, nd non-symmetric densities of
    width nbf // 10 each."""
    shapes = shapes if shapes is not None else uneven_batch_shapes(nmol, seed)
    mols = []
    for m, (n, nd) in enumerate(shapes):
        mols.append(molecule(n, 6 * n, float(n), [(n // 10, False)] * nd,
                             seed * 1000 + m, with_factor))
    return mols


def custom_densities(n: int, ks, seed: int = 0):
    """(X list, Y list) of non-symmetric transition densities of widths ks,
    without a factor (the recipe of transition_density)."""
    XY = [transition_density(n, k, s, seed) for s, k in enumerate(ks)]
    return [x for x, _ in XY], [y for _, y in XY]


def custom(n: int, naux: int, tau: float, ks, sym=None, seed: int = 0) -> Molecule:
    """Arbitrary shapes for tests (ragged sizes, tiny cases)."""
    sym = sym if sym is not None else [False] * len(ks)
    return molecule(n, naux, tau, list(zip(ks, sym)), seed, True)
