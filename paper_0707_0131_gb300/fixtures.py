"""Seeded synthetic inputs: gauge fields, right-hand sides, gauge transformations.

This module only draws inputs.  It holds none of the solver's arithmetic (no
Wilson operator, no Krylov step), so both the CUDA path and the CPU oracle can
consume what it produces without sharing any of the method's code.

Layouts (all complex128, C order):
  gauge  : [V][4][3][3]   U_mu(x), mu = 0..3 <-> x, y, z, t; row-major colour matrix
  spinor : [V][4][3]      spin-major, then colour
  site index s = ((t*Lz + z)*Ly + y)*Lx + x

Gauge recipe (a synthetic stand-in for the paper's dynamical Wilson ensembles,
Sec. 5.1, which are not available): per link draw a 3x3 matrix G with iid
entries (a + ib)/sqrt(2), a, b ~ N(0, 1); form the traceless Hermitian
H = (G + G^H)/2 - tr(.)/3 I; set U = exp(i*eps*H) through the eigendecomposition
of H; then re-project onto SU(3) (Gram-Schmidt of rows 1-2, row 3 =
conj(row1 x row2)) so that unitarity and det U = 1 hold to rounding.
Right-hand sides: iid complex Gaussian entries (a + ib)/sqrt(2).

Random numbers come from numpy's PCG64 generator seeded per input.
"""
from __future__ import annotations

import numpy as np

# Gauge seeds and lattice names of the synthetic workloads.
LATTICES = {
    "4^4": (4, 4, 4, 4),
    "8^4": (8, 8, 8, 8),
    "16^3x32": (16, 16, 16, 32),
    "24^3x64": (24, 24, 24, 64),
}
GAUGE_SEEDS = {"4^4": 101, "8^4": 102, "16^3x32": 103, "24^3x64": 104}
LATTICE_IDS = {"4^4": 1, "8^4": 2, "16^3x32": 3, "24^3x64": 4}


def volume(dims) -> int:
    lx, ly, lz, lt = dims
    return int(lx) * int(ly) * int(lz) * int(lt)


def _su3_project(u: np.ndarray) -> np.ndarray:
    """Gram-Schmidt rows 0 and 1, then row 2 = conj(row0 x row1)."""
    r0 = u[..., 0, :]
    r0 = r0 / np.linalg.norm(r0, axis=-1, keepdims=True)
    r1 = u[..., 1, :]
    r1 = r1 - np.sum(np.conj(r0) * r1, axis=-1, keepdims=True) * r0
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = np.conj(np.cross(r0, r1))
    return np.stack([r0, r1, r2], axis=-2)


def random_su3(rng: np.random.Generator, n: int, eps: float) -> np.ndarray:
    """n SU(3) matrices exp(i*eps*H), H traceless Hermitian Gaussian."""
    g = (rng.standard_normal((n, 3, 3)) + 1j * rng.standard_normal((n, 3, 3))) / np.sqrt(2.0)
    h = 0.5 * (g + np.conj(np.swapaxes(g, -1, -2)))
    tr = np.trace(h, axis1=-2, axis2=-1).real / 3.0
    h = h - tr[:, None, None] * np.eye(3)
    w, W = np.linalg.eigh(h)
    u = (W * np.exp(1j * eps * w)[:, None, :]) @ np.conj(np.swapaxes(W, -1, -2))
    return _su3_project(u)


def make_gauge(dims, seed: int, eps: float = 0.3, chunk: int = 1 << 20) -> np.ndarray:
    """Gauge field [V][4][3][3] complex128 from the recipe above."""
    V = volume(dims)
    n = 4 * V
    rng = np.random.default_rng(seed)
    out = np.empty((n, 3, 3), dtype=np.complex128)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        out[s:e] = random_su3(rng, e - s, eps)
    return out.reshape(V, 4, 3, 3)


def unit_gauge(dims) -> np.ndarray:
    """Free field: every link the identity."""
    V = volume(dims)
    g = np.zeros((V, 4, 3, 3), dtype=np.complex128)
    g[:, :, 0, 0] = g[:, :, 1, 1] = g[:, :, 2, 2] = 1.0
    return g


def make_rhs(dims, seed: int, k: int = 1) -> np.ndarray:
    """k right-hand sides, each [V][4][3] complex128 with iid (a+ib)/sqrt(2) entries.

    Returns shape [k][V][4][3] (RHS-major)."""
    V = volume(dims)
    rng = np.random.default_rng(seed)
    z = rng.standard_normal((k, V, 4, 3, 2))
    return ((z[..., 0] + 1j * z[..., 1]) / np.sqrt(2.0)).astype(np.complex128)


def rhs_seed(lattice: str, r: int) -> int:
    """Seed of right-hand side number r of a run on the named lattice."""
    return 1_000_000 * LATTICE_IDS[lattice] + r


def random_gauge_transform(dims, seed: int) -> np.ndarray:
    """Random SU(3) matrix g(x) per site, [V][3][3] (for covariance tests)."""
    return random_su3(np.random.default_rng(seed), volume(dims), eps=1.0)
