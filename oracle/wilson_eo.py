"""ORACLE -- test infrastructure only.  Odd-even (Schur complement) form of the Wilson
operator, the preconditioned system the paper solves (Sec. 5: "odd-even preconditioned
normal equations", a matrix of half the size).

Sites are split by parity p(x) = (x + y + z + t) mod 2 (every extent even, so the
hopping term only connects opposite parities).  With M = d I + H, d = 4 + m_q and H the
hopping part (H = M - d I, taken from the full operator of wilson.py):

    M_hat   = d I - (1/d) H_oe H_eo                      (on odd sites)
    M x = b  <=>  M_hat x_o = b_o - (1/d) H_oe b_e,   x_e = (b_e - H_eo x_o) / d
    A_hat   = M_hat^H M_hat,   M_hat^H = d I - (1/d) (H^H)_oe (H^H)_eo

and CG runs on A_hat x_o = M_hat^H b_hat.  Half-lattice vectors hold the 12 complex
components of each site of one parity, the sites in natural order (with an even x
extent, odd site s sits at position s // 2).
"""
from __future__ import annotations

import numpy as np

from .wilson import Wilson


class WilsonEO:
    """A_hat = M_hat^H M_hat on the odd sites of one gauge field and quark mass."""

    def __init__(self, dims, m_q: float, gauge: np.ndarray):
        dims = [int(v) for v in dims]
        if any(L % 2 for L in dims):
            raise ValueError("odd-even splitting needs every lattice extent even")
        self.full = Wilson(dims, m_q, gauge)
        self.dims = dims
        self.m_q = float(m_q)
        self.d = 4.0 + self.m_q
        self.V = self.full.V
        self.Vh = self.V // 2
        self.N = self.Vh * 12
        L0, L1, L2, L3 = dims
        t, z, y, x = np.meshgrid(np.arange(L3), np.arange(L2), np.arange(L1), np.arange(L0), indexing="ij")
        par = ((x + y + z + t) % 2).reshape(-1)
        self.sites = {0: np.nonzero(par == 0)[0], 1: np.nonzero(par == 1)[0]}
        self.applies = 0

    # -- half <-> full ---------------------------------------------------------------
    def embed(self, xh: np.ndarray, parity: int) -> np.ndarray:
        out = np.zeros((self.V, 12), dtype=np.complex128)
        out[self.sites[parity]] = np.asarray(xh, dtype=np.complex128).reshape(self.Vh, 12)
        return out.reshape(-1)

    def restrict(self, xf: np.ndarray, parity: int) -> np.ndarray:
        return np.asarray(xf, dtype=np.complex128).reshape(self.V, 12)[self.sites[parity]].reshape(-1)

    # -- hopping blocks ----------------------------------------------------------------
    def H(self, xf: np.ndarray) -> np.ndarray:
        """Hopping part of M: M x - d x."""
        xf = np.asarray(xf, dtype=np.complex128).reshape(-1)
        return self.full.M(xf) - self.d * xf

    def Hdag(self, xf: np.ndarray) -> np.ndarray:
        xf = np.asarray(xf, dtype=np.complex128).reshape(-1)
        return self.full.Mdag(xf) - self.d * xf

    def hop(self, xh: np.ndarray, src: int, dag: bool = False) -> np.ndarray:
        """(H or H^H) restricted to the block from parity src to the other parity."""
        f = self.Hdag if dag else self.H
        return self.restrict(f(self.embed(xh, src)), 1 - src)

    # -- Schur complement ---------------------------------------------------------------
    def Mhat(self, xo: np.ndarray) -> np.ndarray:
        xo = np.asarray(xo, dtype=np.complex128).reshape(-1)
        return self.d * xo - self.hop(self.hop(xo, 1), 0) / self.d

    def Mhat_dag(self, xo: np.ndarray) -> np.ndarray:
        xo = np.asarray(xo, dtype=np.complex128).reshape(-1)
        return self.d * xo - self.hop(self.hop(xo, 1, True), 0, True) / self.d

    def A(self, xo: np.ndarray) -> np.ndarray:
        self.applies += 1
        return self.Mhat_dag(self.Mhat(xo))

    __call__ = A

    # -- the full system ------------------------------------------------------------------
    def prepare(self, b: np.ndarray):
        """b (full lattice) -> (b_hat, M_hat^H b_hat): the odd-site system M_hat x_o = b_hat
        and the right-hand side of its normal equations."""
        be, bo = self.restrict(b, 0), self.restrict(b, 1)
        bhat = bo - self.hop(be, 0) / self.d
        return bhat, self.Mhat_dag(bhat)

    def reconstruct(self, xo: np.ndarray, b: np.ndarray) -> np.ndarray:
        """Full-lattice solution from the odd sites: x_e = (b_e - H_eo x_o) / d."""
        be = self.restrict(b, 0)
        xe = (be - self.hop(xo, 1)) / self.d
        return self.embed(xe, 0) + self.embed(xo, 1)

    def dense(self, which: str = "A") -> np.ndarray:
        """Dense matrix of A_hat (or M_hat) on the odd sites (tiny lattices only)."""
        if self.N > 3072:
            raise ValueError("dense() is for lattices of at most 512 sites")
        f = {"A": self.A, "Mhat": self.Mhat, "Mhat_dag": self.Mhat_dag}[which]
        D = np.empty((self.N, self.N), dtype=np.complex128)
        e = np.zeros(self.N, dtype=np.complex128)
        for k in range(self.N):
            e[k] = 1.0
            D[:, k] = f(e)
            e[k] = 0.0
        return D


def free_field_spectrum_eo(dims, m_q: float) -> np.ndarray:
    """Eigenvalues of A_hat for unit links (closed form, sorted).

    In momentum space D(p) = 2c - 2i gamma.s with c = sum cos p_mu, s_mu = sin p_mu, so
    M_hat(p) = d - (c - i gamma.s)^2 / d = a + i b gamma.s with a = d - (c^2 - s^2)/d,
    b = 2c/d, and A_hat(p) = a^2 + b^2 s^2 (times the 4x4 identity: gamma.s is Hermitian
    with square s^2).  p and p + (pi, pi, pi, pi) give the same value and describe one
    mode of the half lattice, so each class contributes 12 (4 spin x 3 colour) eigenvalues."""
    d = 4.0 + m_q
    axes = [2 * np.pi * np.arange(L) / L for L in dims]
    P = np.meshgrid(*axes, indexing="ij")
    c = sum(np.cos(p) for p in P)
    s2 = sum(np.sin(p) ** 2 for p in P)
    a = d - (c * c - s2) / d
    lam = (a * a + (2 * c / d) ** 2 * s2).reshape(-1)
    # every value appears twice over the full Brillouin zone (p and p + pi): keep half
    lam = np.sort(lam)[::2]
    return np.sort(np.repeat(lam, 12))
