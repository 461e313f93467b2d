"""ORACLE -- test infrastructure only.  Python face of the plain-C Wilson operator.

The operator is the one of Sec. 1: M = m_q I - D, gamma5-Hermitian, and CG is run
on the normal operator A = M^H M.  The convention written out in oracle/wilson.c:
  (M psi)(x) = (4 + m_q) psi(x)
      - 1/2 sum_mu [(I - g_mu) U_mu(x) psi(x+mu) + (I + g_mu) U_mu(x-mu)^H psi(x-mu)].

Vectors are numpy complex128 arrays of V*12 entries (any shape that flattens to
[V][4][3]); results come back flat.
"""
from __future__ import annotations

import numpy as np

from . import _native


def gammas() -> np.ndarray:
    """The oracle's gamma table: shape (5, 4, 4) = g1, g2, g3, g4, g5."""
    out = np.zeros(80, dtype=np.complex128)
    _native.lib().oracle_get_gammas(out.ctypes.data)
    return out.reshape(5, 4, 4)


def num_threads() -> int:
    return int(_native.lib().oracle_num_threads())


class Wilson:
    """A = M^H M of the Wilson-Dirac matrix for one gauge field and quark mass."""

    def __init__(self, dims, m_q: float, gauge: np.ndarray):
        self.dims = np.ascontiguousarray(np.asarray(dims, dtype=np.int32))
        self.m_q = float(m_q)
        self.V = int(np.prod(self.dims.astype(np.int64)))
        g = np.ascontiguousarray(gauge, dtype=np.complex128)
        if g.size != self.V * 36:
            raise ValueError("gauge must hold V*4*3*3 complex entries")
        self.gauge = g
        self.N = self.V * 12
        self._work = np.empty(self.N, dtype=np.complex128)
        self.applies = 0  # number of A applications (matrix-vector products of CG)

    def _vec(self, psi: np.ndarray) -> np.ndarray:
        v = np.ascontiguousarray(psi, dtype=np.complex128).reshape(-1)
        if v.size != self.N:
            raise ValueError("spinor must hold V*12 complex entries")
        return v

    def M(self, psi: np.ndarray) -> np.ndarray:
        v = self._vec(psi)
        out = np.empty(self.N, dtype=np.complex128)
        _native.lib().oracle_wilson_m(self.dims.ctypes.data, self.m_q, self.gauge.ctypes.data,
                                      v.ctypes.data, out.ctypes.data)
        return out

    def Mdag(self, psi: np.ndarray) -> np.ndarray:
        v = self._vec(psi)
        out = np.empty(self.N, dtype=np.complex128)
        _native.lib().oracle_wilson_mdag(self.dims.ctypes.data, self.m_q, self.gauge.ctypes.data,
                                         v.ctypes.data, out.ctypes.data, self._work.ctypes.data)
        return out

    def A(self, psi: np.ndarray) -> np.ndarray:
        v = self._vec(psi)
        out = np.empty(self.N, dtype=np.complex128)
        _native.lib().oracle_wilson_a(self.dims.ctypes.data, self.m_q, self.gauge.ctypes.data,
                                      v.ctypes.data, out.ctypes.data, self._work.ctypes.data)
        self.applies += 1
        return out

    __call__ = A

    def dense(self, which: str = "A") -> np.ndarray:
        """Dense matrix by applying the operator to every unit vector (tiny lattices only)."""
        if self.N > 6144:
            raise ValueError("dense() is for lattices of at most 512 sites")
        f = {"A": self.A, "M": self.M, "Mdag": self.Mdag}[which]
        D = np.empty((self.N, self.N), dtype=np.complex128)
        e = np.zeros(self.N, dtype=np.complex128)
        for k in range(self.N):
            e[k] = 1.0
            D[:, k] = f(e)
            e[k] = 0.0
        return D
