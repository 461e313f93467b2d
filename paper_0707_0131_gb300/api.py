"""Op / Basis handles over the C ABI (argument marshalling only).

    op = Op(gauge, dims, m_q, prec=32, max_rhs=4)       # A = M^H M (Sec. 1)
    basis = Basis(op, 240)
    st = op.eigcg_solve(b, x, nev=10, m=100, tol=1e-8, basis=basis)   # Fig. 1
    basis.grow()                                                       # Sec. 4 box
    sts = op.initcg_solve(B, X, tol=1e-8, restart_tol=1e-6, basis=basis, k=4)   # Eq. 1

Vectors: numpy complex128 (host) or torch complex128 CUDA tensors (device), in
the natural layout [k][V][4][3].
"""
from __future__ import annotations

import numpy as np

from . import _lib


class Op:
    def __init__(self, gauge, dims, m_q, prec=64, compress12=True, max_rhs=1, reliable_delta=0.1, even_odd=False):
        self.dims = tuple(int(d) for d in dims)
        self.V = int(np.prod(self.dims))
        self.even_odd = bool(even_odd)
        self.Vf = self.V // 2 if self.even_odd else self.V  # sites of apply / basis vectors
        self.m_q = float(m_q)
        self.prec = _lib.PREC[prec]
        self.max_rhs = int(max_rhs)
        self.h = _lib.eig_op_create(gauge, self.dims, m_q, prec, 1 if compress12 else 0, max_rhs, reliable_delta,
                                    1 if self.even_odd else 0)

    def close(self):
        if self.h is not None:
            _lib.eig_op_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def trim(self):
        """Releases the workspace (allocated again by the next call); bases keep their vectors."""
        return _lib.eig_op_trim(self.h)

    def apply(self, which, vin, vout, k=1, stream=None):
        _lib.eig_op_apply(self.h, which, vin, vout, k, stream)
        return vout

    def stencil_choice(self, k=1):
        """(variant, link_reals) the autotuner chose for k-RHS stencils."""
        return _lib.eig_op_stencil_choice(self.h, k)

    def _host(self, which, psi, k):
        vin = np.ascontiguousarray(psi, dtype=np.complex128)
        out = np.empty_like(vin)
        return self.apply(which, vin, out, k)

    def M(self, psi, k=1):
        return self._host(0, psi, k)

    def Mdag(self, psi, k=1):
        return self._host(1, psi, k)

    def A(self, psi, k=1):
        return self._host(2, psi, k)

    def eigcg_solve(self, b, x, nev, m, tol, basis=None, max_iter=100000, stream=None):
        return _lib.eig_eigcg_solve(self.h, basis.h if basis is not None else None, b, x, nev, m, tol, max_iter,
                                    stream)

    def eigcg_solve_sp(self, b, x, nev, m, tol, basis, sp_vecs, sp_shift, max_iter=100000, stream=None):
        """eigCG preconditioned by the spectral preconditioner of basis' first sp_vecs vectors."""
        return _lib.eig_eigcg_solve_sp(self.h, basis.h, b, x, nev, m, tol, sp_vecs, sp_shift, max_iter, stream)

    def bicgstab_solve(self, b, x, tol, basis=None, defl_vecs=0, max_iter=100000, stream=None):
        """BiCGSTAB on M x = b, deflated through g5 M with defl_vecs Ritz vectors of the basis."""
        return _lib.eig_bicgstab_solve(self.h, basis.h if basis is not None else None, b, x, tol, max_iter,
                                       defl_vecs, stream)

    def initcg_solve(self, b, x, tol, restart_tol=0.0, basis=None, k=1, max_iter=100000, stream=None):
        return _lib.eig_initcg_solve(self.h, basis.h if basis is not None else None, b, x, tol, restart_tol,
                                     max_iter, k, stream)


class Basis:
    def __init__(self, op: Op, max_vecs: int):
        self.op = op
        self.h = _lib.eig_basis_create(op.h, max_vecs)

    def close(self):
        if self.h is not None:
            _lib.eig_basis_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def size(self) -> int:
        return _lib.eig_basis_size(self.h)

    def truncate(self, l):
        _lib.eig_basis_truncate(self.h, l)

    def grow(self, stream=None):
        _lib.eig_basis_grow(self.h, stream)

    def deflate(self, b, x_in, x0, k=1, stream=None):
        _lib.eig_basis_deflate(self.h, b, x_in, x0, k, stream)
        return x0

    def ritz(self, residuals=True, stream=None):
        return _lib.eig_basis_ritz(self.h, residuals, stream)

    def vector(self, j):
        out = np.zeros(self.op.Vf * 12, dtype=np.complex128)
        _lib.eig_basis_vector(self.h, j, out)
        return out

    def vectors(self):
        return np.stack([self.vector(j) for j in range(self.size)], axis=1)

    def H(self):
        return _lib.eig_basis_h(self.h)

    def pending(self):
        """Ritz values of the pending block of the last eigCG solve."""
        return _lib.eig_basis_pending(self.h)

    def save(self, path, stream=None):
        """Writes U and H to a file (the pending Ritz block is not saved)."""
        _lib.eig_basis_save(self.h, path, stream)

    def load(self, path, stream=None):
        """Replaces U and H with a saved basis of the same operator."""
        _lib.eig_basis_load(self.h, path, stream)
