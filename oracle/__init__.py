"""ORACLE -- test infrastructure, not part of the product.

A plain, slow, FP64 CPU statement of what the solver computes, written from the
paper (Stathopoulos & Orginos, "Computing and deflating eigenvalues while solving
multiple right hand side linear systems ..."):

  wilson.c / wilson.py   M = m_q I - D (Sec. 1), M^H = gamma5 M gamma5, A = M^H M
  wilson_eo.py           odd-even (Schur complement) form: M_hat on odd sites, its normal
                         equations, preparation of b and reconstruction of x (Sec. 5)
  solvers.py             CG and eigCG (Fig. 1, with an optional preconditioner P, Sec. 3),
                         full-history Lanczos (Eq. 4, Sec. 3.1), init-CG (Eq. 1) with its
                         restart (Sec. 5.3), Incremental eigCG and Rayleigh-Ritz on U
                         (Sec. 4 box, Sec. 5.2), the spectral preconditioner from U (Sec. 2),
                         BiCGSTAB on M deflated with eigenvectors of A through g5 M (Sec. 1)

Only tests/, __graft_entry__.smoke() and the CPU-baseline leg of bench.py may
import this package.  It shares no code with the CUDA library; the two meet only
through the seeded input generators (the package's fixtures module).

Parity pins (tests/test_oracle_*.py): free-field spectrum in closed form, plane
waves, gamma5-Hermiticity, Hermiticity and positivity of A, gauge covariance,
dense solves and eigensolves on 4^4, CG/eigCG bit-identity, T = V^H A V, Galerkin
condition of Eq. 1, PCG against CG on the split system, the spectrum of the spectrally
preconditioned operator in closed form, P-orthonormality of the preconditioned eigCG
window, BiCGSTAB against dense solves and the Galerkin / invariant-subspace properties
of the g5 M deflation, the Schur identity against the full operator and the free-field
spectrum of the odd-site normal equations in closed form.  Parity of the eigen part at the paper's own scale (its
figures, on ensembles that are not available) is unpinned.
"""
from .wilson import Wilson, gammas, num_threads  # noqa: F401
from .wilson_eo import WilsonEO, free_field_spectrum_eo  # noqa: F401
from . import solvers  # noqa: F401
