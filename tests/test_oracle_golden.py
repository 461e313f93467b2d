"""The oracle against values fixed by the paper's text (tests/golden/, each file cites
its passage)."""
import os

import numpy as np

import oracle
from paper_0707_0131_gb300 import fixtures as fx

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_gamma5_is_the_papers_diagonal_sign_matrix():
    g5 = np.loadtxt(os.path.join(GOLDEN, "gamma5_sec1.txt"), comments="#")
    G = oracle.gammas()
    assert np.array_equal(G[4], g5.astype(np.complex128))
    # and it is the product of the four Dirac matrices of the operator
    assert np.allclose(G[0] @ G[1] @ G[2] @ G[3], g5, atol=1e-15)
    # gamma5 M = M^H gamma5 on a random field (Sec. 1)
    dims = (4, 2, 2, 2)
    W = oracle.Wilson(dims, 0.1, fx.make_gauge(dims, 63))
    psi = fx.make_rhs(dims, 64).reshape(-1)

    def g5v(v):
        return np.einsum("ab,vbc->vac", g5, v.reshape(-1, 4, 3)).reshape(-1)

    assert np.linalg.norm(g5v(W.M(psi)) - W.Mdag(g5v(psi))) < 1e-13 * np.linalg.norm(psi)
