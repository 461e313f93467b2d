"""GPU parity at the 16^3x32 lattice (1.57M complex unknowns, several thousand tiles).

* Incremental eigCG(10, 100), FP64 GPU vs FP64 oracle, cond(A) ~ 1e3, two RHS:
  iterations per RHS within 10%, true residuals <= tol (oracle operator), lowest
  basis Ritz values within 1e-6, Galerkin condition of Eq. 1 on the GPU's basis.
* Mixed precision (FP32 and FP16 storage, 12-real links) at cond(A) ~ 1e4: the FP64
  true residual recomputed by the oracle meets 1e-8; FP32 iterations within 10% of the
  oracle's FP64 CG.
"""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import solvers
from paper_0707_0131_gb300 import fixtures as fx

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

MASSES = json.load(open(os.path.join(os.path.dirname(__file__), "..", "configs", "masses.json")))
NAME = "16^3x32"


@pytest.fixture(scope="module")
def api():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_0707_0131_gb300 import api as a

    return a


@pytest.fixture(scope="module")
def lattice():
    dims = fx.LATTICES[NAME]
    gauge = fx.make_gauge(dims, fx.GAUGE_SEEDS[NAME])
    bs = [fx.make_rhs(dims, fx.rhs_seed(NAME, r))[0].reshape(-1) for r in range(3)]
    return dims, gauge, bs


def test_incremental_eigcg_fp64_16x32(api, lattice):
    dims, gauge, bs = lattice
    m_q = MASSES[NAME]["1e+03"]["m_q"]
    W = oracle.Wilson(dims, m_q, gauge)
    U0, H0, ores = solvers.incremental_eigcg(W, bs[:2], nev=10, m=100, tol=1e-8)
    op = api.Op(gauge, dims, m_q, prec=64)
    basis = api.Basis(op, 32)
    for r in range(2):
        x = np.zeros_like(bs[r])
        st = op.eigcg_solve(bs[r], x, nev=10, m=100, tol=1e-8, basis=basis)
        assert abs(st["iters"] - ores[r]["iters"]) <= max(1, 0.1 * ores[r]["iters"]), (st, ores[r]["iters"])
        assert np.linalg.norm(bs[r] - W.A(x)) / np.linalg.norm(bs[r]) <= 1e-8
        basis.grow()
    assert basis.size == U0.shape[1]
    th_g, _ = basis.ritz(residuals=False)
    th_o = np.linalg.eigvalsh(H0)
    rel = np.abs(th_g[:4] - th_o[:4]) / th_o[:4]
    assert np.all(rel < 1e-6), rel
    # Galerkin condition of Eq. 1 on the GPU's own basis
    U = basis.vectors()
    X0 = np.zeros((1, bs[2].size), dtype=np.complex128)
    basis.deflate(bs[2].reshape(1, -1).copy(), None, X0, k=1)
    g = U.conj().T @ (bs[2] - W.A(X0[0]))
    assert np.linalg.norm(g) < 1e-10 * np.linalg.norm(bs[2])
    basis.close()
    op.close()


@pytest.mark.parametrize("prec", [32, 16])
def test_mixed_precision_16x32(api, lattice, prec):
    dims, gauge, bs = lattice
    m_q = MASSES[NAME]["1e+04"]["m_q"]
    W = oracle.Wilson(dims, m_q, gauge)
    op = api.Op(gauge, dims, m_q, prec=prec)
    x = np.zeros_like(bs[0])
    st = op.initcg_solve(bs[0], x, tol=1e-8)[0]
    assert st["converged"] == 1
    assert np.linalg.norm(bs[0] - W.A(x)) / np.linalg.norm(bs[0]) <= 1e-8
    if prec == 32:
        o = solvers.cg(W, bs[0], tol=1e-8)
        assert abs(st["iters"] - o["iters"]) <= 0.1 * o["iters"], (st["iters"], o["iters"])
    op.close()
