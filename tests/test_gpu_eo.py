"""Odd-even (Schur complement) operators on the GPU against the oracle (oracle/wilson_eo.py).

* M_hat, M_hat^H and A_hat on odd-site vectors: FP64 <= 1e-12, FP32 <= 1e-6 and FP16
  storage <= 5e-3 relative, k = 1 and 4, on lattices with a ragged last block;
* solves take the full-lattice b and x of M x = b: the reconstructed x satisfies the
  full Wilson equation (oracle M) to within cond(M_hat) times the tolerance of the
  odd-site normal equations, FP64 and mixed precision, single and batched;
* eigCG on the odd sites matches the oracle's eigCG on A_hat (iterations within 10%,
  lowest Ritz values within 1e-6), and a grown basis deflates later solves.
"""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import solvers
from oracle.wilson_eo import WilsonEO
from paper_0707_0131_gb300 import fixtures as fx

pytestmark = pytest.mark.gpu

TOL = {64: 1e-12, 32: 1e-6, 16: 5e-3}
MASSES = json.load(open(os.path.join(os.path.dirname(__file__), "..", "configs", "masses.json")))


@pytest.fixture(scope="module")
def api():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_0707_0131_gb300 import api as a

    return a


def _rand(n, seed, k=None):
    rng = np.random.default_rng(seed)
    shape = (n,) if k is None else (k, n)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2)


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 2, 10), (8, 8, 8, 8)])
@pytest.mark.parametrize("prec", [64, 32, 16])
@pytest.mark.parametrize("k", [1, 4])
def test_eo_matvec_parity(api, dims, prec, k):
    gauge = fx.make_gauge(dims, 71)
    E = WilsonEO(dims, 0.05, gauge)
    op = api.Op(gauge, dims, 0.05, prec=prec, max_rhs=k, even_odd=True)
    psi = _rand(E.N, 72, k)
    for which, f in [(0, E.Mhat), (1, E.Mhat_dag), (2, E.A)]:
        out = np.empty_like(psi)
        op.apply(which, psi, out, k)
        for r in range(k):
            ref = f(psi[r])
            err = np.linalg.norm(out[r] - ref) / np.linalg.norm(ref)
            assert err < TOL[prec], (dims, prec, k, which, r, err)
    op.close()


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("k", [1, 4])
def test_eo_solve_dirac_equation(api, prec, k):
    dims = fx.LATTICES["8^4"]
    m_q = MASSES["8^4"]["1e+03"]["m_q"]
    gauge = fx.make_gauge(dims, fx.GAUGE_SEEDS["8^4"])
    W = oracle.Wilson(dims, m_q, gauge)
    op = api.Op(gauge, dims, m_q, prec=prec, max_rhs=k, even_odd=True)
    B = _rand(W.N, 73, k)
    X = np.zeros_like(B)
    st = op.initcg_solve(B, X, tol=1e-10, k=k)
    for r in range(k):
        assert st[r]["converged"] == 1 and st[r]["true_rel_res"] <= 1e-10, st[r]
        # cond(M) * tol of the normal equations bounds the Dirac residual loosely
        assert np.linalg.norm(W.M(X[r]) - B[r]) / np.linalg.norm(B[r]) < 1e-7, r
    op.close()


def test_eo_eigcg_matches_oracle(api):
    dims = fx.LATTICES["8^4"]
    m_q = MASSES["8^4"]["1e+03"]["m_q"]
    gauge = fx.make_gauge(dims, fx.GAUGE_SEEDS["8^4"])
    E = WilsonEO(dims, m_q, gauge)
    W = oracle.Wilson(dims, m_q, gauge)
    b = _rand(W.N, 74)
    _, rhs = E.prepare(b)
    ref = solvers.eigcg(E, rhs, nev=8, m=24, tol=1e-10)
    op = api.Op(gauge, dims, m_q, prec=64, even_odd=True)
    basis = api.Basis(op, 16)
    x = np.zeros_like(b)
    st = op.eigcg_solve(b, x, nev=8, m=24, tol=1e-10, basis=basis)
    assert abs(st["iters"] - ref["iters"]) <= 0.1 * ref["iters"], (st["iters"], ref["iters"])
    assert np.linalg.norm(W.M(x) - b) / np.linalg.norm(b) < 1e-8
    basis.grow()
    ev, _ = basis.ritz(residuals=False)
    ref_ev = np.sort(ref["ritz"])[:2]
    assert np.max(np.abs(np.sort(ev)[:2] - ref_ev) / ref_ev) < 1e-6, (np.sort(ev)[:2], ref_ev)
    basis.close()
    op.close()


def test_eo_incremental_deflation(api):
    """eigCG grows an odd-site basis; later init-CG batches in mixed precision need fewer
    iterations and still solve M x = b."""
    dims = fx.LATTICES["8^4"]
    m_q = MASSES["8^4"]["1e+04"]["m_q"]
    gauge = fx.make_gauge(dims, fx.GAUGE_SEEDS["8^4"])
    W = oracle.Wilson(dims, m_q, gauge)
    op = api.Op(gauge, dims, m_q, prec=32, max_rhs=4, even_odd=True)
    B0 = _rand(W.N, 75, 4)
    X0 = np.zeros_like(B0)
    plain = op.initcg_solve(B0, X0, tol=1e-8, k=4)
    basis = api.Basis(op, 48)
    for r in range(4):
        b = _rand(W.N, 76 + r)
        x = np.zeros_like(b)
        op.eigcg_solve(b, x, nev=10, m=40, tol=1e-8, basis=basis)
        basis.grow()
    X = np.zeros_like(B0)
    st = op.initcg_solve(B0, X, tol=1e-8, restart_tol=1e-5, basis=basis, k=4)
    for r in range(4):
        assert st[r]["converged"] == 1
        assert np.linalg.norm(W.M(X[r]) - B0[r]) / np.linalg.norm(B0[r]) < 1e-5
        assert st[r]["iters"] < plain[r]["iters"], (st[r]["iters"], plain[r]["iters"])
    basis.close()
    op.close()
