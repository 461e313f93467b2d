"""BiCGSTAB on M (eig_bicgstab_solve) against the oracle (oracle/solvers.py: bicgstab,
deflated_guess_g5), Sec. 1's use of the eigenvectors of A = (g5 M)^2 for later systems.

* FP64, no deflation: iterations within 10% of the oracle's, FP64 residual at tol, the
  same solution to cond * tol;
* FP32 storage: the FP64 residual still reaches tol (restarts from the FP64 residual);
* deflated with the lowest Ritz vectors of a basis grown by eigCG: the oracle, handed the
  GPU basis, runs the same g5 M Galerkin guess and BiCGSTAB; iterations within 10%, fewer
  than without deflation;
* odd-even and FP16 ops are refused.
"""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import solvers
from paper_0707_0131_gb300 import fixtures as fx

pytestmark = pytest.mark.gpu

DIMS = fx.LATTICES["8^4"]
MASSES = json.load(open(os.path.join(os.path.dirname(__file__), "..", "configs", "masses.json")))


@pytest.fixture(scope="module")
def api():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_0707_0131_gb300 import api as a

    return a


def _setup(kappa):
    m_q = MASSES["8^4"][kappa]["m_q"]
    gauge = fx.make_gauge(DIMS, fx.GAUGE_SEEDS["8^4"])
    return m_q, gauge, oracle.Wilson(DIMS, m_q, gauge)


def _rel(W, x, b):
    return np.linalg.norm(b - W.M(x)) / np.linalg.norm(b)


def test_bicgstab_fp64_matches_oracle(api):
    m_q, gauge, W = _setup("1e+03")
    op = api.Op(gauge, DIMS, m_q, prec=64)
    b = fx.make_rhs(DIMS, 400).reshape(-1)
    x = np.zeros_like(b)
    st = op.bicgstab_solve(b, x, tol=1e-10)
    ref = solvers.bicgstab(W.M, b, tol=1e-10)
    assert st["converged"] == 1 and _rel(W, x, b) <= 1e-10 * (1 + 1e-6), st
    assert abs(st["iters"] - ref["iters"]) <= 0.1 * ref["iters"], (st["iters"], ref["iters"])
    assert np.linalg.norm(x - ref["x"]) <= 1e-6 * np.linalg.norm(ref["x"])
    op.close()


def test_bicgstab_fp32_reaches_tol(api):
    m_q, gauge, W = _setup("1e+04")
    op = api.Op(gauge, DIMS, m_q, prec=32)
    b = fx.make_rhs(DIMS, 401).reshape(-1)
    x = np.zeros_like(b)
    st = op.bicgstab_solve(b, x, tol=1e-8)
    assert st["converged"] == 1 and st["true_rel_res"] <= 1e-8, st
    assert _rel(W, x, b) <= 1e-8 * (1 + 1e-6)
    assert st["restarts"] >= 1  # at least one FP64 restart on the way from 1 to 1e-8
    op.close()


@pytest.mark.parametrize("prec", [64, 32])
def test_deflated_bicgstab_matches_oracle(api, prec):
    m_q, gauge, W = _setup("1e+04")
    op = api.Op(gauge, DIMS, m_q, prec=prec)
    basis = api.Basis(op, 40)
    for r in range(3):
        bb = fx.make_rhs(DIMS, 410 + r).reshape(-1)
        xx = np.zeros_like(bb)
        op.eigcg_solve(bb, xx, nev=8, m=24, tol=1e-8, basis=basis)
        basis.grow()
    nz = 16
    U, H = basis.vectors(), basis.H()
    _, S = np.linalg.eigh(H)
    Z = U @ S[:, :nz]
    g5 = oracle.gammas()[4]
    b = fx.make_rhs(DIMS, 420).reshape(-1)
    tol = 1e-10 if prec == 64 else 1e-8
    x = np.zeros_like(b)
    st = op.bicgstab_solve(b, x, tol=tol, basis=basis, defl_vecs=nz)
    assert st["converged"] == 1 and _rel(W, x, b) <= tol * (1 + 1e-6), st
    x0, _ = solvers.deflated_guess_g5(W.M, Z, b, g5)
    ref = solvers.bicgstab(W.M, b, x0, tol=tol)
    plain = solvers.bicgstab(W.M, b, tol=tol)
    assert ref["iters"] < plain["iters"], (ref["iters"], plain["iters"])
    bar = 0.1 if prec == 64 else 0.25  # FP32: restarts from the FP64 residual cost a few iterations
    assert abs(st["iters"] - ref["iters"]) <= bar * ref["iters"], (st["iters"], ref["iters"])
    # the cached Z^H g5 M Z is reused by a second solve and rebuilt after the basis grows
    x2 = np.zeros_like(b)
    st2 = op.bicgstab_solve(b, x2, tol=tol, basis=basis, defl_vecs=nz)
    assert st2["iters"] == st["iters"] or prec == 32
    basis.close()
    op.close()


def test_bicgstab_refusals(api):
    from paper_0707_0131_gb300._lib import EIG_ERR_ARG, EigError

    m_q, gauge, _ = _setup("1e+03")
    b = fx.make_rhs(DIMS, 430).reshape(-1)
    for kw in [dict(prec=32, even_odd=True), dict(prec=16)]:
        op = api.Op(gauge, DIMS, m_q, **kw)
        with pytest.raises(EigError) as e:
            op.bicgstab_solve(b, np.zeros_like(b), tol=1e-8)
        assert e.value.status == EIG_ERR_ARG
        op.close()
