"""Spectrally preconditioned eigCG (eig_eigcg_solve_sp) against the oracle.

The GPU basis U (grown by two plain eigCG solves) and its H are read back and handed
to the oracle, which runs eigCG of Fig. 1 with P^{-1} = (I - U_p U_p^H) + shift U_p
H_p^{-1} U_p^H (oracle/solvers.py: spectral_preconditioner) from the same deflated
initial guess (Eq. 1).  FP64 (tol 1e-10): iterations within 10%, the two lowest
pending Ritz values within 1e-6 relative, the true residual at tol; FP32 storage (tol
1e-8): iterations within 10% and Ritz values within 8 eps_32 ||A||; the basis keeps
growing.  Invalid arguments are refused.
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
M_Q = MASSES["8^4"]["1e+04"]["m_q"]
SHIFT = (8.0 + M_Q) ** 2


@pytest.fixture(scope="module")
def api():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_0707_0131_gb300 import api as a

    return a


@pytest.fixture(scope="module")
def wilson():
    gauge = fx.make_gauge(DIMS, fx.GAUGE_SEEDS["8^4"])
    return gauge, oracle.Wilson(DIMS, M_Q, gauge)


def _basis(api, gauge, prec):
    op = api.Op(gauge, DIMS, M_Q, prec=prec)
    basis = api.Basis(op, 64)
    for r in range(2):
        b = fx.make_rhs(DIMS, 300 + r).reshape(-1)
        x = np.zeros_like(b)
        op.eigcg_solve(b, x, nev=8, m=24, tol=1e-8, basis=basis)
        basis.grow()
    return op, basis


@pytest.mark.parametrize("prec,lp", [(64, 16), (64, 8), (32, 16)])
def test_spectral_eigcg_matches_oracle(api, wilson, prec, lp):
    gauge, W = wilson
    op, basis = _basis(api, gauge, prec)
    l = basis.size
    assert l >= lp
    U = basis.vectors()
    H = basis.H()
    b = fx.make_rhs(DIMS, 310).reshape(-1)
    x = np.zeros_like(b)
    tol = 1e-10 if prec == 64 else 1e-8
    st = op.eigcg_solve_sp(b, x, nev=8, m=24, tol=tol, basis=basis, sp_vecs=lp, sp_shift=SHIFT)
    assert st["converged"] == 1 and st["true_rel_res"] <= tol, st
    assert np.linalg.norm(b - W.A(x)) / np.linalg.norm(b) <= tol * (1 + 1e-6)
    x0 = solvers.deflated_guess(W.A, U, H, b)
    Pinv = solvers.spectral_preconditioner(U[:, :lp], H[:lp, :lp], SHIFT)
    ref = solvers.eigcg(W.A, b, x0, nev=8, m=24, tol=tol, Pinv=Pinv)
    assert abs(st["iters"] - ref["iters"]) <= 0.1 * ref["iters"], (st["iters"], ref["iters"])
    # the pending Ritz values are those of P^{-1} A: the oracle's lowest two.  FP64: 1e-6
    # relative; FP32 arithmetic resolves eigenvalues of A only to about eps_32 ||A||
    # (||A|| ~ SHIFT here), so its bar is 8 eps_32 ||A|| absolute
    pend = np.sort(basis.pending())
    ref_ev = np.sort(ref["ritz"])[:2]
    err = np.abs(pend[:2] - ref_ev)
    if prec == 64:
        assert np.max(err / ref_ev) < 1e-6, (pend[:4], ref_ev)
    else:
        assert np.max(err) < 8 * np.finfo(np.float32).eps * SHIFT, (pend[:4], ref_ev)
    basis.grow()
    assert basis.size > l
    basis.close()
    op.close()


def test_spectral_eigcg_refusals(api, wilson):
    from paper_0707_0131_gb300._lib import EIG_ERR_ARG, EigError

    gauge, _ = wilson
    op, basis = _basis(api, gauge, 64)
    b = fx.make_rhs(DIMS, 320).reshape(-1)
    for kw in [dict(sp_vecs=basis.size + 1, sp_shift=SHIFT), dict(sp_vecs=0, sp_shift=SHIFT),
               dict(sp_vecs=4, sp_shift=0.0), dict(sp_vecs=4, sp_shift=-1.0)]:
        with pytest.raises(EigError) as e:
            op.eigcg_solve_sp(b, np.zeros_like(b), nev=8, m=24, tol=1e-8, basis=basis, **kw)
        assert e.value.status == EIG_ERR_ARG, kw
    basis.close()
    op.close()
    op16 = api.Op(gauge, DIMS, M_Q, prec=16)
    b16 = api.Basis(op16, 32)
    x = np.zeros_like(b)
    op16.eigcg_solve(b, x, nev=8, m=24, tol=1e-5, basis=b16)
    b16.grow()
    with pytest.raises(EigError) as e:
        op16.eigcg_solve_sp(b, np.zeros_like(b), nev=8, m=24, tol=1e-5, basis=b16, sp_vecs=4, sp_shift=SHIFT)
    assert e.value.status == EIG_ERR_ARG
    b16.close()
    op16.close()
