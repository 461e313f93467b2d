"""Pins of the odd-even (Schur complement) oracle against the pinned full operator, the
mathematics of the block decomposition, and a closed form.

* Schur identity: with x_e = -(1/d) H_eo x_o, the full M maps (x_e, x_o) to (0, M_hat x_o);
* the full system M x = b solved through the odd sites (dense M_hat solve, reconstruction)
  equals the dense solve of M on 4^4;
* M_hat^H is the adjoint of M_hat and equals gamma5 M_hat gamma5; A_hat is Hermitian
  positive definite;
* unit links: the spectrum of A_hat is the closed form a(p)^2 + b(p)^2 s(p)^2 (module
  docstring of oracle/wilson_eo.py), each p ~ p + pi class 12-fold;
* CG on A_hat reconstructs a solution of M x = b.
"""
import numpy as np
import pytest

import oracle
from oracle import solvers
from oracle.wilson_eo import WilsonEO, free_field_spectrum_eo
from paper_0707_0131_gb300 import fixtures as fx


def _rand(n, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(n) + 1j * rng.standard_normal(n)) / np.sqrt(2)


@pytest.fixture(scope="module")
def eo44():
    dims = (4, 4, 4, 4)
    gauge = fx.make_gauge(dims, 101)
    return WilsonEO(dims, 0.1, gauge), oracle.Wilson(dims, 0.1, gauge), gauge


def test_schur_identity(eo44):
    E, W, _ = eo44
    xo = _rand(E.N, 1)
    xe = -E.hop(xo, 1) / E.d
    full = W.M(E.embed(xe, 0) + E.embed(xo, 1))
    assert np.linalg.norm(E.restrict(full, 0)) < 1e-13 * np.linalg.norm(full)
    ref = E.Mhat(xo)
    assert np.linalg.norm(E.restrict(full, 1) - ref) < 1e-13 * np.linalg.norm(ref)


def test_full_solve_through_odd_sites(eo44):
    E, W, _ = eo44
    b = _rand(W.N, 2)
    bhat, _ = E.prepare(b)
    xo = np.linalg.solve(E.dense("Mhat"), bhat)
    x = E.reconstruct(xo, b)
    assert np.linalg.norm(W.M(x) - b) < 1e-12 * np.linalg.norm(b)
    xd = np.linalg.solve(W.dense("M"), b)
    assert np.linalg.norm(x - xd) < 1e-11 * np.linalg.norm(xd)


def test_adjoint_and_gamma5(eo44):
    E, _, _ = eo44
    phi, psi = _rand(E.N, 3), _rand(E.N, 4)
    lhs = np.vdot(phi, E.Mhat(psi))
    rhs = np.vdot(E.Mhat_dag(phi), psi)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    g5 = np.tile(np.repeat([1.0, 1.0, -1.0, -1.0], 3), E.Vh)
    assert np.linalg.norm(E.Mhat_dag(psi) - g5 * E.Mhat(g5 * psi)) < 1e-13 * np.linalg.norm(psi)


def test_normal_operator_hpd(eo44):
    E, _, _ = eo44
    A = E.dense("A")
    assert np.linalg.norm(A - A.conj().T) < 1e-12 * np.linalg.norm(A)
    assert np.linalg.eigvalsh(A).min() > 0


@pytest.mark.parametrize("m_q", [0.1, -0.3])
def test_free_field_spectrum(m_q):
    dims = (4, 4, 4, 4)
    E = WilsonEO(dims, m_q, fx.unit_gauge(dims))
    ev = np.linalg.eigvalsh(E.dense("A"))
    ref = free_field_spectrum_eo(dims, m_q)
    assert ev.shape == ref.shape
    assert np.max(np.abs(ev - ref)) < 1e-10 * ref.max()


def test_cg_on_odd_sites_solves_the_dirac_equation():
    dims = (4, 4, 4, 8)
    gauge = fx.make_gauge(dims, 7)
    E = WilsonEO(dims, 0.05, gauge)
    W = oracle.Wilson(dims, 0.05, gauge)
    b = _rand(W.N, 5)
    _, rhs = E.prepare(b)
    out = solvers.cg(E, rhs, tol=1e-12)
    x = E.reconstruct(out["x"], b)
    assert np.linalg.norm(W.M(x) - b) < 1e-9 * np.linalg.norm(b)
