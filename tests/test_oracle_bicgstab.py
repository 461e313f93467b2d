"""Pins of the oracle's BiCGSTAB on M and of its deflation with eigenvectors of A (Sec. 1:
A = M^H M = (g5 M)^2, so the eigenvectors CG/eigCG compute for A are eigenvectors of the
Hermitian g5 M and can deflate BiCGSTAB for later right-hand sides).

* BiCGSTAB solves a random nonsymmetric system to the dense solution, terminates within
  N (+ rounding) steps on a tiny one, takes one step for M = c I, and solves the Wilson
  system M x = b to its tolerance;
* g5 M is Hermitian (so is H5 = U^H g5 M U for any U) and the deflated guess satisfies
  the Galerkin condition U^H g5 (b - M x0) = 0;
* when U spans complete eigenspaces of A (an invariant subspace of g5 M) the guess has
  the exact solution's components in span(U); a random U does not;
* deflating with the lowest eigenvectors of A cuts BiCGSTAB's iterations.
"""
import numpy as np
import pytest

import oracle
from oracle import solvers
from paper_0707_0131_gb300 import fixtures as fx


def _rand(n, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(n) + 1j * rng.standard_normal(n)) / np.sqrt(2)


@pytest.fixture(scope="module")
def wil():
    dims = (4, 2, 2, 2)
    W = oracle.Wilson(dims, -0.3, fx.make_gauge(dims, 62))
    Md = W.dense("M")
    g5 = oracle.gammas()[4]
    lam, X = np.linalg.eigh(W.dense("A"))
    return W, Md, g5, lam, X


def test_bicgstab_dense_and_special_cases():
    rng = np.random.default_rng(3)
    n = 60
    M = np.eye(n) * 4 + (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    b = _rand(n, 4)
    out = solvers.bicgstab(lambda v: M @ v, b, tol=1e-12)
    x = np.linalg.solve(M, b)
    assert out["true_rel_res"] < 1e-11
    assert np.linalg.norm(out["x"] - x) < 1e-10 * np.linalg.cond(M) * np.linalg.norm(x)
    # finite termination on a tiny system
    Ms = M[:6, :6]
    small = solvers.bicgstab(lambda v: Ms @ v, b[:6], tol=1e-13)
    assert small["iters"] <= 8 and small["true_rel_res"] < 1e-12
    # M = c I: one step, exact
    one = solvers.bicgstab(lambda v: 2.5 * v, b, tol=1e-14)
    assert one["iters"] == 1 and np.allclose(one["x"], b / 2.5, rtol=1e-15, atol=0)


def test_bicgstab_wilson(wil):
    W, Md, g5, lam, X = wil
    b = _rand(W.N, 5)
    out = solvers.bicgstab(W.M, b, tol=1e-10)
    assert out["true_rel_res"] < 2e-10
    x = np.linalg.solve(Md, b)
    assert np.linalg.norm(out["x"] - x) < 1e-7 * np.linalg.norm(x)


def test_g5_galerkin(wil):
    W, Md, g5, lam, X = wil
    G = np.stack([solvers.gamma5(c, g5) for c in Md.T], axis=1)  # g5 M, column by column
    assert np.linalg.norm(G - np.conj(G.T)) < 1e-13 * np.linalg.norm(G)
    rng = np.random.default_rng(6)
    U, _ = np.linalg.qr(rng.standard_normal((W.N, 10)) + 1j * rng.standard_normal((W.N, 10)))
    b = _rand(W.N, 7)
    x0, H5 = solvers.deflated_guess_g5(W.M, U, b, g5)
    assert np.linalg.norm(H5 - np.conj(H5.T)) < 1e-13 * np.linalg.norm(H5)
    r0 = b - W.M(x0)
    assert np.linalg.norm(np.conj(U.T) @ solvers.gamma5(r0, g5)) < 1e-12 * np.linalg.norm(b)


def test_invariant_subspace_gives_exact_components(wil):
    W, Md, g5, lam, X = wil
    # the l >= 8 lowest eigenvectors of A, l at a gap so that they span whole eigenspaces
    l = 8
    while lam[l] - lam[l - 1] < 1e-8 * lam[l]:
        l += 1
    U = X[:, :l]
    b = _rand(W.N, 8)
    x = np.linalg.solve(Md, b)
    x0, _ = solvers.deflated_guess_g5(W.M, U, b, g5)
    cx = np.conj(U.T) @ x
    assert np.linalg.norm(np.conj(U.T) @ x0 - cx) < 1e-9 * np.linalg.norm(cx)
    rng = np.random.default_rng(9)
    R, _ = np.linalg.qr(rng.standard_normal((W.N, l)) + 1j * rng.standard_normal((W.N, l)))
    xr, _ = solvers.deflated_guess_g5(W.M, R, b, g5)
    assert np.linalg.norm(np.conj(R.T) @ (xr - x)) > 1e-3 * np.linalg.norm(np.conj(R.T) @ x)


def test_deflation_cuts_iterations(wil):
    W, Md, g5, lam, X = wil
    b = _rand(W.N, 10)
    plain = solvers.bicgstab(W.M, b, tol=1e-10)
    x0, _ = solvers.deflated_guess_g5(W.M, X[:, :24], b, g5)
    defl = solvers.bicgstab(W.M, b, x0, tol=1e-10)
    assert defl["true_rel_res"] < 2e-10
    assert defl["iters"] < plain["iters"], (defl["iters"], plain["iters"])
