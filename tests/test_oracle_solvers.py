"""Pins of the oracle's solvers (CG, eigCG, Lanczos, init-CG, Incremental eigCG).

Each check is a fact fixed by the paper or by the mathematics, not a re-typing of
the oracle's formulas:
  * CG solves A x = b: compared with a dense LU solve on 4^4;
  * CG on the free field ends in at most (number of distinct eigenvalues) steps;
  * eigCG leaves CG untouched (Sec. 1, Sec. 3.1): x, residuals, alpha, beta are
    bit-identical to plain CG;
  * the eigCG window keeps V orthonormal and T = V^H A V (Sec. 3, Sec. 3.1);
  * Ritz values lie above the exact eigenvalues (Cauchy interlacing) and do not
    increase across restarts (Sec. 3.1, monotonic convergence);
  * Eq. 4 from CG scalars equals the tridiagonal of an independent Lanczos run
    started from b/||b|| (up to the sign convention of the off-diagonal);
  * eigCG tracks unrestarted Lanczos and stagnates later for larger (nev, m)
    (the Fig. 2 experiment, on a synthetic 8^4 operator);
  * Eq. 1 satisfies the Galerkin condition U^H (b - A x0) = 0, and with exact
    eigenvectors init-CG runs like CG on the spectrum with them removed;
  * Incremental eigCG recovers eigenvalue multiplicities of the free field
    exactly (each Krylov run sees an eigenspace once; deflation exposes the rest).
"""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import solvers
from paper_0707_0131_gb300 import fixtures as fx

MASSES = json.load(open(os.path.join(os.path.dirname(__file__), "..", "configs", "masses.json")))


@pytest.fixture(scope="module")
def small():
    """4^4, gauge seed 101, cond(A) ~ 1e3; dense A and its eigendecomposition."""
    dims = fx.LATTICES["4^4"]
    W = oracle.Wilson(dims, MASSES["4^4"]["1e+03"]["m_q"], fx.make_gauge(dims, 101))
    A = W.dense("A")
    lam, X = np.linalg.eigh(A)
    b = fx.make_rhs(dims, fx.rhs_seed("4^4", 0))[0].reshape(-1)
    return W, A, lam, X, b


def test_cg_matches_dense_solve(small):
    W, A, lam, X, b = small
    res = solvers.cg(W, b, tol=1e-10)
    x = np.linalg.solve(A, b)
    assert res["true_rel_res"] < 3e-10
    assert np.linalg.norm(res["x"] - x) / np.linalg.norm(x) < 1e-10 * lam[-1] / lam[0] * 10
    assert 50 < res["iters"] < 400


def test_cg_free_field_terminates():
    dims = (4, 4, 4, 4)
    m = 0.1
    W = oracle.Wilson(dims, m, fx.unit_gauge(dims))
    lam = np.linalg.eigvalsh(W.dense("A"))
    distinct = len(np.unique(np.round(lam, 9)))
    b = fx.make_rhs(dims, 77)[0]
    res = solvers.cg(W, b, tol=1e-12)
    # exact arithmetic: zero residual after `distinct` steps; rounding leaves ~1e-9
    assert res["res"][distinct] < 1e-7
    assert res["iters"] <= distinct + 3


def test_eigcg_leaves_cg_untouched(small):
    W, A, lam, X, b = small
    a = solvers.cg(W, b, tol=1e-10)
    e = solvers.eigcg(W, b, nev=8, m=24, tol=1e-10)
    assert e["restarts"] >= 3
    assert a["iters"] == e["iters"]
    assert np.array_equal(a["x"], e["x"])
    assert np.array_equal(a["res"], e["res"])
    assert np.array_equal(a["alphas"], e["alphas"]) and np.array_equal(a["betas"], e["betas"])


def test_eigcg_window_is_orthonormal_projection(small):
    W, A, lam, X, b = small
    checks = []

    def on_restart(j, V, T, ritz):
        AV = A @ V
        checks.append((j, np.max(np.abs(V.conj().T @ V - np.eye(V.shape[1]))),
                       np.max(np.abs(V.conj().T @ AV - T)) / lam[-1]))

    e = solvers.eigcg(W, b, nev=8, m=24, tol=1e-10, on_restart=on_restart)
    assert len(checks) == e["restarts"] >= 3
    # exact to rounding until Ritz vectors converge (Sec. 3.1): first restart
    assert checks[0][1] < 1e-12 and checks[0][2] < 1e-12
    # and still at the level of sqrt(eps) afterwards
    assert max(c[1] for c in checks) < 1e-7
    assert max(c[2] for c in checks) < 1e-7
    # final Ritz vectors: orthonormal and with Ritz values = Rayleigh quotients
    V = e["V"]
    assert np.max(np.abs(V.conj().T @ V - np.eye(V.shape[1]))) < 1e-7
    rq = np.real(np.einsum("ik,ik->k", V.conj(), A @ V))
    assert np.max(np.abs(rq - e["ritz"])) < 1e-8 * lam[-1]


def test_eigcg_ritz_bounds_monotone_and_tracks_lanczos(small):
    W, A, lam, X, b = small
    hist = []
    e = solvers.eigcg(W, b, nev=8, m=24, tol=1e-10,
                      on_restart=lambda j, V, T, ritz: hist.append((j, ritz[:8].copy())))
    H = np.array([h[1] for h in hist])
    # Cauchy interlacing: k-th Ritz value >= k-th eigenvalue
    assert np.all(H >= lam[None, :8] - 1e-10 * lam[-1])
    assert np.all(e["ritz"] >= lam[:8] - 1e-10 * lam[-1])
    # monotone across restarts (Rayleigh-Ritz + thick restart, Sec. 3.1)
    assert np.all(np.diff(H, axis=0) <= 1e-10 * lam[-1])
    # the window's Ritz values equal those of unrestarted Lanczos (Sec. 3.1, Fig. 2):
    # at every restart j (T_{j-1} complete) and at the end
    for j, th in hist:
        ev = np.linalg.eigvalsh(solvers.lanczos_tridiagonal(e["alphas"], e["betas"], j - 1))
        assert np.max(np.abs(th[:4] - ev[:4]) / ev[:4]) < 1e-8
    ev = np.linalg.eigvalsh(solvers.lanczos_tridiagonal(e["alphas"], e["betas"], e["iters"]))
    assert np.max(np.abs(e["ritz"][:4] - ev[:4]) / ev[:4]) < 1e-8


def test_eigcg_restart_is_exact_on_free_field():
    """Free field on 4x6x8x10: 236 distinct eigenvalues, far more than m = 16, so the
    window restarts many times; CG ends when b's Krylov space is exhausted, and eigCG's
    Ritz values are then the lowest distinct levels (m + sum(1-cos p))^2 + sum sin^2 p."""
    import itertools

    dims = (4, 6, 8, 10)
    m = 0.1
    W = oracle.Wilson(dims, m, fx.unit_gauge(dims))
    ps = [2 * np.pi * np.arange(L) / L for L in dims]
    lev = sorted({round((m + np.sum(1 - np.cos(p))) ** 2 + np.sum(np.sin(p) ** 2), 10)
                  for p in map(np.array, itertools.product(*ps))})
    b = fx.make_rhs(dims, 5)[0].reshape(-1)
    e = solvers.eigcg(W, b, nev=6, m=16, tol=1e-12)
    assert e["restarts"] > 10
    assert np.max(np.abs(e["ritz"] - np.array(lev[:6]))) < 1e-8


def test_cg_lanczos_tridiagonal_matches_independent_lanczos(small):
    W, A, lam, X, b = small
    res = solvers.cg(W, b, tol=1e-10)
    k = 25
    T_cg = solvers.lanczos_tridiagonal(res["alphas"], res["betas"], k)
    _, T_l = solvers.lanczos_full_reorth(lambda v: A @ v, b, k)
    assert np.max(np.abs(np.diag(T_cg) - np.diag(T_l))) < 1e-10 * lam[-1]
    # Eq. 4 off-diagonals are -(Lanczos beta) with non-alternating z/sqrt(rho) vectors
    assert np.max(np.abs(np.diag(T_cg, 1) + np.diag(T_l, 1))) < 1e-10 * lam[-1]
    # Ritz values of the full history lie above the spectrum (interlacing)
    ev = np.linalg.eigvalsh(solvers.lanczos_tridiagonal(res["alphas"], res["betas"], res["iters"]))
    assert np.all(ev[:8] >= lam[:8] - 1e-10 * lam[-1])
    # fully re-orthogonalised Lanczos run long enough resolves the clustered bottom
    _, T_long = solvers.lanczos_full_reorth(lambda v: A @ v, b, 400)
    assert np.max(np.abs(np.linalg.eigvalsh(T_long)[:4] - lam[:4])) < 1e-10 * lam[-1]


@pytest.mark.slow
def test_eigcg_tracks_lanczos_and_stagnation_order():
    """Fig. 2 analogue on 8^4 (synthetic, cond ~ 1e4)."""
    dims = fx.LATTICES["8^4"]
    W = oracle.Wilson(dims, MASSES["8^4"]["1e+04"]["m_q"], fx.make_gauge(dims, 102))
    b = fx.make_rhs(dims, fx.rhs_seed("8^4", 0))[0].reshape(-1)
    final = {}
    track = []
    for nev, m in [(1, 3), (3, 9), (8, 20)]:
        hist = []
        e = solvers.eigcg(W, b, nev=nev, m=m, tol=1e-10,
                          on_restart=lambda j, V, T, ritz: hist.append((j, ritz[0])))
        v0 = e["V"][:, 0]
        final[(nev, m)] = np.linalg.norm(W.A(v0) - e["ritz"][0] * v0)
        if (nev, m) == (8, 20):
            track = hist
            cgres = e
    assert final[(1, 3)] > final[(3, 9)] > final[(8, 20)]
    # eigCG(8,20) against the full-history Lanczos Ritz value at the same step:
    # the window is a subspace of the Krylov space, so its Ritz value is never
    # lower, and it stays close to it while converging
    lan_final = np.linalg.eigvalsh(solvers.lanczos_tridiagonal(cgres["alphas"], cgres["betas"],
                                                                cgres["iters"]))[0]
    for j, th in track[: len(track) // 2]:
        lj = np.linalg.eigvalsh(solvers.lanczos_tridiagonal(cgres["alphas"], cgres["betas"], j - 1))[0]
        assert th >= lj - 1e-12
        assert th - lan_final <= 2.0 * (lj - lan_final) + 1e-10


def test_initcg_galerkin_condition(small):
    W, A, lam, X, b = small
    dims = fx.LATTICES["4^4"]
    bs = [fx.make_rhs(dims, fx.rhs_seed("4^4", r))[0].reshape(-1) for r in (1, 2)]
    U, H, _ = solvers.incremental_eigcg(W, bs, nev=8, m=24, tol=1e-10)
    assert U.shape[1] == 16
    xt = fx.make_rhs(dims, 999)[0].reshape(-1)
    x0 = solvers.deflated_guess(W, U, H, b, xt)
    g = U.conj().T @ (b - A @ x0)
    assert np.linalg.norm(g) < 1e-11 * np.linalg.norm(b)
    # without deflation the same quantity is O(||b||): the check is not vacuous
    assert np.linalg.norm(U.conj().T @ (b - A @ xt)) > 1e-2 * np.linalg.norm(b)


def test_initcg_with_exact_eigenvectors_matches_deflated_spectrum(small):
    W, A, lam, X, b = small
    k = 24
    U = X[:, :k]
    H = U.conj().T @ A @ U
    tol = 1e-8
    out = solvers.initcg(W, U, H, b, tol=tol)
    # CG on the diagonal operator of the remaining eigenvalues with the same start residual
    r0 = b - A @ out["x0"]
    c = X.conj().T @ r0
    assert np.linalg.norm(c[:k]) < 1e-10 * np.linalg.norm(c)
    D = lam[k:]
    bd = c[k:]
    ref = solvers.cg(lambda v: D * v, bd, tol=tol * np.linalg.norm(b) / np.linalg.norm(bd))
    assert abs(out["iters"] - ref["iters"]) <= max(1, 0.1 * ref["iters"])
    plain = solvers.cg(W, b, tol=tol)
    assert out["iters"] < 0.8 * plain["iters"]
    assert out["true_rel_res"] < 3 * tol


def test_initcg_restart(small):
    W, A, lam, X, b = small
    dims = fx.LATTICES["4^4"]
    bs = [fx.make_rhs(dims, fx.rhs_seed("4^4", r))[0].reshape(-1) for r in (1, 2, 3)]
    U, H, _ = solvers.incremental_eigcg(W, bs, nev=8, m=24, tol=1e-10)
    out = solvers.initcg(W, U, H, b, tol=1e-10, restart_tol=1e-5)
    assert out["restarted"] and 0 < out["iters_before_restart"] < out["iters"]
    assert out["true_rel_res"] < 3e-10
    plain = solvers.cg(W, b, tol=1e-10)
    assert out["iters"] < plain["iters"]


def test_incremental_recovers_free_field_multiplicities():
    dims = (4, 4, 4, 4)
    m = 0.1
    W = oracle.Wilson(dims, m, fx.unit_gauge(dims))
    bs = [fx.make_rhs(dims, 500 + r)[0].reshape(-1) for r in range(13)]
    U, H, results = solvers.incremental_eigcg(W, bs, nev=2, m=24, tol=1e-12)
    theta, resn, _ = solvers.basis_ritz(W, U, H)
    lam0 = m ** 2  # p = 0, 12-fold
    lam1 = (m + 1.0) ** 2 + 1.0  # one direction at p = pi/2 or 3pi/2, 96-fold
    assert np.max(np.abs(theta[:12] - lam0)) < 1e-10
    assert theta[12] > lam0 + 0.5
    assert np.max(np.abs(theta[12:24] - lam1)) < 1e-9
    assert np.max(resn[:24]) < 1e-8
    # the 13th system has no p = 0 component left after deflation
    assert results[-1]["ritz"][0] > lam0 + 0.5


def test_incremental_basis_invariants(small):
    W, A, lam, X, b = small
    dims = fx.LATTICES["4^4"]
    bs = [fx.make_rhs(dims, fx.rhs_seed("4^4", r))[0].reshape(-1) for r in range(1, 5)]
    U, H, results = solvers.incremental_eigcg(W, bs, nev=8, m=24, tol=1e-10)
    l = U.shape[1]
    assert l == 32
    assert np.max(np.abs(U.conj().T @ U - np.eye(l))) < 1e-10
    assert np.max(np.abs(H - H.conj().T)) < 1e-12 * lam[-1]
    assert np.max(np.abs(H - U.conj().T @ A @ U)) < 1e-12 * lam[-1]
    theta, resn, _ = solvers.basis_ritz(W, U, H)
    assert np.all(theta >= lam[:l] - 1e-10 * lam[-1])
    # deflation helps: later systems take fewer iterations than the first
    assert results[-1]["iters"] < results[0]["iters"]
    # the lowest eigenpairs are found accurately (Sec. 5.2)
    assert np.max(np.abs(theta[:4] - lam[:4]) / lam[:4]) < 1e-8
