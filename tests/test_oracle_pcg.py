"""Pins of the preconditioned CG / eigCG of the oracle (Fig. 1 with P != I, Sec. 3) and
of the spectral preconditioner built from the deflation basis (Sec. 2).

* P = I given as a callable reproduces the unpreconditioned CG and eigCG bit for bit;
* PCG with an HPD P^{-1} = L L^H equals CG on the split system L^H A L y = L^H b
  (same alpha_j, beta_j over the first iterations), converges to the dense solution,
  and a preconditioner close to A^{-1} cuts the iterations;
* with U the lowest exact eigenvectors of A, P^{-1} A has the eigenvalue `shift` on
  span(U) and the other eigenvalues of A unchanged (closed form); for any orthonormal
  U the preconditioner is Hermitian positive definite;
* eigCG with P keeps its window P-orthonormal (V^H P V = I) and T = V^H A V at every
  restart (Sec. 3);
* eigCG spectrally preconditioned with the lowest l eigenvectors finds the next ones:
  its lowest Ritz value is lambda_{l+1} of A and the Ritz vector is an eigenvector of A.
"""
import numpy as np
import pytest

import oracle
from oracle import solvers
from paper_0707_0131_gb300 import fixtures as fx


def _dense_hpd(n, cond, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    ev = np.geomspace(1.0, cond, n)
    return (Q * ev) @ np.conj(Q.T)


def _rand(n, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(n) + 1j * rng.standard_normal(n)) / np.sqrt(2)


@pytest.fixture(scope="module")
def small_wilson():
    dims = (4, 2, 2, 2)
    W = oracle.Wilson(dims, 0.02, fx.make_gauge(dims, 61))
    A = W.dense("A")
    lam, X = np.linalg.eigh(A)
    return W, A, lam, X


def test_identity_preconditioner_is_plain_cg():
    A = _dense_hpd(60, 1e3, 1)
    b = _rand(60, 2)
    f = lambda v: A @ v  # noqa: E731
    ident = lambda r: r.copy()  # noqa: E731
    a, c = solvers.cg(f, b, tol=1e-10), solvers.cg(f, b, tol=1e-10, Pinv=ident)
    assert a["iters"] == c["iters"]
    assert np.array_equal(a["x"], c["x"]) and np.array_equal(a["alphas"], c["alphas"])
    e1 = solvers.eigcg(f, b, nev=4, m=12, tol=1e-10)
    e2 = solvers.eigcg(f, b, nev=4, m=12, tol=1e-10, Pinv=ident)
    assert np.array_equal(e1["x"], e2["x"]) and np.array_equal(e1["ritz"], e2["ritz"])


def test_pcg_equals_cg_on_the_split_system():
    n = 48
    A = _dense_hpd(n, 1e4, 3)
    Pinv = _dense_hpd(n, 30.0, 4)
    L = np.linalg.cholesky(Pinv)  # Pinv = L L^H
    b = _rand(n, 5)
    pcg = solvers.cg(lambda v: A @ v, b, tol=1e-9, Pinv=lambda r: Pinv @ r)
    Ah = np.conj(L.T) @ A @ L
    split = solvers.cg(lambda v: Ah @ v, np.conj(L.T) @ b, tol=1e-30, max_iter=12)
    # the same scalars while rounding has not yet separated the two recurrences
    assert np.allclose(pcg["alphas"][:12], split["alphas"][:12], rtol=1e-9, atol=0)
    assert np.allclose(pcg["betas"][1:12], split["betas"][1:12], rtol=1e-9, atol=0)
    x_ref = np.linalg.solve(A, b)
    assert np.linalg.norm(pcg["x"] - x_ref) <= 1e-4 * np.linalg.norm(x_ref)
    # and it needs fewer iterations than plain CG when P^{-1} approximates A^{-1}
    Pgood = np.linalg.inv(A + np.eye(n))  # cond(P^{-1} A) <= 2
    better = solvers.cg(lambda v: A @ v, b, tol=1e-9, Pinv=lambda r: Pgood @ r)
    plain = solvers.cg(lambda v: A @ v, b, tol=1e-9)
    assert better["iters"] < plain["iters"] // 5, (better["iters"], plain["iters"])


@pytest.mark.parametrize("l", [1, 8])
def test_spectral_preconditioner_closed_form(small_wilson, l):
    W, A, lam, X = small_wilson
    U = X[:, :l]
    H = np.conj(U.T) @ A @ U
    shift = 0.5 * (lam[l] + lam[-1])
    Pinv = solvers.spectral_preconditioner(U, H, shift)
    n = A.shape[0]
    D = np.stack([Pinv(e) for e in np.eye(n, dtype=np.complex128)], axis=1)
    ev = np.sort(np.linalg.eigvals(D @ A).real)
    ref = np.sort(np.concatenate([np.full(l, shift), lam[l:]]))
    assert np.max(np.abs(ev - ref)) <= 1e-9 * lam[-1]
    # any orthonormal U: Hermitian positive definite
    rng = np.random.default_rng(7)
    Ur, _ = np.linalg.qr(rng.standard_normal((n, l)) + 1j * rng.standard_normal((n, l)))
    Dr = np.stack([solvers.spectral_preconditioner(Ur, np.conj(Ur.T) @ A @ Ur, shift)(e)
                   for e in np.eye(n, dtype=np.complex128)], axis=1)
    assert np.linalg.norm(Dr - np.conj(Dr.T)) <= 1e-12 * np.linalg.norm(Dr)
    assert np.linalg.eigvalsh(Dr).min() > 0


def test_preconditioned_eigcg_window(small_wilson):
    W, A, lam, X = small_wilson
    n = A.shape[0]
    rng = np.random.default_rng(8)
    Ur, _ = np.linalg.qr(rng.standard_normal((n, 6)) + 1j * rng.standard_normal((n, 6)))
    Pinv = solvers.spectral_preconditioner(Ur, np.conj(Ur.T) @ A @ Ur, lam[-1])
    Pd = np.stack([Pinv(e) for e in np.eye(n, dtype=np.complex128)], axis=1)
    P = np.linalg.inv(Pd)
    seen = []

    def check(j, V, T, ritz):
        # exact over the first restarts; once Ritz values converge the recurrence loses
        # orthogonality slowly (finite-precision Lanczos: up to ~1e-6 here), orders of
        # magnitude below what an error in the window's contents would show
        bar = 1e-10 if len(seen) < 3 else 1e-5
        seen.append(j)
        assert np.linalg.norm(np.conj(V.T) @ P @ V - np.eye(V.shape[1])) < bar
        assert np.linalg.norm(np.conj(V.T) @ A @ V - T) < bar * np.linalg.norm(T)

    out = solvers.eigcg(lambda v: A @ v, _rand(n, 9), nev=4, m=16, tol=1e-11, on_restart=check, Pinv=Pinv)
    assert len(seen) >= 2 and out["true_rel_res"] < 1e-10


def test_spectral_eigcg_finds_the_next_eigenvalues(small_wilson):
    W, A, lam, X = small_wilson
    l = 8
    U = X[:, :l]
    Pinv = solvers.spectral_preconditioner(U, np.conj(U.T) @ A @ U, lam[-1])
    out = solvers.eigcg(lambda v: A @ v, _rand(A.shape[0], 10), nev=4, m=24, tol=1e-13, Pinv=Pinv)
    theta = out["ritz"][0]
    assert abs(theta - lam[l]) <= 1e-8 * lam[l], (theta, lam[l])
    v = out["V"][:, 0]
    assert np.linalg.norm(A @ v - theta * v) <= 1e-6 * lam[-1] * np.linalg.norm(v)
    assert np.linalg.norm(np.conj(U.T) @ v) <= 1e-6 * np.linalg.norm(v)
