"""The engine's host FP64 linear algebra (small eigensolves of Fig. 1 steps 11.3-11.6,
Cholesky solves with H = U^H A U, Gram-Schmidt) against numpy on the CPU.

The engine's dense.cpp is compiled with g++ into a test shim (no GPU needed)."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
from oracle import solvers
from paper_0707_0131_gb300 import fixtures as fx

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_0707_0131_gb300", "csrc")
OUT = os.path.join(ROOT, "tests", "shim", "_build")


@pytest.fixture(scope="module")
def lib():
    os.makedirs(OUT, exist_ok=True)
    so = os.path.join(OUT, "libdense_shim.so")
    srcs = [os.path.join(ROOT, "tests", "shim", "dense_shim.cpp"), os.path.join(CSRC, "dense.cpp")]
    if not os.path.exists(so) or any(os.path.getmtime(s) > os.path.getmtime(so) for s in srcs):
        subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-I", CSRC, "-o", so, *srcs], check=True)
    L = ctypes.CDLL(so)
    V, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    L.shim_herm_eig_lowest.argtypes = [I, V, I, V, V]
    L.shim_window_lowest.argtypes = [I, V, I, I, I, V, V]
    L.shim_restart_coefficients.argtypes = [I, V, I, I, D, V, V]
    L.shim_cholesky_solve.argtypes = [I, V, V, I]
    L.shim_orth_columns.argtypes = [I, I, V, D, V]
    L.shim_lu_solve.argtypes = [I, V, V, I]
    L.shim_lu_solve.restype = ctypes.c_int
    L.shim_tridiag_eig.argtypes = [I, V, V, I, I, V, V]
    L.shim_restart_coefficients.restype = ctypes.c_int
    L.shim_cholesky_solve.restype = ctypes.c_int
    L.shim_orth_columns.restype = ctypes.c_int
    return L


def P(a):
    return a.ctypes.data


def rand_herm(rng, n, scale=1.0):
    G = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return scale * (G + G.conj().T) / 2


def lowest(lib, A, k):
    n = A.shape[0]
    w = np.zeros(k)
    Y = np.zeros((k, n), dtype=np.complex128)  # column-major n x k
    lib.shim_herm_eig_lowest(n, P(np.ascontiguousarray(A)), k, P(w), P(Y))
    return w, Y.T


@pytest.mark.parametrize("n,k", [(1, 1), (2, 2), (20, 20), (100, 10), (240, 240)])
def test_herm_eig_matches_numpy(lib, n, k):
    rng = np.random.default_rng(n)
    A = rand_herm(rng, n)
    w, Y = lowest(lib, A, k)
    ref = np.linalg.eigvalsh(A)[:k]
    nrm = np.abs(np.linalg.eigvalsh(A)).max()
    assert np.max(np.abs(w - ref)) < 1e-12 * nrm
    assert np.max(np.abs(A @ Y - Y * w)) < 1e-10 * nrm
    assert np.max(np.abs(Y.conj().T @ Y - np.eye(k))) < 1e-10


def test_tridiagonal_clusters_stay_orthonormal(lib):
    """Wilkinson's W21+ has pairs of eigenvalues equal to ~1e-14: the eigenvectors
    from inverse iteration must still be orthonormal."""
    n = 21
    d = np.abs(np.arange(n) - 10).astype(float)
    e = np.ones(n - 1)
    w = np.zeros(n)
    Z = np.zeros((n, n))
    lib.shim_tridiag_eig(n, P(d), P(e), 0, n, P(w), P(Z))
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    Zc = Z  # row q = eigenvector q
    assert np.max(np.abs(w - np.linalg.eigvalsh(T))) < 1e-13 * 10
    assert np.max(np.abs(Zc @ Zc.T - np.eye(n))) < 1e-10
    assert np.max(np.abs(T @ Zc.T - Zc.T * w)) < 1e-10


def structured_T(rng, m, kh):
    """eigCG window after a restart: diagonal Ritz head, arrow row kh, tridiagonal tail."""
    T = np.zeros((m, m), dtype=np.complex128)
    T[np.arange(kh), np.arange(kh)] = np.sort(rng.uniform(0.01, 0.1, kh))
    row = (rng.standard_normal(kh) + 1j * rng.standard_normal(kh)) * 0.05
    T[kh, :kh] = row
    T[:kh, kh] = row.conj()
    d = rng.uniform(0.5, 3.0, m - kh)
    e = -rng.uniform(0.1, 1.0, m - kh - 1)
    T[np.arange(kh, m), np.arange(kh, m)] = d
    T[np.arange(kh + 1, m), np.arange(kh, m - 1)] = e
    T[np.arange(kh, m - 1), np.arange(kh + 1, m)] = e
    return T


@pytest.mark.parametrize("m,kh,n", [(24, 0, 24), (24, 16, 24), (24, 16, 23), (100, 20, 100), (100, 20, 99),
                                    (9, 8, 9), (9, 8, 8), (9, 8, 5)])
def test_window_lowest_matches_dense(lib, m, kh, n):
    rng = np.random.default_rng(m + kh + n)
    T = structured_T(rng, m, kh)
    k = min(5, n)
    w = np.zeros(k)
    Y = np.zeros((k, n), dtype=np.complex128)
    lib.shim_window_lowest(m, P(T), kh, n, k, P(w), P(Y))
    Tn = T[:n, :n]
    ref, R = np.linalg.eigh(Tn)
    assert np.max(np.abs(w - ref[:k])) < 1e-13 * np.abs(ref).max()
    Y = Y.T
    assert np.max(np.abs(Tn @ Y - Y * w)) < 1e-11 * np.abs(ref).max()
    assert np.max(np.abs(Y.conj().T @ Y - np.eye(k))) < 1e-10




def test_restart_coefficients_against_oracle_steps(lib):
    dims = (4, 4, 4, 4)
    W = oracle.Wilson(dims, 0.05, fx.make_gauge(dims, 101))
    b = fx.make_rhs(dims, 7)[0].reshape(-1)
    nev, m = 8, 24
    first = []
    e = solvers.eigcg(W, b, nev=nev, m=m, tol=1e-10,
                      on_restart=lambda j, V, T, ritz: first.append((j, ritz.copy())) if not first else None)
    j, ritz_oracle = first[0]
    T = solvers.lanczos_tridiagonal(e["alphas"], e["betas"], m).astype(np.complex128)
    assert j == m + 1
    QZ = np.zeros((2 * nev, m), dtype=np.complex128)
    M = np.zeros(2 * nev)
    r = lib.shim_restart_coefficients(m, P(np.ascontiguousarray(T)), 0, nev, m * 2.2e-16, P(QZ), P(M))
    assert r == len(ritz_oracle) == 2 * nev
    # the lower half (the Y directions) is well conditioned; the top directions of
    # orth([Y Ybar]) have singular values down to ~1e-12 and are set by rounding
    assert np.max(np.abs(M[:nev] - ritz_oracle[:nev]) / np.abs(ritz_oracle[:nev])) < 1e-11
    QZ = QZ[:r].T
    # QZ has orthonormal columns and diagonalises T
    assert np.max(np.abs(QZ.conj().T @ QZ - np.eye(r))) < 1e-12
    assert np.max(np.abs(QZ.conj().T @ T @ QZ - np.diag(M))) < 1e-11 * np.abs(T).max()


def test_restart_coefficients_drop_dependent_columns(lib):
    """If Y and Ybar coincide (converged Ritz vectors), orth() keeps only the rank."""
    m, nev = 12, 3
    T = np.diag(np.arange(1.0, m + 1)).astype(np.complex128)  # eigenvectors are unit vectors
    QZ = np.zeros((2 * nev, m), dtype=np.complex128)
    M = np.zeros(2 * nev)
    r = lib.shim_restart_coefficients(m, P(T), 0, nev, m * 2.2e-16, P(QZ), P(M))
    assert r == nev
    assert np.allclose(M[:r], [1.0, 2.0, 3.0])


def test_cholesky_solve_and_orth(lib):
    rng = np.random.default_rng(3)
    n = 60
    G = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    H = G @ G.conj().T + n * np.eye(n)
    B = rng.standard_normal((n, 4)) + 1j * rng.standard_normal((n, 4))
    Hc = H.copy()
    Bc = np.ascontiguousarray(B.T)  # column-major n x 4
    assert lib.shim_cholesky_solve(n, P(Hc), P(Bc), 4) == 1
    assert np.max(np.abs(H @ Bc.T - B)) < 1e-10
    Hbad = -np.eye(3, dtype=np.complex128)
    assert lib.shim_cholesky_solve(3, P(Hbad), P(np.zeros(3, dtype=np.complex128)), 1) == 0
    # orth_columns: third column is a combination of the first two -> dropped
    X = rng.standard_normal((3, 50)) + 1j * rng.standard_normal((3, 50))
    X[2] = 0.3 * X[0] - 2.0 * X[1]
    keep = np.zeros(3, dtype=np.int32)
    Xc = np.ascontiguousarray(X)
    r = lib.shim_orth_columns(50, 3, P(Xc), 1e-10, P(keep))
    assert r == 2 and list(keep[:2]) == [0, 1]
    Q = Xc[:2].T
    assert np.max(np.abs(Q.conj().T @ Q - np.eye(2))) < 1e-13


@pytest.mark.parametrize("n", [1, 7, 64, 200])
def test_lu_solve_indefinite(lib, n):
    """Hermitian indefinite systems (the g5-M Galerkin matrix of the BiCGSTAB deflation)
    and a singular one."""
    rng = np.random.default_rng(n)
    A = rand_herm(rng, n)
    B = rng.standard_normal((n, 3)) + 1j * rng.standard_normal((n, 3))
    Af = np.ascontiguousarray(A.copy())
    Bc = np.ascontiguousarray(B.T.copy())  # column-major n x 3
    assert lib.shim_lu_solve(n, P(Af), P(Bc), 3) == 1
    X = np.linalg.solve(A, B)
    assert np.linalg.norm(Bc.T - X) <= 1e-10 * np.linalg.cond(A) * np.linalg.norm(X)
    S = np.zeros((n, n), dtype=np.complex128)  # exactly singular: refused
    S[:, 1:] = A[:, 1:]
    S[0, 0] = 0.0
    S[1:, 0] = 0.0
    if n > 1:
        S[:, 0] = 0.0
    Bs = np.ascontiguousarray(B[:, :1].T.copy())
    assert lib.shim_lu_solve(n, P(np.ascontiguousarray(S)), P(Bs), 1) == 0
