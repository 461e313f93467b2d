"""ORACLE -- test infrastructure only.  Plain FP64 NumPy statement of the paper's solvers.

Each function follows the paper's steps in its order and notation; library
routines (numpy.linalg.eigh, numpy.linalg.qr, numpy.linalg.svd,
numpy.linalg.solve) serve as single steps.  Nothing here is blocked, fused or
reordered.  Only the tests, the smoke check and the benchmark's CPU-baseline leg
may call this module.

Vectors are flat complex128 arrays of length N; ``A`` is any callable x -> A x
(an HPD matrix, here M^H M of oracle.wilson.Wilson).

Readings of points the paper leaves open (each also listed in the design notes):
  * Stopping rule: the loop of Fig. 1 stops on ||r||/||r0||; here it stops on
    the recursive ||r|| <= tol*||b|| (identical for a zero initial guess,
    stricter for deflated starts), and the FP64 true residual is reported.
  * Step 11.1 of Fig. 1 prints T_{j-1,j-1}; the entry written is the diagonal of
    the window column that holds z_{j-1}, i.e. T_{i,i}, with beta_1/alpha_0 := 0.
  * Step 11.10 uses -sqrt(beta_j)/alpha_{j-1} (V holds z/sqrt(rho) with no sign
    alternation); Eq. 4's "+" assumes alternating signs.
  * Step 11.5's orth() is read as Matlab's orth: an orthonormal basis of the
    range from the SVD, dropping singular values below max(m, 2nev)*eps*s_max;
    i becomes that rank.
  * The eigCG output (Sec. 4 box "[x, V, M] = eigCG(...)") is read as the nev
    lowest Ritz pairs of the final window T_i (all of them if i <= nev).
  * init-CG restart (Sec. 5.3): once, when ||r||/||b|| first falls to
    restart_tol, re-deflate from the current x and restart CG.
  * Incremental eigCG (Sec. 4 box): "orthonormalize V against U" is classical
    Gram-Schmidt applied twice followed by a QR of the remainder; a column whose
    remainder norm falls below drop_tol is dropped.
"""
from __future__ import annotations

import numpy as np


def _norm(v: np.ndarray) -> float:
    return float(np.sqrt(np.vdot(v, v).real))


def _lowest_eigpairs(T: np.ndarray, k: int):
    """k algebraically smallest eigenpairs of the Hermitian matrix T (ascending)."""
    w, Y = np.linalg.eigh(T)
    return w[:k], Y[:, :k]


def _orth(X: np.ndarray, m_scale: int) -> np.ndarray:
    """Matlab-style orth(): left singular vectors above max(size)*eps*s_max."""
    Uq, s, _ = np.linalg.svd(X, full_matrices=False)
    if s.size == 0 or s[0] == 0.0:
        return Uq[:, :0]
    tol = max(m_scale, X.shape[1]) * np.finfo(np.float64).eps * s[0]
    rank = int(np.sum(s > tol))
    return Uq[:, :rank]


# ----------------------------------------------------------------------------------------
# CG, Fig. 1 left box, with P = I (z = r)
# ----------------------------------------------------------------------------------------
def cg(A, b, x0=None, tol=1e-10, max_iter=100000, Pinv=None):
    """Conjugate Gradient of Fig. 1 (left box); Pinv (a callable r -> P^{-1} r for an
    HPD preconditioner P) applies step 3, P = I when None.

    Returns dict(x, iters, res (recursive ||r||/||b|| per iteration, entry 0 =
    start), alphas, betas (betas[j-1] = beta_j, beta_1 = 0), true_rel_res)."""
    b = np.asarray(b, dtype=np.complex128).reshape(-1)
    bnorm = _norm(b)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128).reshape(-1)
    r = b - A(x) if x0 is not None else b.copy()  # step 0
    j = 0
    rho = None
    res, alphas, betas = [], [], []
    p = None
    while True:
        rr = np.vdot(r, r).real
        res.append(np.sqrt(rr) / bnorm)
        if np.sqrt(rr) <= tol * bnorm or j >= max_iter:  # step 1
            break
        j += 1  # step 2
        z = r if Pinv is None else np.asarray(Pinv(r), dtype=np.complex128)  # step 3
        rho_prev, rho = rho, (rr if Pinv is None else np.vdot(r, z).real)  # step 4: rho = r^H z
        if j == 1:  # steps 5-6
            p = z.copy()
            beta = 0.0
        else:  # steps 8-9
            beta = rho / rho_prev
            p = z + beta * p
        t = A(p)  # step 11
        alpha = rho / np.vdot(p, t).real  # step 12
        x = x + alpha * p  # step 13
        r = r - alpha * t  # step 14
        alphas.append(alpha)
        betas.append(beta)
    true_rel = _norm(b - A(x)) / bnorm
    return dict(x=x, iters=j, res=np.array(res), alphas=np.array(alphas), betas=np.array(betas),
                true_rel_res=true_rel)


def lanczos_tridiagonal(alphas, betas, j: int) -> np.ndarray:
    """T_j of Eq. 4 from the CG scalars, with the off-diagonal sign of step 11.10.

    T[k,k] = 1/alpha_{k+1} + beta_{k+1}/alpha_k (beta_1/alpha_0 := 0),
    T[k,k+1] = T[k+1,k] = -sqrt(beta_{k+2})/alpha_{k+1}   (0-based k)."""
    T = np.zeros((j, j))
    for k in range(j):
        T[k, k] = 1.0 / alphas[k] + (betas[k] / alphas[k - 1] if k > 0 else 0.0)
        if k + 1 < j:
            T[k, k + 1] = T[k + 1, k] = -np.sqrt(betas[k + 1]) / alphas[k]
    return T


# ----------------------------------------------------------------------------------------
# eigCG(nev, m), Fig. 1 right box
# ----------------------------------------------------------------------------------------
def eigcg(A, b, x0=None, nev=8, m=24, tol=1e-10, max_iter=100000, on_restart=None, Pinv=None):
    """CG of Fig. 1 with the eigCG(nev, m) additions of its right box; Pinv as in cg()
    (the window then holds z / sqrt(r^H z), P-orthonormal, and T = V^H A V, Sec. 3).

    on_restart(j, V, T, ritz) -- optional observer called after each restart with
    the restarted window V (N x i), its projection T (i x i) and the Ritz values.

    Returns the CG dict of cg() plus V (N x k Ritz vectors), ritz (k values),
    restarts, window (final i), Tfinal."""
    if not (m > 2 * nev and nev >= 1):
        raise ValueError("eigCG needs m > 2*nev >= 2")
    b = np.asarray(b, dtype=np.complex128).reshape(-1)
    N = b.size
    bnorm = _norm(b)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128).reshape(-1)
    r = b - A(x) if x0 is not None else b.copy()  # step 0
    V = np.zeros((N, m), dtype=np.complex128)  # step 0.1
    T = np.zeros((m, m), dtype=np.complex128)
    i = 0
    j = 0
    rho = None
    res, alphas, betas = [], [], []
    p = t = t_prev = None
    restarts = 0
    while True:
        rr = np.vdot(r, r).real
        res.append(np.sqrt(rr) / bnorm)
        if np.sqrt(rr) <= tol * bnorm or j >= max_iter:  # step 1
            break
        j += 1  # step 2
        z = r if Pinv is None else np.asarray(Pinv(r), dtype=np.complex128)  # step 3
        rho_prev, rho = rho, (rr if Pinv is None else np.vdot(r, z).real)  # step 4
        if j == 1:  # steps 5-6
            p = z.copy()
            beta = 0.0
        else:  # steps 8-9
            beta = rho / rho_prev
            p = z + beta * p
        if i == m:  # step 10.1
            t_prev = t
        t = A(p)  # step 11
        if j > 1:  # step 11.1: diagonal of the column holding z_{j-1}
            T[i - 1, i - 1] = 1.0 / alphas[-1] + (betas[-1] / alphas[-2] if j > 2 else 0.0)
        if i == m:  # step 11.2
            _, Y = _lowest_eigpairs(T[:m, :m], nev)  # step 11.3
            _, Yb = _lowest_eigpairs(T[:m - 1, :m - 1], nev)
            Yb = np.vstack([Yb, np.zeros((1, nev))])  # step 11.4
            Q = _orth(np.hstack([Y, Yb]), m)  # step 11.5
            H = np.conj(Q.T) @ T[:m, :m] @ Q
            Mv, Z = np.linalg.eigh(H)  # step 11.6
            V[:, :Q.shape[1]] = V[:, :m] @ (Q @ Z)  # step 11.7
            i = Q.shape[1]
            V[:, i:] = 0.0
            T[:, :] = 0.0
            T[:i, :i] = np.diag(Mv)
            w = t - beta * t_prev  # step 11.8
            row = (np.conj(w) @ V[:, :i]) / np.sqrt(rho)  # T_{i+1,1:i} = w^H V / sqrt(rho)
            T[i, :i] = row
            T[:i, i] = np.conj(row)
            restarts += 1
            if on_restart is not None:
                on_restart(j, V[:, :i].copy(), T[:i, :i].copy(), Mv.copy())
        elif i > 0:  # step 11.10
            T[i, i - 1] = T[i - 1, i] = -np.sqrt(beta) / alphas[-1]
        i += 1  # step 11.12
        V[:, i - 1] = z / np.sqrt(rho)  # step 11.13
        alpha = rho / np.vdot(p, t).real  # step 12
        x = x + alpha * p  # step 13
        r = r - alpha * t  # step 14
        alphas.append(alpha)
        betas.append(beta)
    # Output (reading of "[x, V, M] = eigCG(...)"): diagonal of the last column, then
    # the nev lowest Ritz pairs of the final window.
    if i > 0:
        T[i - 1, i - 1] = 1.0 / alphas[-1] + (betas[-1] / alphas[-2] if j > 1 else 0.0)
        k = min(nev, i)
        ritz, Y = _lowest_eigpairs(T[:i, :i], k)
        Vout = V[:, :i] @ Y
    else:
        ritz = np.zeros(0)
        Vout = np.zeros((N, 0), dtype=np.complex128)
    true_rel = _norm(b - A(x)) / bnorm
    return dict(x=x, iters=j, res=np.array(res), alphas=np.array(alphas), betas=np.array(betas),
                true_rel_res=true_rel, V=Vout, ritz=ritz, restarts=restarts, window=i,
                Tfinal=T[:i, :i].copy())


# ----------------------------------------------------------------------------------------
# Unrestarted Lanczos (comparison for eigCG, Sec. 3.1 / Fig. 2)
# ----------------------------------------------------------------------------------------
def lanczos_ritz_from_cg(alphas, betas, steps):
    """Ritz values of the full-history T_j (Eq. 4) built from CG scalars, for each j in steps."""
    return {j: np.linalg.eigvalsh(lanczos_tridiagonal(alphas, betas, j)) for j in steps}


def lanczos_full_reorth(A, v1, steps: int):
    """Unrestarted Lanczos with full re-orthogonalisation from v1.

    Returns (Vl N x k, T k x k) with k <= steps (stops early on breakdown)."""
    v = np.asarray(v1, dtype=np.complex128).reshape(-1)
    v = v / _norm(v)
    N = v.size
    Vl = np.zeros((N, steps), dtype=np.complex128)
    T = np.zeros((steps, steps))
    Vl[:, 0] = v
    beta_prev = 0.0
    k = steps
    for j in range(steps):
        w = A(Vl[:, j])
        a = np.vdot(Vl[:, j], w).real
        T[j, j] = a
        w = w - a * Vl[:, j] - (beta_prev * Vl[:, j - 1] if j > 0 else 0.0)
        for _ in range(2):  # full re-orthogonalisation, twice
            w = w - Vl[:, :j + 1] @ (np.conj(Vl[:, :j + 1].T) @ w)
        bta = _norm(w)
        if j + 1 == steps:
            break
        if bta == 0.0:
            k = j + 1
            break
        T[j, j + 1] = T[j + 1, j] = bta
        Vl[:, j + 1] = w / bta
        beta_prev = bta
    return Vl[:, :k], T[:k, :k]


# ----------------------------------------------------------------------------------------
# init-CG, Eq. 1, and its restart (Sec. 5.3)
# ----------------------------------------------------------------------------------------
def deflated_guess(A, U, H, b, x_tilde=None):
    """Eq. 1: x0 = x~0 + U (U^H A U)^{-1} U^H (b - A x~0), with H = U^H A U given."""
    b = np.asarray(b, dtype=np.complex128).reshape(-1)
    if x_tilde is None:
        x_tilde = np.zeros_like(b)
        r = b
    else:
        x_tilde = np.asarray(x_tilde, dtype=np.complex128).reshape(-1)
        r = b - A(x_tilde)
    if U.shape[1] == 0:
        return x_tilde.copy()
    c = np.conj(U.T) @ r
    y = np.linalg.solve(H, c)
    return x_tilde + U @ y


def initcg(A, U, H, b, x_tilde=None, tol=1e-8, restart_tol=0.0, max_iter=100000):
    """init-CG: Eq. 1 then CG (Fig. 1, P = I); one re-deflation and restart when the
    residual first reaches restart_tol (Sec. 5.3; restart_tol <= tol disables it)."""
    b = np.asarray(b, dtype=np.complex128).reshape(-1)
    bnorm = _norm(b)
    x0 = deflated_guess(A, U, H, b, x_tilde)
    if restart_tol > tol:
        first = cg(A, b, x0, tol=restart_tol, max_iter=max_iter)
        iters1 = first["iters"]
        x1 = deflated_guess(A, U, H, b, first["x"])
        second = cg(A, b, x1, tol=tol, max_iter=max(0, max_iter - iters1))
        out = dict(second)
        out["iters"] = iters1 + second["iters"]
        out["restarted"] = True
        out["iters_before_restart"] = iters1
    else:
        out = cg(A, b, x0, tol=tol, max_iter=max_iter)
        out["restarted"] = False
    out["x0"] = x0
    out["true_rel_res"] = _norm(b - A(out["x"])) / bnorm
    return out


# ----------------------------------------------------------------------------------------
# Incremental eigCG, Sec. 4 box
# ----------------------------------------------------------------------------------------
def orthonormalize_against(V, U, drop_tol=1e-10):
    """V-bar: V minus its U components (classical Gram-Schmidt twice), then an
    orthonormal basis of the remainder (Householder QR), dropping columns whose
    remainder norm (relative to the column's norm) is below drop_tol."""
    Vb = np.array(V, dtype=np.complex128)
    norms0 = np.linalg.norm(Vb, axis=0)
    for _ in range(2):
        if U.shape[1] > 0:
            Vb = Vb - U @ (np.conj(U.T) @ Vb)
    keep = np.linalg.norm(Vb, axis=0) > drop_tol * np.maximum(norms0, 1e-300)
    Vb = Vb[:, keep]
    if Vb.shape[1] == 0:
        return Vb
    Q, R = np.linalg.qr(Vb)
    good = np.abs(np.diag(R)) > drop_tol
    return Q[:, good]


def basis_grow(A, U, H, Vnew, drop_tol=1e-10):
    """Sec. 4 box, last three lines: V-bar, W = A V-bar, H extended, U augmented."""
    Vb = orthonormalize_against(Vnew, U, drop_tol)
    if Vb.shape[1] == 0:
        return U, H
    W = np.stack([A(Vb[:, c]) for c in range(Vb.shape[1])], axis=1)
    UW = np.conj(U.T) @ W
    VW = np.conj(Vb.T) @ W
    l, k = U.shape[1], Vb.shape[1]
    Hn = np.zeros((l + k, l + k), dtype=np.complex128)
    Hn[:l, :l] = H
    Hn[:l, l:] = UW
    Hn[l:, :l] = np.conj(UW.T)
    Hn[l:, l:] = VW
    return np.hstack([U, Vb]), Hn


def incremental_eigcg(A, bs, nev=10, m=100, tol=1e-8, max_iter=100000, drop_tol=1e-10, U=None, H=None):
    """Sec. 4 box: for each b_i, x0 = U H^{-1} U^H b_i, eigCG, orthonormalise, extend H, augment U.

    Returns (U, H, per-RHS results)."""
    N = np.asarray(bs[0]).size
    if U is None:
        U = np.zeros((N, 0), dtype=np.complex128)
        H = np.zeros((0, 0), dtype=np.complex128)
    results = []
    for b in bs:
        x0 = deflated_guess(A, U, H, b) if U.shape[1] > 0 else None
        res = eigcg(A, b, x0, nev=nev, m=m, tol=tol, max_iter=max_iter)
        U, H = basis_grow(A, U, H, res["V"], drop_tol)
        res["basis_size"] = U.shape[1]
        results.append(res)
    return U, H, results


def basis_ritz(A, U, H):
    """Rayleigh-Ritz on U (Sec. 5.2): eigenpairs of H, residual norms ||A u - theta u||."""
    theta, S = np.linalg.eigh(H)
    X = U @ S
    res = np.array([_norm(A(X[:, c]) - theta[c] * X[:, c]) for c in range(X.shape[1])])
    return theta, res, X


# ----------------------------------------------------------------------------------------
# Spectral preconditioner from the deflation basis (Sec. 2, "using U as a spectral
# preconditioner"; Sec. 4 and 5.2 suggest it for eigCG near the critical mass)
# ----------------------------------------------------------------------------------------
def spectral_preconditioner(U, H, shift):
    """P^{-1} = (I - U U^H) + shift * U H^{-1} U^H for an orthonormal U with H = U^H A U.

    HPD for shift > 0.  When U spans an invariant subspace of A, P^{-1} A keeps the
    eigenpairs of A outside span(U) and maps the ones inside to the value shift, so the
    lowest part of the spectrum, the part U has captured, stops slowing CG down.
    Returns the callable r -> P^{-1} r."""
    U = np.asarray(U, dtype=np.complex128)
    H = np.asarray(H, dtype=np.complex128)

    def apply(r):
        c = np.conj(U.T) @ r
        return r - U @ c + shift * (U @ np.linalg.solve(H, c))

    return apply


# ----------------------------------------------------------------------------------------
# BiCGSTAB on M, deflated with eigenvectors of A = M^H M = (g5 M)^2 (Sec. 1: the
# eigenvectors CG computes for A are eigenvectors of the Hermitian g5 M, so they can
# deflate BiCGSTAB for the remaining right-hand sides)
# ----------------------------------------------------------------------------------------
def bicgstab(M, b, x0=None, tol=1e-8, max_iter=100000):
    """BiCGSTAB (van der Vorst, SIAM J. Sci. Stat. Comput. 13, 631 (1992)) on M x = b for a
    callable M, shadow residual r_hat = r_0, stopped on the recursive ||r|| <= tol ||b||.

    Returns dict(x, iters, res (||r||/||b|| per iteration), true_rel_res)."""
    b = np.asarray(b, dtype=np.complex128).reshape(-1)
    bnorm = _norm(b)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128).reshape(-1)
    r = b - M(x) if x0 is not None else b.copy()
    r_hat = r.copy()
    rho = alpha = omega = 1.0 + 0.0j
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    res = [_norm(r) / bnorm]
    j = 0
    while res[-1] > tol and j < max_iter:
        j += 1
        rho_new = np.vdot(r_hat, r)
        beta = (rho_new / rho) * (alpha / omega)
        rho = rho_new
        p = r + beta * (p - omega * v)
        v = M(p)
        alpha = rho / np.vdot(r_hat, v)
        s = r - alpha * v
        if _norm(s) <= tol * bnorm:  # converged at the half step
            x = x + alpha * p
            r = s
            res.append(_norm(r) / bnorm)
            break
        t = M(s)
        omega = np.vdot(t, s) / np.vdot(t, t)
        x = x + alpha * p + omega * s
        r = s - omega * t
        res.append(_norm(r) / bnorm)
    return dict(x=x, iters=j, res=np.array(res), true_rel_res=_norm(b - M(x)) / bnorm)


def gamma5(psi, g5):
    """g5 applied to every site of a [V][4][3] spinor (g5: the 4 x 4 spin matrix)."""
    v = np.asarray(psi, dtype=np.complex128).reshape(-1, 4, 3)
    return np.einsum("ab,vbc->vac", g5, v).reshape(-1)


def deflated_guess_g5(M, U, b, g5, x_tilde=None):
    """Galerkin projection of the Hermitian indefinite system g5 M x = g5 b onto span(U):
    x0 = x~0 + U (U^H g5 M U)^{-1} U^H g5 (b - M x~0), the Eq. 1 construction with g5 M in
    place of A.  Returns (x0, H5 = U^H g5 M U)."""
    b = np.asarray(b, dtype=np.complex128).reshape(-1)
    x_tilde = np.zeros_like(b) if x_tilde is None else np.asarray(x_tilde, dtype=np.complex128).reshape(-1)
    r = b - M(x_tilde)
    W = np.stack([gamma5(M(U[:, c]), g5) for c in range(U.shape[1])], axis=1)
    H5 = np.conj(U.T) @ W
    y = np.linalg.solve(H5, np.conj(U.T) @ gamma5(r, g5))
    return x_tilde + U @ y, H5
