"""Pins of the oracle's Wilson operator against facts the paper and the mathematics fix.

Sec. 1 fixes M = m_q I - D, gamma5 M = M^H gamma5 with gamma5 = diag(+-1), and CG
on A = M^H M.  The rest of the operator is the standard Wilson convention written
out in oracle/wilson.c; these tests pin it with closed forms and invariants:
  * gamma algebra: Hermitian, {g_mu, g_nu} = 2 delta, g1 g2 g3 g4 = diag(1,1,-1,-1);
  * free field (all U = 1): plane waves e^{ipx} chi are mapped to
    [m + sum(1 - cos p) + i sum g_mu sin p_mu] chi e^{ipx}, so the spectrum of A is
    (m + sum(1 - cos p))^2 + sum sin^2 p, each value 12-fold per momentum;
  * gamma5-Hermiticity of the dense M, Hermiticity and positivity of A;
  * gauge covariance, which catches direction, sign and adjoint mistakes that the
    free field cannot see.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_0707_0131_gb300 import fixtures as fx


def _rand_spinor(rng, V):
    return (rng.standard_normal((V, 4, 3)) + 1j * rng.standard_normal((V, 4, 3))).astype(np.complex128)


def test_gamma_algebra():
    g = oracle.gammas()
    eye = np.eye(4)
    for mu in range(4):
        assert np.allclose(g[mu], g[mu].conj().T, atol=0)
        for nu in range(4):
            ac = g[mu] @ g[nu] + g[nu] @ g[mu]
            assert np.allclose(ac, 2.0 * eye * (mu == nu), atol=0)
    g5 = g[0] @ g[1] @ g[2] @ g[3]
    assert np.allclose(g[4], g5, atol=0)
    assert np.allclose(g5, np.diag([1, 1, -1, -1]), atol=0)


def test_gauge_fixture_is_su3():
    U = fx.make_gauge((4, 4, 4, 4), 101).reshape(-1, 3, 3)
    UUh = U @ np.conj(np.swapaxes(U, -1, -2))
    assert np.max(np.abs(UUh - np.eye(3))) < 1e-14
    assert np.max(np.abs(np.linalg.det(U) - 1.0)) < 1e-14
    # the field is not trivial: links are spread around the identity
    assert 0.05 < np.mean(np.abs(U - np.eye(3))) < 1.0


def _free_field_levels(dims, m):
    ps = [2 * np.pi * np.arange(L) / L for L in dims]
    lam = []
    for p in itertools.product(*ps):
        p = np.array(p)
        lam.append((m + np.sum(1 - np.cos(p))) ** 2 + np.sum(np.sin(p) ** 2))
    return np.array(lam)


@pytest.mark.parametrize("m", [0.1, -0.3])
def test_free_field_spectrum_4x4(m):
    dims = (4, 4, 4, 4)
    W = oracle.Wilson(dims, m, fx.unit_gauge(dims))
    ev = np.linalg.eigvalsh(W.dense("A"))
    expect = np.sort(np.repeat(_free_field_levels(dims, m), 12))
    assert np.max(np.abs(ev - expect)) < 1e-12 * expect.max()


def test_free_field_plane_waves():
    dims = (4, 6, 2, 8)  # anisotropic: catches axis mix-ups
    m = 0.137
    W = oracle.Wilson(dims, m, fx.unit_gauge(dims))
    g = oracle.gammas()
    rng = np.random.default_rng(5)
    coords = np.stack(np.meshgrid(*[np.arange(L) for L in dims[::-1]], indexing="ij"), -1)
    coords = coords.reshape(-1, 4)[:, ::-1]  # (x, y, z, t) in site order
    for _ in range(6):
        n = [rng.integers(0, L) for L in dims]
        p = np.array([2 * np.pi * n[k] / dims[k] for k in range(4)])
        chi = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        phase = np.exp(1j * coords @ p)
        psi = phase[:, None, None] * chi[None]
        Mp = (m + np.sum(1 - np.cos(p))) * np.eye(4) + 1j * sum(g[mu] * np.sin(p[mu]) for mu in range(4))
        expect = phase[:, None, None] * (Mp @ chi)[None]
        got = W.M(psi).reshape(-1, 4, 3)
        assert np.max(np.abs(got - expect)) < 1e-13 * np.max(np.abs(expect))


def test_gamma5_hermiticity_dense():
    dims = (4, 4, 4, 4)
    W = oracle.Wilson(dims, 0.05, fx.make_gauge(dims, 101))
    M = W.dense("M")
    G5 = np.kron(np.eye(W.V), np.kron(np.diag([1.0, 1.0, -1.0, -1.0]), np.eye(3)))
    assert np.max(np.abs(G5 @ M @ G5 - M.conj().T)) < 1e-14
    # and M itself is not Hermitian: the test is not vacuous
    assert np.max(np.abs(M - M.conj().T)) > 0.1


def test_A_hermitian_positive_and_normal_form():
    dims = (4, 4, 4, 4)
    W = oracle.Wilson(dims, -0.1, fx.make_gauge(dims, 101))
    A = W.dense("A")
    M = W.dense("M")
    assert np.max(np.abs(A - A.conj().T)) < 1e-13 * np.max(np.abs(A))
    assert np.max(np.abs(A - M.conj().T @ M)) < 1e-13 * np.max(np.abs(A))
    assert np.linalg.eigvalsh(A)[0] > 0


def test_mdag_is_adjoint_8x4():
    dims = (8, 8, 8, 8)
    W = oracle.Wilson(dims, 0.02, fx.make_gauge(dims, 102))
    rng = np.random.default_rng(7)
    phi, psi = _rand_spinor(rng, W.V), _rand_spinor(rng, W.V)
    lhs = np.vdot(phi, W.M(psi))
    rhs = np.vdot(W.Mdag(phi), psi)
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)
    a1 = np.vdot(phi, W.A(psi))
    a2 = np.conj(np.vdot(psi, W.A(phi)))
    assert abs(a1 - a2) < 1e-13 * abs(a1)
    assert np.vdot(psi, W.A(psi)).real > 0


def test_gauge_covariance():
    dims = (4, 2, 6, 4)
    V = fx.volume(dims)
    U = fx.make_gauge(dims, 11)
    g = fx.random_gauge_transform(dims, 12)
    # U'_mu(x) = g(x) U_mu(x) g(x+mu)^H
    Up = np.empty_like(U)
    idx = np.arange(V).reshape(dims[::-1])  # [t][z][y][x]
    for mu in range(4):
        axis = 3 - mu
        fwd = np.roll(idx, -1, axis=axis).reshape(-1)
        Up[:, mu] = g @ U[:, mu] @ np.conj(np.swapaxes(g[fwd], -1, -2))
    rng = np.random.default_rng(3)
    psi = _rand_spinor(rng, V)
    psip = np.einsum("sab,sxb->sxa", g, psi)
    m = 0.07
    out = oracle.Wilson(dims, m, U).M(psi).reshape(V, 4, 3)
    outp = oracle.Wilson(dims, m, Up).M(psip).reshape(V, 4, 3)
    assert np.max(np.abs(outp - np.einsum("sab,sxb->sxa", g, out))) < 1e-13 * np.max(np.abs(out))
    # a wrong transform (g(x-mu) instead of g(x+mu)) must break it: the test has teeth
    Ubad = np.empty_like(U)
    for mu in range(4):
        bwd = np.roll(idx, 1, axis=3 - mu).reshape(-1)
        Ubad[:, mu] = g @ U[:, mu] @ np.conj(np.swapaxes(g[bwd], -1, -2))
    outb = oracle.Wilson(dims, m, Ubad).M(psip).reshape(V, 4, 3)
    assert np.max(np.abs(outb - np.einsum("sab,sxb->sxa", g, out))) > 1e-3
