"""Tensor-core (tcgen05) U^H r of the Eq. 1 deflation against the CUDA-core kernel
and the oracle.

The FP32 contractions run on the tensor cores unless EIG_GEMM_TC=0 (then on CUDA
cores); U^H r of eig_basis_deflate goes through the tcgen05 kernel (TF32 hi/lo split, three products per K step, TMEM accumulators
drained every two K tiles into double-float sums, FP64 sum over CTAs).  On 8^4
each CTA runs 21 K tiles, so the pipeline wraps and several drains happen.  Its result agrees with FP32 arithmetic:
the deflated guess x0 = U H^{-1} U^H b matches the oracle's FP64 evaluation on
the same (FP32-stored) basis to 1e-5 relative -- the FP32 rounding of r and of the
products (~1e-7) amplified by cond(H) (at most ~1e2 for these bases) -- and the
CUDA-core kernel's x0 to the same bar.  Bases of l <= 128 and l > 128 cover one
and two 128-row M tiles; k = 1, 5 and 16 RHS cover N = 16 and N = 32 columns.
"""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import solvers
from paper_0707_0131_gb300 import fixtures as fx

pytestmark = pytest.mark.gpu

MASSES = json.load(open(os.path.join(os.path.dirname(__file__), "..", "configs", "masses.json")))


@pytest.fixture(scope="module")
def grown():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_0707_0131_gb300 import api

    dims = fx.LATTICES["8^4"]
    m_q = MASSES["8^4"]["1e+03"]["m_q"]
    gauge = fx.make_gauge(dims, fx.GAUGE_SEEDS["8^4"])
    W = oracle.Wilson(dims, m_q, gauge)
    op = api.Op(gauge, dims, m_q, prec=32, max_rhs=16)
    basis = api.Basis(op, 160)
    sizes = []
    r = 0
    while basis.size < 140 and r < 40:
        b = fx.make_rhs(dims, 5000 + r)[0].reshape(-1)
        x = np.zeros_like(b)
        op.eigcg_solve(b, x, nev=10, m=30, tol=1e-6, basis=basis)
        basis.grow()
        sizes.append(basis.size)
        r += 1
    yield dims, W, op, basis, sizes
    os.environ.pop("EIG_GEMM_TC", None)
    basis.close()
    op.close()


def _deflate(basis, B, k, tc):
    os.environ["EIG_GEMM_TC"] = "1" if tc else "0"
    X0 = np.zeros_like(B)
    basis.deflate(B, None, X0, k=k)
    return X0


def test_tc_deflation_matches(grown):
    dims, W, op, basis, sizes = grown
    assert basis.size >= 137, sizes
    for l in (137, 40):  # two M tiles, then one (truncation keeps the leading vectors)
        basis.truncate(l)
        U, H = basis.vectors(), basis.H()
        for k in (1, 4, 16):
            B = fx.make_rhs(dims, 6000 + k, k).reshape(k, -1)
            x_tc = _deflate(basis, B, k, True)
            x_cc = _deflate(basis, B, k, False)
            for r in range(k):
                ref = solvers.deflated_guess(W, U, H, B[r])
                e_tc = np.linalg.norm(x_tc[r] - ref) / np.linalg.norm(ref)
                e_cc = np.linalg.norm(x_cc[r] - ref) / np.linalg.norm(ref)
                assert e_tc < 1e-5, (l, k, r, e_tc, e_cc)
                assert e_cc < 1e-5, (l, k, r, e_tc, e_cc)
                assert np.linalg.norm(x_tc[r] - x_cc[r]) / np.linalg.norm(ref) < 1e-5


def test_tc_deflation_twice_same_result(grown):
    """Deterministic: the FP64 sum over chunks runs in a fixed order."""
    dims, W, op, basis, sizes = grown
    B = fx.make_rhs(dims, 6100, 4).reshape(4, -1)
    a = _deflate(basis, B, 4, True)
    b = _deflate(basis, B, 4, True)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("tc", [True, False])
def test_basis_growth_with_tc(tc):
    """Incremental eigCG with every A^H B of the growth step (Gram-Schmidt against U,
    Gram matrices, U^H W) on the tensor cores: U stays orthonormal to FP32 accuracy and
    H matches U^H A U from the oracle, as with the CUDA-core kernel."""
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_0707_0131_gb300 import api

    os.environ["EIG_GEMM_TC"] = "1" if tc else "0"
    try:
        dims = fx.LATTICES["8^4"]
        m_q = MASSES["8^4"]["1e+03"]["m_q"]
        gauge = fx.make_gauge(dims, fx.GAUGE_SEEDS["8^4"])
        W = oracle.Wilson(dims, m_q, gauge)
        op = api.Op(gauge, dims, m_q, prec=32)
        basis = api.Basis(op, 64)
        for r in range(5):
            b = fx.make_rhs(dims, 5200 + r)[0].reshape(-1)
            x = np.zeros_like(b)
            op.eigcg_solve(b, x, nev=10, m=30, tol=1e-6, basis=basis)
            basis.grow()
        U, H = basis.vectors(), basis.H()
        l = U.shape[1]
        assert l >= 40
        assert np.max(np.abs(U.conj().T @ U - np.eye(l))) < 1e-5
        AU = np.stack([W.A(U[:, j]) for j in range(l)], axis=1)
        Href = U.conj().T @ AU
        assert np.linalg.norm(H - Href) / np.linalg.norm(Href) < 1e-5
        basis.close()
        op.close()
    finally:
        os.environ.pop("EIG_GEMM_TC", None)


def test_tc_accuracy_at_scale():
    """16^3x32 (1.57M complex rows, 96 K tiles per CTA): the tensor-core deflation stays
    within 2e-6 of the FP64 evaluation on the same basis, as the CUDA-core kernel
    does (an undrained FP32 accumulator over the whole CTA range lost ~1e-5)."""
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_0707_0131_gb300 import api

    dims = fx.LATTICES["16^3x32"]
    m_q = MASSES["16^3x32"]["1e+03"]["m_q"]
    gauge = fx.make_gauge(dims, fx.GAUGE_SEEDS["16^3x32"])
    op = api.Op(gauge, dims, m_q, prec=32, max_rhs=4)
    basis = api.Basis(op, 40)
    try:
        os.environ["EIG_GEMM_TC"] = "0"
        for r in range(2):
            b = fx.make_rhs(dims, 5300 + r)[0].reshape(-1)
            x = np.zeros_like(b)
            op.eigcg_solve(b, x, nev=10, m=40, tol=1e-6, basis=basis)
            basis.grow()
        U, H = basis.vectors(), basis.H()
        B = fx.make_rhs(dims, 5400, 4).reshape(4, -1)
        ref = U @ np.linalg.solve(H, U.conj().T @ B.T)
        for tc in (True, False):
            X = _deflate(basis, B, 4, tc)
            for q in range(4):
                err = np.linalg.norm(X[q] - ref[:, q]) / np.linalg.norm(ref[:, q])
                assert err < 2e-6, (tc, q, err)
    finally:
        os.environ.pop("EIG_GEMM_TC", None)
        basis.close()
        op.close()


def test_eigcg_restart_on_tensor_cores():
    """eigCG(10, 40) on 8^4: the window restart V <- V QZ (in place, tensor cores) and
    w^H V_new give the same run as the CUDA-core restart kernel: iteration counts within
    2, the lowest 5 pending Ritz values within 1e-5 relative (FP32 window arithmetic) and
    all 10 within 1e-4, both solutions at tol."""
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_0707_0131_gb300 import api

    dims = fx.LATTICES["8^4"]
    m_q = MASSES["8^4"]["1e+04"]["m_q"]
    gauge = fx.make_gauge(dims, fx.GAUGE_SEEDS["8^4"])
    W = oracle.Wilson(dims, m_q, gauge)
    b = fx.make_rhs(dims, 5500)[0].reshape(-1)
    runs = {}
    try:
        for tc in (True, False):
            os.environ["EIG_GEMM_TC"] = "1" if tc else "0"
            op = api.Op(gauge, dims, m_q, prec=32)
            basis = api.Basis(op, 16)
            x = np.zeros_like(b)
            st = op.eigcg_solve(b, x, nev=10, m=40, tol=1e-8, basis=basis)
            basis.grow()
            ev, _ = basis.ritz(residuals=False)
            runs[tc] = (st, np.sort(ev), x)
            assert st["restarts"] >= 3
            assert np.linalg.norm(b - W.A(x)) / np.linalg.norm(b) <= 1e-8
            basis.close()
            op.close()
    finally:
        os.environ.pop("EIG_GEMM_TC", None)
    (s1, e1, _), (s0, e0, _) = runs[True], runs[False]
    assert abs(s1["iters"] - s0["iters"]) <= 2, (s1["iters"], s0["iters"])
    # both restarts run in FP32 window arithmetic: the Ritz values agree to the FP32
    # rounding of A (about eps_32 ||A|| absolute; ~1e-8 here against lambda ~ 6e-3)
    rel = np.abs(e1 - e0) / e0
    assert np.max(rel[:5]) < 1e-5 and np.max(rel) < 1e-4, (e1, e0)
