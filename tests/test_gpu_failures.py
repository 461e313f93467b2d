"""Failure paths of the C ABI, each made without faulting, trapping or hanging a GPU.

* EIG_ERR_TIMEOUT: the tensor-core kernels bound every mbarrier wait and report a
  wait that gave up through an error flag.  The test hook EIG_TEST_INJECT_WAIT=1
  makes CTA 0 of the A^H B contraction wait (at most 5 ms) on a barrier that nothing
  arrives on before it issues any copy; the call must return EIG_ERR_TIMEOUT and the
  next call on the same handles must succeed with a correct result.
* EIG_ERR_BREAKDOWN: a NaN in the right-hand side makes rho non-finite; the solve
  stops and reports it, and the op stays usable.
* EIG_ERR_OOM: the test hook EIG_TEST_ALLOC_LIMIT=<bytes> fakes a failing cudaMalloc
  for larger requests, so the out-of-memory path runs without exhausting a device.
* EIG_ERR_BUDGET: growing a basis past its max_vecs is refused and leaves the basis
  as it was.
"""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import solvers
from paper_0707_0131_gb300 import _lib
from paper_0707_0131_gb300 import fixtures as fx

pytestmark = pytest.mark.gpu

MASSES = json.load(open(os.path.join(os.path.dirname(__file__), "..", "configs", "masses.json")))


@pytest.fixture(scope="module")
def api():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_0707_0131_gb300 import api as a

    return a


@pytest.fixture(scope="module")
def lat8():
    dims = fx.LATTICES["8^4"]
    m_q = MASSES["8^4"]["1e+03"]["m_q"]
    gauge = fx.make_gauge(dims, fx.GAUGE_SEEDS["8^4"])
    return dims, m_q, gauge


class _env:
    def __init__(self, name, value):
        self.name, self.value = name, value

    def __enter__(self):
        os.environ[self.name] = self.value

    def __exit__(self, *exc):
        os.environ.pop(self.name, None)


def test_timeout_status_and_recovery(api, lat8):
    dims, m_q, gauge = lat8
    W = oracle.Wilson(dims, m_q, gauge)
    op = api.Op(gauge, dims, m_q, prec=32)
    basis = api.Basis(op, 8)
    b0 = fx.make_rhs(dims, 31)[0].reshape(-1)
    x = np.zeros_like(b0)
    op.eigcg_solve(b0, x, nev=4, m=12, tol=1e-6, basis=basis)
    basis.grow()
    assert basis.size >= 1
    b = fx.make_rhs(dims, 32)[0].reshape(-1)
    x0 = np.zeros_like(b)
    with _env("EIG_TEST_INJECT_WAIT", "1"):
        with pytest.raises(_lib.EigError) as e:
            basis.deflate(b, None, x0, k=1)
    assert e.value.status == _lib.EIG_ERR_TIMEOUT
    assert "bounded wait" in _lib.eig_last_error()
    # the same handles work afterwards, and the result satisfies the Galerkin condition
    basis.deflate(b, None, x0, k=1)
    U = basis.vectors()
    g = U.conj().T @ (b - W.A(x0))
    assert np.linalg.norm(g) < 1e-4 * np.linalg.norm(b)
    x = np.zeros_like(b)
    st = op.initcg_solve(b, x, tol=1e-8, basis=basis)[0]
    assert st["converged"] == 1
    assert np.linalg.norm(b - W.A(x)) / np.linalg.norm(b) <= 1e-8
    basis.close()
    op.close()


@pytest.mark.parametrize("prec", [64, 32])
def test_nan_rhs_reports_breakdown(api, lat8, prec):
    dims, m_q, gauge = lat8
    W = oracle.Wilson(dims, m_q, gauge)
    op = api.Op(gauge, dims, m_q, prec=prec)
    b = fx.make_rhs(dims, 33)[0].reshape(-1)
    bad = b.copy()
    bad[1234] = np.nan
    x = np.zeros_like(b)
    with pytest.raises(_lib.EigError) as e:
        op.initcg_solve(bad, x, tol=1e-8)
    assert e.value.status == _lib.EIG_ERR_BREAKDOWN
    basis = api.Basis(op, 8)
    with pytest.raises(_lib.EigError) as e:
        op.eigcg_solve(bad, np.zeros_like(b), nev=4, m=12, tol=1e-8, basis=basis)
    assert e.value.status == _lib.EIG_ERR_BREAKDOWN
    # the op is usable afterwards
    x = np.zeros_like(b)
    st = op.initcg_solve(b, x, tol=1e-8)[0]
    assert st["converged"] == 1
    o = solvers.cg(W, b, tol=1e-8)
    assert abs(st["iters"] - o["iters"]) <= max(1, 0.1 * o["iters"])
    assert np.linalg.norm(b - W.A(x)) / np.linalg.norm(b) <= 1e-8
    basis.close()
    op.close()


def test_oom_from_fake_allocator(api, lat8):
    dims, m_q, gauge = lat8
    with _env("EIG_TEST_ALLOC_LIMIT", str(1 << 20)):
        with pytest.raises(_lib.EigError) as e:
            api.Op(gauge, dims, m_q, prec=32, max_rhs=4)
    assert e.value.status == _lib.EIG_ERR_OOM
    assert "test limit" in _lib.eig_last_error()
    op = api.Op(gauge, dims, m_q, prec=32, max_rhs=4)  # nothing leaked or left behind
    with _env("EIG_TEST_ALLOC_LIMIT", str(1 << 20)):
        with pytest.raises(_lib.EigError) as e:
            api.Basis(op, 64)
    assert e.value.status == _lib.EIG_ERR_OOM
    basis = api.Basis(op, 8)
    assert basis.size == 0
    basis.close()
    op.close()


def test_basis_budget(api, lat8):
    dims, m_q, gauge = lat8
    op = api.Op(gauge, dims, m_q, prec=64)
    basis = api.Basis(op, 8)
    for r in range(2):
        b = fx.make_rhs(dims, 40 + r)[0].reshape(-1)
        op.eigcg_solve(b, np.zeros_like(b), nev=6, m=14, tol=1e-8, basis=basis)
        if r == 0:
            basis.grow()
            l1 = basis.size
            H1 = basis.H()
    assert l1 >= 6
    with pytest.raises(_lib.EigError) as e:
        basis.grow()  # l1 + 6 > 8
    assert e.value.status == _lib.EIG_ERR_BUDGET
    assert basis.size == l1
    assert np.array_equal(basis.H(), H1)
    basis.close()
    op.close()
