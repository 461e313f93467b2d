"""Basis files (eig_basis_save / eig_basis_load) on the GPU.

* round trip: a basis grown by Incremental eigCG (FP32 and FP64 ops, full and odd-even
  forms), saved and loaded into a fresh op on the same links, has bit-identical vectors
  and H, and deflates a new right-hand side (Eq. 1) to the same initial guess;
* precision: an FP32 file loads exactly into an FP64 op, and an FP64 file holding
  FP32-representable values loads exactly into an FP32 op;
* refusals: other links, quark mass or form -> EIG_ERR_ARG with the basis unchanged;
  more vectors than max_vecs -> EIG_ERR_BUDGET; a missing or truncated file ->
  EIG_ERR_IO (a truncated one leaves the basis empty).
"""
import os

import numpy as np
import pytest

from paper_0707_0131_gb300 import fixtures as fx

pytestmark = pytest.mark.gpu

DIMS = (8, 8, 8, 8)
M_Q = -0.05


@pytest.fixture(scope="module")
def api():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_0707_0131_gb300 import api as a

    return a


def _grown(api, prec, eo, gauge, nvec=2):
    op = api.Op(gauge, DIMS, M_Q, prec=prec, even_odd=eo)
    basis = api.Basis(op, 32)
    n = op.V * 12
    for r in range(nvec):
        b = fx.make_rhs(DIMS, 200 + r).reshape(-1)[:n]
        x = np.zeros_like(b)
        op.eigcg_solve(b, x, nev=6, m=20, tol=1e-8, basis=basis)
        basis.grow()
    return op, basis


def _deflated(op, basis, seed):
    n = op.Vf * 12
    b = np.random.default_rng(seed).standard_normal(2 * n).view(np.complex128)
    x0 = np.zeros_like(b)
    basis.deflate(b, np.zeros_like(b), x0)
    return x0


@pytest.mark.parametrize("prec,eo", [(32, False), (64, False), (32, True)])
def test_round_trip(api, tmp_path, prec, eo):
    gauge = fx.make_gauge(DIMS, 201)
    op, basis = _grown(api, prec, eo, gauge)
    path = str(tmp_path / "u.basis")
    basis.save(path)
    l = basis.size
    assert l == 12
    nbytes = 64 + l * l * 16 + l * op.Vf * 12 * 2 * (4 if prec == 32 else 8)
    assert os.path.getsize(path) == nbytes
    op2 = api.Op(gauge, DIMS, M_Q, prec=prec, even_odd=eo)
    b2 = api.Basis(op2, 16)
    b2.load(path)
    assert b2.size == l
    assert np.array_equal(b2.H(), basis.H())
    for j in range(l):
        assert np.array_equal(b2.vector(j), basis.vector(j)), j
    x_a, x_b = _deflated(op, basis, 5), _deflated(op2, b2, 5)
    assert np.linalg.norm(x_a - x_b) <= 1e-13 * np.linalg.norm(x_a)
    # the loaded basis keeps growing
    b = fx.make_rhs(DIMS, 210).reshape(-1)[: op2.V * 12]
    x = np.zeros_like(b)
    op2.eigcg_solve(b, x, nev=2, m=20, tol=1e-8, basis=b2)
    b2.grow()
    assert b2.size == l + 2
    for h in (b2, basis):
        h.close()
    op.close()
    op2.close()


def test_precision_conversion(api, tmp_path):
    gauge = fx.make_gauge(DIMS, 202)
    op32, bas32 = _grown(api, 32, False, gauge)
    p32 = str(tmp_path / "f32.basis")
    bas32.save(p32)
    op64 = api.Op(gauge, DIMS, M_Q, prec=64)
    b64 = api.Basis(op64, 32)
    b64.load(p32)
    for j in range(bas32.size):
        assert np.array_equal(b64.vector(j), bas32.vector(j)), j
    p64 = str(tmp_path / "f64.basis")
    b64.save(p64)
    fresh = api.Basis(op32, 32)
    fresh.load(p64)
    for j in range(bas32.size):
        assert np.array_equal(fresh.vector(j), bas32.vector(j)), j  # FP32 -> FP64 -> FP32
    for h in (bas32, b64, fresh):
        h.close()
    op32.close()
    op64.close()


def test_refusals(api, tmp_path):
    from paper_0707_0131_gb300._lib import EIG_ERR_ARG, EIG_ERR_BUDGET, EIG_ERR_IO, EigError

    gauge = fx.make_gauge(DIMS, 203)
    op, basis = _grown(api, 32, False, gauge)
    path = str(tmp_path / "u.basis")
    basis.save(path)
    l = basis.size

    def refused(target, status, p=path):
        with pytest.raises(EigError) as e:
            target.load(p)
        assert e.value.status == status, e.value

    others = [api.Op(fx.make_gauge(DIMS, 204), DIMS, M_Q, prec=32),  # links
              api.Op(gauge, DIMS, M_Q + 1e-12, prec=32),               # quark mass
              api.Op(gauge, DIMS, M_Q, prec=32, even_odd=True)]        # form
    for o in others:
        t = api.Basis(o, 32)
        refused(t, EIG_ERR_ARG)
        assert t.size == 0
        t.close()
        o.close()
    small = api.Basis(op, l - 1)
    refused(small, EIG_ERR_BUDGET)
    small.close()
    refused(basis, EIG_ERR_IO, str(tmp_path / "missing.basis"))
    assert basis.size == l
    cut = str(tmp_path / "cut.basis")
    with open(path, "rb") as f, open(cut, "wb") as g:
        g.write(f.read()[: os.path.getsize(path) - 100])
    refused(basis, EIG_ERR_IO, cut)
    assert basis.size == 0
    basis.close()
    op.close()
