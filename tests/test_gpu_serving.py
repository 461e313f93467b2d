"""Serving form: continuous batching over several operators with resident bases.

* every result meets the FP64 true residual bar (recomputed by the oracle);
* each result equals the solution of the same request solved alone, within the
  tolerance implied by tol and cond(A);
* later requests of an operator are deflated by the basis grown from earlier ones
  (fewer iterations) and, once the basis is full, arrive in batches of several RHS;
* an HBM budget that fits one operator at a time still serves every request
  (idle operators are retired and re-activated).
"""
import json
import os
import time

import numpy as np
import pytest

import oracle
from paper_0707_0131_gb300 import fixtures as fx

pytestmark = pytest.mark.gpu

MASSES = json.load(open(os.path.join(os.path.dirname(__file__), "..", "configs", "masses.json")))


@pytest.fixture(scope="module")
def serving():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_0707_0131_gb300 import serving as s

    return s


def _specs(serving):
    out = []
    for name in ("4^4", "8^4"):
        dims = fx.LATTICES[name]
        out.append(serving.OpSpec(key=name, dims=dims, m_q=MASSES[name]["1e+03"]["m_q"],
                                  gauge=fx.make_gauge(dims, fx.GAUGE_SEEDS[name]), prec=32, max_rhs=4, nev=4, m=12,
                                  basis_max=12, tol=1e-8, restart_tol=1e-6))
    return out


def _check(spec, b, x, tol):
    W = oracle.Wilson(spec.dims, spec.m_q, spec.gauge)
    return np.linalg.norm(b - W.A(x)) / np.linalg.norm(b) <= tol


@pytest.mark.parametrize("budget", ["ample", "one_op"])
def test_mixed_requests(serving, budget):
    specs = _specs(serving)
    by_key = {s.key: s for s in specs}
    cap = 150e9 if budget == "ample" else max(s.footprint() for s in specs) * 1.01
    srv = serving.Server(specs, hbm_budget_bytes=cap)
    reqs = []
    rng = np.random.default_rng(0)
    for i in range(20):
        key = specs[i % 2].key
        b = fx.make_rhs(by_key[key].dims, 7000 + i)[0].reshape(-1)
        reqs.append((key, b, srv.submit(key, b)))
        time.sleep(float(rng.uniform(0, 0.01)))
    results = [(k, b, f.result(timeout=600)) for k, b, f in reqs]
    for key, b, res in results:
        assert res["stats"]["converged"] == 1
        assert _check(by_key[key], b, res["x"], 1e-8)
    # every operator's basis was grown by its first requests and then used to deflate
    for key in by_key:
        kinds = [res["kind"] for k, b, res in results if k == key]
        sizes = [res["basis_size"] for k, b, res in results if k == key]
        assert kinds[0] == "eigcg" and max(sizes) >= by_key[key].basis_max - by_key[key].nev
        assert "initcg" in kinds
    assert srv.max_used <= cap
    p = srv.percentiles()
    assert p["n"] == 20 and p["p99_ms"] >= p["p50_ms"] > 0
    srv.close()


def test_burst_forms_batches_same_as_alone(serving):
    """Once an operator's basis is full, a burst of requests that arrive while its
    first init-CG batch is on the GPU is admitted into the next batch (at least one
    batch of more than one RHS forms).  Each batched result equals the same request
    solved alone through the same deflated path (same operator, same basis, k = 1):
    iteration counts within 10%, and solutions within 10 tol cond(A), the forward error
    that two solutions to tol can differ by."""
    specs = _specs(serving)
    spec = specs[1]  # 8^4, cond(A) ~ 1e3
    srv = serving.Server([spec])
    # grow the basis with the first requests (eigCG), one at a time, until the next
    # request would go to init-CG (the worker's rule: size + nev > basis_max)
    w = srv.workers[spec.key]
    i = 0
    while w.basis is None or w.basis.size + spec.nev <= spec.basis_max:
        r = srv.submit(spec.key, fx.make_rhs(spec.dims, 9100 + i)[0].reshape(-1)).result(timeout=600)
        assert r["kind"] == "eigcg"
        i += 1
        assert i <= 8
    full = w.basis.size
    # burst: 9 requests submitted back to back
    bs = [fx.make_rhs(spec.dims, 9200 + i)[0].reshape(-1) for i in range(9)]
    fs = [srv.submit(spec.key, b) for b in bs]
    res = [f.result(timeout=600) for f in fs]
    assert all(r["kind"] == "initcg" for r in res)
    sizes = [r["batch"] for r in res]
    assert max(sizes) > 1, sizes
    assert w.basis.size == full  # init-CG leaves the basis as it is
    cond = 1e3
    for b, r in zip(bs, res):
        x = np.zeros_like(b)
        st = w.op.initcg_solve(b, x, tol=spec.tol, restart_tol=spec.restart_tol, basis=w.basis, k=1)[0]
        it_a, it_b = st["iters"], r["stats"]["iters"]
        assert abs(it_a - it_b) <= max(1, 0.1 * it_a), (it_a, it_b, r["batch"])
        assert np.linalg.norm(r["x"] - x) / np.linalg.norm(x) <= 10 * spec.tol * cond
        assert _check(spec, b, r["x"], spec.tol)
    srv.close()


def test_result_same_alone_and_in_mix(serving):
    """Requests for two operators interleaved: every result equals the solution of the
    same system solved alone without deflation, within 10 tol cond(A)."""
    from paper_0707_0131_gb300.api import Op

    specs = _specs(serving)
    srv = serving.Server(specs)
    futs = []
    for i in range(16):
        s = specs[i % 2]
        futs.append((s, fx.make_rhs(s.dims, 9000 + i)[0].reshape(-1)))
    fs = [srv.submit(s.key, b) for s, b in futs]
    res = [f.result(timeout=600) for f in fs]
    for (s, b), r in zip(futs, res):
        op = Op(s.gauge, s.dims, s.m_q, prec=32)
        x = np.zeros_like(b)
        op.initcg_solve(b, x, tol=1e-8)
        op.close()
        assert np.linalg.norm(r["x"] - x) / np.linalg.norm(x) <= 10 * 1e-8 * 1e3
    srv.close()


def test_trim_keeps_basis(serving):
    """eig_op_trim gives an operator's workspace back and keeps its basis: the next solve
    allocates the workspace again and deflates exactly as before."""
    from paper_0707_0131_gb300.api import Basis, Op

    spec = _specs(serving)[1]
    op = Op(spec.gauge, spec.dims, spec.m_q, prec=32, max_rhs=4)
    basis = Basis(op, 16)
    for i in range(2):
        b = fx.make_rhs(spec.dims, 9300 + i)[0].reshape(-1)
        op.eigcg_solve(b, np.zeros_like(b), 4, 12, 1e-8, basis=basis)
        basis.grow()
    l = basis.size
    th0, _ = basis.ritz(residuals=False)
    B = np.stack([fx.make_rhs(spec.dims, 9400 + i)[0].reshape(-1) for i in range(4)])
    X0 = np.zeros_like(B)
    st0 = op.initcg_solve(B, X0, tol=1e-8, restart_tol=1e-6, basis=basis, k=4)
    freed = op.trim()
    assert freed > 4 * 12 * fx.volume(spec.dims) * 16  # at least the FP64 staging of k = 4
    assert basis.size == l
    th1, _ = basis.ritz(residuals=False)
    assert np.array_equal(th0, th1)
    X1 = np.zeros_like(B)
    st1 = op.initcg_solve(B, X1, tol=1e-8, restart_tol=1e-6, basis=basis, k=4)
    for r in range(4):
        assert st1[r]["iters"] == st0[r]["iters"]
        assert np.linalg.norm(X1[r] - X0[r]) / np.linalg.norm(X0[r]) < 1e-6
        assert _check(spec, B[r], X1[r], 1e-8)
    basis.close()
    op.close()


def test_trim_while_another_thread_captures(serving):
    """Two operators served from two threads, each on its own stream: every round one
    thread trims its operator (device-wide sync and frees) while the other may be capturing
    the CG graph of its next solve (a trimmed operator captures its graphs again).  Trims
    and captures exclude each other inside the library, so neither call fails and every
    solve reaches its tolerance."""
    import threading

    import torch

    from paper_0707_0131_gb300.api import Op

    spec = _specs(serving)[1]
    errors, done = [], []

    def worker(seed):
        try:
            stream = torch.cuda.Stream()
            op = Op(spec.gauge, spec.dims, spec.m_q, prec=32, max_rhs=4)
            B = np.stack([fx.make_rhs(spec.dims, seed + i)[0].reshape(-1) for i in range(4)])
            for _ in range(12):
                X = np.zeros_like(B)
                sts = op.initcg_solve(B, X, tol=1e-8, k=4, stream=stream)
                assert all(_check(spec, B[r], X[r], 1e-8) for r in range(4)), [s_["iters"] for s_ in sts]
                op.trim()
            op.close()
            done.append(seed)
        except Exception as e:  # reported below; the other thread keeps going
            errors.append(repr(e))

    threads = [threading.Thread(target=worker, args=(9500 + 100 * i,)) for i in range(2)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=600)
    assert not errors, errors
    assert len(done) == 2
