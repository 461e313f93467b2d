"""The serving loop end to end on the host (no GPU): the real Server and worker threads,
admission under the HBM budget, workspace trims and continuous batching, with fake
operators that take a fixed time per solve on one shared device lock.  Nine operators of
the benchmark's three lattice sizes grow their bases by eigCG, then a burst of sixteen
requests per operator is served in full batches of sixteen, and requests that arrive
while their operator is busy join its next batch."""
import contextlib
import threading
import time

import numpy as np
import pytest
import torch

from paper_0707_0131_gb300 import serving

_GPU = threading.Lock()  # one device: solves run one at a time


class _Op:
    def __init__(self, gauge, dims, m_q, prec=32, max_rhs=16):
        self.vol = int(np.prod(dims)) / 884736.0
        self.closed = False

    def eigcg_solve(self, b, x, nev, m, tol, basis=None, stream=None):
        with _GPU:
            time.sleep(0.002 + 0.01 * self.vol)
        return {"iters": 100, "true_rel_res": 1e-9}

    def initcg_solve(self, B, X, tol, rtol, basis=None, k=1, stream=None):
        assert B.shape[0] == k and k <= 16
        with _GPU:
            time.sleep(0.002 + 0.004 * k * self.vol)
        return [{"iters": 50, "true_rel_res": 1e-9}] * k

    def trim(self):
        return 0

    def close(self):
        self.closed = True


class _Basis:
    def __init__(self, op, n):
        self.size = 0

    def grow(self, stream=None):
        self.size += 10

    def close(self):
        pass


@pytest.fixture
def fake_device(monkeypatch):
    monkeypatch.setattr(serving, "Op", _Op)
    monkeypatch.setattr(serving, "Basis", _Basis)
    monkeypatch.setattr(torch.cuda, "Stream", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "stream", lambda s: contextlib.nullcontext())
    to = torch.Tensor.to
    monkeypatch.setattr(torch.Tensor, "to", lambda self, *a, **k: self if a and a[0] == "cuda" else to(self, *a, **k))


def _specs(basis_max):
    return [serving.OpSpec(key=f"{d}/{c}", dims=d, m_q=0.1, gauge=None, prec=32, max_rhs=16, nev=10, m=100,
                           basis_max=basis_max)
            for d in [(8, 8, 8, 8), (16, 16, 16, 32), (24, 24, 24, 64)] for c in range(3)]


def test_growth_then_full_batches_under_the_budget(fake_device):
    specs = _specs(240)  # 24^3x64: 25 GB resident + 35 GB workspace each
    srv = serving.Server(specs, hbm_budget_bytes=150e9)
    b = np.ones(8, dtype=np.complex128)
    try:
        grow = [srv.submit(s.key, b) for _ in range(24) for s in specs]
        res = [f.result(timeout=120) for f in grow]
        assert all(r["kind"] == "eigcg" for r in res) and all(r["batch"] == 1 for r in res)
        assert all(srv.workers[s.key].basis.size == 240 for s in specs)
        srv.records.clear()
        burst = [srv.submit(s.key, b) for _ in range(16) for s in specs]
        res = [f.result(timeout=60) for f in burst]
        assert all(r["kind"] == "initcg" for r in res)
        hist = srv.batch_histogram()
        assert hist.get(16, 0) >= 16 * 6, hist  # at least six operators in one full batch each
        assert srv.max_used <= 150e9 and srv.closes == 0
        assert srv.trims > 0  # the three 24^3x64 operators cannot all hold a workspace at once
    finally:
        srv.close()


def test_requests_arriving_during_a_solve_join_the_next_batch(fake_device):
    spec = _specs(10)[-1]  # one 24^3x64 operator: a batch of k takes 2 + 4k ms
    srv = serving.Server([spec], hbm_budget_bytes=150e9)
    b = np.ones(8, dtype=np.complex128)
    try:
        srv.submit(spec.key, b).result(timeout=60)  # grows the basis to its maximum
        srv.records.clear()
        first = srv.submit(spec.key, b)
        time.sleep(0.001)  # the first request's solve is running
        later = [srv.submit(spec.key, b) for _ in range(10)]
        for f in [first] + later:
            f.result(timeout=60)
        sizes = sorted({r[4] for r in srv.records})
        assert max(sizes) >= 5, sizes  # the later requests were served together
        assert sum(srv.batch_histogram().values()) == 11
    finally:
        srv.close()
