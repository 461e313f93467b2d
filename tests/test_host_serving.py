"""Host logic of the serving loop (no GPU): admission under the HBM budget first takes
workspaces back from idle operators (their bases stay), waits while busy operators'
workspaces would make room, only then closes the least recently used idle operator,
skips operators with queued
requests, and the Poisson arrival generator and latency percentiles behave as stated."""
import queue
import threading
import time

import numpy as np

from paper_0707_0131_gb300 import serving


class _Spec:
    def __init__(self, key, resident, workspace):
        self.key = key
        self.res = resident
        self.ws = workspace
        self.prebuilt = None

    def resident_bytes(self):
        return self.res

    def workspace_bytes(self):
        return self.ws

    def footprint(self):
        return self.res + self.ws


class _FakeWorker:
    def __init__(self, key, resident, workspace, last_used):
        self.spec = _Spec(key, resident, workspace)
        self.active = False
        self.resident = False
        self.busy = False
        self.q = queue.Queue()
        self.last_used = last_used
        self.events = []

    def activate(self):
        self.active = True
        self.resident = True
        self.events.append("activate")

    def trim(self):
        self.active = False
        self.events.append("trim")

    def close(self):
        self.active = False
        self.resident = False
        self.events.append("close")


def _server(budget, workers):
    srv = serving.Server([], hbm_budget_bytes=budget)
    srv.workers = {w.spec.key: w for w in workers}
    return srv


def test_admission_trims_before_it_closes():
    # resident 10 + workspace 30 each (c: 20 + 30), budget 100
    a, b, c = _FakeWorker("a", 10, 30, 1.0), _FakeWorker("b", 10, 30, 2.0), _FakeWorker("c", 20, 30, 3.0)
    srv = _server(100, [a, b, c])
    srv._admit(a)
    srv._admit(b)
    assert srv.used == 80 and a.active and b.active
    srv._admit(c)  # needs 50: the older idle operator (a) gives its workspace back, keeps its basis
    assert a.events == ["activate", "trim"] and a.resident and b.active and c.active
    assert srv.used == 100 and srv.max_used == 100 and srv.trims == 1 and srv.closes == 0
    srv._admit(c)  # already active: nothing changes
    assert srv.used == 100
    # a again: only its workspace is needed (30); b and c give theirs back in LRU order
    b.last_used, c.last_used = 4.0, 5.0
    srv._admit(a)
    assert a.active and b.events[-1] == "trim" and c.active and srv.used == 100


def test_admission_closes_when_trimming_is_not_enough():
    a, b = _FakeWorker("a", 50, 30, 1.0), _FakeWorker("b", 40, 30, 2.0)
    srv = _server(100, [a, b])
    srv._admit(a)  # 80
    srv._admit(b)  # needs 70: trimming a leaves 50 + 70 > 100, so a is closed as well
    assert a.events == ["activate", "trim", "close"] and not a.resident
    assert b.active and srv.used == 70 and srv.trims == 1 and srv.closes == 1


def test_admission_waits_for_busy_operators():
    a, b = _FakeWorker("a", 20, 40, 1.0), _FakeWorker("b", 20, 40, 2.0)
    srv = _server(100, [a, b])
    srv._admit(a)
    a.busy = True

    def release():
        time.sleep(0.2)
        a.busy = False
        srv._released()

    t = threading.Thread(target=release)
    t.start()
    t0 = time.perf_counter()
    srv._admit(b)  # a is busy: b waits until a is idle, then a gives its workspace back
    t.join()
    assert time.perf_counter() - t0 >= 0.15
    assert b.active and not a.active and a.resident and srv.used == 80


def test_admission_waits_for_a_busy_workspace_before_closing_a_basis():
    # a busy (resident 20 + workspace 40), c resident but trimmed (30), budget 130: b needs 60.
    # Closing c would make room at once, but a's workspace will too once a is done, so b
    # waits and c keeps its basis.
    a, b, c = _FakeWorker("a", 20, 40, 1.0), _FakeWorker("b", 20, 40, 2.0), _FakeWorker("c", 30, 10, 0.5)
    srv = _server(130, [a, b, c])
    srv._admit(c)
    c.trim()
    srv.used -= 10
    srv._admit(a)
    a.busy = True
    assert srv.used == 90

    def release():
        time.sleep(0.2)
        a.busy = False
        srv._released()

    th = threading.Thread(target=release)
    th.start()
    t0 = time.perf_counter()
    srv._admit(b)
    th.join()
    assert time.perf_counter() - t0 >= 0.15
    assert b.active and not a.active and a.resident and c.resident and "close" not in c.events
    assert srv.closes == 0 and srv.used == 110


def test_admission_skips_operators_with_queued_requests():
    a, b, c = _FakeWorker("a", 10, 40, 1.0), _FakeWorker("b", 10, 40, 2.0), _FakeWorker("c", 10, 40, 3.0)
    srv = _server(110, [a, b, c])
    srv._admit(a)
    srv._admit(b)
    a.q.put("pending request")  # a is idle but has work waiting: b gives its workspace back
    srv._admit(c)
    assert a.active and not b.active and b.resident and c.active


def test_poisson_arrivals_and_percentiles():
    t = serving.poisson_arrivals(4.0, 20000, 7)
    assert np.all(np.diff(t) > 0)
    assert abs(np.mean(np.diff(t)) - 0.25) < 0.01
    srv = serving.Server([], hbm_budget_bytes=1.0)
    srv.latencies = list(range(1, 101))
    p = srv.percentiles()
    assert p["n"] == 100 and abs(p["p50_ms"] - 50.5) < 1e-9 and abs(p["p99_ms"] - 99.01) < 1e-9


def test_operator_larger_than_budget_is_refused():
    spec = serving.OpSpec(key="big", dims=(24, 24, 24, 64), m_q=0.0, gauge=None)
    try:
        serving.Server([spec], hbm_budget_bytes=1e9)
    except ValueError as e:
        assert "budget" in str(e)
    else:
        raise AssertionError("an operator above the budget must be refused")


def test_failed_solve_fails_its_requests_and_the_worker_goes_on():
    """A solve that raises (here: no GPU to copy the batch to) sets the exception on every
    request of its batch instead of ending the worker thread, so that no caller waits on
    a future that never completes."""

    class _Basis:
        size = 100

    spec = serving.OpSpec(key="x", dims=(4, 4, 4, 4), m_q=0.1, gauge=None, max_rhs=4, nev=4, m=12, basis_max=8)
    w = serving._Worker.__new__(serving._Worker)
    w.spec, w.q, w.stream, w.basis, w.op = spec, queue.Queue(), None, _Basis(), None
    w.policy, w.growing = None, False
    reqs = [serving.Request("x", np.ones(8, dtype=np.complex128)) for _ in range(3)]
    for r in reqs[1:]:
        w.q.put(r)
    w._serve(reqs[0])  # must not raise
    assert all(r.future.done() and r.future.exception() is not None for r in reqs)
    again = serving.Request("x", np.ones(8, dtype=np.complex128))
    w._serve(again)
    assert again.future.exception() is not None
