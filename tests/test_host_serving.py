"""Host logic of the serving loop (no GPU): admission under the HBM budget retires the
least recently used idle operator, waits while the others are busy, and the Poisson
arrival generator and latency percentiles behave as stated."""
import queue
import threading
import time

import numpy as np

from paper_0707_0131_gb300 import serving


class _Spec:
    def __init__(self, key, nbytes):
        self.key = key
        self.nbytes = nbytes

    def footprint(self):
        return self.nbytes


class _FakeWorker:
    def __init__(self, key, nbytes, last_used):
        self.spec = _Spec(key, nbytes)
        self.active = False
        self.busy = False
        self.q = queue.Queue()
        self.last_used = last_used
        self.events = []

    def activate(self):
        self.active = True
        self.events.append("activate")

    def retire(self):
        self.active = False
        self.events.append("retire")


def _server(budget, workers):
    srv = serving.Server([], hbm_budget_bytes=budget)
    srv.workers = {w.spec.key: w for w in workers}
    return srv


def test_admission_retires_least_recently_used_idle_operator():
    a, b, c = _FakeWorker("a", 40, 1.0), _FakeWorker("b", 40, 2.0), _FakeWorker("c", 50, 3.0)
    srv = _server(100, [a, b, c])
    srv._admit(a)
    srv._admit(b)
    assert srv.used == 80 and a.active and b.active
    srv._admit(c)  # needs 50: the older idle operator (a) goes
    assert a.events == ["activate", "retire"] and b.active and c.active
    assert srv.used == 90 and srv.max_used == 90
    srv._admit(c)  # already active: nothing changes
    assert srv.used == 90


def test_admission_waits_for_busy_operators():
    a, b = _FakeWorker("a", 60, 1.0), _FakeWorker("b", 60, 2.0)
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
    srv._admit(b)  # a is busy: b waits until a is idle, then a is retired
    t.join()
    assert time.perf_counter() - t0 >= 0.15
    assert b.active and not a.active and srv.used == 60


def test_admission_skips_operators_with_queued_requests():
    a, b, c = _FakeWorker("a", 50, 1.0), _FakeWorker("b", 50, 2.0), _FakeWorker("c", 50, 3.0)
    srv = _server(100, [a, b, c])
    srv._admit(a)
    srv._admit(b)
    a.q.put("pending request")  # a is idle but has work waiting: b is retired instead
    srv._admit(c)
    assert a.active and not b.active and c.active


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
