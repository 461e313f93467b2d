"""Continuous-batching solve service over many operators (gauge field, quark mass).

Each operator keeps its own deflation basis resident on the device, so earlier
requests deflate later ones (the incremental idea of Sec. 4): while the basis is
still growing a request is solved with eigCG(nev, m) and its Ritz vectors are
added (Sec. 4 box); once the basis is full, or the switch policy (policy.py, for
operators with an expected request count) finds that more growth no longer pays
for itself (Sec. 5.3), every request that is waiting for
that operator is taken into one batched init-CG call (Eq. 1, restarted as in
Sec. 5.3) of up to max_rhs right-hand sides.

Every operator has its own worker thread and CUDA stream, so solves for
different operators overlap on the GPU; requests that arrive while a batch is
running are admitted into the next batch of their operator.  Operators are
admitted under an HBM budget in two tiers: an operator's resident part (links
and deflation basis, the state the incremental method builds up) and its
workspace (Krylov fields, staging, the eigCG window).  An operator is activated
when its workspace (and, the first time, its resident part) fits next to what is
held; otherwise idle operators give their workspace back (eig_op_trim, the basis
stays); while the workspaces of busy operators would make room once they are done, the
request waits for them; only when even that is not enough is the least recently used
idle operator closed and its basis dropped.

This module only schedules calls; all arithmetic runs in libeigcg.so.
"""
from __future__ import annotations

import queue
import threading
import time
from concurrent.futures import Future
from dataclasses import dataclass, field

import numpy as np

from . import _lib
from .api import Basis, Op
from .policy import SwitchPolicy


@dataclass
class OpSpec:
    key: str
    dims: tuple
    m_q: float
    gauge: np.ndarray
    prec: int = 32
    max_rhs: int = 16
    nev: int = 10
    m: int = 100
    basis_max: int = 240
    tol: float = 1e-8
    restart_tol: float = 1e-6
    # expected number of requests for this operator: > 0 lets the switch policy of
    # policy.py (Sec. 5.3) end the eigCG phase before basis_max when more growth no
    # longer pays; 0 grows the basis to basis_max
    expected_requests: int = 0
    eigcg_overhead: float = 1.2
    # an operator and basis that already exist (Op, Basis): served as they are, never
    # trimmed or closed by the server; its footprint still counts against the budget
    prebuilt: tuple = None

    def resident_bytes(self) -> int:
        """Device bytes an operator keeps while idle: links in all forms, the basis."""
        V = int(np.prod(self.dims))
        wide = 192 if self.prec == 64 else 96
        # FP64 links, their double-float copy (mixed precision) and the inner formats
        # (FP32 ops keep both the 12- and the 18-real form, FP16 ops the 12-real one)
        links = V * 4 * (144 + (0 if self.prec == 64 else 144) + {64: 0, 32: 48 + 72, 16: 48}[self.prec])
        basis = V * wide * (self.basis_max + self.nev + 16 + 16)
        return links + basis

    def workspace_bytes(self) -> int:
        """Device bytes of an active operator's workspace: Krylov fields for max_rhs RHS,
        FP64 and natural-layout staging, the eigCG window."""
        V = int(np.prod(self.dims))
        sp = {64: 192, 32: 96, 16: 52}[self.prec]
        wide = 192 if self.prec == 64 else 96
        work = V * self.max_rhs * (3 * sp + 5 * 192 + 2 * wide + 2 * 192) + V * 96 * 4
        window = V * wide * (self.m + 3)
        return work + window

    def footprint(self) -> int:
        """Device bytes of an active operator."""
        return self.resident_bytes() + self.workspace_bytes()


@dataclass
class Request:
    key: str
    b: np.ndarray
    submitted: float = 0.0
    future: Future = field(default_factory=Future)


class _Worker:
    def __init__(self, server: "Server", spec: OpSpec):
        self.server = server
        self.spec = spec
        self.q: "queue.Queue[Request]" = queue.Queue()
        self.op = None
        self.basis = None
        self.stream = None
        self.active = False
        self.busy = False
        self.last_used = time.perf_counter()
        self.policy = SwitchPolicy(spec.expected_requests, spec.eigcg_overhead) if spec.expected_requests > 0 else None
        self.growing = True
        self.thread = threading.Thread(target=self._run, daemon=True, name=f"eig-{spec.key}")
        self.thread.start()

    @property
    def resident(self) -> bool:
        return self.op is not None

    def activate(self):
        import torch

        if self.stream is None:
            self.stream = torch.cuda.Stream()
        s = self.spec
        if self.op is None:
            if s.prebuilt is not None:
                self.op, self.basis = s.prebuilt
            else:
                self.op = Op(s.gauge, s.dims, s.m_q, prec=s.prec, max_rhs=s.max_rhs)
                self.basis = Basis(self.op, s.basis_max + s.nev)
        self.active = True  # a trimmed op allocates its workspace again at its next call

    def trim(self):
        """Gives the workspace back and keeps the basis."""
        if self.op is not None and self.spec.prebuilt is None:
            self.op.trim()
        self.active = False

    def close(self):
        """Drops the operator and its basis."""
        if self.spec.prebuilt is None:
            if self.basis is not None:
                self.basis.close()
            if self.op is not None:
                self.op.close()
        self.op = self.basis = None
        self.active = False
        self.growing = True

    def _take(self, first: Request, limit: int):
        batch = [first]
        while len(batch) < limit:
            try:
                batch.append(self.q.get_nowait())
            except queue.Empty:
                break
        return batch

    def _run(self):
        while True:
            req = self.q.get()
            if req is None:
                return
            self.server._admit(self)
            self.busy = True
            try:
                self._serve(req)
            finally:
                self.busy = False
                self.last_used = time.perf_counter()
                self.server._released()

    def use_eigcg(self, basis_size: int) -> bool:
        """Whether the next request grows the basis (eigCG) or joins an init-CG batch.
        The eigCG phase ends for good at basis_max or when the switch policy says so."""
        s = self.spec
        if self.growing:
            self.growing = basis_size + s.nev <= s.basis_max and (self.policy is None or self.policy.use_eigcg())
        return self.growing

    def _serve(self, req: Request):
        import torch

        s = self.spec
        batch = [req]
        try:
            with torch.cuda.stream(self.stream):
                if self.use_eigcg(self.basis.size):
                    b = torch.from_numpy(req.b).to("cuda", non_blocking=False)
                    x = torch.zeros_like(b)
                    st = self.op.eigcg_solve(b, x, s.nev, s.m, s.tol, basis=self.basis, stream=self.stream)
                    self.basis.grow(stream=self.stream)
                    if self.policy is not None:
                        self.policy.record(st["iters"])
                    self._finish([req], x.reshape(1, -1), [st], "eigcg")
                    return
                batch = self._take(req, s.max_rhs)
                k = 1
                while k < len(batch):
                    k *= 2
                B = np.zeros((k, req.b.size), dtype=np.complex128)
                for i, r in enumerate(batch):
                    B[i] = r.b
                Bd = torch.from_numpy(B).to("cuda")
                Xd = torch.zeros_like(Bd)
                sts = self.op.initcg_solve(Bd, Xd, s.tol, s.restart_tol, basis=self.basis, k=k, stream=self.stream)
                self._finish(batch, Xd, sts[: len(batch)], "initcg")
        except Exception as e:  # the requests of this call fail; the worker serves the next ones
            for r in batch:
                if not r.future.done():
                    r.future.set_exception(e)

    def _finish(self, batch, X, sts, kind):
        X = X.cpu().numpy()
        now = time.perf_counter()
        for i, r in enumerate(batch):
            res = {"x": X[i].copy(), "stats": sts[i], "kind": kind, "latency_ms": (now - r.submitted) * 1e3,
                   "basis_size": self.basis.size, "batch": len(batch)}
            self.server._record(r.key, res)
            r.future.set_result(res)


class Server:
    """submit(key, b) -> Future[dict(x, stats, kind, latency_ms, basis_size, batch)]."""

    def __init__(self, specs, hbm_budget_bytes: float = 150e9):
        self.budget = float(hbm_budget_bytes)
        self.specs = {s.key: s for s in specs}
        for s in specs:
            if s.footprint() > self.budget:
                raise ValueError(f"operator {s.key} alone needs {s.footprint() / 1e9:.1f} GB > budget")
        self.cv = threading.Condition()
        self.used = 0.0
        self.workers = {s.key: _Worker(self, s) for s in specs}
        self.latencies = []
        self.records = []
        self.max_used = 0.0
        self.trims = 0   # workspaces given back by idle operators
        self.closes = 0  # idle operators closed (basis dropped)

    def submit(self, key: str, b: np.ndarray) -> Future:
        req = Request(key, np.ascontiguousarray(b, dtype=np.complex128).reshape(-1))
        req.submitted = time.perf_counter()
        self.workers[key].q.put(req)
        return req.future

    # admission by HBM budget: activate the operator; first take workspaces back from idle
    # operators (their bases stay), then close the least recently used idle operator
    def _admit(self, w: _Worker):
        with self.cv:
            while not w.active:
                need = w.spec.workspace_bytes() + (0 if w.resident else w.spec.resident_bytes())
                if self.used + need <= self.budget:
                    self.used += need
                    self.max_used = max(self.max_used, self.used)
                    w.activate()
                    break
                idle = [o for o in self.workers.values()
                        if o is not w and not o.busy and o.q.empty() and o.spec.prebuilt is None]
                active_idle = [o for o in idle if o.active]
                if active_idle:
                    victim = min(active_idle, key=lambda o: o.last_used)
                    victim.trim()
                    self.used -= victim.spec.workspace_bytes()
                    self.trims += 1
                    continue
                # a basis is the work of all the eigCG solves that grew it: rather than close
                # one, wait while the workspaces of busy operators would make room once freed
                busy_ws = sum(o.spec.workspace_bytes() for o in self.workers.values()
                              if o is not w and o.active and o.spec.prebuilt is None)
                if busy_ws > 0 and self.used - busy_ws + need <= self.budget:
                    self.cv.wait(timeout=0.05)
                    continue
                resident_idle = [o for o in idle if o.resident and not o.active]
                if resident_idle:
                    victim = min(resident_idle, key=lambda o: o.last_used)
                    victim.close()
                    self.used -= victim.spec.resident_bytes()
                    self.closes += 1
                    continue
                self.cv.wait(timeout=0.05)

    def _released(self):
        with self.cv:
            self.cv.notify_all()

    def _record(self, key, res):
        with self.cv:
            self.latencies.append(res["latency_ms"])
            self.records.append((key, res["kind"], res["stats"]["iters"], res["latency_ms"], res["batch"]))

    def percentiles(self):
        a = np.array(self.latencies)
        return {"p50_ms": float(np.percentile(a, 50)), "p99_ms": float(np.percentile(a, 99)), "n": int(a.size)}

    def batch_histogram(self):
        """{batch size: number of requests served in batches of that size}."""
        with self.cv:
            sizes = [rec[4] for rec in self.records]
        return {int(b): int(sum(1 for x in sizes if x == b)) for b in sorted(set(sizes))}

    def close(self):
        for w in self.workers.values():
            w.q.put(None)
        for w in self.workers.values():
            w.thread.join(timeout=60)
            w.close()


def poisson_arrivals(rate_per_s: float, n: int, seed: int) -> np.ndarray:
    """n arrival times (seconds from 0) of a Poisson process of the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=n))
