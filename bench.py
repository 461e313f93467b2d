"""Benchmark: RHS solved per second at a 1e-8 FP64 true residual, 24^3x64 Wilson lattice.

One step is one pass of the whole hot path over one batch of synthetic input:
  1. eigCG(10, 100) on one new RHS, deflated by the resident basis (Eq. 1 + Fig. 1),
     then basis_grow (Sec. 4 box) and a rollback of the basis to its base size so
     that every step does the same work;
  2. init-CG on a batch of k = 16 RHS through the multi-RHS dslash, deflated by the
     basis and restarted once at 1e-6 (Sec. 5.3).
Storage FP32 (12-real links) with FP64 reliable updates and FP64 true residuals.
The basis (up to 240 vectors, as in Sec. 5) is grown by Incremental eigCG before
the warm-up steps.  Inputs are synthetic (gauge recipe and Gaussian RHS of the
fixtures module), every field far larger than L2.

Also reported: plain FP64 eigCG (no deflation, no batching, FP64 storage) on the
same GPU, the dominant kernel's roofline, the end-to-end rate through the C ABI
with host buffers, and the FP64 CPU oracle's rate on the host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_0707_0131_gb300 import fixtures as fx  # noqa: E402

METRIC = "RHS solved/s at 1e-8 residual (24^3x64)"
UNIT = "RHS/s"
LATTICE = "24^3x64"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--lattice", default=LATTICE)
    ap.add_argument("--k", type=int, default=16)
    ap.add_argument("--basis", type=int, default=240)
    ap.add_argument("--nev", type=int, default=10)
    ap.add_argument("--m", type=int, default=100)
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--restart-tol", type=float, default=1e-6)
    ap.add_argument("--kappa", default="1e+05")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-serve", action="store_true", help="skip the short serving phase of the solve benchmark")
    ap.add_argument("--no-eo", action="store_true", help="skip the odd-even arm of the solve benchmark")
    ap.add_argument("--serve-requests", type=int, default=48, help="solve mode: requests of the serving phase")
    ap.add_argument("--mode", default="solve", choices=["solve", "dslash", "serve", "bicgstab", "oracle"],
                    help="dslash: only repeated matvecs through eig_op_apply (kernel GB/s); "
                         "serve: Poisson requests over 9 operators through the serving loop")
    ap.add_argument("--requests", type=int, default=200, help="serve mode: number of requests")
    ap.add_argument("--serve-lattices", default="8^4,16^3x32,24^3x64")
    ap.add_argument("--serve-basis", type=int, default=40)
    ap.add_argument("--serve-policy", action="store_true",
                    help="serve mode: end each operator's eigCG phase by the switch policy (expected requests "
                         "= requests / operators) instead of at --serve-basis")
    ap.add_argument("--budget-gb", type=float, default=150.0)
    ap.add_argument("--prec", type=int, default=32)
    ap.add_argument("--reliable-delta", type=float, default=0.01,
                    help="residual replacement when ||r|| fell by this factor since the last one")
    ap.add_argument("--links", type=int, default=12, choices=[12, 18],
                    help="FP32 link storage: 12 reals (third row rebuilt) or all 18")
    ap.add_argument("--which", type=int, default=2, help="dslash mode: 0 M, 1 M^H, 2 A")
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--defl-vecs", type=int, default=64, help="bicgstab mode: Ritz vectors in the g5 M deflation")
    return ap.parse_args()


def mass_for(lattice, kappa):
    masses = json.load(open(os.path.join(ROOT, "configs", "masses.json")))
    if lattice in masses and kappa in masses[lattice]:
        return masses[lattice][kappa]["m_q"], f"{lattice} calibration"
    # bulk critical mass of this gauge recipe is volume independent: take the
    # largest calibrated lattice's mass for the same target condition number
    for name in ("16^3x32", "8^4"):
        if name in masses and kappa in masses[name]:
            return masses[name][kappa]["m_q"], f"{name} calibration"
    raise KeyError(f"no mass for {lattice} cond {kappa}")


def rank_info():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def max_over_ranks(ms, world, device):
    """The slowest rank's time (every rank gets it): replicas finish when the last one does."""
    if world == 1:
        return float(ms)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, steps, rhs_per_step, ms):
    """Whole-job RHS/s: every replica solves steps * rhs_per_step RHS in the slowest time."""
    return world * steps * rhs_per_step / (ms / 1e3)


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([v.strip() for v in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm = [float(s[0]) for s in self.samples if len(s) >= 8 and s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if len(s) >= 8 and s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            if len(s) < 8:
                continue
            for i, n in enumerate(names):
                if s[4 + i].lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_rate(dims, m_q, gauge, seconds):
    """FP64 CPU oracle: seconds per CG iteration (one A application + vector updates)."""
    import oracle
    from oracle import solvers

    W = oracle.Wilson(dims, m_q, gauge)
    b = fx.make_rhs(dims, fx.rhs_seed(LATTICE if tuple(dims) == fx.LATTICES[LATTICE] else "8^4", 999))[0]
    t0 = time.perf_counter()
    solvers.cg(W, b, tol=1e-30, max_iter=1)  # warm
    per = time.perf_counter() - t0
    n = max(2, int(seconds / max(per, 1e-3)))
    t0 = time.perf_counter()
    res = solvers.cg(W, b, tol=1e-30, max_iter=n)
    dt = time.perf_counter() - t0
    # cg() also spends one A application on the final true residual
    return dt / (res["iters"] + 1), res["iters"], oracle.num_threads()


def run_reference(a):
    rank, world, _ = rank_info()
    if rank != 0:
        return
    dims = fx.LATTICES[a.lattice]
    m_q, _ = mass_for(a.lattice, a.kappa)
    gauge = fx.make_gauge(dims, fx.GAUGE_SEEDS[a.lattice])
    cfg = json.load(open(os.path.join(ROOT, "configs", "bench.json")))
    iters_per_rhs = cfg["iters_per_rhs"]
    per_step = max(2.0, min(a.cpu_seconds, 60.0) / max(1, a.steps))
    oracle_rate(dims, m_q, gauge, 1.0)  # warm-up
    times = []
    for _ in range(a.steps):
        t_it, n, cores = oracle_rate(dims, m_q, gauge, per_step)
        times.append(t_it)
    t_it = float(np.mean(times))
    value = 1.0 / (t_it * iters_per_rhs)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
           "steps": a.steps, "warmup": a.warmup, "ms_per_step": t_it * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"{a.lattice} Wilson, cond(A)~{a.kappa}, k={a.k}, basis {a.basis}, tol {a.tol}"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"FP64 oracle CG iterations on one RHS of the {a.lattice} workload, "
                                      f"{per_step:.0f} s per step; RHS/s = 1/(s per iteration x "
                                      f"{iters_per_rhs} iterations per RHS, configs/bench.json)"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_oracle(a):
    """Timings of the FP64 CPU oracle on this machine's host cores (a reported baseline, not
    the target): full CG and eigCG solves at 4^4, 8^4 and 16^3x32 and a full CG solve at
    24^3x64, all at cond(A) ~ 1e3 and tol 1e-8, plus seconds per CG iteration at 24^3x64."""
    import oracle
    from oracle import solvers

    rows = []
    for name in ("4^4", "8^4", "16^3x32", "24^3x64"):
        dims = fx.LATTICES[name]
        m_q, src = mass_for(name, "1e+03")
        W = oracle.Wilson(dims, m_q, fx.make_gauge(dims, fx.GAUGE_SEEDS[name]))
        b = fx.make_rhs(dims, fx.rhs_seed(name, 0))[0].reshape(-1)
        for kind in ("cg", "eigcg"):
            if kind == "eigcg" and name == "24^3x64":
                continue
            t0 = time.perf_counter()
            o = solvers.cg(W, b, tol=1e-8) if kind == "cg" else solvers.eigcg(W, b, nev=10, m=100, tol=1e-8)
            dt = time.perf_counter() - t0
            rows.append({"lattice": name, "solver": kind, "iters": int(o["iters"]), "seconds": dt,
                         "s_per_iter": dt / max(1, o["iters"]), "true_rel_res": float(o["true_rel_res"]),
                         "mass": src})
            print(json.dumps(rows[-1]), flush=True)
    print(json.dumps({"mode": "oracle", "cores": oracle.num_threads(), "solves": rows}), flush=True)


def run_dslash(a):
    """Repeated matvecs on device-resident fields: per-kernel launches, time and GB/s."""
    import torch

    from paper_0707_0131_gb300 import _lib
    from paper_0707_0131_gb300.api import Op

    torch.cuda.set_device(0)
    dims = fx.LATTICES[a.lattice]
    m_q, _ = mass_for(a.lattice, a.kappa)
    gauge = fx.make_gauge(dims, fx.GAUGE_SEEDS[a.lattice])
    op = Op(gauge, dims, m_q, prec=a.prec, max_rhs=a.k, compress12=a.links == 12)
    x = torch.from_numpy(fx.make_rhs(dims, 7, a.k)).cuda()
    y = torch.empty_like(x)
    for _ in range(3):
        op.apply(a.which, x, y, a.k)
    _lib.eig_profile_reset()
    _lib.eig_profile_enable(True)
    for _ in range(a.reps):
        op.apply(a.which, x, y, a.k)
    _lib.eig_profile_enable(False)
    prof = _lib.eig_profile_read()
    peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"] \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 6800.0
    out = {"mode": "dslash", "lattice": a.lattice, "k": a.k, "prec": a.prec, "links": a.links, "which": a.which,
           "kernels": {}}
    for n, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"]):
        gbs = v["bytes"] / (v["ms"] / 1e3) / 1e9 if v["ms"] > 0 else None
        out["kernels"][n] = {"launches": v["launches"], "ms_per_launch": v["ms"] / max(1, v["launches"]),
                             "GBps": gbs, "frac_of_hbm": gbs / peak if gbs else None,
                             "bytes_per_launch": v["bytes"] / max(1, v["launches"])}
    print(json.dumps(out), flush=True)
    op.close()


def run_bicgstab(a):
    """Deflated BiCGSTAB on M (Sec. 1) next to init-CG on A: a basis is grown by
    Incremental eigCG as in the solve mode, then each of a.steps new right-hand sides of
    M x = b is solved by BiCGSTAB without and with the g5 M deflation, and by init-CG on
    A x = M^H b with the same basis (one RHS per call)."""
    import torch

    from paper_0707_0131_gb300.api import Basis, Op

    torch.cuda.set_device(0)
    dims = fx.LATTICES[a.lattice]
    m_q, mass_src = mass_for(a.lattice, a.kappa)
    gauge = fx.make_gauge(dims, fx.GAUGE_SEEDS[a.lattice])
    op = Op(gauge, dims, m_q, prec=32, max_rhs=1)
    basis = Basis(op, a.basis + a.nev)
    r = 0
    while basis.size + a.nev <= a.basis:
        b = torch.from_numpy(fx.make_rhs(dims, fx.rhs_seed(a.lattice, r))[0].reshape(-1)).cuda()
        op.eigcg_solve(b, torch.zeros_like(b), a.nev, a.m, a.tol, basis=basis)
        basis.grow()
        r += 1
    rows = {"bicgstab": [], "bicgstab_deflated": [], "initcg": []}
    nz = min(a.defl_vecs, basis.size)
    for i in range(a.steps):
        b = torch.from_numpy(fx.make_rhs(dims, fx.rhs_seed(a.lattice, 500 + i))[0].reshape(-1)).cuda()
        bA = b.clone()
        op.apply(1, b, bA)  # A x = M^H b has the same solution
        for kind in rows:
            x = torch.zeros_like(b)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if kind == "initcg":
                st = op.initcg_solve(bA, x, a.tol, a.restart_tol, basis=basis)[0]
            else:
                st = op.bicgstab_solve(b, x, a.tol, basis=basis if kind != "bicgstab" else None, defl_vecs=nz)
            torch.cuda.synchronize()
            rows[kind].append({"ms": (time.perf_counter() - t0) * 1e3, "iters": st["iters"],
                               "true_rel_res": st["true_rel_res"]})
    out = {"mode": "bicgstab", "lattice": a.lattice, "m_q": m_q, "basis": basis.size, "defl_vecs": nz,
           "tol": a.tol, "note": "first BiCGSTAB with deflation includes building Z and Z^H g5 M Z"}
    for kind, v in rows.items():
        out[kind] = {"ms_mean": float(np.mean([e["ms"] for e in v])), "iters_mean": float(np.mean([e["iters"] for e in v])),
                     "max_true_rel_res": float(max(e["true_rel_res"] for e in v)), "runs": v}
    print(json.dumps(out), flush=True)
    basis.close()
    op.close()


def run_serve(a):
    """Serving form: single-RHS requests over 3 lattices x 3 masses, continuous batching with
    per-operator resident bases under an HBM budget.  Three phases: the requests that grow
    every basis to its maximum (eigCG, incremental), a burst of one full batch per operator
    that measures the steady-state capacity, then Poisson arrivals at 0.8x that capacity,
    from which the rate, the latency percentiles and the batch sizes are reported."""
    import torch

    from paper_0707_0131_gb300 import serving
    from paper_0707_0131_gb300.api import Op

    torch.cuda.set_device(0)
    specs = []
    names = a.serve_lattices.split(",")
    expected = a.requests // (3 * len(names)) if a.serve_policy else 0
    for name in names:
        dims = fx.LATTICES[name]
        gauge = fx.make_gauge(dims, fx.GAUGE_SEEDS[name])
        for kappa in ("1e+03", "1e+04", "1e+05"):
            m_q, _ = mass_for(name, kappa)
            specs.append(serving.OpSpec(key=f"{name}/{kappa}", dims=dims, m_q=m_q, gauge=gauge, prec=32,
                                        max_rhs=a.k, nev=a.nev, m=a.m, basis_max=a.serve_basis, tol=a.tol,
                                        restart_tol=a.restart_tol, expected_requests=expected))
    by_key = {s.key: s for s in specs}
    rng = np.random.default_rng(105)
    keys = [specs[i].key for i in rng.integers(0, len(specs), size=a.requests)]
    # eight Gaussian RHS per operator, generated once before anything is timed (requests
    # reuse them in turn)
    rhs_cache = {s_.key: [fx.make_rhs(s_.dims, 4_000_000 + j)[0].reshape(-1) for j in range(8)] for s_ in specs}

    def rhs_of(key, j):
        return rhs_cache[key][j % 8]

    def rhs(i):
        return rhs_of(keys[i], i)

    # plain FP64 eigCG per request (same GPU, no deflation, no batching): one solve per operator
    plain_ms = {}
    if not a.no_plain:
        for s_ in specs:
            op64 = Op(s_.gauge, s_.dims, s_.m_q, prec=64)
            b = torch.from_numpy(rhs_of(s_.key, 0)).cuda()
            x = torch.zeros_like(b)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            op64.eigcg_solve(b, x, s_.nev, s_.m, s_.tol, max_iter=50000)
            torch.cuda.synchronize()
            plain_ms[s_.key] = (time.perf_counter() - t0) * 1e3
            op64.close()

    srv = serving.Server(specs, hbm_budget_bytes=a.budget_gb * 1e9)
    # phase 1, growth: each operator serves the requests that grow its basis to basis_max
    # (eigCG(nev, m) per request, Sec. 4), all submitted at once and queued per operator
    n_grow = max(1, a.serve_basis // a.nev)
    t0 = time.perf_counter()
    grow = [srv.submit(s_.key, rhs_of(s_.key, j)) for j in range(n_grow) for s_ in specs]
    grow_res = [f.result() for f in grow]
    grow_wall = time.perf_counter() - t0
    print(f"serve: growth phase {len(grow_res)} requests in {grow_wall:.1f} s", file=sys.stderr, flush=True)
    grow_lat = srv.percentiles()
    # phase 2, capacity: a burst of max_rhs requests per operator (one full batch each)
    srv.latencies.clear()
    srv.records.clear()
    t0 = time.perf_counter()
    burst = [srv.submit(s_.key, rhs_of(s_.key, 100 + j)) for j in range(a.k) for s_ in specs]
    for f in burst:
        f.result()
    cap = len(burst) / (time.perf_counter() - t0)
    rate = 0.8 * cap
    print(f"serve: capacity {cap:.1f} RHS/s from a burst of {len(burst)}; Poisson at {rate:.1f}/s",
          file=sys.stderr, flush=True)
    # phase 3, timed: Poisson arrivals at 0.8x that capacity; latencies and batch sizes are
    # taken from this phase only
    srv.latencies.clear()
    srv.records.clear()
    arrivals = serving.poisson_arrivals(rate, a.requests, 105)
    futs = []
    t0 = time.perf_counter()
    for i, ta in enumerate(arrivals):
        now = time.perf_counter() - t0
        if ta > now:
            time.sleep(ta - now)
        futs.append((keys[i], srv.submit(keys[i], rhs(i))))
    res = [(k_, f.result()) for k_, f in futs]
    wall = time.perf_counter() - t0
    pct = srv.percentiles()
    plain_mean = float(np.mean([plain_ms[k_] for k_, _ in res])) if plain_ms else None
    out = {"mode": "serve", "metric": "RHS/s and latency under Poisson load", "value": len(res) / wall,
           "unit": UNIT, "p50_ms": pct["p50_ms"], "p99_ms": pct["p99_ms"], "requests": len(res),
           "arrival_rate_per_s": rate, "capacity_estimate_per_s": cap,
           "plain_fp64_eigcg_ms_per_request_mean": plain_mean,
           "max_true_rel_res": float(max(r["stats"]["true_rel_res"] for _, r in res)),
           "batched_fraction": float(np.mean([r["batch"] > 1 for _, r in res])),
           "batch_histogram": srv.batch_histogram(),
           "max_hbm_used_gb": srv.max_used / 1e9, "budget_gb": a.budget_gb,
           "workspaces_released": srv.trims, "operators_closed": srv.closes,
           "eigcg_solves": int(sum(r["kind"] == "eigcg" for _, r in res)),
           "growth_phase": {"requests": len(grow_res), "wall_s": grow_wall,
                            "eigcg_solves": int(sum(r["kind"] == "eigcg" for r in grow_res)),
                            "max_true_rel_res": float(max(r["stats"]["true_rel_res"] for r in grow_res)),
                            "p50_ms": grow_lat["p50_ms"], "p99_ms": grow_lat["p99_ms"],
                            "basis_sizes": {s_.key: int(srv.workers[s_.key].basis.size)
                                            for s_ in specs if srv.workers[s_.key].basis is not None}},
           "config": {"workload": f"{len(specs)} operators ({a.serve_lattices} x cond 1e3/1e4/1e5), basis "
                                  f"<= {a.serve_basis}, eigCG({a.nev},{a.m}) then init-CG batches of <= {a.k}, tol {a.tol}",
                      "switch": f"policy, {expected} expected requests per operator" if expected else "basis full"}}
    srv.close()
    print(json.dumps(out), flush=True)


def main():
    a = parse()
    if a.mode == "serve":
        run_serve(a)
        return
    if a.impl == "reference":
        run_reference(a)
        return
    if a.mode == "dslash":
        run_dslash(a)
        return
    if a.mode == "oracle":
        run_oracle(a)
        return
    if a.mode == "bicgstab":
        run_bicgstab(a)
        return
    import torch

    from paper_0707_0131_gb300 import _lib
    from paper_0707_0131_gb300.api import Basis, Op

    rank, world, local = rank_info()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()
        torch.cuda.synchronize()

    dims = fx.LATTICES[a.lattice]
    V = fx.volume(dims)
    m_q, mass_src = mass_for(a.lattice, a.kappa)
    gauge = fx.make_gauge(dims, fx.GAUGE_SEEDS[a.lattice])
    k = a.k
    if a.prec not in (32, 16):
        raise SystemExit("the solve benchmark stores spinors in FP32 or FP16 (--prec 32|16)")
    op = Op(gauge, dims, m_q, prec=a.prec, max_rhs=k, compress12=a.links == 12, reliable_delta=a.reliable_delta)
    basis = Basis(op, a.basis + a.nev)
    nrhs_id = [0]

    def next_rhs(n):
        out = []
        for _ in range(n):
            out.append(fx.make_rhs(dims, fx.rhs_seed(a.lattice, 1000 * rank + nrhs_id[0]))[0])
            nrhs_id[0] += 1
        return np.stack(out)

    # --- setup: Incremental eigCG until the basis holds a.basis vectors -------------------
    t0 = time.perf_counter()
    phase1 = []
    while basis.size + a.nev <= a.basis:
        b = torch.from_numpy(next_rhs(1)[0]).to(dev)
        x = torch.zeros_like(b)
        st = op.eigcg_solve(b, x, a.nev, a.m, a.tol, basis=basis)
        basis.grow()
        phase1.append(st["iters"])
    setup_s = time.perf_counter() - t0
    l0 = basis.size

    # arithmetic roofs of this GPU (FMA throughput), for the FP64 kernels
    alu = {}
    try:
        alu = {"fp64_tflops": _lib.eig_profile_alu_peak(64), "fp32_tflops": _lib.eig_profile_alu_peak(32),
               "how": "independent FMA chains over 8 CTAs x 256 threads per SM, best of two (FP32 as packed pairs)"}
    except Exception as ex:  # measurement aid only
        alu = {"error": str(ex)}

    # step inputs: fresh RHS per step, resident on the device
    nsteps = a.warmup + a.steps
    B1 = [torch.from_numpy(next_rhs(1)[0]).to(dev) for _ in range(nsteps)]
    Bk = [torch.from_numpy(next_rhs(k)).to(dev) for _ in range(nsteps)]
    iters = {"eigcg": [], "initcg": []}
    status = {"true_res": []}

    def step(i, b1, x1, bk, xk, record):
        st = op.eigcg_solve(b1, x1, a.nev, a.m, a.tol, basis=basis)
        basis.grow()
        basis.truncate(l0)
        sts = op.initcg_solve(bk, xk, a.tol, a.restart_tol, basis=basis, k=k)
        if record:
            iters["eigcg"].append(st["iters"])
            iters["initcg"].extend(s["iters"] for s in sts)
            status["true_res"].extend([st["true_rel_res"]] + [s["true_rel_res"] for s in sts])

    for i in range(a.warmup):
        step(i, B1[i], torch.zeros_like(B1[i]), Bk[i], torch.zeros_like(Bk[i]), False)
    X1 = [torch.zeros_like(B1[i]) for i in range(nsteps)]
    Xk = [torch.zeros_like(Bk[i]) for i in range(nsteps)]
    clocks = ClockSampler(local)
    _lib.eig_profile_reset()
    _lib.eig_profile_enable(True)
    barrier()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for i in range(a.warmup, nsteps):
        step(i, B1[i], X1[i], Bk[i], Xk[i], True)
    ev1.record()
    barrier()
    clk = clocks.stop()
    _lib.eig_profile_enable(False)
    prof = _lib.eig_profile_read()
    ms = max_over_ranks(ev0.elapsed_time(ev1), world, dev)
    rhs_per_step = 1 + k
    value = job_rate(world, a.steps, rhs_per_step, ms)
    launches = int(sum(v["launches"] for v in prof.values()))
    # roofline of the dominant kernel: the one with the most device time in the timed
    # region, whatever it is; every kernel of the path is HBM-bound at this size except
    # the FP64 / double-float stencils (arithmetic), reported against the FMA roofs below
    kern = max(prof, key=lambda n: prof[n]["ms"])
    kp = prof[kern]
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(peaks_path):
        peak = json.load(open(peaks_path))["hbm_gbs"]
        peak_src = "measured"
    else:
        peak, peak_src = 6800.0, "fallback"
    achieved = (kp["bytes"] / kp["launches"]) / (kp["ms"] / kp["launches"] / 1e3) / 1e9
    # the stencil variant and link form the autotuner chose for that kernel's batch width
    kk = int(kern.rsplit("_k", 1)[1]) if "_k" in kern else 1
    kvar, klinks = op.stencil_choice(kk)
    # DRAM traffic from an ncu capture of this kernel (configs/traffic_from_ncu.py): the
    # measured DRAM / algorithmic byte ratio, valid while the stencil sources, the variant
    # and the link form match the capture's
    traffic = None
    tfile = os.path.join(ROOT, "configs", "traffic.json")
    if os.path.exists(tfile):
        h = hashlib.sha1()
        for f in ("dslash32.cuh", "dslash32.cu", "dslash32d_rb1.cu", "dslash32d_rb2.cu", "dslash32pp.cuh",
                  "dslash32p2.cu", "dslash32p3.cu", "dslash32p3f.cu"):
            h.update(open(os.path.join(ROOT, "paper_0707_0131_gb300", "csrc", f), "rb").read())
        for tj in json.load(open(tfile)).get(kern, []):
            if (tj.get("stencil_sha1") == h.hexdigest() and tj.get("variant") == kvar
                    and tj.get("link_reals") == klinks):
                traffic = tj["dram_over_algorithmic"] * kp["bytes"] / kp["launches"]
    roofline = {"bound": "hbm", "kernel": kern, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_src, "traffic": traffic,
                "variant": kvar, "link_reals": klinks,
                "algorithmic_bytes_per_launch": kp["bytes"] / kp["launches"],
                "avg_launch_ms": kp["ms"] / kp["launches"], "launches": kp["launches"]}
    kernels = {}
    for n, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"]):
        gbs = (v["bytes"] / (v["ms"] / 1e3) / 1e9) if v["ms"] > 0 else None
        e = {"launches": v["launches"], "ms": round(v["ms"], 3), "GBps": gbs,
             "frac_of_hbm": (gbs / peak) if gbs else None}
        # FP64 stencils: ~1320 flop per site and RHS for one M (spin-projected count)
        if n.startswith("dslash_") and "f64" in n and v["ms"] > 0 and alu.get("fp64_tflops"):
            kk_ = int(n.rsplit("_k", 1)[1]) if "_k" in n else 1
            tf = 1320.0 * V * kk_ * v["launches"] / (v["ms"] / 1e3) / 1e12
            e["fp64_tflops"] = tf
            e["frac_of_fp64_fma"] = tf / alu["fp64_tflops"]
        kernels[n] = e

    # --- end to end: same steps with pinned host buffers -----------------------------
    e2e = None
    if not a.no_e2e:
        hb1 = [torch.from_numpy(next_rhs(1)[0]).pin_memory() for _ in range(a.steps)]
        hbk = [torch.from_numpy(next_rhs(k)).pin_memory() for _ in range(a.steps)]
        hx1 = [torch.zeros_like(t).pin_memory() for t in hb1]
        hxk = [torch.zeros_like(t).pin_memory() for t in hbk]
        barrier()
        t0 = time.perf_counter()
        for i in range(a.steps):
            step(i, hb1[i], hx1[i], hbk[i], hxk[i], False)
        barrier()
        e2e_s = time.perf_counter() - t0
        bytes_in = (1 + k) * V * 12 * 16 * 2  # b and the initial guess x
        bytes_out = (1 + k) * V * 12 * 16
        e2e = {"value": world * a.steps * rhs_per_step / e2e_s, "unit": UNIT, "h2d_bytes_per_step": bytes_in,
               "d2h_bytes_per_step": bytes_out}

    # --- what each part of the method buys on this GPU (one call each, synchronised) ----
    def timed(fn):
        torch.cuda.synchronize()
        t0_ = time.perf_counter()
        out_ = fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t0_, out_

    arms = {}
    if not a.no_plain:
        bk, xk0 = Bk[0], torch.zeros_like(Bk[0])
        dt, sts = timed(lambda: op.initcg_solve(bk, xk0, a.tol, a.restart_tol, basis=basis, k=k))
        arms[f"deflated_initcg_fp32_k{k}"] = {"value": k / dt, "unit": UNIT,
                                              "iters_mean": float(np.mean([q["iters"] for q in sts]))}
        xk0 = torch.zeros_like(Bk[0])
        dt, sts = timed(lambda: op.initcg_solve(bk, xk0, a.tol, k=k, max_iter=20000))
        arms[f"plain_cg_fp32_k{k}"] = {"value": k / dt, "unit": UNIT,
                                       "iters_mean": float(np.mean([q["iters"] for q in sts]))}
        b1, x10 = B1[0], torch.zeros_like(B1[0])
        dt, sts = timed(lambda: op.initcg_solve(b1, x10, a.tol, k=1, max_iter=20000))
        arms["plain_cg_fp32_k1"] = {"value": 1 / dt, "unit": UNIT, "iters_mean": float(sts[0]["iters"])}
        x10 = torch.zeros_like(B1[0])
        dt, sts = timed(lambda: op.initcg_solve(b1, x10, a.tol, a.restart_tol, basis=basis, k=1))
        arms["deflated_initcg_fp32_k1"] = {"value": 1 / dt, "unit": UNIT, "iters_mean": float(sts[0]["iters"])}

    # --- the odd-even form (Sec. 5's operator): M x = b through the odd-site Schur complement,
    # Incremental eigCG to the same basis size on A_hat = M_hat^H M_hat, then a k-RHS init-CG
    if not a.no_plain and not a.no_eo:
        op_eo = Op(gauge, dims, m_q, prec=a.prec, max_rhs=k, compress12=a.links == 12,
                   reliable_delta=a.reliable_delta, even_odd=True)
        basis_eo = Basis(op_eo, a.basis + a.nev)
        t0 = time.perf_counter()
        grow_iters = []
        while basis_eo.size + a.nev <= a.basis:
            b = torch.from_numpy(next_rhs(1)[0]).to(dev)
            st = op_eo.eigcg_solve(b, torch.zeros_like(b), a.nev, a.m, a.tol, basis=basis_eo)
            basis_eo.grow()
            grow_iters.append(st["iters"])
        setup_eo = time.perf_counter() - t0
        bk = torch.from_numpy(next_rhs(k)).to(dev)
        xk0 = torch.zeros_like(bk)
        dt, sts = timed(lambda: op_eo.initcg_solve(bk, xk0, a.tol, a.restart_tol, basis=basis_eo, k=k))
        arms[f"eo_deflated_initcg_fp32_k{k}"] = {
            "value": k / dt, "unit": UNIT, "iters_mean": float(np.mean([q["iters"] for q in sts])),
            "max_true_rel_res": float(max(q["true_rel_res"] for q in sts)), "basis": basis_eo.size,
            "setup_s": setup_eo, "eigcg_iters_first_last": [grow_iters[0], grow_iters[-1]] if grow_iters else None,
            "system": "M x = b on the full lattice, solved through the odd-site Schur complement "
                      "(CG on M_hat^H M_hat, residual of those normal equations <= tol)"}
        xk0 = torch.zeros_like(bk)
        dt, sts = timed(lambda: op_eo.initcg_solve(bk, xk0, a.tol, k=k, max_iter=20000))
        arms[f"eo_plain_cg_fp32_k{k}"] = {"value": k / dt, "unit": UNIT,
                                          "iters_mean": float(np.mean([q["iters"] for q in sts]))}
        basis_eo.close()
        op_eo.close()

    # --- serving: Poisson single-RHS requests on this operator and basis --------------
    serve = None
    if not a.no_serve and rank == 0 and arms:
        from paper_0707_0131_gb300 import serving

        spec = serving.OpSpec(key=a.lattice, dims=dims, m_q=m_q, gauge=gauge, prec=a.prec, max_rhs=k, nev=a.nev,
                              m=a.m, basis_max=l0, tol=a.tol, restart_tol=a.restart_tol, prebuilt=(op, basis))
        srv = serving.Server([spec], hbm_budget_bytes=a.budget_gb * 1e9)
        cap = arms[f"deflated_initcg_fp32_k{k}"]["value"]
        rate = 0.8 * cap
        arrivals = serving.poisson_arrivals(rate, a.serve_requests, 105)
        reqs = [next_rhs(1)[0].reshape(-1) for _ in range(a.serve_requests)]
        futs = []
        t0 = time.perf_counter()
        for i, ta in enumerate(arrivals):
            now = time.perf_counter() - t0
            if ta > now:
                time.sleep(ta - now)
            futs.append(srv.submit(spec.key, reqs[i]))
        res = [f.result() for f in futs]
        wall = time.perf_counter() - t0
        pct = srv.percentiles()
        serve = {"value": len(res) / wall, "unit": UNIT, "p50_ms": pct["p50_ms"], "p99_ms": pct["p99_ms"],
                 "requests": len(res), "arrival_rate_per_s": rate,
                 "capacity_per_s": cap, "batch_histogram": srv.batch_histogram(),
                 "max_true_rel_res": float(max(r["stats"]["true_rel_res"] for r in res)),
                 "workload": f"Poisson arrivals at 0.8 x the k={k} deflated init-CG rate, one RHS per request, "
                             f"continuous batching into init-CG calls of <= {k} RHS on the resident {l0}-vector basis"}
        srv.close()

    # --- plain FP64 eigCG on the same GPU ---------------------------------------------
    plain = None
    if not a.no_plain:
        op64 = Op(gauge, dims, m_q, prec=64)
        b = B1[0]
        x = torch.zeros_like(b)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = op64.eigcg_solve(b, x, a.nev, a.m, a.tol, max_iter=20000)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        plain = {"value": 1.0 / dt, "unit": UNIT, "iters": st["iters"], "true_rel_res": st["true_rel_res"]}
        op64.close()

    # --- CPU oracle on a bounded sample ------------------------------------------------
    cpu = None
    all_iters = iters["eigcg"] + iters["initcg"]
    mean_iters = float(np.mean(all_iters))
    if not a.no_cpu and rank == 0:
        t_it, n, cores = oracle_rate(dims, m_q, gauge, a.cpu_seconds)
        cpu = {"value": 1.0 / (t_it * mean_iters), "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{n} FP64 oracle CG iterations on one RHS of this workload ({t_it:.3f} s each); "
                         f"RHS/s = 1/(s per iteration x {mean_iters:.0f} mean iterations per RHS of the timed steps)"}

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
               "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": {"workload": f"{a.lattice} Wilson, m_q={m_q} ({mass_src}, cond(A)~{a.kappa}), "
                                      f"per step 1 eigCG({a.nev},{a.m}) + grow + k={k} batched init-CG, "
                                      f"basis {l0} FP32 vectors, tol {a.tol}, restart {a.restart_tol}",
                          "lattice": a.lattice, "k": k, "basis": l0, "storage": ("fp32 spinors, fp32 links (12- and 18-real resident, chosen per k by the autotuner), " if a.prec == 32 else
                                     "fp16 spinors with one fp32 scale per site and RHS, fp32 12-real links, fp32 eigCG window and basis, ") +
                          f"double-float residual replacements (delta {a.reliable_delta}), fp64 final residual", "l2": "inputs larger than L2 (each field >= 85 MB)",
                          "parallelism": f"replicas{world}"},
               "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
               "clocks": clk, "p50_ms": serve["p50_ms"] if serve else None,
               "p99_ms": serve["p99_ms"] if serve else None, "serving": serve, "arms": arms, "alu_peaks": alu,
               "plain_fp64_eigcg": plain,
               "vs_plain_fp64_eigcg": (value / world / plain["value"]) if plain else None,
               "iters_per_rhs": {"eigcg_mean": float(np.mean(iters["eigcg"])),
                                 "initcg_mean": float(np.mean(iters["initcg"])),
                                 "phase1_first": phase1[0] if phase1 else None, "phase1_last": phase1[-1] if phase1 else None},
               "max_true_rel_res": float(np.max(status["true_res"])), "setup_s": setup_s, "kernels": kernels}
        print(json.dumps(out), flush=True)
    basis.close()
    op.close()
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
