"""Writes configs/masses.json: the quark mass m_q giving a target cond(A), A = M^H M.

The paper's masses are specific to its ensembles (critical mass -0.4188, Sec. 5.1);
the synthetic gauge fields here need their own.  For each lattice (gauge seed
fixed) and each target condition number kappa, m_q is found by secant steps on
log cond(A)(m_q), starting from the model lambda_min ~ (m_q - m_c)^2 fitted at
m_q = 0.  cond(A) comes from the oracle only:
  * 4^4: dense eigensolve of A;
  * larger lattices: extreme Ritz values of the full-history CG-Lanczos
    tridiagonal (Eq. 4) of an oracle CG solve to 1e-11 (Ritz values bound the
    spectrum from inside; the extremes converge well before CG does).

Usage: python configs/calibrate_masses.py [lattice ...]   (default: all)
It merges into an existing masses.json, so lattices can be run separately.
"""
from __future__ import annotations

import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from oracle import solvers  # noqa: E402
from paper_0707_0131_gb300 import fixtures as fx  # noqa: E402

OUT = os.path.join(ROOT, "configs", "masses.json")
TARGETS = {"4^4": [1e3], "8^4": [1e3, 1e4, 1e5], "16^3x32": [1e3, 1e4, 1e5], "24^3x64": [1e5]}


def spectrum_extremes(name, gauge, m):
    dims = fx.LATTICES[name]
    W = oracle.Wilson(dims, m, gauge)
    if name == "4^4":
        ev = np.linalg.eigvalsh(W.dense("A"))
        return float(ev[0]), float(ev[-1])
    b = fx.make_rhs(dims, fx.rhs_seed(name, 0))[0]
    res = solvers.cg(W, b, tol=1e-11, max_iter=20000)
    T = solvers.lanczos_tridiagonal(res["alphas"], res["betas"], res["iters"])
    ev = np.linalg.eigvalsh(T)
    return float(ev[0]), float(ev[-1])


def calibrate(name, targets):
    dims = fx.LATTICES[name]
    gauge = fx.make_gauge(dims, fx.GAUGE_SEEDS[name])
    lo0, hi0 = spectrum_extremes(name, gauge, 0.0)
    # model: sqrt(lambda_min) = (m - m_c) with unit slope
    m_c = -math.sqrt(lo0)
    out = {}
    for kappa in targets:
        m = m_c + math.sqrt(hi0 / kappa)
        hist = []
        for _ in range(6):
            lo, hi = spectrum_extremes(name, gauge, m)
            k = hi / lo
            hist.append((m, k))
            print(f"{name} target {kappa:.0e}: m={m:.6f} cond={k:.4g}", flush=True)
            if abs(math.log(k / kappa)) < math.log(1.05):
                break
            # secant in sqrt(lambda_min) ~ (m - m_c): re-fit m_c from this point
            m_c = m - math.sqrt(lo)
            m = m_c + math.sqrt(hi / kappa)
        m_best, k_best = min(hist, key=lambda mk: abs(math.log(mk[1] / kappa)))
        out[f"{kappa:.0e}"] = {"m_q": round(m_best, 6), "cond": float(f"{k_best:.4g}")}
    return out


def main(names):
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            data = json.load(f)
    for name in names:
        t = time.time()
        entry = calibrate(name, TARGETS[name])
        entry["gauge_seed"] = fx.GAUGE_SEEDS[name]
        entry["eps"] = 0.3
        data[name] = entry
        print(f"{name}: {entry} ({time.time() - t:.0f} s)", flush=True)
        with open(OUT, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:] or list(TARGETS))
