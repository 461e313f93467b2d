"""CUDA-graph replay of init-CG's plain CG iterations.

Blocks of 16 iterations (p update, the two stencil passes with their CG epilogues)
are captured once per buffer set and replayed; the kernels read the block's first
iteration index from device memory.  The replayed solve runs the same kernels in
the same order as the eagerly launched one, so solutions, iteration counts and
residuals must be identical bit for bit (EIG_CG_GRAPH=0 switches graphs off).
"""
import os

import numpy as np
import pytest

import oracle
from paper_0707_0131_gb300 import fixtures as fx

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,k", [(64, 1), (32, 4), (16, 2)])
def test_graph_replay_identical(prec, k):
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_0707_0131_gb300 import api

    dims = (8, 8, 8, 8)
    gauge = fx.make_gauge(dims, 61)
    W = oracle.Wilson(dims, 0.02, gauge)
    B = fx.make_rhs(dims, 62, k).reshape(k, -1)
    out = {}
    try:
        for mode in ("0", "1"):
            os.environ["EIG_CG_GRAPH"] = mode
            op = api.Op(gauge, dims, 0.02, prec=prec, max_rhs=k)
            X = np.zeros_like(B)
            st = op.initcg_solve(B, X, tol=1e-9, k=k)
            # a second solve on the same op replays the cached graph
            X2 = np.zeros_like(B)
            st2 = op.initcg_solve(B, X2, tol=1e-9, k=k)
            op.close()
            out[mode] = (X, st, X2, st2)
    finally:
        os.environ.pop("EIG_CG_GRAPH", None)
    X0, st0, _, _ = out["0"]
    X1, st1, X1b, st1b = out["1"]
    assert st0[0]["iters"] > 40  # several replayed blocks
    assert np.array_equal(X0, X1) and np.array_equal(X1, X1b)
    for q in range(k):
        assert st0[q]["iters"] == st1[q]["iters"] == st1b[q]["iters"]
        assert st0[q]["true_rel_res"] == st1[q]["true_rel_res"]
        assert np.linalg.norm(B[q] - W.A(X1[q])) / np.linalg.norm(B[q]) <= 1e-9
