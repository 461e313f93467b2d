"""Every variant of the FP32-arithmetic stencil against the oracle.

The library picks the fastest of the stencil variants (staged or direct loads, one or two
RHS per thread, register budgets, L1 prefetch, lexicographic or tiled site traversal:
variants 8 + v, tiled on 8^4 and untiled on the ragged lattice; the pipelined-pair
variants 16-21 with 256-bit loads, k >= 2 only) per lattice and k;
EIG_DSLASH_VARIANT forces one
for the whole process (EIG_DSLASH_LINKS the FP32 link format: 12 or 18 reals), so
each variant runs in a subprocess of its own.  Each one
must meet the FP32 (1e-6) and FP16 (5e-3) matvec bars of test_gpu_dslash.py for M,
M^H and A, on a lattice with a ragged last block and on 8^4, with k = 1 and 4, and
with the CG epilogue (an init-CG solve reaching 1e-8 in mixed precision); the op
reports the forced variant and link form as its choice.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

CHILD = r"""
import numpy as np, oracle
from paper_0707_0131_gb300 import api, fixtures as fx
TOL = {32: 1e-6, 16: 5e-3}
for dims in [(6, 4, 2, 10), (8, 8, 8, 8)]:
    gauge = fx.make_gauge(dims, 51)
    W = oracle.Wilson(dims, -0.1, gauge)
    for prec in (32, 16):
        for k in (1, 4):
            op = api.Op(gauge, dims, -0.1, prec=prec, max_rhs=k)
            psi = fx.make_rhs(dims, 52, k)
            for which, f in [(0, W.M), (1, W.Mdag), (2, W.A)]:
                out = np.empty_like(psi)
                op.apply(which, psi, out, k)
                for r in range(k):
                    ref = f(psi[r])
                    err = np.linalg.norm(out[r].reshape(-1) - ref) / np.linalg.norm(ref)
                    assert err < TOL[prec], (dims, prec, k, which, r, err)
            op.close()
dims = (8, 8, 8, 8)
gauge = fx.make_gauge(dims, 53)
W = oracle.Wilson(dims, 0.05, gauge)
op = api.Op(gauge, dims, 0.05, prec=32, max_rhs=4)
B = fx.make_rhs(dims, 54, 4).reshape(4, -1)
X = np.zeros_like(B)
st = op.initcg_solve(B, X, tol=1e-8, k=4)
for r in range(4):
    assert np.linalg.norm(B[r] - W.A(X[r])) / np.linalg.norm(B[r]) <= 1e-8, (r, st[r])
# the reported choice is the forced one
import os
v, g = op.stencil_choice(4)
assert v == int(os.environ["EIG_DSLASH_VARIANT"]), v
assert g == int(os.environ.get("EIG_DSLASH_LINKS", "0")) or (g in (12, 18) and "EIG_DSLASH_LINKS" not in os.environ), g
op.close()
print("variant ok")
"""


@pytest.mark.parametrize("variant,links", [(v, None) for v in range(8)] + [(v, "18") for v in (2, 4, 6)]
                         + [(v, None) for v in (10, 12, 14, 15)] + [(14, "18")]
                         + [(v, None) for v in (16, 17, 18, 19, 20, 21)] + [(16, "18"), (18, "18"), (21, "18")])
def test_variant_parity(variant, links):
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    env = dict(os.environ, EIG_DSLASH_VARIANT=str(variant))
    if links:
        env["EIG_DSLASH_LINKS"] = links  # FP32 ops: 12- or 18-real links
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    p = subprocess.run([sys.executable, "-c", CHILD], env=env, cwd=root, capture_output=True, text=True,
                       timeout=600)
    assert p.returncode == 0 and "variant ok" in p.stdout, p.stdout[-2000:] + p.stderr[-4000:]


def test_stencil_choice_reported():
    """FP64 ops and untuned shapes report no choice; after a solve the autotuner's pick
    is one of the variants valid for the batch width."""
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_0707_0131_gb300 import api, fixtures as fx

    dims = (4, 6, 4, 8)
    gauge = fx.make_gauge(dims, 55)
    op64 = api.Op(gauge, dims, 0.1, prec=64, max_rhs=2)
    assert op64.stencil_choice(2) == (-1, 0)
    op64.close()
    op = api.Op(gauge, dims, 0.1, prec=32, max_rhs=2)
    assert op.stencil_choice(2) == (-1, 0)
    B = fx.make_rhs(dims, 56, 2).reshape(2, -1)
    X = np.zeros_like(B)
    op.initcg_solve(B, X, tol=1e-6, k=2)
    v, g = op.stencil_choice(2)
    assert 0 <= v <= 21 and g in (12, 18), (v, g)
    v1, g1 = op.stencil_choice(1)
    assert (v1, g1) == (-1, 0)  # k = 1 not solved yet
    with pytest.raises(Exception):
        op.stencil_choice(3)
    op.close()
