"""The allocation-free entry point eig_wilson_apply_noalloc against eig_op_apply
and the oracle.

It serves callers that may not allocate device memory (memory owned by another
allocator, a device reserved in full).  Both entry points apply the same FP64
operator; the allocation-free one works on caller-owned device buffers with its
intermediate in a static device array shared by all calls.  Two calls in a row (the
second one finds the first one's data in the array) must each match eig_op_apply
and the FP64 oracle within the FP64 matvec tolerance of the other tests.  Argument
errors are rejected on the host before anything reaches the GPU.
"""
import numpy as np
import pytest

import oracle
from paper_0707_0131_gb300 import _lib
from paper_0707_0131_gb300 import fixtures as fx

TOL64 = 1e-12


def _relerr(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.gpu
@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 2, 10), (16, 16, 16, 16)])
def test_noalloc_matches_op_apply(dims):
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    m_q = -0.1
    gauge = fx.make_gauge(dims, 41)
    op = _lib.eig_op_create(gauge, dims, m_q, spinor_prec=64)
    d_gauge = torch.from_numpy(np.ascontiguousarray(gauge)).cuda()
    V = fx.volume(dims)
    W = oracle.Wilson(dims, m_q, gauge)
    try:
        for call in range(2):
            psi = fx.make_rhs(dims, 42 + call, 1)[0]
            d_in = torch.from_numpy(psi).cuda()
            for which in (2, 0, 1):
                ref = np.empty_like(psi)
                _lib.eig_op_apply(op, which, psi, ref, 1)
                d_out = torch.empty_like(d_in)
                _lib.eig_wilson_apply_noalloc(d_gauge, dims, m_q, which, d_in, d_out)
                torch.cuda.synchronize()
                out = d_out.cpu().numpy()
                assert out.shape == (V, 4, 3)
                err = _relerr(out.reshape(-1), ref.reshape(-1))
                assert err < TOL64, (call, which, err)
                o = (W.M, W.Mdag, W.A)[which](psi.reshape(-1))
                err_o = _relerr(out.reshape(-1), o)
                assert err_o < TOL64, (call, which, err_o)
    finally:
        _lib.eig_op_destroy(op)


@pytest.mark.gpu
def test_noalloc_two_calls_on_a_stream():
    """A on two RHS back to back on one side stream: the second call overwrites the
    shared intermediate only after the first call's kernels have read it."""
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    dims = (8, 8, 8, 8)
    m_q = 0.05
    gauge = fx.make_gauge(dims, 43)
    op = _lib.eig_op_create(gauge, dims, m_q, spinor_prec=64)
    try:
        d_gauge = torch.from_numpy(np.ascontiguousarray(gauge)).cuda()
        psis = fx.make_rhs(dims, 44, 2)
        d_in = [torch.from_numpy(p).cuda() for p in psis]
        d_out = [torch.empty_like(t) for t in d_in]
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        for r in range(2):
            _lib.eig_wilson_apply_noalloc(d_gauge, dims, m_q, 2, d_in[r], d_out[r], stream=s)
        s.synchronize()
        for r in range(2):
            ref = np.empty_like(psis[r])
            _lib.eig_op_apply(op, 2, psis[r], ref, 1)
            assert _relerr(d_out[r].cpu().numpy().reshape(-1), ref.reshape(-1)) < TOL64
    finally:
        _lib.eig_op_destroy(op)


def test_noalloc_rejects_bad_arguments_on_the_host():
    """Checked before any CUDA call: runs without a GPU."""
    dims = (4, 4, 4, 4)
    g = np.zeros((fx.volume(dims), 4, 3, 3), dtype=np.complex128)
    v = np.zeros((fx.volume(dims), 4, 3), dtype=np.complex128)
    with pytest.raises(_lib.EigError) as e:
        _lib.eig_wilson_apply_noalloc(g, dims, 0.1, 3, v, v.copy())
    assert e.value.status == _lib.EIG_ERR_ARG
    with pytest.raises(_lib.EigError) as e:
        _lib.eig_wilson_apply_noalloc(g, (4, 4, 1, 4), 0.1, 0, v, v.copy())
    assert e.value.status == _lib.EIG_ERR_ARG
    for big in ((32, 32, 32, 8), (16, 16, 16, 17)):  # 262144 and 69632 sites > 65536
        with pytest.raises(_lib.EigError) as e:
            _lib.eig_wilson_apply_noalloc(g, big, 0.1, 0, v, v.copy())
        assert e.value.status == _lib.EIG_ERR_BUDGET
        assert "65536" in _lib.eig_last_error()


@pytest.mark.gpu
def test_noalloc_rejects_host_buffers():
    """Host (numpy) buffers are refused before launch: the kernels read their
    arguments directly and would otherwise fault."""
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    dims = (4, 4, 4, 4)
    g = fx.make_gauge(dims, 45)
    v = fx.make_rhs(dims, 46, 1)[0]
    with pytest.raises(_lib.EigError) as e:
        _lib.eig_wilson_apply_noalloc(g, dims, 0.1, 0, v, np.empty_like(v))
    assert e.value.status == _lib.EIG_ERR_ARG
    # device buffers, but out overlapping in or the gauge field: refused before launch
    d_g = torch.from_numpy(np.ascontiguousarray(g)).cuda()
    d_v = torch.from_numpy(v).cuda()
    for out in (d_v, d_g.view(-1)[: v.size].view(v.shape)):
        with pytest.raises(_lib.EigError) as e:
            _lib.eig_wilson_apply_noalloc(d_g, dims, 0.1, 2, d_v, out)
        assert e.value.status == _lib.EIG_ERR_ARG
        assert "overlap" in _lib.eig_last_error()
