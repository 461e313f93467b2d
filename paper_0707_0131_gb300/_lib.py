"""ctypes binding of libeigcg.so (include/eigcg.h).  Argument marshalling only.

Vector arguments may be numpy complex128 arrays (host memory) or torch
complex128 CUDA tensors (device memory); both are passed as raw pointers and the
library detects which is which.  The library must be built (build.py); nothing
here falls back to another implementation: if libeigcg.so cannot be loaded the
import of the functions below raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

EIG_OK = 0
EIG_NOT_CONVERGED = 1
EIG_ERR_ARG = -1
EIG_ERR_OOM = -2
EIG_ERR_BUDGET = -3
EIG_ERR_CUDA = -4
EIG_ERR_BREAKDOWN = -5
EIG_ERR_TIMEOUT = -6
EIG_ERR_IO = -7

PREC = {"f64": 64, "f32": 32, "f16": 16, 64: 64, 32: 32, 16: 16}


class EigError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"eig status {status}: {msg}")
        self.status = status


class OpOpts(ctypes.Structure):
    _fields_ = [("spinor_prec", ctypes.c_int), ("link_compress12", ctypes.c_int), ("max_rhs", ctypes.c_int),
                ("reliable_delta", ctypes.c_double), ("even_odd", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("restarts", ctypes.c_int), ("reliable_updates", ctypes.c_int),
                ("converged", ctypes.c_int), ("true_rel_res", ctypes.c_double), ("ms", ctypes.c_double),
                ("n_ritz", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 40), ("launches", ctypes.c_long), ("ms", ctypes.c_double),
                ("bytes", ctypes.c_double)]


# every symbol declared in include/eigcg.h, with its ctypes signature
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
SIGNATURES = {
    "eig_op_create": [_P, _P, _D, _P, _P],
    "eig_op_destroy": [_P],
    "eig_op_apply": [_P, _I, _P, _P, _I, _P],
    "eig_op_stencil_choice": [_P, _I, _P, _P],
    "eig_basis_create": [_P, _I, _P],
    "eig_basis_destroy": [_P],
    "eig_basis_size": [_P, _P],
    "eig_basis_truncate": [_P, _I],
    "eig_eigcg_solve": [_P, _P, _P, _P, _I, _I, _D, _I, _P, _P],
    "eig_eigcg_solve_sp": [_P, _P, _P, _P, _I, _I, _D, _I, _I, _D, _P, _P],
    "eig_basis_grow": [_P, _P],
    "eig_basis_deflate": [_P, _P, _P, _P, _I, _P],
    "eig_bicgstab_solve": [_P, _P, _P, _P, _D, _I, _I, _P, _P],
    "eig_initcg_solve": [_P, _P, _P, _P, _D, _D, _I, _I, _P, _P],
    "eig_basis_ritz": [_P, _P, _P, _P, _P],
    "eig_basis_vector": [_P, _I, _P, _P],
    "eig_basis_h": [_P, _P],
    "eig_basis_pending": [_P, _P, _P],
    "eig_basis_save": [_P, ctypes.c_char_p, _P],
    "eig_basis_load": [_P, ctypes.c_char_p, _P],
    "eig_profile_enable": [_I],
    "eig_profile_reset": [],
    "eig_profile_read": [_P, _I, _P],
    "eig_op_trim": [_P, _P],
    "eig_profile_alu_peak": [_I, _P, _P],
    "eig_wilson_apply_noalloc": [_P, _P, _D, _I, _P, _P, _P],
    "eig_last_error": [],
}

_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Loads libeigcg.so (building it first if it is missing and nvcc exists)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing:
            _build.build()
        if not os.path.exists(_build.LIB):
            raise ImportError("libeigcg.so is not built; run paper_0707_0131_gb300.build.build()")
        L = ctypes.CDLL(_build.LIB)
        for name, args in SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_char_p if name == "eig_last_error" else ctypes.c_int
        _lib = L
    return _lib


def _ptr(a) -> int:
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.complex128 or not a.flags["C_CONTIGUOUS"]:
            raise TypeError("host vectors must be C-contiguous complex128 numpy arrays")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):  # torch tensor
        import torch

        if a.dtype != torch.complex128 or not a.is_contiguous():
            raise TypeError("device vectors must be contiguous complex128 torch tensors")
        return a.data_ptr()
    if isinstance(a, int):
        return a
    raise TypeError(f"unsupported vector type {type(a)}")


def _check(status: int) -> int:
    if status < 0:
        raise EigError(status, load().eig_last_error().decode())
    return status


def _stream(stream) -> int:
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


# ------------------------------------------------------------------------------------------
# functions with the C names
# ------------------------------------------------------------------------------------------
def eig_op_create(gauge: np.ndarray, dims, m_q: float, spinor_prec=64, link_compress12=1, max_rhs=1,
                  reliable_delta=0.1, even_odd=0) -> ctypes.c_void_p:
    g = np.ascontiguousarray(gauge, dtype=np.complex128)
    d = (ctypes.c_int * 4)(*[int(v) for v in dims])
    opts = OpOpts(PREC[spinor_prec], int(link_compress12), int(max_rhs), float(reliable_delta), int(even_odd))
    h = ctypes.c_void_p()
    _check(load().eig_op_create(g.ctypes.data, d, float(m_q), ctypes.byref(opts), ctypes.byref(h)))
    return h


def eig_op_destroy(op) -> None:
    _check(load().eig_op_destroy(op))


def eig_op_apply(op, which: int, vin, vout, k: int = 1, stream=None) -> None:
    _check(load().eig_op_apply(op, int(which), _ptr(vin), _ptr(vout), int(k), _stream(stream)))


def eig_op_stencil_choice(op, k: int = 1):
    """(variant, link_reals) the stencil autotuner chose for k-RHS products; (-1, 0)
    for FP64 ops or before the first solve with k RHS."""
    v, g = ctypes.c_int(), ctypes.c_int()
    _check(load().eig_op_stencil_choice(op, int(k), ctypes.byref(v), ctypes.byref(g)))
    return v.value, g.value


def eig_basis_create(op, max_vecs: int) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load().eig_basis_create(op, int(max_vecs), ctypes.byref(h)))
    return h


def eig_basis_destroy(basis) -> None:
    _check(load().eig_basis_destroy(basis))


def eig_basis_size(basis) -> int:
    n = ctypes.c_int()
    _check(load().eig_basis_size(basis, ctypes.byref(n)))
    return n.value


def eig_basis_truncate(basis, l: int) -> None:
    _check(load().eig_basis_truncate(basis, int(l)))


def eig_eigcg_solve(op, basis, b, x, nev: int, m: int, tol: float, max_iter: int = 100000, stream=None):
    st = Stats()
    status = _check(load().eig_eigcg_solve(op, basis, _ptr(b), _ptr(x), int(nev), int(m), float(tol),
                                           int(max_iter), ctypes.byref(st), _stream(stream)))
    d = st.as_dict()
    d["status"] = status
    return d


def eig_eigcg_solve_sp(op, basis, b, x, nev: int, m: int, tol: float, sp_vecs: int, sp_shift: float,
                       max_iter: int = 100000, stream=None):
    st = Stats()
    status = _check(load().eig_eigcg_solve_sp(op, basis, _ptr(b), _ptr(x), int(nev), int(m), float(tol),
                                              int(max_iter), int(sp_vecs), float(sp_shift), ctypes.byref(st),
                                              _stream(stream)))
    d = st.as_dict()
    d["status"] = status
    return d


def eig_bicgstab_solve(op, basis, b, x, tol: float, max_iter: int = 100000, defl_vecs: int = 0, stream=None):
    st = Stats()
    status = _check(load().eig_bicgstab_solve(op, basis, _ptr(b), _ptr(x), float(tol), int(max_iter),
                                              int(defl_vecs), ctypes.byref(st), _stream(stream)))
    d = st.as_dict()
    d["status"] = status
    return d


def eig_basis_grow(basis, stream=None) -> None:
    _check(load().eig_basis_grow(basis, _stream(stream)))


def eig_basis_deflate(basis, b, x_in, x0, k: int = 1, stream=None) -> None:
    _check(load().eig_basis_deflate(basis, _ptr(b), _ptr(x_in), _ptr(x0), int(k), _stream(stream)))


def eig_initcg_solve(op, basis, b, x, tol: float, restart_tol: float = 0.0, max_iter: int = 100000, k: int = 1,
                     stream=None):
    st = (Stats * k)()
    status = _check(load().eig_initcg_solve(op, basis, _ptr(b), _ptr(x), float(tol), float(restart_tol),
                                            int(max_iter), int(k), st, _stream(stream)))
    out = [s.as_dict() for s in st]
    for d in out:
        d["status"] = status
    return out


def eig_basis_ritz(basis, residuals: bool = True, stream=None):
    l = eig_basis_size(basis)
    ev = np.zeros(max(l, 1))
    rn = np.zeros(max(l, 1))
    n = ctypes.c_int()
    _check(load().eig_basis_ritz(basis, ev.ctypes.data, rn.ctypes.data if residuals else None, ctypes.byref(n),
                                 _stream(stream)))
    return ev[: n.value], (rn[: n.value] if residuals else None)


def eig_basis_vector(basis, j: int, out, stream=None) -> None:
    _check(load().eig_basis_vector(basis, int(j), _ptr(out), _stream(stream)))


def eig_basis_h(basis) -> np.ndarray:
    l = eig_basis_size(basis)
    out = np.zeros((l, l), dtype=np.complex128)
    _check(load().eig_basis_h(basis, out.ctypes.data))
    return out


def eig_basis_pending(basis) -> np.ndarray:
    n = ctypes.c_int()
    _check(load().eig_basis_pending(basis, None, ctypes.byref(n)))
    ev = np.zeros(n.value)
    _check(load().eig_basis_pending(basis, ev.ctypes.data, ctypes.byref(n)))
    return ev


def eig_basis_save(basis, path, stream=None) -> None:
    _check(load().eig_basis_save(basis, os.fsencode(path), _stream(stream)))


def eig_basis_load(basis, path, stream=None) -> None:
    _check(load().eig_basis_load(basis, os.fsencode(path), _stream(stream)))


def eig_profile_enable(on: bool = True) -> None:
    _check(load().eig_profile_enable(1 if on else 0))


def eig_op_trim(op) -> int:
    """Releases the op's workspace (bases keep their vectors); returns the bytes freed."""
    v = ctypes.c_size_t(0)
    _check(load().eig_op_trim(op, ctypes.byref(v)))
    return int(v.value)


def eig_profile_alu_peak(prec: int, stream=None) -> float:
    """Measured FMA throughput of the GPU in TFLOP/s (prec 64 or 32)."""
    v = ctypes.c_double(0.0)
    _check(load().eig_profile_alu_peak(int(prec), ctypes.byref(v), _stream(stream)))
    return float(v.value)


def eig_profile_reset() -> None:
    _check(load().eig_profile_reset())


def eig_profile_read() -> dict:
    """{kernel name: {"launches", "ms", "bytes"}} (synchronises the device)."""
    n = ctypes.c_int()
    _check(load().eig_profile_read(None, 0, ctypes.byref(n)))
    arr = (KernelStat * max(n.value, 1))()
    _check(load().eig_profile_read(arr, n.value, ctypes.byref(n)))
    return {a.name.decode(): {"launches": a.launches, "ms": a.ms, "bytes": a.bytes} for a in arr[: n.value]}


def eig_wilson_apply_noalloc(gauge, dims, m_q: float, which: int, vin, vout, stream=None) -> None:
    """M, M^H or A on one RHS without any device allocation.  gauge, vin and vout
    are complex128 CUDA tensors in the natural layout (gauge [V][4][3][3], vectors
    [V][4][3]); vin and vout must not overlap.  Asynchronous on `stream`."""
    d = (ctypes.c_int * 4)(*[int(v) for v in dims])
    _check(load().eig_wilson_apply_noalloc(_ptr(gauge), d, float(m_q), int(which), _ptr(vin), _ptr(vout),
                                           _stream(stream)))


def eig_last_error() -> str:
    return load().eig_last_error().decode()
