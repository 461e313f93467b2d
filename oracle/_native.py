"""ORACLE -- test infrastructure only.  Builds and loads the plain-C oracle library.

Compiles oracle/wilson.c with gcc (-O2, OpenMP, IEEE semantics: no fast-math)
into oracle/_build/liboracle_wilson.so the first time it is needed, or when the
source is newer than the library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wilson.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle_wilson.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle's C code; returns the library path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    stale = force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
    if stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            P = ctypes.c_void_p
            L.oracle_wilson_m.argtypes = [P, ctypes.c_double, P, P, P]
            L.oracle_wilson_mdag.argtypes = [P, ctypes.c_double, P, P, P, P]
            L.oracle_wilson_a.argtypes = [P, ctypes.c_double, P, P, P, P]
            L.oracle_get_gammas.argtypes = [P]
            L.oracle_num_threads.restype = ctypes.c_int
            _lib = L
    return _lib
