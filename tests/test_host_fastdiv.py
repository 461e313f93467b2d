"""The stencil's division by the lattice extents (multiply-high and shift with
host-computed magic numbers, Granlund-Montgomery) against exact integer division.

The stencil divides site indices (< V <= 2^27) by Lx, Ly, Lz (2..4096).  Checked
exhaustively for every n below 2^20 and for all n in windows at the top of the
31-bit range and around every multiple of d near 2^27, for every extent 2..64 and
the larger ones the lattices use; the host build of the same header is called
through a g++ shim (no GPU)."""
import ctypes
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_0707_0131_gb300", "csrc")
OUT = os.path.join(ROOT, "tests", "shim", "_build")


@pytest.fixture(scope="module")
def lib():
    os.makedirs(OUT, exist_ok=True)
    so = os.path.join(OUT, "libfastdiv_shim.so")
    srcs = [os.path.join(ROOT, "tests", "shim", "fastdiv_shim.cpp"), os.path.join(CSRC, "fastdiv.h")]
    if not os.path.exists(so) or any(os.path.getmtime(s) > os.path.getmtime(so) for s in srcs):
        subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-o", so, srcs[0]], check=True)
    L = ctypes.CDLL(so)
    U = ctypes.c_uint
    L.fd_make.argtypes = [U, ctypes.POINTER(U), ctypes.POINTER(U)]
    L.fd_div.argtypes = [U, U]
    L.fd_div.restype = U
    L.fd_check_range.argtypes = [U, U, U]
    L.fd_check_range.restype = ctypes.c_long
    return L


DIVISORS = list(range(2, 65)) + [96, 100, 127, 128, 129, 255, 256, 1000, 1023, 1024, 1025, 4095, 4096]


@pytest.mark.parametrize("d", DIVISORS)
def test_fastdiv_exact(lib, d):
    m, sh = ctypes.c_uint(), ctypes.c_uint()
    lib.fd_make(d, ctypes.byref(m), ctypes.byref(sh))
    assert 0 < m.value < 2**32
    assert lib.fd_check_range(d, 0, 1 << 20) == 0
    top = (1 << 31)
    assert lib.fd_check_range(d, top - (1 << 16), top) == 0
    for c in range(((1 << 27) // d) - 3, ((1 << 27) // d) + 3):
        lo = max(0, c * d - 2)
        assert lib.fd_check_range(d, lo, lo + 5) == 0
    assert lib.fd_div(2**31 - 1, d) == (2**31 - 1) // d
