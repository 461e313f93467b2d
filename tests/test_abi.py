"""The C ABI library builds, loads without a GPU and exports every symbol of include/eigcg.h;
the oracle and the CUDA path share no code."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "eigcg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(eig_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["eig_op_create", "eig_eigcg_solve", "eig_basis_grow", "eig_basis_deflate", "eig_initcg_solve"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_0707_0131_gb300 import _lib

    L = _lib.load()
    for n in _declared():
        assert hasattr(L, n), n
        assert n in _lib.SIGNATURES, n
    assert set(_lib.SIGNATURES) == set(_declared())


def test_last_error_is_empty_initially():
    from paper_0707_0131_gb300 import _lib

    assert _lib.load().eig_last_error() in (b"",)


def test_argument_errors_need_no_gpu():
    """Validation happens before any CUDA call: bad sizes return EIG_ERR_ARG."""
    from paper_0707_0131_gb300 import _lib

    L = _lib.load()
    h = ctypes.c_void_p()
    dims = (ctypes.c_int * 4)(1, 4, 4, 4)
    g = (ctypes.c_double * 8)()
    assert L.eig_op_create(ctypes.addressof(g), dims, 0.1, None, ctypes.byref(h)) == _lib.EIG_ERR_ARG
    assert b"extents" in L.eig_last_error()
    assert L.eig_op_apply(None, 0, None, None, 1, None) == _lib.EIG_ERR_ARG


def test_oracle_and_cuda_path_share_no_code():
    pkg = os.path.join(ROOT, "paper_0707_0131_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle", txt, re.M), f
                assert "oracle/" not in txt and "oracle_wilson" not in txt, f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c")):
            txt = open(os.path.join(ROOT, "oracle", f)).read()
            assert "paper_0707_0131_gb300" not in txt, f
            assert "csrc" not in txt, f


def test_header_is_plain_c(tmp_path):
    """include/eigcg.h compiles as C99 and as C++ (no CUDA or torch types in the boundary)."""
    import subprocess

    src = tmp_path / "use.c"
    src.write_text('#include "eigcg.h"\nint main(void) { eig_op op = 0; (void)op; return EIG_OK; }\n')
    inc = os.path.join(ROOT, "include")
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-fsyntax-only", "-I", inc, str(src)], check=True)
    cpp = tmp_path / "use.cpp"
    cpp.write_text(src.read_text())
    subprocess.run(["g++", "-std=c++17", "-Wall", "-Werror", "-fsyntax-only", "-I", inc, str(cpp)], check=True)
