"""C ABI checks that need no GPU: the library builds, loads and exports every
function include/sl1m.h declares; the binding declares the same set."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(sl1m_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib_path():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1310_2078_gb300 import sl1m
    return sl1m.LIB_PATH


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    names = declared_functions()
    assert len(names) >= 20
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header(lib_path):
    from paper_1310_2078_gb300 import sl1m
    assert set(sl1m.EXPORTS) == declared_functions()
    lib = sl1m.load()
    assert lib.sl1m_version() >= 100
    assert lib.sl1m_status_string(0) == b"ok"
    assert lib.sl1m_status_string(4) == b"non-finite value"


def test_null_arguments_are_rejected_without_gpu(lib_path):
    from paper_1310_2078_gb300 import sl1m
    lib = sl1m.load()
    assert lib.sl1m_create(None, 0, None) == sl1m.ERR_ARG
    assert lib.sl1m_destroy(None) == sl1m.ERR_ARG
    assert lib.sl1m_problem_destroy(None) == sl1m.ERR_ARG
    assert lib.sl1m_forward(None, None, None, 1) == sl1m.ERR_ARG
    assert lib.sl1m_solve(None, None, None, None) == sl1m.ERR_ARG


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    """No CPU fallback: without libsl1m.so the binding raises, both when
    loading and when a context is created."""
    from paper_1310_2078_gb300 import sl1m
    monkeypatch.setattr(sl1m, "_lib", None)
    monkeypatch.setattr(sl1m, "LIB_PATH", str(tmp_path / "libsl1m.so"))
    with pytest.raises(RuntimeError, match="not found"):
        sl1m.load()
    with pytest.raises(RuntimeError, match="not found"):
        sl1m.Context(0)


def _sources(top, exts):
    for dirpath, dirs, files in os.walk(top):
        dirs[:] = [d for d in dirs if d not in ("_build", "__pycache__")]
        for f in files:
            if f.endswith(exts):
                yield os.path.join(dirpath, f)


def test_product_and_oracle_share_nothing():
    """The package (Python, C++ and CUDA) never imports, includes or loads the
    oracle, and the oracle never touches the package or its headers."""
    pkg = os.path.join(ROOT, "paper_1310_2078_gb300")
    exts = (".py", ".cu", ".cuh", ".cpp", ".h", ".c")
    for path in _sources(pkg, exts):
        txt = open(path).read()
        assert not re.search(r"^\s*(import|from)\s+oracle\b|sl1m_oracle|orc_[a-z]+\(", txt, re.M), path
    for path in _sources(os.path.join(ROOT, "oracle"), exts):
        txt = open(path).read()
        assert not re.search(r"^\s*(import|from)\s+paper_1310_2078_gb300|^\s*#include\s+\"sl1m|"
                             r"CDLL\([^)]*libsl1m\.so|\bsl1m_[a-z_]+\(", txt, re.M), path
