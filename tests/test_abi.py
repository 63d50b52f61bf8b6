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
