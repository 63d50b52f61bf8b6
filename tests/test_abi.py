"""C ABI checks that need no GPU: the library builds, loads and exports every
function include/sl1m.h declares; the binding declares the same set, raises
without the library, and refuses arrays of the wrong length; the package and
the oracle share no code."""
import ctypes
import os
import re

import numpy as np
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


class _FakeLib:
    """Stands in for libsl1m: records the calls, returns OK."""

    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        def f(*args):
            self.calls.append(name)
            return 0
        return f


class _FakeCtx:
    h = 1

    def __init__(self, lib):
        self.lib = lib

    def check(self, st):
        assert st == 0


class _FakeTensor:
    def __init__(self, n, dtype="torch.float64"):
        self.n, self.dtype, self.is_cuda = n, dtype, True

    def numel(self):
        return self.n

    def is_contiguous(self):
        return True

    def data_ptr(self):
        return 4096


def _fake_problem(n_vis, n_pix):
    from paper_1310_2078_gb300 import sl1m
    lib = _FakeLib()
    P = sl1m.Problem.__new__(sl1m.Problem)
    P.ctx, P.lib, P.h, P.n_vis, P.n_pix = _FakeCtx(lib), lib, 1, n_vis, n_pix
    return P, lib


def test_binding_refuses_arrays_of_the_wrong_length():
    """The library reads host and device arrays without a size argument: the
    binding checks every length against the problem before the call, and
    passes arrays of the right length through."""
    P, lib = _fake_problem(5, 3)
    bad = [lambda: P.forward(np.zeros(4)), lambda: P.adjoint(np.zeros(6, complex)),
           lambda: P.set_vis_data(np.zeros(4, complex)), lambda: P.solve(1.0, x0=np.zeros(2)),
           lambda: P.set_gains(np.ones((4, 2), complex)), lambda: P.set_gains(np.ones(3, complex)),
           lambda: P.set_pixels(np.zeros((3, 2)), sigma=np.zeros(2)),
           lambda: P.set_pixels(np.zeros((3, 2)), kind=np.zeros(4)),
           lambda: P.set_visibilities(np.zeros((5, 3)), weights=np.ones(4)),
           lambda: P.set_visibilities(np.zeros((5, 3)), vis=np.zeros(4, complex)),
           lambda: P.set_visibilities(np.zeros((5, 3)), ant_pair=np.zeros((4, 2))),
           lambda: P.forward_dev(_FakeTensor(4), _FakeTensor(10)),
           lambda: P.forward_dev(_FakeTensor(3), _FakeTensor(9)),
           lambda: P.forward_dev(_FakeTensor(3, "torch.float32"), _FakeTensor(10)),
           lambda: P.forward_noalloc(_FakeTensor(3), _FakeTensor(8)),
           lambda: P.adjoint_dev(_FakeTensor(10), _FakeTensor(2))]
    for call in bad:
        with pytest.raises(ValueError):
            call()
    assert lib.calls == []
    P.forward(np.zeros(3))
    P.adjoint(np.zeros(5, complex))
    P.set_vis_data(np.zeros(5, complex))
    P.solve(1.0, x0=np.zeros(3))
    P.set_gains(np.ones((3, 2), complex))
    P.forward_dev(_FakeTensor(3), _FakeTensor(10))
    P.forward_noalloc(_FakeTensor(3), _FakeTensor(10))
    P.adjoint_dev(_FakeTensor(10), _FakeTensor(3))
    P.set_pixels(np.zeros((4, 2)), sigma=np.zeros(4), kind=np.zeros(4))
    P.set_visibilities(np.zeros((6, 3)), np.zeros(6, complex), np.ones(6), np.zeros((6, 2)))
    assert lib.calls == ["sl1m_forward", "sl1m_adjoint", "sl1m_set_vis_data", "sl1m_solve", "sl1m_set_gains",
                         "sl1m_forward_dev", "sl1m_forward_noalloc", "sl1m_adjoint_dev", "sl1m_set_pixels",
                         "sl1m_set_visibilities"]
    # with a side not set yet the call goes through: the library reports the missing data
    Q, qlib = _fake_problem(0, 0)
    Q.forward(np.zeros(1))
    assert qlib.calls == ["sl1m_forward"]
