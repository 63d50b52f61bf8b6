"""FP64 CPU oracle for the SL1M hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product (the CUDA library
``libsl1m`` and its binding ``paper_1310_2078_gb300``) never imports, links or
calls it, and this package imports nothing from the product.

The arithmetic lives in ``sl1m_oracle.c`` (plain C99, FP64, single-threaded
unless a Problem asks for threads over its outer loops);
this module only compiles it with gcc and marshals numpy arrays through
ctypes.  Every function cites the passage of Hardy (2013) it follows:

* :func:`entry`    -- operator entry, Eq. deltam / Eq. samlm4 / Eq. samlm5
* :func:`forward`  -- Vhat = A x, Eq. sme
* :func:`adjoint`  -- Re(A^H r), the back-projection of Sect. 3
* :func:`power`    -- L = largest eigenvalue of Re(A^H W A), Sect. 3.1
* :func:`fista`    -- the FISTA box of Sect. 3 with Eq. threshp
* :func:`mfista`   -- the monotone FISTA that Sect. 3 names (Beck & Teboulle 2009b)
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

DIRAC, GAUSS_PARAXIAL, GAUSS_WIDE = 0, 1, 2

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sl1m_oracle.c")
_LIB = os.path.join(_HERE, "libsl1m_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library in place (plain gcc, no -ffast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-std=c99", "-O2", "-fno-fast-math", "-ffp-contract=off", "-pthread",
             "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Problem(C.Structure):
    _fields_ = [
        ("n_vis", C.c_long), ("uvw", C.c_void_p), ("weights", C.c_void_p),
        ("ant_pair", C.c_void_p),
        ("n_pix", C.c_long), ("lm", C.c_void_p), ("sigma", C.c_void_p),
        ("kind", C.c_void_p),
        ("n_ant", C.c_int), ("gains", C.c_void_p), ("n_threads", C.c_int),
    ]


class Stats(C.Structure):
    _fields_ = [
        ("iters", C.c_int), ("converged", C.c_int), ("E", C.c_double),
        ("E_paper", C.c_double), ("resid2", C.c_double), ("l1", C.c_double),
        ("nnz", C.c_long), ("t_final", C.c_double),
    ]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.POINTER(_Problem)
            d = C.POINTER(C.c_double)
            lp = C.POINTER(C.c_long)
            lib.orc_entry.argtypes = [C.c_int] + [C.c_double] * 6 + [d]
            lib.orc_entry_kj.argtypes = [P, C.c_long, C.c_long, d]
            lib.orc_forward_rows.argtypes = [P, d, C.c_long, lp, d]
            lib.orc_adjoint_cols.argtypes = [P, d, C.c_long, lp, d]
            lib.orc_power.argtypes = [P, C.c_int, C.c_double, d, C.POINTER(C.c_int)]
            lib.orc_fista.argtypes = [P, d, C.c_double, C.c_double, C.c_int,
                                      C.c_double, d, d, C.POINTER(Stats)]
            lib.orc_mfista.argtypes = [P, d, C.c_double, C.c_double, C.c_int,
                                       C.c_double, d, d, C.POINTER(Stats), d]
            for f in ("orc_entry", "orc_entry_kj", "orc_forward_rows",
                      "orc_adjoint_cols", "orc_power", "orc_fista", "orc_mfista"):
                getattr(lib, f).restype = C.c_int
            _lib = lib
    return _lib


def _f64(a, shape=None):
    if a is None:
        return None
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def _i32(a, shape=None):
    if a is None:
        return None
    a = np.ascontiguousarray(np.asarray(a, dtype=np.int32))
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a):
    return None if a is None else a.ctypes.data


def _dp(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_double))


class Problem:
    """Inputs of one deconvolution problem, held as contiguous numpy arrays.

    uvw     [n_vis, 3] wavelengths;  weights [n_vis] or None;
    ant_pair[n_vis, 2] int or None;  lm [n_pix, 2] direction cosines;
    sigma   [n_pix] or None;         kind [n_pix] int (0 Dirac, 1 paraxial
    Gaussian, 2 wide-field Gaussian) or None;  gains [n_pix, n_ant] complex or
    None (unit gains).  threads: threads for the outer loops of the forward
    (rows) and adjoint (columns), also inside power / fista / mfista; every
    output is still one sum in the single-threaded order, so results are
    bitwise the same for any count (1 = single-threaded, the default).
    """

    def __init__(self, uvw, lm, sigma=None, kind=None, weights=None,
                 ant_pair=None, gains=None, threads=1):
        self.uvw = _f64(uvw, (-1, 3))
        self.lm = _f64(lm, (-1, 2))
        self.sigma = _f64(sigma)
        self.kind = _i32(kind)
        self.weights = _f64(weights)
        self.ant_pair = _i32(ant_pair, (-1, 2)) if ant_pair is not None else None
        if gains is not None:
            g = np.asarray(gains, dtype=np.complex128)
            self.n_ant = g.shape[1]
            self.gains = np.ascontiguousarray(
                np.stack([g.real, g.imag], axis=-1).astype(np.float64))
        else:
            self.n_ant = 0
            self.gains = None
        self.n_vis = self.uvw.shape[0]
        self.n_pix = self.lm.shape[0]
        self._c = _Problem(self.n_vis, _ptr(self.uvw), _ptr(self.weights),
                           _ptr(self.ant_pair), self.n_pix, _ptr(self.lm),
                           _ptr(self.sigma), _ptr(self.kind), self.n_ant,
                           _ptr(self.gains), int(threads))

    @property
    def c(self):
        return C.byref(self._c)


def _check(st, what):
    if st != 0:
        raise ValueError(f"oracle {what} failed with status {st}")


def entry(kind, l, m, sigma, u, v, w) -> complex:
    """One operator entry without gain: Eq. deltam / samlm4 / samlm5."""
    out = np.zeros(2)
    _check(_load().orc_entry(int(kind), l, m, sigma, u, v, w, _dp(out)), "entry")
    return complex(out[0], out[1])


def entry_kj(P: Problem, k: int, j: int) -> complex:
    """A_kj including the gain product G[j][a_k] conj(G[j][b_k])."""
    out = np.zeros(2)
    _check(_load().orc_entry_kj(P.c, k, j, _dp(out)), "entry_kj")
    return complex(out[0], out[1])


def forward(P: Problem, x, rows=None) -> np.ndarray:
    """Vhat_k = sum_j A_kj x_j (Eq. sme) for all k, or for the listed rows."""
    x = _f64(x)
    n = P.n_vis if rows is None else len(rows)
    out = np.zeros((n, 2))
    r = None if rows is None else np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    rp = None if r is None else r.ctypes.data_as(C.POINTER(C.c_long))
    _check(_load().orc_forward_rows(P.c, _dp(x), n, rp, _dp(out)), "forward")
    return out[:, 0] + 1j * out[:, 1]


def adjoint(P: Problem, r, cols=None) -> np.ndarray:
    """g_j = sum_k Re(conj(A_kj) r_k) for all j, or for the listed cols."""
    r = np.asarray(r, dtype=np.complex128)
    rr = np.ascontiguousarray(np.stack([r.real, r.imag], axis=-1))
    n = P.n_pix if cols is None else len(cols)
    out = np.zeros(n)
    c = None if cols is None else np.ascontiguousarray(np.asarray(cols, dtype=np.int64))
    cp = None if c is None else c.ctypes.data_as(C.POINTER(C.c_long))
    _check(_load().orc_adjoint_cols(P.c, _dp(rr), n, cp, _dp(out)), "adjoint")
    return out


def power(P: Problem, max_iter=50, tol=1e-6):
    """(L, iterations): power iteration on Re(A^H W A), Sect. 3.1."""
    L = C.c_double(0.0)
    it = C.c_int(0)
    _check(_load().orc_power(P.c, int(max_iter), float(tol), C.byref(L), C.byref(it)), "power")
    return L.value, it.value


def fista(P: Problem, vis, lam, L, max_iter, tol=0.0, x0=None):
    """(image, stats dict): the FISTA box of Sect. 3 with Eq. threshp."""
    v = np.asarray(vis, dtype=np.complex128)
    vv = np.ascontiguousarray(np.stack([v.real, v.imag], axis=-1))
    img = np.zeros(P.n_pix)
    st = Stats()
    x0 = _f64(x0)
    _check(_load().orc_fista(P.c, _dp(vv), float(lam), float(L), int(max_iter),
                             float(tol), _dp(x0), _dp(img), C.byref(st)), "fista")
    return img, st.as_dict()


def mfista(P: Problem, vis, lam, L, max_iter, tol=0.0, x0=None, trace=False):
    """(image, stats dict[, trace]): monotone FISTA (Beck & Teboulle 2009b),
    the variant Sect. 3 names.  With ``trace`` the third value holds, per
    step k, a dict of arrays y, z, x [iters, n_pix] and t, Fz, Fx [iters]."""
    v = np.asarray(vis, dtype=np.complex128)
    vv = np.ascontiguousarray(np.stack([v.real, v.imag], axis=-1))
    img = np.zeros(P.n_pix)
    st = Stats()
    x0 = _f64(x0)
    n = P.n_pix
    tr = np.zeros((max(int(max_iter), 1), 3 * n + 3)) if trace else None
    _check(_load().orc_mfista(P.c, _dp(vv), float(lam), float(L), int(max_iter),
                              float(tol), _dp(x0), _dp(img), C.byref(st), _dp(tr)), "mfista")
    d = st.as_dict()
    if not trace:
        return img, d
    tr = tr[:d["iters"]]
    return img, d, {"y": tr[:, :n], "z": tr[:, n:2 * n], "x": tr[:, 2 * n:3 * n],
                    "t": tr[:, 3 * n], "Fz": tr[:, 3 * n + 1], "Fx": tr[:, 3 * n + 2]}
