"""Python binding of libsl1m (include/sl1m.h): argument marshalling only.

Every step of the hot path runs in the library's CUDA kernels; this module
only converts numpy arrays / torch CUDA tensors to pointers and back.  It
raises if ``libsl1m.so`` is missing -- there is no CPU fallback.

Low-level: the C functions are reachable under their own names via
:func:`load` (``lib.sl1m_forward`` ...).  The thin wrappers below keep the
same names without the ``sl1m_`` prefix (``Problem.forward`` ->
``sl1m_forward``).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsl1m.so")

OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_NONFINITE, ERR_TIMEOUT, ERR_BUSY, ERR_STATE = range(8)
FP64, MIXED = 0, 1
FISTA, MFISTA = 0, 1
_ALGOS = {"fista": FISTA, "mfista": MFISTA, FISTA: FISTA, MFISTA: MFISTA}
DIRAC, GAUSS_PARAXIAL, GAUSS_WIDE = 0, 1, 2
ADMIT_TWO_LANES, ADMIT_ARRIVAL = 0, 1
KERNEL_IDS = {"fwd_fp64": 0, "adj_fp64": 1, "fwd_mixed": 2, "adj_mixed": 3,
              "fwd_finish": 4, "adj_finish": 5, "other": 6}

EXPORTS = [
    "sl1m_version", "sl1m_status_string", "sl1m_create", "sl1m_destroy", "sl1m_last_error",
    "sl1m_problem_create", "sl1m_problem_destroy", "sl1m_set_visibilities",
    "sl1m_set_vis_data", "sl1m_set_pixels", "sl1m_set_gains", "sl1m_forward", "sl1m_adjoint",
    "sl1m_forward_dev", "sl1m_adjoint_dev", "sl1m_max_eig", "sl1m_solve",
    "sl1m_profile_enable", "sl1m_profile_reset", "sl1m_profile_read", "sl1m_problem_bytes",
    "sl1m_counters", "sl1m_counters_reset", "sl1m_plan_preview", "sl1m_granule_order",
    "sl1m_granule_layout",
    "sl1m_server_start", "sl1m_server_submit", "sl1m_server_poll", "sl1m_server_wait",
    "sl1m_server_stop", "sl1m_server_info", "sl1m_forward_noalloc", "sl1m_autotune",
    "sl1m_dirty_image", "sl1m_solve_refine", "sl1m_get_solution", "sl1m_set_tile_shape",
    "sl1m_exact_tile_share", "sl1m_selftest_bounded_wait", "sl1m_measure_sfu",
]


class SolveOpts(C.Structure):
    _fields_ = [("lambda_", C.c_double), ("L", C.c_double), ("rel_tol", C.c_double),
                ("max_iter", C.c_int32), ("precision", C.c_int32),
                ("power_max_iter", C.c_int32), ("power_tol", C.c_double),
                ("x0", C.c_void_p), ("algorithm", C.c_int32)]


class ServerOpts(C.Structure):
    _fields_ = [("mem_budget_bytes", C.c_int64), ("max_slots", C.c_int32),
                ("ticks_per_round", C.c_int32), ("precision", C.c_int32), ("admission", C.c_int32),
                ("max_pairs_per_tick", C.c_double)]


class ServerInfo(C.Structure):
    _fields_ = [("queued", C.c_int64), ("active", C.c_int64), ("finished", C.c_int64),
                ("max_active", C.c_int64), ("bytes_in_use", C.c_int64),
                ("bytes_budget", C.c_int64), ("ticks", C.c_int64), ("rounds", C.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class RefineOpts(C.Structure):
    _fields_ = [("levels", C.c_int32), ("refine_frac", C.c_double), ("keep_unrefined", C.c_int32)]


class SolveStats(C.Structure):
    _fields_ = [("iters", C.c_int32), ("converged", C.c_int32), ("E", C.c_double),
                ("E_paper", C.c_double), ("resid2", C.c_double), ("l1", C.c_double),
                ("nnz", C.c_int64), ("L", C.c_double), ("power_iters", C.c_int32),
                ("seconds", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class RefineStats(C.Structure):
    _fields_ = [("levels_done", C.c_int32), ("n_pix", C.c_int64 * 17), ("iters", C.c_int32 * 17),
                ("power_iters", C.c_int32 * 17), ("final_n_pix", C.c_int64),
                ("total_pair_evals", C.c_double), ("last", SolveStats)]

    def as_dict(self):
        n = self.levels_done
        return {"levels_done": n, "n_pix": list(self.n_pix)[:n], "iters": list(self.iters)[:n],
                "power_iters": list(self.power_iters)[:n], "final_n_pix": self.final_n_pix,
                "total_pair_evals": self.total_pair_evals, "last": self.last.as_dict()}


_lib = None
_lock = threading.Lock()


class SL1MError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libsl1m status {status}: {msg}")
        self.status = status


def load():
    """Load libsl1m.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libsl1m.so not found at {LIB_PATH}; run __graft_entry__.build()")
        lib = C.CDLL(LIB_PATH)
        vp, d, i64, i32 = C.c_void_p, C.c_double, C.c_int64, C.c_int32
        pvp = C.POINTER(C.c_void_p)
        sig = {
            "sl1m_version": ([], C.c_int),
            "sl1m_status_string": ([C.c_int], C.c_char_p),
            "sl1m_create": ([pvp, C.c_int, vp], C.c_int),
            "sl1m_destroy": ([vp], C.c_int),
            "sl1m_last_error": ([vp], C.c_char_p),
            "sl1m_problem_create": ([vp, pvp], C.c_int),
            "sl1m_problem_destroy": ([vp], C.c_int),
            "sl1m_set_visibilities": ([vp, i64, vp, vp, vp, vp], C.c_int),
            "sl1m_set_vis_data": ([vp, vp], C.c_int),
            "sl1m_set_pixels": ([vp, i64, vp, vp, vp], C.c_int),
            "sl1m_set_gains": ([vp, i32, vp], C.c_int),
            "sl1m_forward": ([vp, vp, vp, C.c_int], C.c_int),
            "sl1m_adjoint": ([vp, vp, vp, C.c_int], C.c_int),
            "sl1m_forward_dev": ([vp, vp, vp, C.c_int], C.c_int),
            "sl1m_forward_noalloc": ([vp, vp, vp, C.c_int], C.c_int),
            "sl1m_autotune": ([vp, C.c_int, vp, vp, vp], C.c_int),
            "sl1m_set_tile_shape": ([vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int], C.c_int),
            "sl1m_dirty_image": ([vp, C.c_int, vp, C.POINTER(d)], C.c_int),
            "sl1m_solve_refine": ([vp, C.POINTER(SolveOpts), C.POINTER(RefineOpts), d, C.POINTER(RefineStats)],
                                  C.c_int),
            "sl1m_get_solution": ([vp, C.POINTER(i64), vp, vp], C.c_int),
            "sl1m_adjoint_dev": ([vp, vp, vp, C.c_int], C.c_int),
            "sl1m_max_eig": ([vp, C.c_int, d, C.c_int, C.POINTER(d), C.POINTER(C.c_int)], C.c_int),
            "sl1m_solve": ([vp, C.POINTER(SolveOpts), vp, C.POINTER(SolveStats)], C.c_int),
            "sl1m_profile_enable": ([vp, C.c_int], C.c_int),
            "sl1m_profile_reset": ([vp], C.c_int),
            "sl1m_profile_read": ([vp, C.c_int, C.POINTER(d), C.POINTER(i64), C.POINTER(d),
                                   C.POINTER(d)], C.c_int),
            "sl1m_problem_bytes": ([vp, C.POINTER(i64)], C.c_int),
            "sl1m_exact_tile_share": ([vp, C.POINTER(d), C.POINTER(i64)], C.c_int),
            "sl1m_selftest_bounded_wait": ([vp, C.POINTER(i64), C.POINTER(i64)], C.c_int),
            "sl1m_measure_sfu": ([vp, C.POINTER(d), C.POINTER(d)], C.c_int),
            "sl1m_counters": ([vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64)], C.c_int),
            "sl1m_counters_reset": ([vp], C.c_int),
            "sl1m_plan_preview": ([i32, vp, vp, i32, vp, C.POINTER(i32), C.POINTER(i64), C.POINTER(i32),
                                   vp, vp, vp, vp], C.c_int),
            "sl1m_granule_order": ([i64, vp, vp, C.POINTER(i64)], C.c_int),
            "sl1m_granule_layout": ([i64, vp, vp, i64, vp, vp, vp, vp, vp, vp, vp], C.c_int),
            "sl1m_server_start": ([vp, C.POINTER(ServerOpts)], C.c_int),
            "sl1m_server_submit": ([vp, vp, C.POINTER(SolveOpts), C.POINTER(C.c_uint64)], C.c_int),
            "sl1m_server_poll": ([vp, C.c_uint64, C.POINTER(C.c_int)], C.c_int),
            "sl1m_server_wait": ([vp, C.c_uint64, d, vp, C.POINTER(SolveStats)], C.c_int),
            "sl1m_server_stop": ([vp], C.c_int),
            "sl1m_server_info": ([vp, C.POINTER(ServerInfo)], C.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
        return lib


def _f64(a, shape=None):
    if a is None:
        return None
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    return a.reshape(shape) if shape is not None else a


def _cplx_interleaved(a):
    if a is None:
        return None
    a = np.asarray(a)
    if np.iscomplexobj(a):
        return np.ascontiguousarray(np.stack([a.real, a.imag], axis=-1).astype(np.float64))
    return _f64(a)


def _ptr(a):
    return None if a is None else a.ctypes.data


def _need(a, n, what):
    """The library reads host and device arrays without a size argument, so
    an array of the wrong length would be read past its end: refuse it here.
    n == 0 (the problem's side not set yet) leaves the check to the library,
    which reports the missing data."""
    if a is None or not n:
        return
    size = a.numel() if hasattr(a, "numel") else a.size
    if size != n:
        raise ValueError(f"{what}: expected {n} values, got {size}")


def _dev_f64(t, n, what):
    """Device pointer of a contiguous float64 CUDA tensor of n values."""
    if str(getattr(t, "dtype", "")) != "torch.float64":
        raise ValueError(f"{what}: expected a float64 tensor")
    _need(t, n, what)
    return _tptr(t)


def _tptr(t):
    """Device pointer of a contiguous torch CUDA tensor."""
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def plan_preview(owned_blocks, streamed_granules, max_ctas, unit_costs=None):
    """Host-only stream-K schedule (sl1m_plan_preview)."""
    lib = load()
    nb = np.ascontiguousarray(np.asarray(owned_blocks, np.int32))
    ns = np.ascontiguousarray(np.asarray(streamed_granules, np.int32))
    nbt = int(nb.sum())
    fc = np.zeros(max(1, nbt), np.int32)
    nc = np.zeros(max(1, nbt), np.int32)
    fs = np.zeros(max(1, nbt), np.int32)
    cu = np.zeros(max(1, int(max_ctas)) + 1, np.int64)
    uc = None if unit_costs is None else np.ascontiguousarray(np.asarray(unit_costs, np.float32))
    C_, U, S = C.c_int32(), C.c_int64(), C.c_int32()
    st = lib.sl1m_plan_preview(len(nb), _ptr(nb), _ptr(ns), int(max_ctas), _ptr(uc), C.byref(C_), C.byref(U),
                               C.byref(S), _ptr(fc), _ptr(nc), _ptr(fs), _ptr(cu))
    if st != OK:
        raise SL1MError(st, "sl1m_plan_preview failed")
    return {"n_ctas": C_.value, "n_units": U.value, "n_slots": S.value,
            "first_cta": fc[:nbt], "n_ctas_blk": nc[:nbt], "first_slot": fs[:nbt],
            "cta_first_unit": cu[:C_.value + 1]}


def granule_order(xy):
    """Host-only granule order (sl1m_granule_order): indices, -1 = padding."""
    lib = load()
    xy = _f64(xy, (-1, 2))
    npad = C.c_int64()
    st = lib.sl1m_granule_order(xy.shape[0], _ptr(xy), None, C.byref(npad))
    if st != OK:
        raise SL1MError(st, "sl1m_granule_order failed")
    out = np.zeros(npad.value, np.int32)
    lib.sl1m_granule_order(xy.shape[0], _ptr(xy), _ptr(out), C.byref(npad))
    return out


def granule_layout(xyzw, order):
    """Host-only FP32 layout of one side (sl1m_granule_layout): a dict of
    hi, lo, off, offlo [n_pad, 4] and cen_hi, cen_lo, ext [n_pad / 64, 4]."""
    lib = load()
    xyzw = _f64(xyzw, (-1, 4))
    order = np.ascontiguousarray(order, np.int32)
    npad = order.shape[0]
    out = {k: np.zeros((npad, 4), np.float32) for k in ("hi", "lo", "off", "offlo")}
    out.update({k: np.zeros((npad // 64, 4), np.float32) for k in ("cen_hi", "cen_lo", "ext")})
    st = lib.sl1m_granule_layout(xyzw.shape[0], _ptr(xyzw), _ptr(order), npad,
                                 *(_ptr(out[k]) for k in ("hi", "lo", "off", "offlo", "cen_hi", "cen_lo", "ext")))
    if st != OK:
        raise SL1MError(st, "sl1m_granule_layout failed")
    return out


class Context:
    """sl1m_create / sl1m_destroy.  `stream`: a torch.cuda.Stream, a raw
    cudaStream_t as int, or None (the context makes its own)."""

    def __init__(self, device: int = 0, stream=None):
        self.lib = load()
        h = C.c_void_p()
        s = None
        if stream is not None:
            s = getattr(stream, "cuda_stream", stream)
        st = self.lib.sl1m_create(C.byref(h), int(device), s)
        if st != OK:
            raise SL1MError(st, "sl1m_create failed (no CUDA device?)")
        self.h = h
        self.device = device
        self._problems = []

    def check(self, st):
        if st != OK:
            raise SL1MError(st, self.lib.sl1m_last_error(self.h).decode())

    def problem(self) -> "Problem":
        p = Problem(self)
        self._problems.append(p)
        return p

    def profile_enable(self, on=True):
        self.check(self.lib.sl1m_profile_enable(self.h, int(bool(on))))

    def profile_reset(self):
        self.check(self.lib.sl1m_profile_reset(self.h))

    def profile_read(self, kernel):
        kid = KERNEL_IDS[kernel] if isinstance(kernel, str) else int(kernel)
        ms, n, pairs, by = C.c_double(), C.c_int64(), C.c_double(), C.c_double()
        self.check(self.lib.sl1m_profile_read(self.h, kid, C.byref(ms), C.byref(n),
                                              C.byref(pairs), C.byref(by)))
        return {"ms": ms.value, "launches": n.value, "pairs": pairs.value, "bytes": by.value}

    def counters(self):
        n, a, b = C.c_int64(), C.c_int64(), C.c_int64()
        self.check(self.lib.sl1m_counters(self.h, C.byref(n), C.byref(a), C.byref(b)))
        return {"launches": n.value, "h2d_bytes": a.value, "d2h_bytes": b.value}

    def counters_reset(self):
        self.check(self.lib.sl1m_counters_reset(self.h))

    def measure_sfu(self):
        """sl1m_measure_sfu: {"sincos_per_s": ..., "ex2_per_s": ...} (results/s, device)."""
        a, b = C.c_double(), C.c_double()
        self.check(self.lib.sl1m_measure_sfu(self.h, C.byref(a), C.byref(b)))
        return {"sincos_per_s": a.value, "ex2_per_s": b.value}

    def selftest_bounded_wait(self):
        """sl1m_selftest_bounded_wait: (status, waited_ns, limit_ns); status
        SL1M_ERR_CUDA is the expected outcome (the wait gave up)."""
        w, lim = C.c_int64(), C.c_int64()
        st = self.lib.sl1m_selftest_bounded_wait(self.h, C.byref(w), C.byref(lim))
        return st, w.value, lim.value

    # ---- continuous-batching server (sl1m_server_*)
    def server_start(self, mem_budget_bytes=0, max_slots=0, ticks_per_round=0, precision=MIXED,
                     max_pairs_per_tick=0.0, admission=ADMIT_TWO_LANES):
        o = ServerOpts(int(mem_budget_bytes), int(max_slots), int(ticks_per_round), int(precision),
                       int(admission), float(max_pairs_per_tick))
        self.check(self.lib.sl1m_server_start(self.h, C.byref(o)))

    def server_submit(self, problem, lam, L=0.0, max_iter=200, rel_tol=0.0, x0=None,
                      power_max_iter=0, power_tol=0.0, algorithm="fista"):
        x0a = _f64(x0)
        _need(x0a, problem.n_pix, "x0")
        o = SolveOpts(float(lam), float(L), float(rel_tol), int(max_iter), MIXED,
                      int(power_max_iter), float(power_tol), _ptr(x0a), _ALGOS[algorithm])
        t = C.c_uint64()
        self.check(self.lib.sl1m_server_submit(self.h, problem.h, C.byref(o), C.byref(t)))
        return t.value

    def server_poll(self, ticket):
        d = C.c_int()
        self.check(self.lib.sl1m_server_poll(self.h, C.c_uint64(ticket), C.byref(d)))
        return bool(d.value)

    def server_wait(self, ticket, problem, timeout_s=-1.0):
        img = np.zeros(problem.n_pix)
        st = SolveStats()
        self.check(self.lib.sl1m_server_wait(self.h, C.c_uint64(ticket), float(timeout_s), _ptr(img),
                                             C.byref(st)))
        return img, st.as_dict()

    def server_stop(self):
        self.check(self.lib.sl1m_server_stop(self.h))

    def server_info(self):
        i = ServerInfo()
        self.check(self.lib.sl1m_server_info(self.h, C.byref(i)))
        return i.as_dict()

    def close(self):
        if getattr(self, "h", None):
            self.lib.sl1m_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Problem:
    """One deconvolution problem (sl1m_problem_*)."""

    def __init__(self, ctx: Context):
        self.ctx = ctx
        self.lib = ctx.lib
        h = C.c_void_p()
        ctx.check(self.lib.sl1m_problem_create(ctx.h, C.byref(h)))
        self.h = h
        self.n_vis = self.n_pix = 0

    def set_visibilities(self, uvw, vis=None, weights=None, ant_pair=None):
        uvw = _f64(uvw, (-1, 3))
        n = uvw.shape[0]
        v = _cplx_interleaved(vis)
        w = _f64(weights)
        ap = None if ant_pair is None else np.ascontiguousarray(np.asarray(ant_pair, np.int32).reshape(-1, 2))
        _need(v, 2 * n, "vis")
        _need(w, n, "weights")
        _need(ap, 2 * n, "ant_pair")
        self.ctx.check(self.lib.sl1m_set_visibilities(self.h, n, _ptr(uvw), _ptr(v), _ptr(w), _ptr(ap)))
        self.n_vis = n

    def set_vis_data(self, vis):
        v = _cplx_interleaved(vis)
        _need(v, 2 * self.n_vis, "vis")
        self.ctx.check(self.lib.sl1m_set_vis_data(self.h, _ptr(v)))

    def set_pixels(self, lm, sigma=None, kind=None):
        lm = _f64(lm, (-1, 2))
        s = _f64(sigma)
        k = None if kind is None else np.ascontiguousarray(np.asarray(kind, np.int32))
        _need(s, lm.shape[0], "sigma")
        _need(k, lm.shape[0], "kind")
        self.ctx.check(self.lib.sl1m_set_pixels(self.h, lm.shape[0], _ptr(lm), _ptr(s), _ptr(k)))
        self.n_pix = lm.shape[0]

    def set_gains(self, gains):
        if gains is None:
            self.ctx.check(self.lib.sl1m_set_gains(self.h, 0, None))
            return
        g = np.asarray(gains, dtype=np.complex128)
        if g.ndim != 2 or (self.n_pix and g.shape[0] != self.n_pix):
            raise ValueError(f"gains: expected an array [n_pix = {self.n_pix}, n_ant], got {g.shape}")
        gi = _cplx_interleaved(g)
        self.ctx.check(self.lib.sl1m_set_gains(self.h, g.shape[1], _ptr(gi)))

    def forward(self, x, precision=MIXED):
        x = _f64(x)
        _need(x, self.n_pix, "x")
        out = np.zeros((self.n_vis, 2))
        self.ctx.check(self.lib.sl1m_forward(self.h, _ptr(x), _ptr(out), int(precision)))
        return out[:, 0] + 1j * out[:, 1]

    def adjoint(self, r, precision=MIXED):
        rr = _cplx_interleaved(np.asarray(r, dtype=np.complex128))
        _need(rr, 2 * self.n_vis, "r")
        out = np.zeros(self.n_pix)
        self.ctx.check(self.lib.sl1m_adjoint(self.h, _ptr(rr), _ptr(out), int(precision)))
        return out

    def forward_dev(self, x_t, out_t, precision=MIXED):
        """x_t: float64 CUDA tensor [n_pix]; out_t: float64 CUDA tensor [n_vis, 2]."""
        self.ctx.check(self.lib.sl1m_forward_dev(self.h, _dev_f64(x_t, self.n_pix, "x"),
                                                 _dev_f64(out_t, 2 * self.n_vis, "out"), int(precision)))

    def forward_noalloc(self, x_t, out_t, precision=MIXED):
        """sl1m_forward_noalloc: like forward_dev, scratch in a static device array."""
        self.ctx.check(self.lib.sl1m_forward_noalloc(self.h, _dev_f64(x_t, self.n_pix, "x"),
                                                     _dev_f64(out_t, 2 * self.n_vis, "out"), int(precision)))

    def adjoint_dev(self, r_t, out_t, precision=MIXED):
        """r_t: float64 CUDA tensor [n_vis, 2]; out_t: float64 CUDA tensor [n_pix]."""
        self.ctx.check(self.lib.sl1m_adjoint_dev(self.h, _dev_f64(r_t, 2 * self.n_vis, "r"),
                                                 _dev_f64(out_t, self.n_pix, "out"), int(precision)))

    def dirty_image(self, precision=MIXED):
        """sl1m_dirty_image: (Re A^H W V, lambda_max)."""
        img = np.zeros(self.n_pix)
        lm = C.c_double()
        self.ctx.check(self.lib.sl1m_dirty_image(self.h, int(precision), _ptr(img), C.byref(lm)))
        return img, lm.value

    def max_eig(self, max_iter=50, tol=1e-6, precision=MIXED):
        L, it = C.c_double(), C.c_int()
        self.ctx.check(self.lib.sl1m_max_eig(self.h, int(max_iter), float(tol), int(precision),
                                             C.byref(L), C.byref(it)))
        return L.value, it.value

    def solve(self, lam, L=0.0, max_iter=200, rel_tol=0.0, precision=MIXED, x0=None,
              power_max_iter=0, power_tol=0.0, algorithm="fista"):
        x0a = _f64(x0)
        _need(x0a, self.n_pix, "x0")
        o = SolveOpts(float(lam), float(L), float(rel_tol), int(max_iter), int(precision),
                      int(power_max_iter), float(power_tol), _ptr(x0a), _ALGOS[algorithm])
        img = np.zeros(self.n_pix)
        st = SolveStats()
        self.ctx.check(self.lib.sl1m_solve(self.h, C.byref(o), _ptr(img), C.byref(st)))
        return img, st.as_dict()

    def autotune(self, precision=MIXED):
        """sl1m_autotune: returns {"nst": [fwd, adj], "ctas_per_sm": [fwd, adj],
        "npoly": [fwd, adj]}."""
        nst = np.zeros(2, np.int32)
        k = np.zeros(2, np.int32)
        npoly = np.zeros(2, np.int32)
        self.ctx.check(self.lib.sl1m_autotune(self.h, int(precision), _ptr(nst), _ptr(k), _ptr(npoly)))
        return {"nst": nst.tolist(), "ctas_per_sm": k.tolist(), "npoly": npoly.tolist()}

    def set_tile_shape(self, op, nst, ctas_per_sm, npoly=0, precision=MIXED):
        """sl1m_set_tile_shape (op 0 forward, 1 adjoint)."""
        self.ctx.check(self.lib.sl1m_set_tile_shape(self.h, int(precision), int(op), int(nst),
                                                    int(ctas_per_sm), int(npoly)))

    def solve_refine(self, lam, delta0, levels, refine_frac=0.01, keep_unrefined=True, L=0.0,
                     max_iter=200, rel_tol=0.0, precision=MIXED):
        """sl1m_solve_refine: returns (lm [n,2], image [n], stats)."""
        o = SolveOpts(float(lam), float(L), float(rel_tol), int(max_iter), int(precision), 0, 0.0, None,
                      FISTA)
        ro = RefineOpts(int(levels), float(refine_frac), int(bool(keep_unrefined)))
        st = RefineStats()
        self.ctx.check(self.lib.sl1m_solve_refine(self.h, C.byref(o), C.byref(ro), float(delta0), C.byref(st)))
        n = C.c_int64()
        self.ctx.check(self.lib.sl1m_get_solution(self.h, C.byref(n), None, None))
        lm = np.zeros((n.value, 2))
        img = np.zeros(n.value)
        self.ctx.check(self.lib.sl1m_get_solution(self.h, C.byref(n), _ptr(lm), _ptr(img)))
        self.n_pix = n.value
        return lm, img, st.as_dict()

    def bytes(self):
        b = C.c_int64()
        self.ctx.check(self.lib.sl1m_problem_bytes(self.h, C.byref(b)))
        return b.value

    def exact_tile_share(self):
        """sl1m_exact_tile_share: (share of tiles on the exact phase path, tiles)."""
        sh, n = C.c_double(), C.c_int64()
        self.ctx.check(self.lib.sl1m_exact_tile_share(self.h, C.byref(sh), C.byref(n)))
        return sh.value, n.value

    def close(self):
        if getattr(self, "h", None) and self.ctx.h:
            self.lib.sl1m_problem_destroy(self.h)
            self.h = None


def problem_from(ctx: Context, w, vis=None):
    """Problem from a synth.Workload (and optional visibilities)."""
    P = ctx.problem()
    P.set_visibilities(w.uvw, vis, w.weights, w.ant_pair)
    P.set_pixels(w.lm, w.sigma, w.kind)
    if w.gains is not None:
        P.set_gains(w.gains)
    return P
