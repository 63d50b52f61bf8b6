"""The FMA-pipe sincos of the mixed kernels (Chebyshev interpolants of
sqrt(2) sin(pi f) and sqrt(2) cos(pi f) in f^2, then the double-angle
formulas): the committed header is what the generator writes, the
interpolants pass through their Chebyshev points, and an FP32 evaluation in
the kernel's operation order stays within the SFU-sized error bound."""
import importlib.util
import os

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1310_2078_gb300", "csrc")


def _gen():
    spec = importlib.util.spec_from_file_location("gen_sincos_poly", os.path.join(CSRC, "gen_sincos_poly.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _fma32(a, b, c):
    """One rounding, as the FP32 fma (float64 product of two floats is exact)."""
    return (np.float64(a) * np.float64(b) + np.float64(c)).astype(np.float32) if np.ndim(a) == 0 else \
        (a.astype(np.float64) * b.astype(np.float64) + np.asarray(c, np.float64)).astype(np.float32)


def _sincos32(ph):
    """The kernel's sincos_fma in FP32 arithmetic, step by step."""
    P, Q = _gen().coefficients()
    ph = ph.astype(np.float32)
    t = (ph * np.float32(0.15915494309189535)).astype(np.float32)
    M = np.float32(12582912.0)
    f = (t - ((t + M).astype(np.float32) - M).astype(np.float32)).astype(np.float32)
    z = (f * f).astype(np.float32)
    hp = np.full_like(z, P[4])
    for c in P[3::-1]:
        hp = _fma32(hp, z, np.full_like(z, c))
    h = (f * hp).astype(np.float32)
    q = np.full_like(z, Q[4])
    for c in Q[3::-1]:
        q = _fma32(q, z, np.full_like(z, c))
    s = (h * q).astype(np.float32)
    co = _fma32(-h, h, np.ones_like(h))
    return f, s, co


def test_header_is_the_generator_output():
    with open(os.path.join(CSRC, "sl1m_sincos_poly.h")) as fh:
        assert fh.read() == _gen().header_text()


def test_interpolants_pass_through_the_chebyshev_points():
    g = _gen()
    P, Q = g.coefficients()
    k = np.arange(g.DEG + 1)
    x = np.cos((2 * k + 1) * np.pi / (2 * (g.DEG + 1)))
    z = g.Z_MAX * (x + 1) / 2
    f = np.sqrt(z)
    hp = np.polynomial.polynomial.polyval(z, P.astype(np.float64))
    qp = np.polynomial.polynomial.polyval(z, Q.astype(np.float64))
    assert np.allclose(hp, np.sqrt(2) * np.sin(np.pi * f) / f, rtol=2e-7, atol=0)
    assert np.allclose(qp, np.sqrt(2) * np.cos(np.pi * f), rtol=0, atol=2e-7)


def test_fp32_evaluation_error_bound_over_the_kernel_phase_range():
    # the kernels pass |phase| <= 2 pi (1.5 + 6) rad; sample densely, with the ends
    ph = np.concatenate([np.linspace(-48.0, 48.0, 2_000_001), [0.0, np.pi, -np.pi, np.pi / 2]])
    ph = ph.astype(np.float32).astype(np.float64)          # the kernel's FP32 phase
    f, s, c = _sincos32(ph)
    # reference: sin and cos of the FP32 reduced argument (the reduction's own
    # rounding is the same as the SFU path's and is checked separately)
    ref = 2 * np.pi * f.astype(np.float64)
    assert np.max(np.abs(s - np.sin(ref))) < 6e-7
    assert np.max(np.abs(c - np.cos(ref))) < 6e-7
    # against the FP32 phase itself, the conversion to turns included: the
    # FP32 constant 1/(2 pi) (relative error <= 2^-24) and the product's
    # rounding (half an ulp of <= 7.6 turns) give <= 6.9e-7 turns = 4.3e-6 rad
    # at the largest phases, the size of the FP32 phase's own rounding there
    assert np.max(np.abs(s - np.sin(ph))) < 4.4e-6
    assert np.max(np.abs(c - np.cos(ph))) < 4.4e-6
    small = np.abs(ph) < 2 * np.pi             # a phase of one turn or less
    assert np.max(np.abs(s - np.sin(ph))[small]) < 1e-6
    assert np.max(np.abs(s * s + c * c - 1.0)) < 2e-6
