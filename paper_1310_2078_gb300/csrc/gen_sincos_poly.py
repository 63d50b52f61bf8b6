"""Writes sl1m_sincos_poly.h: polynomial sin/cos for the FMA pipe.

Method: Chebyshev interpolation (interpolation at the Chebyshev points of the
first kind, then conversion to monomials; see L. N. Trefethen, *Approximation
Theory and Approximation Practice*, SIAM 2013, ch. 3-4).  With f the phase in
turns reduced to [-1/2, 1/2] and a = pi f,

    h(f) = sqrt(2) sin(pi f) = f * P(f^2),   q(f) = sqrt(2) cos(pi f) = Q(f^2),

each fitted as a degree-4 polynomial in z = f^2 on [0, 1/4]; then
sin(2 pi f) = h q and cos(2 pi f) = 1 - h^2 (double-angle formulas), which
is why both carry the factor sqrt(2).  Run as a script to regenerate the
header; tests re-derive the coefficients and check the FP32 error bound.
"""
import os

import numpy as np
from numpy.polynomial import chebyshev as _ch
from numpy.polynomial import polynomial as _po

DEG = 4
Z_MAX = 0.25


def _interp_monomial(fun, deg, a, b):
    """Coefficients (constant first) in z of the degree-`deg` interpolant of
    fun at the Chebyshev points of the first kind mapped to [a, b]."""
    k = np.arange(deg + 1)
    x = np.cos((2 * k + 1) * np.pi / (2 * (deg + 1)))
    z = a + (b - a) * (x + 1) / 2
    c = _ch.chebfit(x, fun(z), deg)
    px = _ch.cheb2poly(c)
    lin = _po.Polynomial([-(a + b) / (b - a), 2 / (b - a)])      # x as a function of z
    out = _po.Polynomial([0.0])
    for i, ci in enumerate(px):
        out = out + ci * lin ** i
    return np.asarray(out.coef, dtype=np.float64)


def _h_over_f(z):
    f = np.sqrt(z)
    safe = np.where(f > 0, f, 1.0)
    return np.sqrt(2.0) * np.where(f > 0, np.sin(np.pi * f) / safe, np.pi)


def _q(z):
    return np.sqrt(2.0) * np.cos(np.pi * np.sqrt(z))


def coefficients():
    """(P, Q) as float32 arrays, constant term first."""
    P = _interp_monomial(_h_over_f, DEG, 0.0, Z_MAX).astype(np.float32)
    Q = _interp_monomial(_q, DEG, 0.0, Z_MAX).astype(np.float32)
    return P, Q


def header_text():
    P, Q = coefficients()
    lines = [
        "// sl1m_sincos_poly.h -- generated by gen_sincos_poly.py (Chebyshev interpolation,",
        "// degree 4 in z = f^2 on [0, 1/4]); do not edit by hand.",
        "//   sqrt(2) sin(pi f) = f * P(z),  sqrt(2) cos(pi f) = Q(z),  f in [-1/2, 1/2]",
        "#pragma once",
        "",
        "namespace sl1m {",
    ]
    for name, C in (("SCP", P), ("SCQ", Q)):
        for i, c in enumerate(C):
            lines.append(f"constexpr float {name}{i} = {float(c)!r}f;")
    lines += ["", "}  // namespace sl1m", ""]
    return "\n".join(lines)


if __name__ == "__main__":
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "sl1m_sincos_poly.h")
    with open(path, "w") as f:
        f.write(header_text())
    print(path)
