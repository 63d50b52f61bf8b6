"""The mixed kernels' exact phase split, carried out in FP32 on the CPU.

The mixed-precision operator kernels never form u l in FP64.  Each coordinate
is an FP32 pair (hi, lo); elements are grouped into granules with centres
Xc, Yc; and the phase of a pair (turns) is split exactly as

    X.Y = X.Yc + Xc.(Y - Yc) + (X - Xc).(Y - Yc) = C + B + D.

C and B are reduced to fractional turns by FP32 TwoProducts and a whole-turn
rounding that adds and removes 1.5 * 2^23; B goes to radians; D is one FP32
fma chain on offsets held in radians, as long as the granules' extents bound
|D| by D_MAX = 6 turns; beyond that D is reduced like C and B.  C rotates the
tile's sum, so the pair's phase is 2 pi C + (2 pi B + 2 pi D).

This test performs those steps with numpy float32 (every operation rounded
to FP32; a fused multiply-add as the exact product plus the addend, rounded
once to FP64 and then to FP32), on coordinates drawn like the wide-field and
paper-scale workloads and at the largest products the library accepts, and
checks the phase against the FP64 phase: within 1e-6 turn, with an rms far
below it.  It also checks the two facts the split rests on: whole-turn
rounding is exact below 2^22, and an FP32 D past D_MAX would break the bound.

The adjoint's output is real, so the kernel takes one cosine per pair,
Re(conj(A) r) = |r| cos(theta + arg r), with arg r folded into B and every
other term taken as -cos(theta + pi); the last two tests carry that form out
in FP32 against the FP64 Re(conj(A) r), and show why the signs alternate.
"""
import math

import numpy as np

f32 = np.float32
TWO_PI_F = f32(6.283185307179586)
INV_TWO_PI_F = f32(0.15915494309189535)
M = f32(12582912.0)                          # 1.5 * 2^23
D_MAX = 6.0


def fma32(a, b, c):
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(f32)


def frac_turns(x):
    return x - ((x + M) - M)


def tp_frac(ah, al, bh, bl):
    p = ah * bh
    e = fma32(ah, bh, -p)
    return frac_turns(p) + fma32(ah, bl, fma32(al, bh, e))


def frac_dot3(ah, al, bh, bl):
    s = tp_frac(ah[:, 0], al[:, 0], bh[:, 0], bl[:, 0]) + tp_frac(ah[:, 1], al[:, 1], bh[:, 1], bl[:, 1])
    return frac_turns(s + tp_frac(ah[:, 2], al[:, 2], bh[:, 2], bl[:, 2]))


def split(x):
    hi = x.astype(f32)
    return hi, (x - hi.astype(np.float64)).astype(f32)


def draw(rng, n, uv, w, lm, ext_x, ext_y):
    """Visibilities X = Xc + dX and pixels Y = Yc + dY (Y = (l, m, n - 1))
    with |dX| <= ext_x, |dY| <= ext_y per axis, in FP64."""
    xc = np.stack([rng.uniform(-uv, uv, n), rng.uniform(-uv, uv, n), rng.uniform(-w, w, n)], axis=1)
    x = xc + rng.uniform(-1, 1, (n, 3)) * ext_x
    lmc = rng.uniform(-lm, lm, (n, 2))
    lmv = lmc + rng.uniform(-1, 1, (n, 2)) * ext_y[:2]

    def with_n(p):
        r2 = (p ** 2).sum(axis=1)
        return np.column_stack([p, -r2 / (1 + np.sqrt(1 - r2))])

    return xc, x, with_n(lmc), with_n(lmv)


def phase_error(xc, x, yc, y, exact=False):
    """FP32 phase (turns) of every pair minus the FP64 one, wrapped to (-1/2, 1/2]."""
    xh, xl = split(x)
    xch, xcl = split(xc)
    ych, ycl = split(yc)
    dxh, dxl = split(x - xc)
    dyh, dyl = split(y - yc)
    C = frac_dot3(xh, xl, ych, ycl)                          # per owned element and granule
    B = frac_dot3(xch, xcl, dyh, dyl)                        # per owned granule and element
    b = B * TWO_PI_F                                         # radians
    if exact:
        ph = frac_turns(fma32(b, INV_TWO_PI_F, frac_dot3(dxh, dxl, dyh, dyl))) * TWO_PI_F
    else:
        dx = dxh * TWO_PI_F                                  # owned offsets in radians
        ph = fma32(dx[:, 2], dyh[:, 2], fma32(dx[:, 1], dyh[:, 1], fma32(dx[:, 0], dyh[:, 0], b)))
    got = C.astype(np.float64) + ph.astype(np.float64) / (2 * math.pi)
    want = (x * y).sum(axis=1)
    return (got - want + 0.5) % 1.0 - 0.5


def test_whole_turn_rounding_is_exact_below_2_pow_22():
    rng = np.random.default_rng(1)
    x = (rng.uniform(-1, 1, 200000) * 2.0 ** rng.uniform(-4, 22, 200000)).astype(f32)
    x = np.concatenate([x, f32([0.5, -0.5, 1.5, 2.5, 4194303.5, -4194303.5, 4194304.0])])
    ref = x.astype(np.float64) - np.rint(x.astype(np.float64))      # ties to even, like the add
    np.testing.assert_array_equal(frac_turns(x).astype(np.float64), ref)


def test_wide_field_geometry_within_a_micro_turn():
    """Baselines up to 2,000 wavelengths, |l|, |m| < 1/2, granule extents up to
    the D_MAX bound."""
    rng = np.random.default_rng(2)
    for ext_x, ext_y in (((40.0, 40.0, 15.0), (0.0156, 0.0156, 0.005)),
                         ((150.0, 150.0, 50.0), (0.0156, 0.0156, 0.01))):
        ex, ey = np.array(ext_x), np.array(ext_y)
        assert float(ex @ ey) <= D_MAX
        err = phase_error(*draw(rng, 200000, 2000.0, 500.0, 0.45, ex, ey))
        assert np.max(np.abs(err)) < 1e-6
        assert np.sqrt(np.mean(err ** 2)) < 1.2e-7


def test_paper_scale_geometry_within_a_micro_turn():
    rng = np.random.default_rng(3)
    err = phase_error(*draw(rng, 200000, 1000.0, 250.0, 0.28, np.array([30.0, 30.0, 10.0]),
                            np.array([0.0024, 0.0024, 0.0008])))
    assert np.max(np.abs(err)) < 1e-6


def test_largest_accepted_products_within_a_micro_turn():
    """|u| max|l| just below the 2^21 turns the library accepts."""
    rng = np.random.default_rng(4)
    uv = 0.99 * 2.0 ** 21 / 0.5
    err = phase_error(*draw(rng, 100000, uv, uv / 4, 0.45, np.array([40.0, 40.0, 15.0]),
                            np.array([0.0156, 0.0156, 0.005])))
    assert np.max(np.abs(err)) < 1e-6


def test_exact_path_keeps_the_bound_where_the_fp32_chain_does_not():
    """Granules whose extents bound |D| far above D_MAX: D in one FP32 fma
    chain errs by several micro-turns; reduced exactly, it stays within one."""
    rng = np.random.default_rng(5)
    data = draw(rng, 100000, 2000.0, 500.0, 0.45, np.array([1500.0, 1500.0, 400.0]),
                np.array([0.05, 0.05, 0.02]))
    plain = phase_error(*data)
    exact = phase_error(*data, exact=True)
    assert np.max(np.abs(plain)) > 2e-6
    assert np.max(np.abs(exact)) < 1e-6


# ---- the adjoint's polar form: one cosine per pair

def adjoint_terms(xc, x, yc, y, r, alternate=True, bias=0.0):
    """The mixed adjoint's FP32 term of every pair, carried out as the kernel
    does with roles swapped (owned X = pixels, streamed Y = visibilities):
    r in polar form {|r|, arg r in turns} (FP64, rounded once), arg r added to
    the streamed element's B term in turns (plus half a turn for odd k when
    `alternate`), the phase C + B' + D in radians, one cosine (here exact in
    FP64 of the FP32 argument, plus `bias`), and the term |r| cos (negated
    for odd k)."""
    xh, xl = split(x)
    ych, ycl = split(yc)
    dxh, _ = split(x - xc)
    xch, xcl = split(xc)
    dyh, dyl = split(y - yc)
    C = frac_dot3(xh, xl, ych, ycl)
    B = frac_dot3(xch, xcl, dyh, dyl)
    rabs = np.hypot(r.real, r.imag).astype(f32)
    rho = (np.arctan2(r.imag, r.real) / (2 * math.pi)).astype(f32)
    odd = (np.arange(len(r)) % 2 == 1) & alternate
    b = B + np.where(odd, f32(0.5), f32(0.0))
    bp = frac_turns(b + rho) * TWO_PI_F                       # B + arg r (+ pi), radians
    dx = dxh * TWO_PI_F
    ph = fma32(dx[:, 2], dyh[:, 2], fma32(dx[:, 1], dyh[:, 1], fma32(dx[:, 0], dyh[:, 0], C * TWO_PI_F + bp)))
    cs = (np.cos(ph.astype(np.float64)) + bias).astype(f32)
    return np.where(odd, -rabs, rabs) * cs


def test_adjoint_polar_term_is_re_conj_a_r():
    """|r| cos(theta + arg r), with arg r folded into B and every other term
    taken as -cos(theta + pi), equals Re(conj(A) r) = Re(e^{2 pi i X.Y} r) to
    the phase split's micro-turn, at the wide-field and the largest accepted
    products."""
    rng = np.random.default_rng(6)
    for uv, w in ((2000.0, 500.0), (0.99 * 2.0 ** 21 / 0.5, 0.99 * 2.0 ** 19)):
        xc, x, yc, y = draw(rng, 200000, uv, w, 0.45, np.array([40.0, 40.0, 15.0]),
                            np.array([0.0156, 0.0156, 0.005]))
        # pixels own: X = (l, m, n - 1), Y = (u, v, w)
        r = rng.normal(size=len(x)) + 1j * rng.normal(size=len(x))
        got = adjoint_terms(yc, y, xc, x, r).astype(np.float64)
        want = (np.exp(2j * math.pi * (x * y).sum(axis=1)) * r).real
        err = np.abs(got - want) / np.abs(r)
        assert np.max(err) < 4e-6                  # 2 pi x the micro-turn phase bound, and rounding
        assert np.sqrt(np.mean(err ** 2)) < 4e-7


def test_alternating_signs_cancel_a_bias_of_the_cosine():
    """With the weights |r| all positive, a bias of the cosine adds up over a
    column's N terms; taking every other term as -cos(theta + pi) makes it
    cancel in pairs.  Over 400,000 terms a bias of 2e-8 moves the plain sum
    by ~1e-2 (N E|r| bias) and the alternated one by far less."""
    rng = np.random.default_rng(7)
    xc, x, yc, y = draw(rng, 400000, 1000.0, 250.0, 0.28, np.array([30.0, 30.0, 10.0]),
                        np.array([0.0024, 0.0024, 0.0008]))
    r = rng.normal(size=len(x)) + 1j * rng.normal(size=len(x))
    bias = 2e-8
    plain = adjoint_terms(yc, y, xc, x, r, alternate=False, bias=bias).astype(np.float64).sum()
    plain0 = adjoint_terms(yc, y, xc, x, r, alternate=False).astype(np.float64).sum()
    alt = adjoint_terms(yc, y, xc, x, r, alternate=True, bias=bias).astype(np.float64).sum()
    alt0 = adjoint_terms(yc, y, xc, x, r, alternate=True).astype(np.float64).sum()
    assert abs((plain - plain0) - bias * np.abs(r).sum()) < 0.05 * bias * np.abs(r).sum()
    assert abs(alt - alt0) < 0.02 * abs(plain - plain0)
