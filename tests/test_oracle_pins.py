"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these compares the oracle with itself re-typed: the expected values
come from hand-worked examples (tests/golden), numerical quadrature of the
paper's integrals, textbook closed forms, the adjoint identity, a dense
eigensolver, and brute-force enumeration of the L1 problem's supports.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1310_2078_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
DIRAC, PAR, WIDE = oracle.DIRAC, oracle.GAUSS_PARAXIAL, oracle.GAUSS_WIDE


def _quad_1d(f, x0, sigma, h_div=200, half=9.0):
    x = x0 + np.arange(-half * sigma, half * sigma + sigma / h_div / 2, sigma / h_div)
    return np.sum(f(x)) * (sigma / h_div)


def gaussian_paraxial_quadrature(l0, m0, sigma, u, v, w):
    """Eq. samlm3 integral with gain and 1/n frozen at the pixel centre.

    The integrand factorises into an l- and an m-integral; each is done by the
    trapezoid rule on a fine grid (spectrally accurate for a Gaussian)."""
    n0 = math.sqrt(1 - l0 * l0 - m0 * m0)

    def fl(x):
        return np.exp(-math.pi * (x - l0) ** 2 / sigma ** 2 + 1j * math.pi * w * x ** 2
                      - 2j * math.pi * u * x) / sigma

    def fm(x):
        return np.exp(-math.pi * (x - m0) ** 2 / sigma ** 2 + 1j * math.pi * w * x ** 2
                      - 2j * math.pi * v * x) / sigma

    return _quad_1d(fl, l0, sigma) * _quad_1d(fm, m0, sigma) / n0


def exact_gaussian_quadrature(l0, m0, sigma, u, v, w, h_div=60):
    """Eq. samlm integral of one unit Gaussian pixel with the exact n(l, m)
    everywhere (no Taylor step); 2-D trapezoid rule."""
    ax = np.arange(-7 * sigma, 7 * sigma + sigma / h_div / 2, sigma / h_div)
    L, M = np.meshgrid(l0 + ax, m0 + ax, indexing="ij")
    n = np.sqrt(1 - L ** 2 - M ** 2)
    f = np.exp(-math.pi * ((L - l0) ** 2 + (M - m0) ** 2) / sigma ** 2) / sigma ** 2
    g = f / n * np.exp(-2j * math.pi * (u * L + v * M + w * (n - 1)))
    # 1/n and the gain are taken at the centre by the closed form; undo the
    # variation of 1/n so that only the phase approximation is compared
    n0 = math.sqrt(1 - l0 * l0 - m0 * m0)
    return np.sum(g * n / n0) * (sigma / h_div) ** 2


# ---------------------------------------------------------------- Dirac entry

def test_dirac_hand_worked_values():
    rows = np.loadtxt(os.path.join(GOLDEN, "dirac_entries.txt"))
    for l, m, u, v, w, re, im in rows:
        a = oracle.entry(DIRAC, l, m, 0.0, u, v, w)
        assert abs(a - complex(re, im)) < 1e-13, (l, m, u, v, w, a)
    # the fixture's case 5: l^2 + m^2 = 1 is off the sky (n would be 0), refused
    with pytest.raises(ValueError):
        oracle.entry(DIRAC, -0.28, 0.96, 0.0, 1.0, 1.0, 1.0)


def test_phase_centre_source_gives_constant_visibilities():
    """A point source at the phase centre: V_k = flux for every baseline (n=1)."""
    d = synth.random_problem(1, 50, 7, uv_max=2000, w_max=500)
    lm = d["lm"].copy()
    lm[3] = 0.0
    P = oracle.Problem(d["uvw"], lm)
    x = np.zeros(7)
    x[3] = 2.5
    V = oracle.forward(P, x)
    assert np.max(np.abs(V - 2.5)) < 1e-13


def test_n_minus_one_is_cancellation_free():
    """n - 1 recovered from the w-phase matches its series to 1e-12 even at
    r^2 = 1e-8, where sqrt(1 - r^2) - 1 loses ~8 digits."""
    for r2 in (1e-8, 1e-6, 1e-3):
        l = math.sqrt(r2)
        exact = -r2 / 2 - r2 ** 2 / 8 - r2 ** 3 / 16 - 5 * r2 ** 4 / 128 - 7 * r2 ** 5 / 256
        w = 0.25 / abs(exact)                    # phase w (n - 1) = -0.25 turn
        a = oracle.entry(DIRAC, l, 0.0, 0.0, 0.0, 0.0, w)
        n = math.sqrt(1 - r2)
        # a = (1/n) exp(-2 pi i w (n-1)):  arg(a) = -2 pi w (n - 1)
        nm1 = -math.atan2(a.imag, a.real) / (2 * math.pi * w)
        assert abs(nm1 - exact) <= 1e-12 * abs(exact)
        assert abs(abs(a) - 1 / n) < 1e-15


# ----------------------------------------------------------- Gaussian entries

GAUSS_CASES = [
    # sigma, l, m, u, v, w
    (0.01, 0.03, -0.02, 150.0, -80.0, 60.0),
    (0.004, -0.1, 0.05, 400.0, 250.0, -300.0),
    (0.02, 0.0, 0.0, 30.0, 10.0, 500.0),
    (0.001, 0.2, 0.3, -900.0, 700.0, 200.0),
]


@pytest.mark.parametrize("case", GAUSS_CASES)
def test_gaussian_paraxial_matches_quadrature(case):
    """Eq. samlm4 (without the printed 1/sigma^2) equals the Eq. samlm3 integral."""
    s, l, m, u, v, w = case
    q = gaussian_paraxial_quadrature(l, m, s, u, v, w)
    a = oracle.entry(PAR, l, m, s, u, v, w)
    assert abs(a - q) <= 1e-10 * max(abs(q), 1e-300) + 1e-14


def test_gaussian_w0_is_fourier_transform_of_gaussian():
    """w -> 0: the textbook FT of a unit Gaussian, exp(-pi s^2 |u|^2) e^{-2 pi i u.x0}."""
    rng = np.random.default_rng(5)
    for _ in range(20):
        s = rng.uniform(1e-4, 0.02)
        l, m = rng.uniform(-0.3, 0.3, 2)
        u, v = rng.uniform(-300, 300, 2)
        n = math.sqrt(1 - l * l - m * m)
        ft = math.exp(-math.pi * s * s * (u * u + v * v)) * np.exp(-2j * math.pi * (u * l + v * m)) / n
        a = oracle.entry(PAR, l, m, s, u, v, 0.0)
        assert abs(a - ft) < 1e-13


@pytest.mark.parametrize("case", GAUSS_CASES)
def test_gaussian_wide_matches_frozen_phase_quadrature(case):
    """Eq. samlm5 = the integral whose non-quadratic phase is frozen at the
    pixel centre, i.e. the paraxial integral times exp(-2 pi i w (n0-1+r0^2/2))."""
    s, l, m, u, v, w = case
    r2 = l * l + m * m
    n0 = math.sqrt(1 - r2)
    frozen = np.exp(-2j * math.pi * w * (n0 - 1 + r2 / 2))
    q = gaussian_paraxial_quadrature(l, m, s, u, v, w) * frozen
    a = oracle.entry(WIDE, l, m, s, u, v, w)
    assert abs(a - q) <= 1e-10 * max(abs(q), 1e-300) + 1e-14


def test_gaussian_wide_sigma_to_zero_is_dirac():
    """sigma -> 0 of Eq. samlm5 is Eq. deltam exactly (this fixes the sign of
    the r^2/2 term; the printed sign would leave a phase exp(2 pi i w r^2))."""
    rng = np.random.default_rng(7)
    for _ in range(50):
        l, m = rng.uniform(-0.6, 0.6, 2)
        u, v, w = rng.uniform(-1500, 1500, 3)
        a = oracle.entry(WIDE, l, m, 1e-9, u, v, w)
        d = oracle.entry(DIRAC, l, m, 0.0, u, v, w)
        assert abs(a - d) < 1e-9 * abs(d)


def test_gaussian_paraxial_sigma_to_zero_is_paraxial_dirac():
    """sigma -> 0 of Eq. samlm4 is the paraxial point source: at small (l, m)
    it approaches Eq. deltam with an error that falls like w r^4."""
    for r in (0.02, 0.01, 0.005):
        l, m, u, v, w = r * 0.6, r * 0.8, 120.0, -40.0, 300.0
        a = oracle.entry(PAR, l, m, 1e-9, u, v, w)
        d = oracle.entry(DIRAC, l, m, 0.0, u, v, w)
        # phase of exp(-2 pi i w (n-1+r^2/2)) ~ 2 pi w r^4 / 8
        assert abs(a - d) / abs(d) < 2 * math.pi * w * r ** 4 / 8 * 1.1 + 1e-12


def test_gaussian_wide_converges_to_exact_integral():
    """Against Eq. samlm with the exact n(l, m) inside the integral, the
    wide-field pixel error shrinks as the pixel shrinks (its only
    approximation is the Taylor step inside one pixel)."""
    l, m, u, v, w = 0.35, 0.2, 150.0, -80.0, 60.0
    errs = []
    for s in (0.008, 0.004, 0.002):
        ex = exact_gaussian_quadrature(l, m, s, u, v, w)
        a = oracle.entry(WIDE, l, m, s, u, v, w)
        errs.append(abs(a - ex) / abs(ex))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.3 * errs[0]
    assert errs[2] < 1e-2


# ------------------------------------------------------------------ gains

def test_phase_ramp_gain_equals_uv_shift():
    """G[j][a] = exp(2 pi i (alpha_a l + beta_a m)) makes g_jk a phase ramp:
    for Dirac pixels the gained entry equals the ungained one at
    (u - (alpha_a - alpha_b), v - (beta_a - beta_b), w)."""
    rng = np.random.default_rng(11)
    d = synth.random_problem(3, 40, 12, n_ant=6)
    al, be = rng.uniform(-2, 2, 6), rng.uniform(-2, 2, 6)
    lm = d["lm"]
    G = np.exp(2j * np.pi * (lm[:, 0:1] * al[None] + lm[:, 1:2] * be[None]))
    P = oracle.Problem(d["uvw"], lm, ant_pair=d["ant_pair"], gains=G)
    for k in range(40):
        a, b = d["ant_pair"][k]
        u, v, w = d["uvw"][k]
        for j in range(12):
            want = oracle.entry(DIRAC, lm[j, 0], lm[j, 1], 0.0,
                                u - (al[a] - al[b]), v - (be[a] - be[b]), w)
            assert abs(oracle.entry_kj(P, k, j) - want) < 1e-12


def test_real_gains_scale_by_product_and_swap_conjugates():
    d = synth.random_problem(4, 30, 9, kinds=(DIRAC, PAR, WIDE), gains=True, n_ant=5)
    P = oracle.Problem(d["uvw"], d["lm"], d["sigma"], d["kind"], ant_pair=d["ant_pair"],
                       gains=d["gains"])
    P0 = oracle.Problem(d["uvw"], d["lm"], d["sigma"], d["kind"])
    ap_sw = d["ant_pair"][:, ::-1].copy()
    Psw = oracle.Problem(d["uvw"], d["lm"], d["sigma"], d["kind"], ant_pair=ap_sw,
                         gains=d["gains"])
    G = d["gains"]
    for k in range(30):
        a, b = d["ant_pair"][k]
        for j in range(9):
            g = G[j, a] * np.conj(G[j, b])
            e = oracle.entry_kj(P, k, j)
            e0 = oracle.entry_kj(P0, k, j)
            assert abs(abs(e) - abs(G[j, a]) * abs(G[j, b]) * abs(e0)) < 1e-12
            # swapping the antennas conjugates the gain product
            esw = oracle.entry_kj(Psw, k, j)
            assert abs(esw * g - e * np.conj(g)) < 1e-12


# ------------------------------------------------------ forward / adjoint

def _dense(P):
    return np.array([[oracle.entry_kj(P, k, j) for j in range(P.n_pix)] for k in range(P.n_vis)])


def _problem(seed, nv, npx, **kw):
    d = synth.random_problem(seed, nv, npx, **kw)
    return oracle.Problem(d["uvw"], d["lm"], d["sigma"], d["kind"], d["weights"],
                          d["ant_pair"], d["gains"]), d


@pytest.mark.parametrize("kw", [dict(), dict(kinds=(DIRAC, PAR, WIDE)),
                                dict(kinds=(DIRAC, WIDE), gains=True, weights=True)])
def test_forward_and_adjoint_match_dense_matrix(kw):
    P, d = _problem(21, 37, 23, **kw)
    A = _dense(P)
    rng = np.random.default_rng(0)
    x = rng.normal(size=23)
    x[rng.random(23) < 0.3] = 0.0
    assert np.allclose(oracle.forward(P, x), A @ x, rtol=0, atol=1e-12 * np.abs(A).sum())
    r = rng.normal(size=37) + 1j * rng.normal(size=37)
    assert np.allclose(oracle.adjoint(P, r), (A.conj().T @ r).real, rtol=0,
                       atol=1e-12 * np.abs(A).sum() * np.abs(r).max())
    rows = [5, 0, 36]
    assert np.allclose(oracle.forward(P, x, rows=rows), (A @ x)[rows], rtol=0, atol=1e-11)
    cols = [22, 3]
    assert np.allclose(oracle.adjoint(P, r, cols=cols), (A.conj().T @ r).real[cols],
                       rtol=0, atol=1e-11)


@pytest.mark.parametrize("kw", [dict(), dict(kinds=(DIRAC, PAR, WIDE), gains=True)])
def test_adjoint_identity(kw):
    """<A x, y>_R = <x, Re A^H y> to 1e-12 relative, all kinds, with gains."""
    P, d = _problem(31, 300, 200, uv_max=1500, w_max=400, **kw)
    rng = np.random.default_rng(1)
    for _ in range(3):
        x = rng.normal(size=200)
        y = rng.normal(size=300) + 1j * rng.normal(size=300)
        lhs = np.real(np.vdot(y, oracle.forward(P, x)))
        rhs = np.dot(x, oracle.adjoint(P, y))
        scale = np.abs(x).sum() * np.abs(y).sum()
        assert abs(lhs - rhs) <= 1e-12 * scale


# ------------------------------------------------------------------- L

def test_power_iteration_single_pixel_is_exact():
    P, d = _problem(41, 60, 1, weights=True, gains=True, kinds=(WIDE,))
    A = _dense(P)[:, 0]
    L, it = oracle.power(P, max_iter=5, tol=1e-14)
    assert abs(L - np.sum(d["weights"] * np.abs(A) ** 2)) < 1e-12 * L


def test_power_iteration_from_the_unit_start_vector():
    """N_p Dirac pixels all at the phase centre: every entry is exactly 1, so
    Re(A^H W A) = (sum_k W_k) J, whose top eigenvector is the start vector
    1/sqrt(N_p) (reading R8).  One step gives L = N_p sum W exactly, and the
    second step, which changes nothing, ends the iteration."""
    rng = np.random.default_rng(44)
    n_vis, n_pix = 37, 9
    W = rng.uniform(0.5, 2.0, n_vis)
    P = oracle.Problem(rng.uniform(-50, 50, size=(n_vis, 3)), np.zeros((n_pix, 2)), weights=W)
    want = n_pix * W.sum()
    L1, it1 = oracle.power(P, max_iter=1)
    assert it1 == 1 and abs(L1 - want) <= 1e-12 * want
    L, it = oracle.power(P, max_iter=50, tol=1e-6)
    assert it == 2 and abs(L - want) <= 1e-12 * want


def test_power_iteration_rises_each_step_and_is_scale_free():
    """For the symmetric positive semidefinite B = Re(A^H W A), each power
    step raises ||B x|| / ||x|| strictly until x is an eigenvector, and never
    above lambda_max.  The stopping rule is relative (reading R8): weights
    scaled by 1024 scale B, and every mu, exactly in binary floating point,
    so the iteration stops at the same step with L scaled by 1024; and L is
    the last step's estimate, the one a run of that many steps returns."""
    P, d = _problem(45, 70, 30, kinds=(DIRAC, PAR), weights=True, uv_max=120, w_max=30, sigma_max=0.02)
    A = _dense(P)
    W = d["weights"]
    lam = np.linalg.eigvalsh((A.conj().T @ (W[:, None] * A)).real)[-1]
    Lk = [oracle.power(P, max_iter=k, tol=0.0)[0] for k in range(1, 7)]
    assert np.all(np.diff(Lk) > 1e-9 * lam) and Lk[-1] <= lam * (1 + 1e-12)
    P2 = oracle.Problem(d["uvw"], d["lm"], d["sigma"], d["kind"], 1024.0 * W)
    for tol in (1e-3, 1e-6):
        L1, it1 = oracle.power(P, max_iter=500, tol=tol)
        L2, it2 = oracle.power(P2, max_iter=500, tol=tol)
        assert it1 == it2 < 500 and L2 == 1024.0 * L1
        # L is the estimate of the last step taken: the rule only decides when to stop
        assert oracle.power(P, max_iter=it1, tol=0.0)[0] == L1


@pytest.mark.parametrize("kw", [dict(), dict(kinds=(DIRAC, PAR), weights=True, gains=True)])
def test_power_iteration_matches_dense_eigensolver(kw):
    P, d = _problem(43, 80, 40, **kw)
    A = _dense(P)
    W = d["weights"] if d["weights"] is not None else np.ones(80)
    B = (A.conj().T @ (W[:, None] * A)).real
    lam = np.linalg.eigvalsh(B)[-1]
    L, it = oracle.power(P, max_iter=20000, tol=1e-15)
    assert abs(L - lam) < 1e-7 * lam
    # and the default stopping rule gives a lower bound close to it
    L6, _ = oracle.power(P, max_iter=50, tol=1e-6)
    assert L6 <= lam * (1 + 1e-12) and L6 > 0.9 * lam


# ----------------------------------------------------------------- FISTA

def _normal_eqs(A, W, V):
    B = (A.conj().T @ (W[:, None] * A)).real
    c = (A.conj().T @ (W * V)).real
    return B, c


def brute_force_l1(A, W, V, lam):
    """argmin_{x>=0} 1/2 sum W|Ax - V|^2 + lam sum x by enumerating supports."""
    B, c = _normal_eqs(A, W, V)
    n = B.shape[0]
    best, best_F = None, np.inf
    for mask in range(1 << n):
        S = [j for j in range(n) if mask >> j & 1]
        x = np.zeros(n)
        if S:
            xs = np.linalg.solve(B[np.ix_(S, S)], c[S] - lam)
            if np.any(xs <= 0):
                continue
            x[S] = xs
        grad = B @ x - c
        off = [j for j in range(n) if j not in S]
        if off and np.min(grad[off]) < -lam - 1e-9:
            continue
        r = A @ x - V
        F = 0.5 * np.sum(W * np.abs(r) ** 2) + lam * x.sum()
        if F < best_F:
            best, best_F = x, F
    return best, best_F


def test_fista_single_pixel_closed_form():
    """N_p = 1 with L = ||a||_W^2: one step reaches max(0, (Re a^H W V - lam)/||a||^2)."""
    P, d = _problem(51, 25, 1, weights=True)
    a = _dense(P)[:, 0]
    W = d["weights"]
    rng = np.random.default_rng(2)
    V = 3.0 * a + 0.1 * (rng.normal(size=25) + 1j * rng.normal(size=25))
    L = np.sum(W * np.abs(a) ** 2)
    for lam in (0.0, 1.0, 20.0, 1e4):
        want = max(0.0, (np.real(np.vdot(a, W * V)) - lam) / L)
        img, st = oracle.fista(P, V, lam, L, max_iter=1)
        assert abs(img[0] - want) < 1e-12 * max(1.0, want)
        img5, _ = oracle.fista(P, V, lam, L, max_iter=5)
        assert abs(img5[0] - want) < 1e-12 * max(1.0, want)


def test_fista_zero_above_lambda_max():
    """lam >= max_j Re(A^H W V)_j: the solution is exactly zero."""
    P, d = _problem(53, 60, 30, weights=True)
    A = _dense(P)
    rng = np.random.default_rng(3)
    V = A @ (np.abs(rng.normal(size=30)) * (rng.random(30) < 0.2))
    dirty = (A.conj().T @ (d["weights"] * V)).real
    L, _ = oracle.power(P)
    img, st = oracle.fista(P, V, dirty.max() * 1.0001, L, max_iter=50)
    assert np.all(img == 0.0) and st["nnz"] == 0


@pytest.mark.parametrize("seed", [61, 62, 63])
def test_fista_matches_brute_force_and_rate_bound(seed):
    """Small strictly convex problems: FISTA reaches the enumerated minimiser,
    and F(I_k) - F* <= 2 L ||I_0 - I*||^2 / (k+1)^2 (Beck & Teboulle 2009,
    Thm 4.4) holds along the way."""
    P, d = _problem(seed, 30, 6, kinds=(DIRAC, PAR), weights=True, uv_max=40, w_max=10,
                    extent=0.2, sigma_max=0.02)
    A = _dense(P)
    W = d["weights"]
    rng = np.random.default_rng(seed)
    xt = np.abs(rng.normal(size=6)) * (rng.random(6) < 0.5)
    V = A @ xt + 0.05 * (rng.normal(size=30) + 1j * rng.normal(size=30))
    lam = 0.5
    xs, Fs = brute_force_l1(A, W, V, lam)
    B, _ = _normal_eqs(A, W, V)
    L = np.linalg.eigvalsh(B)[-1]
    for k in (1, 2, 5, 10, 30, 100):
        img, st = oracle.fista(P, V, lam, L, max_iter=k)
        assert st["E"] - Fs <= 2 * L * np.sum(xs ** 2) / (k + 1) ** 2 + 1e-9
    img, st = oracle.fista(P, V, lam, L, max_iter=20000)
    assert np.max(np.abs(img - xs)) < 1e-7 * max(1.0, xs.max())
    assert abs(st["E"] - Fs) < 1e-10 * Fs


@pytest.mark.parametrize("solver", ["fista", "mfista"])
def test_warm_start_at_the_minimiser_is_a_fixed_point(solver):
    """Started at the enumerated minimiser x*, which the proximal gradient
    step T(x - grad/L) leaves in place (its optimality conditions), the
    first step returns x*: FISTA's I_1 and MFISTA's proximal point z_1.
    Started at zero, the same step lands elsewhere."""
    P, d = _problem(62, 30, 6, kinds=(DIRAC, PAR), weights=True, uv_max=40, w_max=10,
                    extent=0.2, sigma_max=0.02)
    A = _dense(P)
    W = d["weights"]
    rng = np.random.default_rng(62)
    xt = np.abs(rng.normal(size=6)) * (rng.random(6) < 0.5)
    V = A @ xt + 0.05 * (rng.normal(size=30) + 1j * rng.normal(size=30))
    lam = 0.5
    xs, _ = brute_force_l1(A, W, V, lam)
    B, _ = _normal_eqs(A, W, V)
    L = np.linalg.eigvalsh(B)[-1]
    if solver == "fista":
        warm, _ = oracle.fista(P, V, lam, L, max_iter=1, x0=xs)
        cold, _ = oracle.fista(P, V, lam, L, max_iter=1)
    else:
        warm = oracle.mfista(P, V, lam, L, 1, x0=xs, trace=True)[2]["z"][0]
        cold = oracle.mfista(P, V, lam, L, 1, trace=True)[2]["z"][0]
    assert np.max(np.abs(warm - xs)) < 1e-9 * max(1.0, xs.max())
    assert np.max(np.abs(cold - xs)) > 1e-3 * xs.max()


def test_fista_kkt_at_convergence():
    """I_j > 0 => Re(A^H W(AI - V))_j = -lam;  I_j = 0 => >= -lam."""
    P, d = _problem(71, 120, 40, kinds=(DIRAC, WIDE), gains=True, uv_max=60, w_max=20,
                    extent=0.2, sigma_max=0.02)
    A = _dense(P)
    rng = np.random.default_rng(4)
    xt = np.zeros(40)
    xt[rng.choice(40, 5, replace=False)] = rng.uniform(1, 3, 5)
    V = A @ xt
    lam = 0.3
    L, _ = oracle.power(P, max_iter=2000, tol=1e-14)
    img, st = oracle.fista(P, V, lam, L * 1.000001, max_iter=20000)
    g = (A.conj().T @ (A @ img - V)).real
    on = img > 0
    assert on.sum() >= 1
    assert np.max(np.abs(g[on] + lam)) < 1e-6 * lam
    assert np.min(g[~on]) > -lam * (1 + 1e-6)


def test_lambda_sweep_has_the_shape_of_table1():
    """Table 1 (Sect. 4.1, noise-free point sources) for its shape only (its
    values need the ASKAP layout): at the minimiser, the flux sum never
    exceeds the true one (the true image is feasible, so F(x*) <= F(x_true)),
    falls as lambda grows while the residual grows (both monotone along the
    L1 path), and tends to the true flux as lambda -> 0; convergence to a
    1e-6 relative change of E takes fewer steps at large lambda."""
    w = synth.config1(scale=0.25)              # 8x8 grid, 2,208 visibilities, 10 sources
    P = oracle.Problem(w.uvw, w.lm)
    V = oracle.forward(P, w.x_true)
    L, _ = oracle.power(P)
    lmax = oracle.adjoint(P, V).max()
    true_l1 = w.x_true.sum()
    runs = [oracle.fista(P, V, f * lmax, L, 6000, tol=1e-6)[1] for f in (1e-4, 1e-3, 1e-2, 1e-1, 3e-1)]
    l1 = np.array([st["l1"] for st in runs])
    r2 = np.array([st["resid2"] for st in runs])
    its = np.array([st["iters"] for st in runs])
    assert all(st["converged"] for st in runs)
    assert np.all(l1 <= true_l1 * (1 + 1e-6))
    assert np.all(np.diff(l1) < 0) and np.all(np.diff(r2) > 0)
    assert l1[0] > 0.999 * true_l1
    assert its[-1] < its[0]


def test_noise_free_isolated_sources_are_recovered():
    """Noise-free, isolated point sources on pixel centres, small lam: the
    recovered fluxes sit within the L1 bias (~lam/||a_j||^2) of the truth."""
    w = synth.config1(scale=0.5)           # 16x16 grid, 2,208 visibilities
    P = oracle.Problem(w.uvw, w.lm)
    V = oracle.forward(P, w.x_true)
    L, _ = oracle.power(P)
    lam = 1.0
    img, st = oracle.fista(P, V, lam, L, max_iter=1500)
    on = w.x_true > 0
    colnorm2 = np.array([np.sum(np.abs(oracle.forward(P, np.eye(1, w.n_pix, j)[0])) ** 2)
                         for j in np.flatnonzero(on)])
    bias = lam / colnorm2
    err = np.abs(img[on] - w.x_true[on])
    assert np.all(err < 5 * bias + 1e-3 * w.x_true[on].max())
    assert img[~on].sum() < 1e-2 * w.x_true.sum()
    assert st["l1"] < w.x_true.sum()


def test_stopping_rule_relative_change_of_E():
    P, d = _problem(81, 80, 30, uv_max=60, w_max=10)
    A = _dense(P)
    rng = np.random.default_rng(5)
    V = A @ (np.abs(rng.normal(size=30)) * (rng.random(30) < 0.3))
    L, _ = oracle.power(P)
    img, st = oracle.fista(P, V, 0.2, L, max_iter=5000, tol=1e-6)
    assert st["converged"] == 1 and st["iters"] < 5000
    # one more step changes E by no more than the tolerance's order
    img2, st2 = oracle.fista(P, V, 0.2, L, max_iter=st["iters"] - 1)
    assert abs(st["E"] - st2["E"]) <= 1e-6 * st2["E"] * (1 + 1e-9)
    # and it is the first step that does: the one before changed E by more
    assert st["iters"] >= 3
    _, st1 = oracle.fista(P, V, 0.2, L, max_iter=st["iters"] - 2)
    assert abs(st2["E"] - st1["E"]) > 1e-6 * st1["E"]
    # the rule is relative: V and lambda scaled by 1024 scale every iterate
    # and E (by 2^20) exactly, so the solve stops at the same step
    img3, st3 = oracle.fista(P, 1024.0 * V, 0.2 * 1024.0, L, max_iter=5000, tol=1e-6)
    assert st3["iters"] == st["iters"] and np.array_equal(img3, 1024.0 * img)
    assert st["E_paper"] == pytest.approx(st["resid2"] + 0.2 * st["l1"])


# ---------------------------------------------------------------- MFISTA

def _mfista_case(seed, lam=0.05):
    """A small ill-conditioned problem on which FISTA's objective oscillates,
    so that MFISTA rejects some proximal points."""
    P, d = _problem(seed, 30, 6, kinds=(DIRAC, PAR), weights=True, uv_max=40, w_max=10,
                    extent=0.2, sigma_max=0.02)
    A = _dense(P)
    W = d["weights"]
    rng = np.random.default_rng(seed)
    xt = np.abs(rng.normal(size=6)) * (rng.random(6) < 0.6)
    V = A @ xt + 0.02 * (rng.normal(size=30) + 1j * rng.normal(size=30))
    B, _ = _normal_eqs(A, W, V)
    L = np.linalg.eigvalsh(B)[-1]
    return P, A, W, V, L, lam


def _F(A, W, V, lam, x):
    return 0.5 * np.sum(W * np.abs(A @ x - V) ** 2) + lam * x.sum()


@pytest.mark.parametrize("seed", [61, 64])
def test_mfista_is_fista_until_the_first_rejection(seed):
    """While every proximal point is accepted, MFISTA's y-update reduces to
    FISTA's, so its iterates equal FISTA's bit for bit."""
    P, A, W, V, L, lam = _mfista_case(seed)
    _, st, tr = oracle.mfista(P, V, lam, L, 200, trace=True)
    rej = np.flatnonzero(tr["Fz"] > np.r_[_F(A, W, V, lam, np.zeros(6)), tr["Fx"][:-1]])
    assert len(rej) >= 1                        # the case does exercise a rejection
    first = rej[0]                              # step first+1 is the first rejected one
    assert first >= 2
    for k in (1, first):
        img, _ = oracle.fista(P, V, lam, L, max_iter=k)
        assert np.array_equal(img, tr["x"][k - 1])


@pytest.mark.parametrize("seed", [61, 64])
def test_mfista_steps_follow_the_estimate_sequence(seed):
    """Each step of the trace checked against forms other than the update the
    oracle codes: F recomputed from the dense matrix; x_k the better of z_k and
    x_{k-1}; z_k the KKT point of the proximal step at y_k; and y_{k+1} in the
    estimate-sequence form of the convergence proof,
        y_{k+1} = (1 - 1/t_{k+1}) x_k + u_k / t_{k+1},
        u_k = x_{k-1} + t_k (z_k - x_{k-1})."""
    P, A, W, V, L, lam = _mfista_case(seed)
    _, st, tr = oracle.mfista(P, V, lam, L, 120, trace=True)
    B, c = _normal_eqs(A, W, V)
    x_prev = np.zeros(6)
    Fx_prev = _F(A, W, V, lam, x_prev)
    n_rej = 0
    for k in range(len(tr["t"])):
        y, z, x, t = tr["y"][k], tr["z"][k], tr["x"][k], tr["t"][k]
        Fz = _F(A, W, V, lam, z)
        assert abs(Fz - tr["Fz"][k]) <= 1e-12 * Fz
        # z: for each j, either z_j > 0 and L (y - z)_j - grad_j = lam, or z_j = 0
        # and L y_j - grad_j <= lam, with grad = B y - c at y
        s = L * y - (B @ y - c)
        on = z > 0
        assert np.allclose(L * z[on], s[on] - lam, rtol=0, atol=1e-9 * (1 + np.abs(s).max()))
        assert np.all(s[~on] <= lam + 1e-9 * (1 + np.abs(s).max()))
        if Fz <= Fx_prev:
            assert np.array_equal(x, z)
        else:
            n_rej += 1
            assert np.array_equal(x, x_prev)
        if k + 1 < len(tr["t"]):
            tn = tr["t"][k + 1]
            assert tn == pytest.approx((1 + math.sqrt(1 + 4 * t * t)) / 2, rel=1e-15)
            u = x_prev + t * (z - x_prev)
            assert np.allclose(tr["y"][k + 1], (1 - 1 / tn) * x + u / tn, rtol=0,
                               atol=1e-12 * (1 + np.abs(u).max()))
        x_prev, Fx_prev = x, min(Fz, Fx_prev)
    assert n_rej >= 1


@pytest.mark.parametrize("seed", [61, 62, 63, 64])
def test_mfista_is_monotone_and_meets_the_rate_bound(seed):
    """F(x_k) never rises, F(x_k) - F* <= 2 L ||x_0 - x*||^2 / (k+1)^2
    (Beck & Teboulle 2009b), and the brute-force minimiser is reached."""
    P, A, W, V, L, lam = _mfista_case(seed, lam=0.5)
    xs, Fs = brute_force_l1(A, W, V, lam)
    _, st, tr = oracle.mfista(P, V, lam, L, 300, trace=True)
    Fx = np.array([_F(A, W, V, lam, x) for x in tr["x"]])
    assert np.all(np.diff(Fx) <= 1e-14 * Fx[0])
    k = np.arange(1, len(Fx) + 1)
    assert np.all(Fx - Fs <= 2 * L * np.sum(xs ** 2) / (k + 1) ** 2 + 1e-9)
    img, st = oracle.mfista(P, V, lam, L, max_iter=20000)
    assert np.max(np.abs(img - xs)) < 1e-7 * max(1.0, xs.max())
    assert abs(st["E"] - Fs) < 1e-10 * Fs


def test_mfista_single_pixel_closed_form():
    """N_p = 1 with L = ||a||_W^2: the first step reaches the minimiser and
    every later proximal point equals it."""
    P, d = _problem(51, 25, 1, weights=True)
    a = _dense(P)[:, 0]
    W = d["weights"]
    rng = np.random.default_rng(2)
    V = 3.0 * a + 0.1 * (rng.normal(size=25) + 1j * rng.normal(size=25))
    L = np.sum(W * np.abs(a) ** 2)
    for lam in (0.0, 1.0, 20.0, 1e4):
        want = max(0.0, (np.real(np.vdot(a, W * V)) - lam) / L)
        for k in (1, 5):
            img, st = oracle.mfista(P, V, lam, L, max_iter=k)
            assert abs(img[0] - want) < 1e-12 * max(1.0, want)


def test_mfista_stopping_rule():
    """With tol, MFISTA stops at the first step whose proposed objective
    change |F(z_k) - F(x_{k-1})| is within tol of F(x_{k-1})."""
    P, A, W, V, L, lam = _mfista_case(64, lam=0.2)
    _, _, tr = oracle.mfista(P, V, lam, L, 3000, trace=True)
    Fprev = np.r_[_F(A, W, V, lam, np.zeros(6)), tr["Fx"][:-1]]
    hit = np.flatnonzero(np.abs(tr["Fz"] - Fprev) <= 1e-6 * Fprev)
    assert len(hit) >= 1
    img, st = oracle.mfista(P, V, lam, L, 3000, tol=1e-6)
    assert st["converged"] == 1 and st["iters"] == hit[0] + 1
    assert np.array_equal(img, tr["x"][hit[0]])
    # the rule is relative: V and lambda times 1024 scale every iterate and F exactly
    img2, st2 = oracle.mfista(P, 1024.0 * V, 1024.0 * lam, L, 3000, tol=1e-6)
    assert st2["iters"] == st["iters"] and np.array_equal(img2, 1024.0 * img)
