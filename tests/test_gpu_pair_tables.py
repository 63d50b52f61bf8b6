"""Gains through the per-granule antenna-pair tables and through the
per-visibility gathers they fall back to, in one problem.

With gains, each visibility granule's members are sorted by antenna pair; a
granule with at most 28 distinct pairs takes the pair-table forward, one with
more takes per-visibility gathers, and the adjoint forms each pair's gain
product once per run of equal pairs.  Here the visibilities with u below the
median use three antenna pairs (few pairs per granule) and the rest draw
random pairs among 16 antennas (up to 120 pairs), so a problem mixes both
forward paths and long and short runs in the adjoint.  Parity against the
FP64 oracle: max |d| / max |oracle| <= 1e-5 (mixed), 1e-10 (FP64).
"""
import numpy as np
import pytest

import oracle
from paper_1310_2078_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {0: 1e-10, 1: 1e-5}
DIRAC, PAR, WIDE = 0, 1, 2


def nmax_err(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


@pytest.fixture(scope="module")
def ctx(gpu_lib):
    c = gpu_lib.Context(0)
    yield c
    c.close()


def mixed_pairs(seed, n_vis, n_pix, kinds, uv_max, extent):
    d = synth.random_problem(seed, n_vis, n_pix, kinds=kinds, gains=True, n_ant=16, uv_max=uv_max,
                             w_max=uv_max / 3, extent=extent, sigma_max=0.01)
    few = np.array([[0, 1], [2, 5], [3, 4]], np.int32)
    low = d["uvw"][:, 0] < np.median(d["uvw"][:, 0])
    d["ant_pair"][low] = few[np.arange(low.sum()) % len(few)]
    return d


@pytest.mark.parametrize("kinds,uv_max,extent", [
    ((DIRAC,), 120.0, 0.1),                 # compact: few exact-phase tiles
    ((DIRAC, WIDE), 900.0, 0.4),            # wide: many exact-phase tiles
    ((DIRAC, PAR, WIDE), 400.0, 0.3)])
@pytest.mark.parametrize("prec", [0, 1])
def test_pair_tables_and_gather_fallback_match_oracle(ctx, kinds, uv_max, extent, prec):
    d = mixed_pairs(21, 3000, 700, kinds, uv_max, extent)
    P = ctx.problem()
    P.set_visibilities(d["uvw"], None, None, d["ant_pair"])
    P.set_pixels(d["lm"], d["sigma"], d["kind"])
    P.set_gains(d["gains"])
    O = oracle.Problem(d["uvw"], d["lm"], d["sigma"], d["kind"], None, d["ant_pair"], d["gains"])
    rng = np.random.default_rng(5)
    x = rng.normal(size=700)                # signed: the table folds x_j / n_j in
    assert nmax_err(P.forward(x, prec), oracle.forward(O, x)) <= TOL[prec]
    r = rng.normal(size=3000) + 1j * rng.normal(size=3000)
    assert nmax_err(P.adjoint(r, prec), oracle.adjoint(O, r)) <= TOL[prec]
    P.close()


def test_pair_tables_solve_matches_oracle(ctx):
    """A short FISTA solve on the mixed problem: same L and lambda, images
    within 1e-4 of the oracle's peak."""
    d = mixed_pairs(22, 1500, 400, (DIRAC, WIDE), 400.0, 0.3)
    O = oracle.Problem(d["uvw"], d["lm"], d["sigma"], d["kind"], None, d["ant_pair"], d["gains"])
    x_true = np.zeros(400)
    x_true[[7, 111, 250]] = [2.0, 1.0, 0.5]
    V = oracle.forward(O, x_true)
    P = ctx.problem()
    P.set_visibilities(d["uvw"], V, None, d["ant_pair"])
    P.set_pixels(d["lm"], d["sigma"], d["kind"])
    P.set_gains(d["gains"])
    L = 1.5 * oracle.power(O, max_iter=8)[0]
    lam = 0.05 * oracle.adjoint(O, V).max()
    img, _ = P.solve(lam, L=L, max_iter=12)
    img_o, _ = oracle.fista(O, V, lam, L, 12)
    assert np.max(np.abs(img - img_o)) <= 1e-4 * img_o.max()
    P.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_most_antennas_fit_and_match_oracle(ctx, gpu_lib, prec):
    """300 antennas, the most the gains kernels' shared memory holds (one
    pixel granule's table of 300 rows, the adjoint's per-warp slices and
    records): forward and adjoint against the oracle; 301 is refused."""
    d = synth.random_problem(31, 1500, 300, kinds=(DIRAC, WIDE), gains=True, n_ant=300, uv_max=300,
                             w_max=100, extent=0.3, sigma_max=0.01)
    P = ctx.problem()
    P.set_visibilities(d["uvw"], None, None, d["ant_pair"])
    P.set_pixels(d["lm"], d["sigma"], d["kind"])
    P.set_gains(d["gains"])
    O = oracle.Problem(d["uvw"], d["lm"], d["sigma"], d["kind"], None, d["ant_pair"], d["gains"])
    rng = np.random.default_rng(6)
    x = rng.normal(size=300)
    assert nmax_err(P.forward(x, prec), oracle.forward(O, x)) <= TOL[prec]
    r = rng.normal(size=1500) + 1j * rng.normal(size=1500)
    assert nmax_err(P.adjoint(r, prec), oracle.adjoint(O, r)) <= TOL[prec]
    with pytest.raises(gpu_lib.SL1MError) as e:
        P.set_gains(np.ones((300, 301), complex))
    assert e.value.status == gpu_lib.ERR_ARG
    P.close()
