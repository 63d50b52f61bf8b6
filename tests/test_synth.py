"""The seeded synthetic inputs follow their stated recipe (CPU only).

The checks rest on facts that do not depend on the generator's code: the
sizes the workloads name; the geometry of the sky (a source at zenith sees,
at hour angle 0, each baseline's east, north and up components as its u, v
and w; the projection on the Earth's axis is constant while the equatorial
part turns at the sidereal rate; rotations keep |b|); a pixel exactly at the
phase centre; and the stated distributions of positions, fluxes, noise and
arrivals.
"""
import math

import numpy as np
import pytest

from paper_1310_2078_gb300 import synth

LAMBDA = synth.WAVELENGTH_150MHZ


@pytest.mark.parametrize("cfg,n_pix,n_vis", [(1, 1024, 2208), (2, 65536, 40320), (3, 65536, 32000),
                                             (4, 1048576, 406400)])
def test_workload_sizes(cfg, n_pix, n_vis):
    w = synth.CONFIGS[cfg]()
    assert (w.n_pix, w.n_vis) == (n_pix, n_vis)
    assert w.noise.shape == (n_vis,) and w.x_true.shape == (n_pix,)
    assert w.ant_pair.shape == (n_vis, 2)


def test_sources_sit_on_pixels_in_the_inner_region():
    for cfg, n_src in ((1, 10), (2, 200)):
        w = synth.CONFIGS[cfg]()
        n = w.meta["n_side"]
        on = np.flatnonzero(w.x_true)
        assert on.size == n_src and np.all(w.x_true[on] > 0)
        assert set(on) <= set(synth.inner_pixels(n))
    w = synth.config4()
    s = w.x_true[w.x_true > 0]
    assert s.size == 2000 and s.min() >= 0.01 and s.max() <= 10.0


def test_zenith_source_at_hour_angle_zero_sees_the_enu_baseline():
    rng = synth.rng_for(7)
    enu = synth.antennas(rng, 6, 300.0, 10.0)
    uvw, ap = synth.uvw_tracks(enu, -30.0, 4)
    nb = 15
    d = enu[ap[:nb, 1]] - enu[ap[:nb, 0]]
    np.testing.assert_allclose(uvw[:nb] * LAMBDA, d, rtol=0, atol=1e-9)


@pytest.mark.parametrize("dec", [-30.0, 10.0, -70.0])
def test_earth_rotation_turns_the_equatorial_part_and_keeps_the_rest(dec):
    rng = synth.rng_for(8)
    enu = synth.antennas(rng, 7, 2000.0, 50.0)
    n_t = 6
    uvw, ap = synth.uvw_tracks(enu, dec, n_t)
    nb = 21
    t = uvw.reshape(n_t, nb, 3)
    sd, cd = math.sin(math.radians(dec)), math.cos(math.radians(dec))
    # |b| is kept
    L0 = np.linalg.norm(t[0], axis=1)
    for i in range(n_t):
        np.testing.assert_allclose(np.linalg.norm(t[i], axis=1), L0, rtol=1e-13)
    # the component along the Earth's axis, v cos(dec) + w sin(dec), is constant
    ax = t[..., 1] * cd + t[..., 2] * sd
    np.testing.assert_allclose(ax, np.broadcast_to(ax[0], ax.shape), rtol=0, atol=1e-9 * L0.max())
    # the equatorial part (w cos(dec) - v sin(dec), u) turns by H = 2 pi t / sidereal day
    ang = np.arctan2(t[..., 0], t[..., 2] * cd - t[..., 1] * sd)
    for i in range(n_t):
        H = 2 * math.pi * (i * 3600.0 / n_t) / synth.SIDEREAL_DAY_S
        dang = np.angle(np.exp(1j * (ang[i] - ang[0])))
        np.testing.assert_allclose(dang, H, rtol=0, atol=1e-9)


def test_records_are_time_major_with_a_below_b():
    w = synth.config1()
    n_ant, n_t = 24, 8
    nb = n_ant * (n_ant - 1) // 2
    assert w.n_vis == nb * n_t
    a, b = np.triu_indices(n_ant, k=1)
    for i in range(n_t):
        np.testing.assert_array_equal(w.ant_pair[i * nb:(i + 1) * nb], np.stack([a, b], axis=1))
    assert np.all(w.ant_pair[:, 0] < w.ant_pair[:, 1])


def test_antennas_fill_a_disk_with_gaussian_heights():
    rng = synth.rng_for(9)
    enu = synth.antennas(rng, 20000, 1000.0, 30.0)
    r = np.hypot(enu[:, 0], enu[:, 1])
    assert r.max() <= 1000.0
    # uniform in area: P(r < R/2) = 1/4
    assert abs(np.mean(r < 500.0) - 0.25) < 0.015
    assert abs(np.std(enu[:, 2]) - 30.0) < 1.0 and abs(np.mean(enu[:, 2])) < 1.0


def test_regular_grid_has_a_pixel_at_the_phase_centre():
    n, ext = 16, 0.3
    lm = synth.regular_grid(n, ext)
    delta = 2 * ext / n
    assert np.all(lm[(n // 2) * n + n // 2] == 0.0)
    assert lm[:, 0].min() == pytest.approx(-ext) and lm[:, 0].max() == pytest.approx(ext - delta)
    # row-major: l runs along a row, m along a column
    np.testing.assert_allclose(lm[1, 0] - lm[0, 0], delta)
    np.testing.assert_allclose(lm[n, 1] - lm[0, 1], delta)
    assert lm[1, 1] == lm[0, 1] and lm[n, 0] == lm[0, 0]


def test_jittered_multiscale_pixels_and_beam_gains():
    w = synth.config3()
    n = w.meta["n_side"]
    npb = n * n
    delta = 2 * w.meta["extent"] / n
    grid = synth.regular_grid(n, w.meta["extent"])
    for s, scale in enumerate(w.meta["scales"]):
        part = slice(s * npb, (s + 1) * npb)
        assert np.max(np.abs(w.lm[part] - grid)) <= 0.3 * delta
        np.testing.assert_allclose(w.sigma[part], scale * delta)
        assert np.all(w.kind[part] == (synth.DIRAC if scale == 0 else synth.GAUSS_WIDE))
    assert w.gains.shape == (4 * npb, 64)
    # |G_ja| = exp(-r^2 / (2 theta_a^2)) with theta_a in [0.2, 0.3]
    r2 = (w.lm ** 2).sum(axis=1)[:, None]
    amp = np.abs(w.gains)
    assert np.all(amp <= np.exp(-r2 / (2 * 0.3 ** 2)) * (1 + 1e-12))
    assert np.all(amp >= np.exp(-r2 / (2 * 0.2 ** 2)) * (1 - 1e-12))


def test_power_law_fluxes_follow_their_cdf():
    stats = pytest.importorskip("scipy.stats")
    rng = synth.rng_for(10)
    s = synth.power_law_fluxes(rng, 20000, index=-1.8, smin=0.01, smax=10.0)
    a = -0.8

    def cdf(x):
        return (np.clip(x, 0.01, 10.0) ** a - 0.01 ** a) / (10.0 ** a - 0.01 ** a)

    assert s.min() >= 0.01 and s.max() <= 10.0
    assert stats.kstest(s, cdf).pvalue > 1e-3


def test_noise_is_independent_on_real_and_imaginary_parts():
    rng = synth.rng_for(11)
    z = synth.complex_noise(rng, 200000, 0.02)
    assert abs(np.std(z.real) - 0.02) < 4e-4 and abs(np.std(z.imag) - 0.02) < 4e-4
    assert abs(np.corrcoef(z.real, z.imag)[0, 1]) < 0.01


def test_serving_stream_sizes_and_arrivals():
    for i in range(12):
        w = synth.serving_request(i)
        assert 60 ** 2 <= w.n_pix <= 513 ** 2
        assert 2048 <= w.n_vis <= 100000
        assert w.kind is None or np.all(w.kind == synth.GAUSS_WIDE)
    t = synth.arrivals(256, 20.0)
    assert np.all(np.diff(t) > 0)
    assert abs(np.mean(np.diff(np.concatenate([[0.0], t]))) - 0.05) < 0.015


def test_equal_seeds_give_equal_inputs():
    a, b = synth.config1(), synth.config1()
    for f in ("uvw", "lm", "x_true", "noise"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f))
    c = synth.random_problem(5, 50, 20, gains=True, weights=True)
    d = synth.random_problem(5, 50, 20, gains=True, weights=True)
    for k in c:
        if c[k] is not None:
            np.testing.assert_array_equal(c[k], d[k])


def test_table1_setting_has_the_papers_sizes():
    """The noise-free sweep of Table 1: 1024^2 pixels of 30 arcsec, 36 antennas
    sampled every minute for an hour (630 x 60 = 37,800 visibilities), 50
    sources of 0.2-2.0 on pixel centres in the inner 80%, no noise."""
    w = synth.table1()
    assert (w.n_pix, w.n_vis) == (1024 * 1024, 37800)
    delta = 30.0 / 206264.806
    assert np.allclose(np.diff(np.unique(w.lm[:, 0])), delta)
    on = np.flatnonzero(w.x_true)
    assert on.size == 50 and np.all((w.x_true[on] >= 0.2) & (w.x_true[on] <= 2.0))
    assert set(on) <= set(synth.inner_pixels(1024))
    assert np.all(w.noise == 0)
    assert np.array_equal(w.ant_pair[:630], np.stack(np.triu_indices(36, 1), axis=1))
