"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds array geometry, pixel layouts and random draws only -- none
of the deconvolution method's arithmetic.  It does NOT compute visibilities:
the caller forms  V = A x_true + noise  with the operator of its choice (the
test suite with the FP64 oracle, the benchmark with the library's own
forward).  Both the oracle tests and the GPU path draw their inputs here.

Geometry (Sect. 4.1 of Hardy 2013 describes the structure, not the numbers):
antennas uniform in a disk with Gaussian height scatter, snapshots every
T/N_t over one hour, the field centre at zenith at the first snapshot (so the
latitude equals the declination), no primary beam unless gains are enabled,
and Gaussian noise added to the real and imaginary parts separately.

uvw follow the textbook rotation of a local east-north-up baseline into the
(u, v, w) frame of a source at hour angle H and declination dec (Thompson,
Moran & Swenson, Interferometry and Synthesis in Radio Astronomy, ch. 4).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

C_LIGHT = 299_792_458.0
WAVELENGTH_150MHZ = C_LIGHT / 150e6          # 1.99862 m
SIDEREAL_DAY_S = 86164.0905
BASE_SEED = 13102078

DIRAC, GAUSS_PARAXIAL, GAUSS_WIDE = 0, 1, 2


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def antennas(rng, n_ant: int, radius_m: float, height_sigma_m: float) -> np.ndarray:
    """[n_ant, 3] east/north/up positions: uniform in a disk, N(0, h) heights."""
    r = radius_m * np.sqrt(rng.random(n_ant))
    th = 2.0 * math.pi * rng.random(n_ant)
    up = rng.normal(0.0, height_sigma_m, n_ant)
    return np.stack([r * np.cos(th), r * np.sin(th), up], axis=1)


def uvw_tracks(enu: np.ndarray, dec_deg: float, n_times: int,
               duration_s: float = 3600.0, wavelength_m: float = WAVELENGTH_150MHZ):
    """uvw [n_vis, 3] (wavelengths) and ant_pair [n_vis, 2], time-major, a < b.

    Latitude = declination, so the field centre is at zenith at t = 0.
    """
    lat = math.radians(dec_deg)
    dec = lat
    n_ant = enu.shape[0]
    a_idx, b_idx = np.triu_indices(n_ant, k=1)
    d = enu[b_idx] - enu[a_idx]                      # baseline b - a, metres
    e, n, u_ = d[:, 0], d[:, 1], d[:, 2]
    # local (E, N, U) -> equatorial (X toward H=0 on the equator, Y east, Z pole)
    X = -n * math.sin(lat) + u_ * math.cos(lat)
    Y = e
    Z = n * math.cos(lat) + u_ * math.sin(lat)
    out, pairs = [], []
    sd, cd = math.sin(dec), math.cos(dec)
    for i in range(n_times):
        t = i * duration_s / n_times
        H = 2.0 * math.pi * t / SIDEREAL_DAY_S
        sh, ch = math.sin(H), math.cos(H)
        uu = sh * X + ch * Y
        vv = -sd * ch * X + sd * sh * Y + cd * Z
        ww = cd * ch * X - cd * sh * Y + sd * Z
        out.append(np.stack([uu, vv, ww], axis=1) / wavelength_m)
        pairs.append(np.stack([a_idx, b_idx], axis=1))
    return np.concatenate(out).astype(np.float64), np.concatenate(pairs).astype(np.int32)


def regular_grid(n_side: int, extent: float) -> np.ndarray:
    """[n_side^2, 2] (l, m): l_i = (i - N/2) Delta, Delta = 2 extent / N.

    Linear index k = row * N + col, l from col = k mod N and m from
    row = floor(k / N); a pixel sits exactly at the phase centre.
    """
    delta = 2.0 * extent / n_side
    idx = np.arange(n_side * n_side)
    l = (idx % n_side - n_side // 2) * delta
    m = (idx // n_side - n_side // 2) * delta
    return np.stack([l, m], axis=1).astype(np.float64)


def inner_pixels(n_side: int, frac: float = 0.8) -> np.ndarray:
    """Linear indices of the pixels in the central `frac` of each axis."""
    lo = int(round(n_side * (1.0 - frac) / 2.0))
    hi = n_side - lo
    r, c = np.meshgrid(np.arange(lo, hi), np.arange(lo, hi), indexing="ij")
    return (r * n_side + c).ravel()


def complex_noise(rng, n: int, sigma: float) -> np.ndarray:
    """Independent N(0, sigma) on the real and the imaginary part."""
    if sigma <= 0:
        return np.zeros(n, dtype=np.complex128)
    return rng.normal(0.0, sigma, n) + 1j * rng.normal(0.0, sigma, n)


def beam_gains(rng, lm: np.ndarray, n_ant: int, theta=(0.2, 0.3), ramp=1.0) -> np.ndarray:
    """G[j][a] = exp(-(l^2+m^2)/(2 theta_a^2)) * exp(2 pi i (alpha_a l + beta_a m)).

    theta_a ~ U(theta), alpha_a, beta_a ~ U(-ramp, ramp): a Gaussian primary
    beam per antenna times a seeded phase ramp (a pointing/ionospheric shift).
    """
    th = rng.uniform(theta[0], theta[1], n_ant)
    al = rng.uniform(-ramp, ramp, n_ant)
    be = rng.uniform(-ramp, ramp, n_ant)
    r2 = (lm ** 2).sum(axis=1)[:, None]
    amp = np.exp(-r2 / (2.0 * th[None, :] ** 2))
    ph = 2.0 * math.pi * (lm[:, 0:1] * al[None, :] + lm[:, 1:2] * be[None, :])
    return amp * np.exp(1j * ph)


def power_law_fluxes(rng, n: int, index: float = -1.8, smin=0.01, smax=10.0) -> np.ndarray:
    """dN/dS proportional to S^index on [smin, smax], by inverse CDF."""
    a = index + 1.0
    u = rng.random(n)
    return (smin ** a + u * (smax ** a - smin ** a)) ** (1.0 / a)


@dataclass
class Workload:
    """One synthetic deconvolution problem (inputs only, no visibilities)."""
    name: str
    uvw: np.ndarray
    ant_pair: np.ndarray
    lm: np.ndarray
    x_true: np.ndarray
    noise: np.ndarray
    sigma: np.ndarray | None = None
    kind: np.ndarray | None = None
    gains: np.ndarray | None = None
    weights: np.ndarray | None = None
    n_iter: int = 200
    lambda_frac: float = 0.02
    precision: str = "mixed"
    meta: dict = field(default_factory=dict)

    @property
    def n_vis(self):
        return self.uvw.shape[0]

    @property
    def n_pix(self):
        return self.lm.shape[0]

    @property
    def pairs(self):
        return self.n_vis * self.n_pix


def _array(rng, n_ant, radius, hsig, dec, n_times, max_vis=None):
    enu = antennas(rng, n_ant, radius, hsig)
    uvw, ap = uvw_tracks(enu, dec, n_times)
    if max_vis is not None:
        uvw, ap = uvw[:max_vis], ap[:max_vis]
    return uvw, ap


def config1(scale: float = 1.0) -> Workload:
    """32x32 Dirac grid over +/-0.05, 24 antennas (R=500 m, h=5 m), dec -30,
    8 snapshots -> 2,208 visibilities, 10 point sources (Exp(1 Jy)) on pixel
    centres, noise 0.01 Jy, FP64, 200 iterations."""
    rng = rng_for(BASE_SEED + 1)
    n_side = max(4, int(round(32 * scale)))
    uvw, ap = _array(rng, 24, 500.0, 5.0, -30.0, 8)
    lm = regular_grid(n_side, 0.05)
    x = np.zeros(n_side * n_side)
    src = rng.choice(inner_pixels(n_side), size=min(10, n_side * n_side // 4), replace=False)
    x[src] = rng.exponential(1.0, src.size)
    return Workload("plain-fp64-dirac-32x32-2208vis", uvw, ap, lm, x,
                    complex_noise(rng, uvw.shape[0], 0.01), precision="fp64",
                    meta={"n_side": n_side, "extent": 0.05})


def config2(n_side: int = 256, n_ant: int = 64, n_times: int = 20) -> Workload:
    """256x256 Dirac grid over +/-0.5 (w-term significant), 64 antennas
    (R=2 km, h=50 m), 20 snapshots -> 40,320 visibilities, 200 point sources
    (Exp(1 Jy)), noise 0.02 Jy, mixed precision."""
    rng = rng_for(BASE_SEED + 2)
    uvw, ap = _array(rng, n_ant, 2000.0, 50.0, -30.0, n_times)
    lm = regular_grid(n_side, 0.5)
    x = np.zeros(n_side * n_side)
    src = rng.choice(inner_pixels(n_side), size=min(200, n_side * n_side // 8), replace=False)
    x[src] = rng.exponential(1.0, src.size)
    return Workload(f"wide-field-dirac-{n_side}x{n_side}-{uvw.shape[0]}vis", uvw, ap, lm, x,
                    complex_noise(rng, uvw.shape[0], 0.02), precision="mixed",
                    meta={"n_side": n_side, "extent": 0.5})


def config3(n_side: int = 128, n_ant: int = 64, n_times: int = 16,
            max_vis: int | None = 32000) -> Workload:
    """128x128 jittered grid over +/-0.25 (jitter U(+/-0.3 Delta)) replicated at
    Dirac and wide-field Gaussian sigma = 1, 2, 4 Delta (65,536 pixels);
    per-antenna beam x phase-ramp gains; 64 antennas (R=1 km, h=20 m) x 16
    snapshots truncated to 32,000 visibilities; 50 points + 10 Gaussian blobs;
    noise 0.02 Jy; mixed precision."""
    rng = rng_for(BASE_SEED + 3)
    extent = 0.25
    delta = 2 * extent / n_side
    uvw, ap = _array(rng, n_ant, 1000.0, 20.0, -30.0, n_times, max_vis)
    base = regular_grid(n_side, extent)
    base = base + rng.uniform(-0.3 * delta, 0.3 * delta, base.shape)
    scales = [0.0, 1.0, 2.0, 4.0]
    lm = np.concatenate([base] * len(scales))
    sigma = np.concatenate([np.full(base.shape[0], s * delta) for s in scales])
    kind = np.concatenate([np.full(base.shape[0], DIRAC if s == 0 else GAUSS_WIDE, np.int32)
                           for s in scales])
    npb = base.shape[0]
    x = np.zeros(lm.shape[0])
    inner = inner_pixels(n_side)
    pts = rng.choice(inner, size=min(50, inner.size // 4), replace=False)
    x[pts] = rng.exponential(1.0, pts.size)
    blobs = rng.choice(inner, size=min(10, inner.size // 8), replace=False)
    which = rng.integers(2, 4, blobs.size)                # sigma = 2 or 4 Delta
    x[which * npb + blobs] = rng.exponential(2.0, blobs.size)
    gains = beam_gains(rng, lm, n_ant)
    return Workload(f"gains-multiscale-{lm.shape[0]}px-{uvw.shape[0]}vis", uvw, ap, lm, x,
                    complex_noise(rng, uvw.shape[0], 0.02), sigma=sigma, kind=kind,
                    gains=gains, precision="mixed",
                    meta={"n_side": n_side, "extent": extent, "scales": scales})


def config4(n_side: int = 1024, n_ant: int = 128, n_times: int = 50) -> Workload:
    """1024x1024 Dirac grid over +/-0.3, 128 antennas (R=1 km, h=30 m) x 50
    snapshots -> 406,400 visibilities, 2,000 power-law sources
    (S^-1.8 on [0.01, 10] Jy), noise 0.01 Jy, mixed precision."""
    rng = rng_for(BASE_SEED + 4)
    uvw, ap = _array(rng, n_ant, 1000.0, 30.0, -30.0, n_times)
    lm = regular_grid(n_side, 0.3)
    x = np.zeros(n_side * n_side)
    src = rng.choice(inner_pixels(n_side), size=min(2000, n_side * n_side // 8), replace=False)
    x[src] = power_law_fluxes(rng, src.size)
    return Workload(f"paper-scale-dirac-{n_side}x{n_side}-{uvw.shape[0]}vis", uvw, ap, lm, x,
                    complex_noise(rng, uvw.shape[0], 0.01), precision="mixed",
                    meta={"n_side": n_side, "extent": 0.3})


def table1(n_side: int = 1024, n_ant: int = 36, n_times: int = 60) -> Workload:
    """The setting of the noise-free lambda sweep (Sect. 4.1, Table 1): a
    1024x1024 Dirac grid of 30 arcsec pixels (+/-0.0745 in l,m), 36 antennas,
    one hour sampled every minute -> 630 baselines x 60 = 37,800 visibilities,
    declination -22.5 deg with the field at zenith at the start, 50 point
    sources of flux U(0.2, 2.0) on pixel centres in the inner 80%, no noise.
    The paper's antenna layout is not available: antennas are uniform in a
    3 km-radius disk with 5 m height scatter (readings), at 150 MHz."""
    rng = rng_for(BASE_SEED + 6)
    uvw, ap = _array(rng, n_ant, 3000.0, 5.0, -22.5, n_times)
    delta = 30.0 / 206264.806
    lm = regular_grid(n_side, 0.5 * n_side * delta)
    x = np.zeros(n_side * n_side)
    src = rng.choice(inner_pixels(n_side), size=min(50, n_side * n_side // 8), replace=False)
    x[src] = rng.uniform(0.2, 2.0, src.size)
    return Workload(f"table1-dirac-{n_side}x{n_side}-{uvw.shape[0]}vis", uvw, ap, lm, x,
                    np.zeros(uvw.shape[0], np.complex128), precision="mixed",
                    meta={"n_side": n_side, "extent": 0.5 * n_side * delta, "noise_free": True})


def serving_request(i: int, np_range=(4096, 262144), nv_range=(2048, 100_000),
                    seed_base: int = BASE_SEED + 5) -> Workload:
    """Request i of the serving stream: its own seed, pixels ~ logU(np_range),
    visibilities ~ logU(nv_range), Dirac or wide-Gaussian (50/50), gains on
    for 50%, 200 iterations or relative change of E below 1e-6."""
    rng = rng_for(seed_base * 1000 + i)
    n_pix = int(round(math.exp(rng.uniform(math.log(np_range[0]), math.log(np_range[1])))))
    n_vis = int(round(math.exp(rng.uniform(math.log(nv_range[0]), math.log(nv_range[1])))))
    n_side = max(8, int(round(math.sqrt(n_pix))))
    n_times = 10
    n_ant = max(4, int(math.ceil((1 + math.sqrt(1 + 8 * n_vis / n_times)) / 2)))
    uvw, ap = _array(rng, n_ant, 1000.0, 20.0, -30.0, n_times, n_vis)
    extent = 0.1
    lm = regular_grid(n_side, extent)
    gauss = bool(rng.random() < 0.5)
    sigma = kind = None
    if gauss:
        kind = np.full(lm.shape[0], GAUSS_WIDE, np.int32)
        sigma = np.full(lm.shape[0], 1.5 * 2 * extent / n_side)
    gains = beam_gains(rng, lm, n_ant) if rng.random() < 0.5 else None
    x = np.zeros(lm.shape[0])
    src = rng.choice(inner_pixels(n_side), size=min(20, lm.shape[0] // 8), replace=False)
    x[src] = rng.exponential(1.0, src.size)
    return Workload(f"request-{i}", uvw, ap, lm, x, complex_noise(rng, uvw.shape[0], 0.01),
                    sigma=sigma, kind=kind, gains=gains, n_iter=200, precision="mixed",
                    meta={"n_side": n_side, "tol": 1e-6})


def arrivals(n: int = 256, rate_hz: float = 20.0, seed: int = BASE_SEED + 5) -> np.ndarray:
    """Poisson arrival times (seconds) of the serving stream."""
    rng = rng_for(seed)
    return np.cumsum(rng.exponential(1.0 / rate_hz, n))


CONFIGS = {1: config1, 2: config2, 3: config3, 4: config4}


def random_problem(seed: int, n_vis: int, n_pix: int, kinds=(DIRAC,), gains=False,
                   weights=False, n_ant: int = 8, uv_max: float = 300.0,
                   w_max: float = 100.0, extent: float = 0.3, sigma_max: float = 0.01):
    """Small unstructured problem for unit tests: uniform uvw and pixel
    positions, per-pixel kind drawn from `kinds`, optional gains/weights.
    Returns a dict of arrays (uvw, lm, sigma, kind, weights, ant_pair, gains)."""
    rng = rng_for(seed)
    uvw = np.stack([rng.uniform(-uv_max, uv_max, n_vis), rng.uniform(-uv_max, uv_max, n_vis),
                    rng.uniform(-w_max, w_max, n_vis)], axis=1)
    r = extent * np.sqrt(rng.random(n_pix))
    th = 2 * math.pi * rng.random(n_pix)
    lm = np.stack([r * np.cos(th), r * np.sin(th)], axis=1)
    kind = rng.choice(np.asarray(kinds, dtype=np.int32), n_pix)
    sigma = np.where(kind == DIRAC, 0.0, rng.uniform(0.1, 1.0, n_pix) * sigma_max)
    a = rng.integers(0, n_ant, n_vis)
    b = (a + rng.integers(1, n_ant, n_vis)) % n_ant
    ant_pair = np.stack([np.minimum(a, b), np.maximum(a, b)], axis=1).astype(np.int32)
    out = dict(uvw=uvw, lm=lm, sigma=sigma, kind=kind.astype(np.int32), ant_pair=ant_pair,
               weights=None, gains=None)
    if weights:
        out["weights"] = rng.uniform(0.5, 2.0, n_vis)
    if gains:
        out["gains"] = beam_gains(rng, lm, n_ant, theta=(0.3, 0.5), ramp=0.5)
    return out
