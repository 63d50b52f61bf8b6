"""Adaptive quadtree refinement (Sect. 4.4) on the GPU against the same rule
driven by oracle solves, and its saving against a solve on the full fine grid."""
import numpy as np
import pytest

import oracle
from paper_1310_2078_gb300 import synth

pytestmark = pytest.mark.gpu


def oracle_refine(uvw, V, lm0, delta0, lam, levels, frac, iters):
    """The refinement rule of sl1m_solve_refine, with oracle solves."""
    lm = lm0.copy()
    delta = np.full(len(lm), delta0)
    x0 = None
    margins = []
    for level in range(levels + 1):
        O = oracle.Problem(uvw, lm)
        L, _ = oracle.power(O)
        img, st = oracle.fista(O, V, lam, L, iters, x0=x0)
        if level == levels:
            break
        thr = frac * img.max()
        margins.append(np.min(np.abs(img - thr)) / thr)
        sel = img > thr
        nlm, nd, nx = [], [], []
        for j in range(len(lm)):
            if sel[j]:
                q = 0.25 * delta[j]
                for dl, dm in ((-q, -q), (q, -q), (-q, q), (q, q)):
                    nlm.append((lm[j, 0] + dl, lm[j, 1] + dm))
                    nd.append(0.5 * delta[j])
                    nx.append(0.25 * img[j])
            else:
                nlm.append(tuple(lm[j]))
                nd.append(delta[j])
                nx.append(img[j])
        lm, delta, x0 = np.array(nlm), np.array(nd), np.array(nx)
    return lm, img, min(margins) if margins else 1.0


def scene(n_coarse=8, extent=0.05, fine_side=64):
    rng = np.random.default_rng(7)
    ant = synth.antennas(rng, 16, 400.0, 3.0)
    uvw, ap = synth.uvw_tracks(ant, -30.0, 6)
    fine = synth.regular_grid(fine_side, extent)
    src = [fine_side * 20 + 22, fine_side * 40 + 41, fine_side * 45 + 12]
    x = np.zeros(fine_side * fine_side)
    x[src] = [1.0, 0.7, 0.4]
    V = oracle.forward(oracle.Problem(uvw, fine), x)
    coarse = synth.regular_grid(n_coarse, extent)
    return uvw, V, coarse, 2 * extent / n_coarse, fine, x


def test_refinement_matches_oracle_driven_refinement(gpu_lib):
    uvw, V, coarse, d0, fine, x = scene()
    lam, levels, frac, iters = 2.0, 2, 0.05, 80
    lm_o, img_o, margin = oracle_refine(uvw, V, coarse, d0, lam, levels, frac, iters)
    assert margin > 1e-3                 # no refinement decision sits on the threshold
    ctx = gpu_lib.Context(0)
    P = ctx.problem()
    P.set_visibilities(uvw, V)
    P.set_pixels(coarse)
    lm, img, st = P.solve_refine(lam, d0, levels, refine_frac=frac, max_iter=iters)
    assert st["levels_done"] == levels + 1
    assert lm.shape == lm_o.shape and np.allclose(lm, lm_o, rtol=0, atol=1e-15)
    assert np.max(np.abs(img - img_o)) <= 1e-4 * img_o.max()
    ctx.close()


def blob_scene(fine_side=128, extent=0.1, n_coarse=16):
    """Extended emission (three Gaussian blobs drawn on the fine grid, 2-3
    fine pixels wide), the kind of sky the paper refines (an HI galaxy)."""
    rng = np.random.default_rng(7)
    ant = synth.antennas(rng, 16, 400.0, 3.0)
    uvw, ap = synth.uvw_tracks(ant, -30.0, 6)
    fine = synth.regular_grid(fine_side, extent)
    d = 2 * extent / fine_side
    blobs = [((-0.04, -0.03), 3 * d, 3.0), ((0.03, 0.024), 2 * d, 2.0), ((-0.05, 0.044), 2.5 * d, 1.5)]
    x = np.zeros(len(fine))
    for c, s, f in blobs:
        p = np.exp(-((fine[:, 0] - c[0]) ** 2 + (fine[:, 1] - c[1]) ** 2) / (2 * s * s))
        p[p < np.exp(-4.5)] = 0
        x += f * p / p.sum()
    V = oracle.forward(oracle.Problem(uvw, fine), x)
    coarse = synth.regular_grid(n_coarse, extent)
    return uvw, V, coarse, 2 * extent / n_coarse, fine, blobs


def test_refinement_needs_far_fewer_pairs_than_the_fine_grid(gpu_lib):
    """Three levels from a 16x16 grid reach the 128x128 grid's spacing where
    there is emission: far fewer pair evaluations than the fine-grid solve,
    the same total flux, and most of each blob's flux where the fine-grid
    solve puts it."""
    uvw, V, coarse, d0, fine, blobs = blob_scene()
    lam, iters = 7.0, 150
    ctx = gpu_lib.Context(0)
    P = ctx.problem()
    P.set_visibilities(uvw, V)
    P.set_pixels(coarse)
    lm, img, st = P.solve_refine(lam, d0, 3, refine_frac=0.1, max_iter=iters)
    Q = ctx.problem()
    Q.set_visibilities(uvw, V)
    Q.set_pixels(fine)                    # the grid the refinement reaches (d0 / 8)
    img_f, st_f = Q.solve(lam, max_iter=iters)
    full = (2 * st_f["iters"] + 2 * st_f["power_iters"] + 2) * len(uvw) * len(fine)
    assert st["total_pair_evals"] < full / 3
    assert st["final_n_pix"] < len(fine) / 4
    assert abs(img.sum() - img_f.sum()) < 0.1 * img_f.sum()
    for c, s, f in blobs:
        r = 2 * s + d0 / 8
        a = img[np.hypot(lm[:, 0] - c[0], lm[:, 1] - c[1]) < r].sum()
        b = img_f[np.hypot(fine[:, 0] - c[0], fine[:, 1] - c[1]) < r].sum()
        assert a > 0.5 * b
    ctx.close()
