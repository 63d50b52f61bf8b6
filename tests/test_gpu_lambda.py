"""Dirty image, lambda_max, a lambda sweep with the shape of Table 1 (Sect.
4.1: noise-free point sources), and warm starts (Sect. 4.4)."""
import numpy as np
import pytest

import oracle
from paper_1310_2078_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup(gpu_lib):
    w = synth.config1()                          # 32x32 Dirac grid, 2,208 visibilities
    O = oracle.Problem(w.uvw, w.lm)
    V = oracle.forward(O, w.x_true)              # noise-free, as Table 1
    ctx = gpu_lib.Context(0)
    P = ctx.problem()
    P.set_visibilities(w.uvw, V)
    P.set_pixels(w.lm)
    yield ctx, P, O, V, w
    ctx.close()


def test_dirty_image_and_lambda_max(gpu_lib, setup):
    ctx, P, O, V, w = setup
    for prec in (gpu_lib.FP64, gpu_lib.MIXED):
        img, lmax = P.dirty_image(prec)
        want = oracle.adjoint(O, V)
        tol = 1e-10 if prec == gpu_lib.FP64 else 1e-5
        assert np.max(np.abs(img - want)) <= tol * np.max(np.abs(want))
        assert lmax == pytest.approx(want.max(), rel=tol)
    L, _ = P.max_eig()
    img0, st0 = P.solve(1.0001 * lmax, L=L, max_iter=20)
    assert st0["nnz"] == 0 and np.all(img0 == 0)
    img1, st1 = P.solve(0.98 * lmax, L=L, max_iter=20)
    assert st1["nnz"] >= 1


def test_lambda_sweep_has_the_shape_of_table1(gpu_lib, setup):
    """Noise-free: for small lambda the L1 term approaches the true flux from
    below, the L2 term grows with lambda, and iterations to a 1e-6 relative
    change of E fall as lambda grows (Table 1)."""
    ctx, P, O, V, w = setup
    true_l1 = w.x_true.sum()
    _, lmax = P.dirty_image()
    L, _ = P.max_eig()
    fracs = [1e-4, 1e-3, 1e-2, 1e-1, 3e-1]
    res = []
    for f in fracs:
        img, st = P.solve(f * lmax, L=L, max_iter=6000, rel_tol=1e-6)
        res.append((f, img, st))
    l1 = np.array([st["l1"] for _, _, st in res])
    r2 = np.array([st["resid2"] for _, _, st in res])
    its = np.array([st["iters"] for _, _, st in res])
    assert np.all(l1 <= true_l1 * (1 + 1e-6))                 # the L1 bias is downward
    assert l1[0] > 0.97 * true_l1 and l1[1] > 0.9 * true_l1
    assert np.all(np.diff(l1) < 0) and np.all(np.diff(r2) > 0)
    assert its[-1] < its[0]
    # the recovered peaks sit on the true sources for small lambda
    on = w.x_true > 0
    err = np.abs(res[0][1] - w.x_true)
    assert err[on].max() < 0.05 * w.x_true[on].max()


def test_warm_start_along_the_sweep_saves_iterations(gpu_lib, setup):
    ctx, P, O, V, w = setup
    _, lmax = P.dirty_image()
    L, _ = P.max_eig()
    cold, warm = 0, 0
    prev = None
    for f in (1e-1, 3e-2, 1e-2):
        img_c, st_c = P.solve(f * lmax, L=L, max_iter=6000, rel_tol=1e-6)
        img_w, st_w = P.solve(f * lmax, L=L, max_iter=6000, rel_tol=1e-6, x0=prev)
        cold += st_c["iters"]
        warm += st_w["iters"]
        assert st_w["E"] <= st_c["E"] * (1 + 1e-4)
        prev = img_w
    assert warm < cold
