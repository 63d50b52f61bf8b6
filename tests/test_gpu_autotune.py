"""The tile-shape autotuner: it picks a valid shape, and the operator and the
solve keep parity with the FP64 oracle under the tuned shape."""
import numpy as np
import pytest

import oracle
from paper_1310_2078_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kw", [dict(), dict(kinds=(0, 2), sigma_max=0.005)])
def test_autotune_choice_is_valid_and_keeps_parity(gpu_lib, kw):
    d = synth.random_problem(123, 6000, 5000, uv_max=900, w_max=250, extent=0.4, **kw)
    ctx = gpu_lib.Context(0)
    P = ctx.problem()
    P.set_visibilities(d["uvw"])
    P.set_pixels(d["lm"], d["sigma"], d["kind"])
    O = oracle.Problem(d["uvw"], d["lm"], d["sigma"], d["kind"])
    ch = P.autotune(gpu_lib.MIXED)
    assert ch["nst"][0] in (2, 4, 8) and ch["nst"][1] in (2, 4)
    assert all(1 <= k <= 4 for k in ch["ctas_per_sm"])
    assert all(n in (0, 1, 2) for n in ch["npoly"])
    rng = np.random.default_rng(9)
    x = np.abs(rng.normal(size=5000))
    f, fo = P.forward(x, gpu_lib.MIXED), oracle.forward(O, x)
    assert np.max(np.abs(f - fo)) / np.max(np.abs(fo)) <= 1e-5
    r = rng.normal(size=6000) + 1j * rng.normal(size=6000)
    a, ao = P.adjoint(r, gpu_lib.MIXED), oracle.adjoint(O, r)
    assert np.max(np.abs(a - ao)) / np.max(np.abs(ao)) <= 1e-5
    # a solve built after tuning uses the tuned plans and still matches
    V = oracle.forward(O, (rng.random(5000) < 0.002) * 2.0)
    P.set_vis_data(V)
    # parity holds at any common step constant; 1.5x a short power iteration
    # keeps the steps stable without paying for a converged one on the CPU
    L = 1.5 * oracle.power(O, max_iter=5)[0]
    lam = 0.05 * oracle.adjoint(O, V).max()
    img, st = P.solve(lam, L=L, max_iter=8)
    img_o, _ = oracle.fista(O, V, lam, L, 8)
    assert np.max(np.abs(img - img_o)) <= 1e-4 * img_o.max()
    ctx.close()
