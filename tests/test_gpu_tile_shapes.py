"""Every tile shape of the mixed operator kernels -- streamed granules per
stage, CTAs per SM, and the share of pairs whose sincos runs on the FMA pipe
(a Chebyshev interpolant) instead of the SFU -- keeps parity with the FP64
oracle; shapes that do not exist are refused."""
import numpy as np
import pytest

import oracle
from paper_1310_2078_gb300 import synth

pytestmark = pytest.mark.gpu

NV, NP = 3001, 2503      # ragged: several granules and blocks plus a tail


@pytest.fixture(scope="module")
def case(gpu_lib):
    d = synth.random_problem(77, NV, NP, uv_max=900, w_max=250, extent=0.4)
    O = oracle.Problem(d["uvw"], d["lm"])
    rng = np.random.default_rng(5)
    x = np.abs(rng.normal(size=NP))
    r = rng.normal(size=NV) + 1j * rng.normal(size=NV)
    ctx = gpu_lib.Context(0)
    P = ctx.problem()
    P.set_visibilities(d["uvw"])
    P.set_pixels(d["lm"])
    yield ctx, P, x, r, oracle.forward(O, x), oracle.adjoint(O, r)
    ctx.close()


SHAPES = [(0, nst, npoly) for nst in (2, 4, 8) for npoly in (0, 1, 2)] + \
         [(1, nst, npoly) for nst in (2, 4) for npoly in (0, 1, 2)]


@pytest.mark.parametrize("op,nst,npoly", SHAPES)
def test_shape_keeps_parity(gpu_lib, case, op, nst, npoly):
    ctx, P, x, r, fo, ao = case
    for k in (1, 2):
        P.set_tile_shape(op, nst, k, npoly)
        if op == 0:
            got, want = P.forward(x, gpu_lib.MIXED), fo
        else:
            got, want = P.adjoint(r, gpu_lib.MIXED), ao
        assert np.max(np.abs(got - want)) / np.max(np.abs(want)) <= 1e-5, (op, nst, npoly, k)


def test_fma_sincos_changes_results_only_at_rounding_level(gpu_lib, case):
    ctx, P, x, r, fo, ao = case
    P.set_tile_shape(0, 8, 2, 0)
    f0 = P.forward(x, gpu_lib.MIXED)
    P.set_tile_shape(0, 8, 2, 2)
    f2 = P.forward(x, gpu_lib.MIXED)
    assert 0 < np.max(np.abs(f2 - f0)) <= 3e-6 * np.max(np.abs(fo))


def test_bad_shapes_are_refused(gpu_lib, case):
    ctx, P, *_ = case
    for args in ((0, 3, 1, 0), (1, 0, 1, 0), (0, 4, 1, 3), (2, 4, 1, 0), (0, 4, 99, 0), (0, 0, 1, 0), (1, 8, 1, 0)):
        with pytest.raises(gpu_lib.SL1MError) as e:
            P.set_tile_shape(*args)
        assert e.value.status == gpu_lib.ERR_ARG
