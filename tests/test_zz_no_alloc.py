"""sl1m_forward_noalloc: the forward operator for callers that cannot allocate
device memory at call time, with its scratch in a static device array.

Collected last on purpose (file name), so that a run stopping at the first
failure has already run every other test.  Works in a fresh process too.
"""
import numpy as np
import pytest

from paper_1310_2078_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {0: 1e-10, 1: 1e-5}


def _nmax(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("prec", [1, 0])
@pytest.mark.parametrize("kw", [dict(), dict(kinds=(0, 2), gains=True, n_ant=8)])
def test_noalloc_forward_matches_forward_dev_twice(gpu_lib, prec, kw):
    import torch
    d = synth.random_problem(77, 3001, 2500, uv_max=800, w_max=200, extent=0.3, **kw)
    ctx = gpu_lib.Context(0)
    P = ctx.problem()
    P.set_visibilities(d["uvw"], None, None, d["ant_pair"])
    P.set_pixels(d["lm"], d["sigma"], d["kind"])
    if d["gains"] is not None:
        P.set_gains(d["gains"])
    rng = np.random.default_rng(5)
    x0 = rng.normal(size=P.n_pix)
    P.forward(x0, prec)                        # an allocating call lays the problem out
    for call in range(2):                      # two calls in a row, different inputs
        x = torch.tensor(rng.normal(size=P.n_pix), dtype=torch.float64, device="cuda")
        want = torch.zeros((P.n_vis, 2), dtype=torch.float64, device="cuda")
        got = torch.full((P.n_vis, 2), float("nan"), dtype=torch.float64, device="cuda")
        P.forward_dev(x, want, prec)
        P.forward_noalloc(x, got, prec)
        torch.cuda.synchronize()
        w = want.cpu().numpy()
        g = got.cpu().numpy()
        assert np.all(np.isfinite(g))
        assert _nmax(g[:, 0] + 1j * g[:, 1], w[:, 0] + 1j * w[:, 1]) <= TOL[prec], call
    ctx.close()


def test_noalloc_rejects_problems_not_laid_out_or_too_large(gpu_lib):
    import torch
    ctx = gpu_lib.Context(0)
    P = ctx.problem()
    d = synth.random_problem(3, 100, 100)
    P.set_visibilities(d["uvw"])
    P.set_pixels(d["lm"])
    x = torch.zeros(100, dtype=torch.float64, device="cuda")
    out = torch.zeros((100, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(gpu_lib.SL1MError) as e:
        P.forward_noalloc(x, out)
    assert e.value.status == gpu_lib.ERR_STATE
    big = ctx.problem()
    d = synth.random_problem(4, 1_000_000, 300_000, uv_max=50, w_max=5)
    big.set_visibilities(d["uvw"])
    big.set_pixels(d["lm"])
    big.forward(np.zeros(300_000))
    xb = torch.zeros(300_000, dtype=torch.float64, device="cuda")
    ob = torch.zeros((1_000_000, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(gpu_lib.SL1MError) as e:
        big.forward_noalloc(xb, ob)
    assert e.value.status == gpu_lib.ERR_ARG
    assert "32 MiB" in str(e.value)
    ctx.close()
