"""sl1m_forward_noalloc: the forward operator for callers that cannot allocate
device memory when they call it (device memory owned by a pool or another
framework, or a loop that must not enter the allocator), with its scratch in
a static device array.

Checks, on two calls in a row: the output equals sl1m_forward_dev's within
the parity tolerance and the FP64 oracle's within the oracle tolerance; no
device memory is allocated (the library's own byte count and torch's
allocator are unchanged); the call returns while earlier work on its stream
is still running (it enqueues, it does not wait).

Collected last on purpose (file name), so that a run stopping at the first
failure has already run every other test.  Works in a fresh process too.
"""
import time

import numpy as np
import pytest

import oracle
from paper_1310_2078_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {0: 1e-10, 1: 1e-5}


def _nmax(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("prec", [1, 0])
@pytest.mark.parametrize("kw", [dict(), dict(kinds=(0, 2), gains=True, n_ant=8)])
def test_noalloc_forward_matches_forward_dev_and_oracle_twice(gpu_lib, prec, kw):
    import torch
    d = synth.random_problem(77, 3001, 2500, uv_max=800, w_max=200, extent=0.3, **kw)
    O = oracle.Problem(d["uvw"], d["lm"], d["sigma"], d["kind"], None, d["ant_pair"], d["gains"], threads=8)
    ctx = gpu_lib.Context(0, stream=torch.cuda.Stream())
    P = ctx.problem()
    P.set_visibilities(d["uvw"], None, None, d["ant_pair"])
    P.set_pixels(d["lm"], d["sigma"], d["kind"])
    if d["gains"] is not None:
        P.set_gains(d["gains"])
    rng = np.random.default_rng(5)
    x0 = rng.normal(size=P.n_pix)
    P.forward(x0, prec)                        # an allocating call lays the problem out
    for call in range(2):                      # two calls in a row, different inputs
        xh = rng.normal(size=P.n_pix)
        x = torch.tensor(xh, dtype=torch.float64, device="cuda")
        want = torch.zeros((P.n_vis, 2), dtype=torch.float64, device="cuda")
        got = torch.full((P.n_vis, 2), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()               # the fills (torch's stream) before the library's kernels
        P.forward_dev(x, want, prec)
        torch.cuda.synchronize()
        bytes_lib, bytes_torch = P.bytes(), torch.cuda.memory_allocated()
        P.forward_noalloc(x, got, prec)
        torch.cuda.synchronize()
        assert P.bytes() == bytes_lib and torch.cuda.memory_allocated() == bytes_torch
        w = want.cpu().numpy()
        g = got.cpu().numpy()
        assert np.all(np.isfinite(g))
        gc, wc = g[:, 0] + 1j * g[:, 1], w[:, 0] + 1j * w[:, 1]
        assert _nmax(gc, wc) <= TOL[prec], call
        assert _nmax(gc, oracle.forward(O, xh)) <= TOL[prec], call
    ctx.close()


def test_noalloc_returns_without_waiting_for_the_stream(gpu_lib):
    """Queued behind a long forward on the same stream, the call returns
    while that forward still runs, and its result is right afterwards."""
    import torch
    stream = torch.cuda.Stream()               # the context's stream (a handle the test can query)
    ctx = gpu_lib.Context(0, stream=stream)
    big = ctx.problem()
    db = synth.random_problem(8, 400_000, 200_000, uv_max=300, w_max=50)
    big.set_visibilities(db["uvw"])
    big.set_pixels(db["lm"])
    xb = torch.ones(200_000, dtype=torch.float64, device="cuda")
    ob = torch.zeros((400_000, 2), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    big.forward_dev(xb, ob)                    # lays it out (allocating call)
    small = ctx.problem()
    d = synth.random_problem(9, 500, 300)
    small.set_visibilities(d["uvw"])
    small.set_pixels(d["lm"])
    small.forward(np.zeros(300))
    x = torch.tensor(np.linspace(0, 1, 300), dtype=torch.float64, device="cuda")
    got = torch.zeros((500, 2), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    for _ in range(3):
        big.forward_dev(xb, ob)                # tens of milliseconds of GPU work
    t0 = time.perf_counter()
    small.forward_noalloc(x, got)
    dt = time.perf_counter() - t0
    busy = not stream.query()
    torch.cuda.synchronize()
    assert busy, "the stream drained before the call returned"
    assert dt < 0.5
    want = torch.zeros((500, 2), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    small.forward_dev(x, want)
    torch.cuda.synchronize()
    w, g = want.cpu().numpy(), got.cpu().numpy()
    assert _nmax(g[:, 0] + 1j * g[:, 1], w[:, 0] + 1j * w[:, 1]) <= TOL[1]
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
