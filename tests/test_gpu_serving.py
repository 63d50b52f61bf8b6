"""Continuous-batching server on the GPU: every result is the same alone and
in the mix (within the image tolerance, 1e-4 of peak), requests that arrive
while others run join them, admission respects the memory budget, waits are
bounded, and the solve matches the FP64 oracle."""
import time

import numpy as np
import pytest

import oracle
from paper_1310_2078_gb300 import synth

pytestmark = pytest.mark.gpu


def small_requests(n, seed=0):
    """Uneven small problems: Dirac / wide Gaussian, gains on some."""
    out = []
    rng = np.random.default_rng(seed)
    for i in range(n):
        nv = int(rng.integers(300, 2500))
        npx = int(rng.integers(200, 1500))
        kinds = (0,) if i % 2 == 0 else (2,)
        d = synth.random_problem(1000 + i, nv, npx, kinds=kinds, gains=(i % 3 == 0), n_ant=8,
                                 uv_max=150, w_max=40, extent=0.15, sigma_max=0.005)
        x = np.zeros(npx)
        x[rng.choice(npx, 6, replace=False)] = rng.uniform(0.5, 2.0, 6)
        out.append((d, x))
    return out


def build(ctx, d, V):
    P = ctx.problem()
    P.set_visibilities(d["uvw"], V, d.get("weights"), d.get("ant_pair"))
    P.set_pixels(d["lm"], d.get("sigma"), d.get("kind"))
    if d.get("gains") is not None:
        P.set_gains(d["gains"])
    return P


def oracle_data(d, x, rng):
    O = oracle.Problem(d["uvw"], d["lm"], d["sigma"], d["kind"], None, d["ant_pair"], d["gains"])
    V = oracle.forward(O, x)
    V = V + 0.01 * np.abs(V).max() * (rng.normal(size=V.size) + 1j * rng.normal(size=V.size))
    return O, V


@pytest.fixture(scope="module")
def reqs():
    rng = np.random.default_rng(1)
    out = []
    for d, x in small_requests(10):
        O, V = oracle_data(d, x, rng)
        L, _ = oracle.power(O)
        lam = 0.05 * oracle.adjoint(O, V).max()
        out.append(dict(d=d, x=x, O=O, V=V, L=L, lam=lam))
    return out


def test_alone_vs_in_the_mix(gpu_lib, reqs):
    # alone: one context, sequential single solves
    ctx1 = gpu_lib.Context(0)
    alone = []
    for r in reqs:
        P = build(ctx1, r["d"], r["V"])
        img, st = P.solve(r["lam"], L=r["L"], max_iter=120, precision=gpu_lib.MIXED)
        alone.append((img, st))
    ctx1.close()
    # in the mix: a server; half submitted up front, the rest while it runs
    ctx = gpu_lib.Context(0)
    ctx.server_start(max_slots=16, ticks_per_round=4)
    probs = [build(ctx, r["d"], r["V"]) for r in reqs]
    tickets = [ctx.server_submit(probs[i], reqs[i]["lam"], L=reqs[i]["L"], max_iter=120)
               for i in range(5)]
    time.sleep(0.02)
    tickets += [ctx.server_submit(probs[i], reqs[i]["lam"], L=reqs[i]["L"], max_iter=120)
                for i in range(5, 10)]
    for i, t in enumerate(tickets):
        img, st = ctx.server_wait(t, probs[i], timeout_s=120.0)
        a, sa = alone[i]
        assert st["iters"] == sa["iters"] == 120
        assert np.max(np.abs(img - a)) <= 1e-4 * max(a.max(), 1e-30), i
        assert st["E"] == pytest.approx(sa["E"], rel=1e-6)
        # and both match the FP64 oracle at equal iteration count
        img_o, _ = oracle.fista(reqs[i]["O"], reqs[i]["V"], reqs[i]["lam"], reqs[i]["L"], 120)
        assert np.max(np.abs(img - img_o)) <= 1e-4 * img_o.max(), i
        assert st["seconds"] > 0
    info = ctx.server_info()
    assert info["finished"] == 10 and info["max_active"] >= 2
    ctx.server_stop()
    ctx.close()


def test_power_iteration_inside_the_server(gpu_lib, reqs):
    ctx = gpu_lib.Context(0)
    ctx.server_start(max_slots=4)
    probs = [build(ctx, r["d"], r["V"]) for r in reqs[:4]]
    tickets = [ctx.server_submit(P, r["lam"], L=0.0, max_iter=40) for P, r in zip(probs, reqs)]
    for P, r, t in zip(probs, reqs, tickets):
        img, st = ctx.server_wait(t, P, timeout_s=120.0)
        Lo, _ = oracle.power(r["O"])
        assert abs(st["L"] - Lo) <= 1e-5 * Lo
        img_o, _ = oracle.fista(r["O"], r["V"], r["lam"], st["L"], 40)
        assert np.max(np.abs(img - img_o)) <= 1e-4 * img_o.max()
    ctx.server_stop()
    ctx.close()


def test_admission_by_memory_budget_and_timeouts(gpu_lib):
    """Equal-size problems under a budget of about two: they queue and run."""
    ctx = gpu_lib.Context(0)
    rng = np.random.default_rng(3)
    probs, lams = [], []
    for i in range(8):
        d = synth.random_problem(2000 + i, 1500, 900, uv_max=150, w_max=40, extent=0.15)
        x = np.zeros(900)
        x[rng.choice(900, 5, replace=False)] = 1.0
        O = oracle.Problem(d["uvw"], d["lm"])
        V = oracle.forward(O, x)
        P = build(ctx, d, V)
        probs.append(P)
        lams.append(0.05 * np.abs(V).max())
    probs[0].forward(np.zeros(900))              # lay one out to measure its footprint
    budget = int(2.5 * probs[0].bytes())
    ctx.server_start(mem_budget_bytes=budget, max_slots=64, ticks_per_round=2)
    tickets = [ctx.server_submit(P, lam, L=0.0, max_iter=60) for P, lam in zip(probs, lams)]
    with pytest.raises(gpu_lib.SL1MError) as e:
        ctx.server_wait(tickets[-1], probs[-1], timeout_s=0.0)
    assert e.value.status == gpu_lib.ERR_TIMEOUT
    with pytest.raises(gpu_lib.SL1MError) as e:
        probs[0].forward(np.zeros(900))          # operator calls are refused while serving
    assert e.value.status == gpu_lib.ERR_BUSY
    for P, t in zip(probs, tickets):
        img, st = ctx.server_wait(t, P, timeout_s=120.0)
        assert st["iters"] == 60
    info = ctx.server_info()
    assert 1 <= info["max_active"] <= 3
    assert info["bytes_budget"] == budget and info["finished"] == 8
    big = ctx.problem()
    d = synth.random_problem(5, 200000, 2000)
    big.set_visibilities(d["uvw"])
    big.set_pixels(d["lm"])
    with pytest.raises(gpu_lib.SL1MError) as e:
        ctx.server_submit(big, 1.0, L=1.0, max_iter=1)
    assert e.value.status == gpu_lib.ERR_BUSY
    ctx.server_stop()
    ctx.close()


def test_stop_drains_queue(gpu_lib, reqs):
    ctx = gpu_lib.Context(0)
    ctx.server_start(max_slots=2, ticks_per_round=8)
    probs = [build(ctx, r["d"], r["V"]) for r in reqs[:6]]
    tickets = [ctx.server_submit(P, r["lam"], L=r["L"], max_iter=30) for P, r in zip(probs, reqs)]
    ctx.server_stop()                     # finishes everything queued
    for P, t in zip(probs, tickets):
        assert ctx.server_poll(t)
        img, st = ctx.server_wait(t, P, timeout_s=0.0)
        assert st["iters"] == 30
    # the context serves ordinary calls again
    img, st = probs[0].solve(reqs[0]["lam"], L=reqs[0]["L"], max_iter=5)
    assert st["iters"] == 5
    ctx.close()


@pytest.mark.parametrize("admission", ["two_lanes", "arrival"])
def test_small_request_passes_a_large_one_that_waits(gpu_lib, admission):
    """Admission lanes.  Under a work budget that one large request fills, a
    second large request waits for the first; a small request submitted after
    both is admitted at once under the two-lane policy (it finishes while the
    first large one still runs), but under arrival-order admission it waits
    behind the second large one (the first has finished by then).  Either
    way its image is the one it gets alone."""
    mode = gpu_lib.ADMIT_TWO_LANES if admission == "two_lanes" else gpu_lib.ADMIT_ARRIVAL
    ctx = gpu_lib.Context(0)
    rng = np.random.default_rng(7)
    probs, lams = [], []
    for i, (nv, npx) in enumerate([(4000, 3000), (4000, 3000), (300, 200)]):
        d = synth.random_problem(3000 + i, nv, npx, uv_max=150, w_max=40, extent=0.15)
        x = np.zeros(npx)
        x[rng.choice(npx, 5, replace=False)] = 1.0
        V = oracle.forward(oracle.Problem(d["uvw"], d["lm"]), x)
        probs.append(build(ctx, d, V))
        lams.append(0.05 * np.abs(V).max())
    # L above each problem's ||A||_F^2 (>= its largest eigenvalue): a valid FISTA step
    alone, _ = probs[2].solve(lams[2], L=1e5, max_iter=20)
    ctx.server_start(max_slots=8, ticks_per_round=4, max_pairs_per_tick=1.3e7, admission=mode)
    big = [ctx.server_submit(probs[i], lams[i], L=2e7, max_iter=400) for i in range(2)]
    small = ctx.server_submit(probs[2], lams[2], L=1e5, max_iter=20)
    img, st = ctx.server_wait(small, probs[2], timeout_s=120.0)
    first_large_done = ctx.server_poll(big[0])
    assert first_large_done == (admission == "arrival")
    assert np.max(np.abs(img - alone)) <= 1e-4 * max(alone.max(), 1e-30)
    for i, t in enumerate(big):
        ctx.server_wait(t, probs[i], timeout_s=120.0)
    ctx.server_stop()
    ctx.close()
