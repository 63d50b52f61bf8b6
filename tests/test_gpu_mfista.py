"""MFISTA (the monotone FISTA of Beck & Teboulle 2009b that Sect. 3 names) on
the GPU: images and objective against the FP64 oracle at equal iteration
count, the objective never rising, the same result alone and in a server mix
beside FISTA solves, and the iteration count to a 1e-6 relative change."""
import numpy as np
import pytest

import oracle
from paper_1310_2078_gb300 import synth

pytestmark = pytest.mark.gpu


def case(seed=2, nv=600, npx=100, **kw):
    """An ill-conditioned problem whose MFISTA run rejects proximal points
    with a clear margin (steps 8, 9 and 16 for seed 2)."""
    d = synth.random_problem(seed, nv, npx, uv_max=40, w_max=10, extent=0.2, **kw)
    O = oracle.Problem(d["uvw"], d["lm"], d["sigma"], d["kind"], d["weights"], d["ant_pair"],
                       d["gains"])
    rng = np.random.default_rng(seed)
    xt = np.abs(rng.normal(size=npx)) * (rng.random(npx) < 0.1)
    V = oracle.forward(O, xt) + 0.01 * (rng.normal(size=nv) + 1j * rng.normal(size=nv))
    L, _ = oracle.power(O)
    lam = 0.01 * oracle.adjoint(O, V).max()
    return d, O, V, L, lam


def load(ctx, d, V):
    P = ctx.problem()
    P.set_visibilities(d["uvw"], V, d["weights"], d["ant_pair"])
    P.set_pixels(d["lm"], d["sigma"], d["kind"])
    if d["gains"] is not None:
        P.set_gains(d["gains"])
    return P


def rejections(O, V, lam, L, k, weights=None):
    _, _, tr = oracle.mfista(O, V, lam, L, k, trace=True)
    W = 1.0 if weights is None else weights
    Fprev = np.r_[0.5 * np.sum(W * np.abs(V) ** 2), tr["Fx"][:-1]]
    return np.flatnonzero((tr["Fz"] - Fprev) / Fprev > 1e-6) + 1


@pytest.mark.parametrize("kw", [dict(), dict(kinds=(0, 2), gains=True, weights=True, sigma_max=0.02)])
def test_mfista_matches_oracle(gpu_lib, kw):
    d, O, V, L, lam = case(**kw)
    assert len(rejections(O, V, lam, L, 20, d["weights"])) >= 1   # the reject branch runs
    ctx = gpu_lib.Context(0)
    P = load(ctx, d, V)
    for k in (1, 5, 12, 20):
        want, sw = oracle.mfista(O, V, lam, L, k)
        peak = max(want.max(), 1e-300)
        for prec, tol_img, tol_E in ((gpu_lib.FP64, 1e-9, 1e-11), (gpu_lib.MIXED, 1e-4, 1e-6)):
            img, st = P.solve(lam, L=L, max_iter=k, precision=prec, algorithm="mfista")
            assert st["iters"] == k
            assert np.max(np.abs(img - want)) <= tol_img * peak, (k, prec)
            assert abs(st["E"] - sw["E"]) <= tol_E * sw["E"], (k, prec)
            assert st["nnz"] == sw["nnz"] or prec == gpu_lib.MIXED
    ctx.close()


def test_mfista_objective_never_rises(gpu_lib):
    """Separate solves of 1..25 steps replay the same deterministic sequence;
    their E(x_k) is non-increasing, while FISTA's E(I_k) on the same problem
    rises somewhere."""
    d, O, V, L, lam = case()
    ctx = gpu_lib.Context(0)
    P = load(ctx, d, V)
    Em = [P.solve(lam, L=L, max_iter=k, algorithm="mfista")[1]["E"] for k in range(1, 26)]
    Ef = [P.solve(lam, L=L, max_iter=k)[1]["E"] for k in range(1, 26)]
    assert np.all(np.diff(Em) <= 0.0)
    assert np.any(np.diff(Ef) > 1e-6 * Ef[0])
    ctx.close()


def test_mfista_alone_and_in_a_mix_with_fista(gpu_lib):
    probs = [case(seed=s, nv=600 + 100 * s, npx=100 + 20 * s) for s in (2, 3, 4, 5)]
    ctx = gpu_lib.Context(0)
    Ps = [load(ctx, d, V) for d, O, V, L, lam in probs]
    algos = ["mfista", "fista", "mfista", "fista"]
    alone = [P.solve(c[4], L=c[3], max_iter=60, algorithm=a)
             for P, c, a in zip(Ps, probs, algos)]
    ctx.server_start(max_slots=8, ticks_per_round=3)
    tickets = [ctx.server_submit(P, c[4], L=c[3], max_iter=60, algorithm=a)
               for P, c, a in zip(Ps, probs, algos)]
    mixed = [ctx.server_wait(t, P, timeout_s=120.0) for t, P in zip(tickets, Ps)]
    ctx.server_stop()
    for (ia, sa), (im, sm), c, a in zip(alone, mixed, probs, algos):
        assert sm["iters"] == sa["iters"] == 60
        assert np.max(np.abs(ia - im)) <= 1e-4 * ia.max()
        want, sw = (oracle.mfista if a == "mfista" else oracle.fista)(c[1], c[2], c[4], c[3], 60)
        assert np.max(np.abs(im - want)) <= 1e-4 * want.max()
    ctx.close()


def test_mfista_iterations_to_tolerance(gpu_lib):
    """Both solvers stop on a 1e-6 relative change of E and reach the same
    objective; MFISTA's count is reported beside FISTA's."""
    w = synth.config1()
    O = oracle.Problem(w.uvw, w.lm)
    V = oracle.forward(O, w.x_true) + w.noise
    ctx = gpu_lib.Context(0)
    P = ctx.problem()
    P.set_visibilities(w.uvw, V)
    P.set_pixels(w.lm)
    _, lmax = P.dirty_image()
    L, _ = P.max_eig()
    _, sf = P.solve(0.02 * lmax, L=L, max_iter=5000, rel_tol=1e-6)
    _, sm = P.solve(0.02 * lmax, L=L, max_iter=5000, rel_tol=1e-6, algorithm="mfista")
    assert sf["converged"] and sm["converged"]
    assert abs(sm["E"] - sf["E"]) <= 1e-4 * sf["E"]
    print(f"iterations to 1e-6: FISTA {sf['iters']}, MFISTA {sm['iters']}")
    ctx.close()
