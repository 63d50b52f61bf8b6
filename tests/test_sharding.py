"""Multi-process sharding arithmetic on CPU (gloo, world_size 2).

A single SL1M solve shards two ways, each with one exchange per iteration:

* by visibilities: each rank holds N_v/P visibilities and a replica of the
  image; the forward is local, the adjoint yields partial images that are
  all-reduced (N_p reals), and the FISTA update is replicated;
* by pixels: each rank holds N_p/P pixels and their image entries; the
  forward yields partial visibilities that are all-reduced (2 N_v reals),
  the residual is replicated, and the adjoint and the threshold step are
  local.

The cheaper split exchanges min(N_p, 2 N_v) reals per iteration.  These tests
run the FP64 oracle on each rank's shard and check the all-reduced results
against the unsharded oracle.  (Every box this build runs on has one GPU, so
the sharded paths are exercised here, on CPU ranks.)
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _problem():
    from paper_1310_2078_gb300 import synth
    d = synth.random_problem(91, 301, 120, kinds=(0, 2), gains=True, weights=True, n_ant=6,
                             uv_max=80, w_max=20, extent=0.2, sigma_max=0.01)
    rng = np.random.default_rng(91)
    x = np.zeros(120)
    x[rng.choice(120, 6, replace=False)] = rng.uniform(0.5, 2, 6)
    return d, x, rng


def _shard(d, rank, world):
    idx = np.array_split(np.arange(d["uvw"].shape[0]), world)[rank]
    sub = dict(d)
    for k in ("uvw", "weights", "ant_pair"):
        sub[k] = None if d[k] is None else d[k][idx]
    return sub, idx


def _worker(rank, world, port, results):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    d, x, rng = _problem()
    Ofull = oracle.Problem(d["uvw"], d["lm"], d["sigma"], d["kind"], d["weights"], d["ant_pair"],
                           d["gains"])
    V = oracle.forward(Ofull, x) + 0.01 * (rng.normal(size=301) + 1j * rng.normal(size=301))
    sub, idx = _shard(d, rank, world)
    O = oracle.Problem(sub["uvw"], d["lm"], d["sigma"], d["kind"], sub["weights"],
                       sub["ant_pair"], d["gains"])
    Vs = V[idx]
    W = sub["weights"]
    # partial adjoint of the local residual, all-reduced
    r = W * (oracle.forward(O, x) - Vs)
    g = torch.from_numpy(oracle.adjoint(O, r))
    dist.all_reduce(g)
    # replicated FISTA over sharded gradients (same L, lambda on all ranks)
    L, _ = oracle.power(Ofull, max_iter=500, tol=1e-13)
    lam = 0.05
    I_prev = np.zeros(120)
    y = I_prev.copy()
    t = 1.0
    for _ in range(30):
        rl = W * (oracle.forward(O, y) - Vs)
        gl = torch.from_numpy(oracle.adjoint(O, rl))
        dist.all_reduce(gl)
        v = y - gl.numpy() / L
        I = np.where(v > lam / L, v - lam / L, 0.0)
        tn = 0.5 * (1 + np.sqrt(1 + 4 * t * t))
        y = I + (t - 1) / tn * (I - I_prev)
        I_prev, t = I, tn
    if rank == 0:
        full_g = oracle.adjoint(Ofull, d["weights"] * (oracle.forward(Ofull, x) - V))
        img, _ = oracle.fista(Ofull, V, lam, L, 30)
        results["grad_err"] = float(np.max(np.abs(g.numpy() - full_g)) / np.max(np.abs(full_g)))
        results["img_err"] = float(np.max(np.abs(I - img)) / max(img.max(), 1e-300))
    dist.barrier()
    dist.destroy_process_group()


def _worker_pix(rank, world, port, results):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    d, x, rng = _problem()
    Ofull = oracle.Problem(d["uvw"], d["lm"], d["sigma"], d["kind"], d["weights"], d["ant_pair"],
                           d["gains"])
    V = oracle.forward(Ofull, x) + 0.01 * (rng.normal(size=301) + 1j * rng.normal(size=301))
    n_pix = d["lm"].shape[0]
    idx = np.array_split(np.arange(n_pix), world)[rank]
    O = oracle.Problem(d["uvw"], d["lm"][idx], d["sigma"][idx], d["kind"][idx], d["weights"],
                       d["ant_pair"], d["gains"][idx])
    W = d["weights"]
    exchanged = [0]

    def forward_sum(xl):
        # partial visibilities of the local pixels, all-reduced as 2 N_v reals
        v = oracle.forward(O, xl)
        t = torch.from_numpy(np.stack([v.real, v.imag], axis=-1))
        dist.all_reduce(t)
        exchanged[0] += t.numel()
        return t[:, 0].numpy() + 1j * t[:, 1].numpy()

    Ax = forward_sum(x[idx])
    g = oracle.adjoint(O, W * (Ax - V))       # local columns of the gradient
    L, _ = oracle.power(Ofull, max_iter=500, tol=1e-13)
    lam = 0.05
    I_prev = np.zeros(len(idx))
    y = I_prev.copy()
    t = 1.0
    exchanged[0] = 0
    for _ in range(30):
        gl = oracle.adjoint(O, W * (forward_sum(y) - V))
        v = y - gl / L
        I = np.where(v > lam / L, v - lam / L, 0.0)
        tn = 0.5 * (1 + np.sqrt(1 + 4 * t * t))
        y = I + (t - 1) / tn * (I - I_prev)
        I_prev, t = I, tn
    img_parts = torch.zeros(n_pix, dtype=torch.float64)
    img_parts[idx] = torch.from_numpy(I)
    dist.all_reduce(img_parts)                 # gather: disjoint supports
    g_parts = torch.zeros(n_pix, dtype=torch.float64)
    g_parts[idx] = torch.from_numpy(g)
    dist.all_reduce(g_parts)
    if rank == 0:
        full_V = oracle.forward(Ofull, x)
        full_g = oracle.adjoint(Ofull, W * (full_V - V))
        img, _ = oracle.fista(Ofull, V, lam, L, 30)
        results["fwd_err"] = float(np.max(np.abs(Ax - full_V)) / np.max(np.abs(full_V)))
        results["grad_err"] = float(np.max(np.abs(g_parts.numpy() - full_g)) / np.max(np.abs(full_g)))
        results["img_err"] = float(np.max(np.abs(img_parts.numpy() - img)) / max(img.max(), 1e-300))
        results["reals_per_iter"] = exchanged[0] / 30
    dist.barrier()
    dist.destroy_process_group()


def _run(target, world=2):
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    results = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=target, args=(r, world, port, results)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    return dict(results)


def test_visibility_split_allreduce_matches_unsharded_oracle():
    results = _run(_worker)
    assert results["grad_err"] < 1e-12
    assert results["img_err"] < 1e-10


def test_pixel_split_allreduce_matches_unsharded_oracle():
    """The forward's partial sums over each rank's pixels, all-reduced, are
    the full forward; the local adjoint columns and threshold steps then give
    the unsharded gradient and FISTA image; one exchange of 2 N_v reals per
    iteration."""
    results = _run(_worker_pix)
    assert results["fwd_err"] < 1e-12
    assert results["grad_err"] < 1e-12
    assert results["img_err"] < 1e-10
    assert results["reals_per_iter"] == 2 * 301
