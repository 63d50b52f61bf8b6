"""Multi-process sharding arithmetic on CPU (gloo, world_size 2).

A single SL1M solve shards by visibilities: each rank holds N_v/P
visibilities and a replica of the image; the forward is local, the adjoint
yields partial images that are all-reduced (one exchange of N_p reals per
iteration), and the FISTA update is replicated.  These tests run the FP64
oracle on each rank's shard and check the all-reduced results against the
unsharded oracle.  (Every box this build runs on has one GPU, so the sharded
path is exercised here, on CPU ranks.)
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


def test_visibility_split_allreduce_matches_unsharded_oracle():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    results = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, results)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    assert results["grad_err"] < 1e-12
    assert results["img_err"] < 1e-10
