"""The bench's roofline arithmetic, its bookkeeping of ncu counters and its
multi-rank totals (no GPU; the totals over gloo ranks on CPU)."""
import os
import shutil
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


class W:
    def __init__(self, kind):
        self.kind = None if kind is None else np.asarray(kind)
        self.n_pix = 100 if kind is None else len(kind)


def test_sfu_peak_dirac_and_fma_sincos_bound():
    peak, basis, alt = bench.sfu_peak(W(None))
    # 152 SMs x 16 MUFU/clk x 2.07 GHz / 2 MUFU per pair
    assert peak == pytest.approx(152 * 16 * 2.07 / 2 * 1e0, rel=1e-12)
    # LP optimum: x = 1/16 SFU-path and y = (1 - 8/16)/21 FMA-path warp-pairs per clock
    # and sub-partition, 4 x 32 pairs per warp-pair and SM
    per_sm_clk = 4 * 32 * (1 / 16 + 0.5 / 21)
    assert alt["peak"] == pytest.approx(152 * 2.07 * per_sm_clk, rel=1e-12)
    assert alt["peak"] > peak


def test_sfu_peak_of_a_kind_mix_adds_time_per_pair():
    kinds = [0] * 25 + [2] * 75          # 25% Dirac (2 MUFU), 75% Gaussian (3 MUFU)
    peak, basis, alt = bench.sfu_peak(W(kinds))
    assert peak == pytest.approx(152 * 16 * 2.07 / 2.75, rel=1e-12)
    assert alt is None


def test_sfu_peak_of_the_adjoint_counts_one_cosine():
    """The adjoint's output is real, so a pair takes a cosine alone: the
    Dirac bound is twice the forward's, and its LP stays MUFU-bound with a
    small FMA-path share (7 instructions per SFU-path pair leave 1/8 of the
    issue slots)."""
    peak, basis, alt = bench.sfu_peak(W(None), "adj")
    assert peak == pytest.approx(152 * 16 * 2.07, rel=1e-12)
    per_sm_clk = 4 * 32 * (1 / 8 + (1 - 7 / 8) / 16)
    assert alt["peak"] == pytest.approx(152 * 2.07 * per_sm_clk, rel=1e-12)
    kinds = [0] * 25 + [2] * 75          # 1 MUFU for Dirac, 2 for Gaussian (cos + exp2)
    assert bench.sfu_peak(W(kinds), "adj")[0] == pytest.approx(152 * 16 * 2.07 / 1.75, rel=1e-12)
    r = 16 * bench.N_SM * bench.SM_MAX_MHZ * 1e6
    m = bench.sfu_peak_measured(W(kinds), {"sincos_per_s": r, "ex2_per_s": 2 * r}, "adj")
    assert m["peak"] == pytest.approx(1e-9 / (1 / r + 0.75 / (2 * r)))


def test_kernel_source_hash_ignores_comments_only(tmp_path):
    src = os.path.join(ROOT, "paper_1310_2078_gb300", "csrc")
    for f in bench.KERNEL_SOURCES:
        shutil.copy(os.path.join(src, f), tmp_path / f)
    h0 = bench.kernel_source_hash(str(tmp_path))
    assert h0 == bench.kernel_source_hash()
    p = tmp_path / "sl1m_mixed.cu"
    text = p.read_text()
    p.write_text("// a new comment\n/* and a\n block one */\n" + text.replace("\n", "\n  ", 3))
    assert bench.kernel_source_hash(str(tmp_path)) == h0
    assert "__launch_bounds__(NTHREADS, 3)" in text
    p.write_text(text.replace("__launch_bounds__(NTHREADS, 3)", "__launch_bounds__(NTHREADS, 2)", 1))
    assert bench.kernel_source_hash(str(tmp_path)) != h0


def test_ncu_traffic_matches_kernel_shape_workload_and_source():
    wl = "wide-field-dirac-256x256-40320vis"
    got = bench.ncu_traffic("adj_mixed", 4, 1, 456, wl)
    assert got is None or got > 0          # None once the kernels change after a capture
    assert bench.ncu_traffic("adj_mixed", 8, 1, 456, wl) is None
    assert bench.ncu_traffic("adj_mixed", 4, 2, 456, wl) is None
    assert bench.ncu_traffic("adj_mixed", 4, 1, 304, wl) is None
    assert bench.ncu_traffic("adj_mixed", 4, 1, 456, "another-workload") is None


def _totals_worker(rank, world, port, results):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    import bench as b
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r took 1.5 + r seconds for 10 * (r + 1) units
    results[rank] = b.job_totals(1.5 + rank, 10.0 * (rank + 1), world)
    dist.barrier()
    dist.destroy_process_group()


def test_job_totals_take_the_slowest_rank_and_all_ranks_work():
    """With several ranks the bench's figures are all ranks' units over the
    slowest rank's time, the same on every rank; with one rank, its own."""
    import socket
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    results = ctx.Manager().dict()
    world = 3
    procs = [ctx.Process(target=_totals_worker, args=(r, world, port, results)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    for r in range(world):
        assert results[r] == (3.5, 60.0)
    assert bench.job_totals(2.0, 7.0, 1) == (2.0, 7.0)


def test_reference_arm_under_torchrun_prints_one_line_from_rank_0():
    """`bench.py --impl reference` launched as the multi-GPU bench is (torchrun,
    two ranks): rank 0 times the oracle and prints one JSON line; the other
    rank exits 0 without work."""
    import json
    import socket
    import subprocess
    pytest.importorskip("torch")
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600,
                       env=dict(os.environ, OMP_NUM_THREADS="1"))
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, p.stdout
    out = json.loads(lines[0])
    assert out["impl"] == "reference" and out["n_gpus"] == 2 and out["value"] > 0
    assert out["cpu_baseline"]["kind"] == "oracle" and out["e2e"]["h2d_bytes_per_step"] == 0
    args = bench.parse(["--gpus", "2"])
    assert out["config"] == bench.bench_config(args, bench.workload(args.config))


def test_cpu_baseline_leg_times_the_oracle_and_measures_the_error():
    """The bench's CPU-baseline leg on a small workload: the single-threaded
    and the threaded oracle runs agree bit for bit, and the error it reports
    for given operator outputs is max |diff| / max |oracle| over its sample."""
    import oracle
    from paper_1310_2078_gb300 import synth
    w = synth.config1(scale=0.5)
    x, r = bench.baseline_inputs(w)
    O = oracle.Problem(w.uvw, w.lm)
    fwd, adj = oracle.forward(O, x), oracle.adjoint(O, r)
    out = bench.cpu_baseline(w, fwd * (1 + 3e-7), adj, budget_s=0.2)
    assert out["kind"] == "oracle" and out["cores"] == 1 and out["value"] > 0
    assert out["unit"] == "pairs/s" and w.name in out["sample"]
    th = out["threaded"]
    assert th["bitwise_identical_to_single_thread"] is True
    assert th["cores"] == (os.cpu_count() or 1) and th["value"] > 0
    err = out["gpu_error_vs_oracle"]
    assert err["forward"] == pytest.approx(3e-7, rel=1e-6)
    assert err["adjoint"] == 0.0


def test_clock_sampler_names_the_gpu_as_nvidia_smi_does(monkeypatch):
    monkeypatch.delenv("CUDA_VISIBLE_DEVICES", raising=False)
    assert bench.smi_id(0) == "0"
    monkeypatch.setenv("CUDA_VISIBLE_DEVICES", "3,5")
    assert bench.smi_id(0) == "3" and bench.smi_id(1) == "5"
    monkeypatch.setenv("CUDA_VISIBLE_DEVICES", "GPU-1234abcd")
    assert bench.smi_id(0) == "GPU-1234abcd"


def test_oracle_stream_estimate_scales_the_sampled_rate_to_the_stream():
    """The serving line's oracle estimate: the samples' total pairs over their
    total time (not a mean of rates of requests of very different sizes),
    applied to the whole stream; the samples run single-threaded only."""
    from paper_1310_2078_gb300 import synth
    reqs = [synth.config1(scale=0.25), synth.config1(scale=0.5), synth.config1(scale=0.25)]
    stream_pairs = 1e9
    est = bench.oracle_stream_estimate(reqs, [0, 1], stream_pairs, budget_s=0.1)
    assert est["kind"] == "oracle" and est["cores"] == 1 and est["unit"] == "solves/s"
    assert [s["request"] for s in est["samples"]] == [0, 1]
    assert all("threaded" not in s for s in est["samples"])
    rate = sum(s["pairs"] for s in est["samples"]) / sum(s["seconds"] for s in est["samples"])
    assert est["pairs_per_s"] == pytest.approx(rate)
    assert est["est_wall_s"] == pytest.approx(stream_pairs / rate)
    assert est["value"] == pytest.approx(3 / (stream_pairs / rate))


def test_default_workload_is_paper_scale_and_ranks_share_its_shape():
    """The bench's default workload is the paper-scale one (1024^2 Dirac
    pixels x 406,400 visibilities) with a step of 5 FISTA steps at a fixed L;
    under several ranks each rank solves the same geometry with its own
    noise (weak scaling)."""
    args = bench.parse([])
    assert args.config == 4 and args.iters == 5 and not args.full_solve
    assert bench.parse(["--full-solve"]).iters == 200
    w = bench.workload(args.config)
    assert w.name == "paper-scale-dirac-1024x1024-406400vis" and (w.n_pix, w.n_vis) == (1048576, 406400)
    w1 = bench.workload(args.config, rank=1)
    assert (w1.n_pix, w1.n_vis) == (w.n_pix, w.n_vis)
    np.testing.assert_array_equal(w1.uvw, w.uvw)
    assert not np.array_equal(w1.noise, w.noise)


def test_both_arms_print_the_same_config():
    """The reference arm's `config` is the one the GPU arm prints."""
    args = bench.parse(["--gpus", "2"])
    w = bench.workload(args.config)
    c = bench.bench_config(args, w)
    assert c["workload"] == w.name and c["parallelism"] == "replicas2"
    assert "5 FISTA steps at a fixed L" in c["step"] and c["precision"] == "mixed"
    assert bench.bench_config(bench.parse(["--ops-only"]), w)["step"].startswith("one forward")


def test_measured_sfu_peak_weighs_the_pixel_kinds():
    """With the measured rates at the table's 16 per clock per SM, the
    measured bound equals the table bound for Dirac and for a Dirac/Gaussian
    mix (exp2 at the same rate)."""
    class W:
        def __init__(self, kind):
            self.kind = kind
            self.n_pix = 4 if kind is None else len(kind)
    r = 16 * bench.N_SM * bench.SM_MAX_MHZ * 1e6
    sfu = {"sincos_per_s": r, "ex2_per_s": r}
    for kinds in (None, np.array([0, 2, 2, 2])):
        m = bench.sfu_peak_measured(W(kinds), sfu)
        assert m["peak"] == pytest.approx(bench.sfu_peak(W(kinds))[0])
        assert m["per_clk_per_sm_at_max_clock"]["sincos_per_s"] == pytest.approx(16.0)
    m = bench.sfu_peak_measured(W(None), {"sincos_per_s": r / 2, "ex2_per_s": r})
    assert m["peak"] == pytest.approx(bench.sfu_peak(W(None))[0] / 2)


def test_profiles_hold_dram_traffic_for_the_default_workload():
    """The committed launch-list summary of the default workload carries the
    one-pass DRAM lines the bench reads for `roofline.traffic`."""
    import re
    w = bench.workload(bench.parse([]).config)
    prof = open(os.path.join(ROOT, "profiles", "launch_list_paper_scale_dirac_1024x1024_406400vis.md")).read()
    lines = re.findall(r"^traffic: kernel=(\S+) .* workload=(\S+) src=\S+ dram_bytes_per_launch=(\d+)$", prof, re.M)
    assert {k for k, wl, _ in lines if wl == w.name} == {"fwd_mixed", "adj_mixed"}
