"""Benchmark of the SL1M hot path on GB300.

Workload (default): the paper-scale configuration -- 1024x1024 = 1,048,576
Dirac pixels over l,m in +/-0.3, 128 antennas (R = 1 km, 30 m height
scatter) x 50 snapshots -> 406,400 visibilities, 2,000 power-law sources +
noise, mixed precision (FP32 operator, FP64 solver scalars).  L is computed
once by power iteration (untimed); one step = `--iters` FISTA steps (default
5) at that L through the C ABI's solve call, each one forward and one
adjoint over all 4.26e11 pixel-visibility pairs, plus the forward of I_0.
Metric: pixel-visibility pairs evaluated per second by the forward and
adjoint kernels (pairs/s), whole job.

value   : inputs resident in HBM when the timed region starts; each step
          timed with CUDA events on the library's stream, L2 flushed between
          steps.
e2e     : the same steps through the C ABI from HOST buffers: setting the
          visibilities and pixels (layout + H2D) and reading the image back
          are inside the timed region.
serving : a shortened serving stream (independent solves of uneven sizes
          arriving as a Poisson process) through the continuous-batching
          server: solves/s, p50/p99 latency, and the FP64 plain single-solve
          path on the same requests.
--impl reference : the FP64 CPU oracle on the host cores, bounded sample.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

MUFU_PER_SM_CLK = 16          # sin/cos/ex2 per clock per SM (CUDA guide throughput table)
# MUFU results per pair, per operator: the forward takes a sine and a cosine
# (its output is complex), the adjoint a cosine alone (its output is real:
# Re(conj(A) r) = |r| cos(theta + arg r)); a Gaussian pixel adds an exp2.
SFU_OPS_PER_PAIR = {"fwd": {"dirac": 2, "gauss": 3}, "adj": {"dirac": 1, "gauss": 2}}
# The fewest instructions a Dirac pair takes with its trigonometry on the
# SFU and on the FMA pipe.  Forward: 3 FFMA phase, 1 FMUL argument scale,
# 2 MUFU, 2 FFMA accumulate; 21 with the 16-instruction sincos.  Adjoint: 1
# FADD + 3 FFMA phase, 1 FMUL, 1 MUFU, 1 FFMA; 16 with the 11-instruction
# cosine.
INSTR_PER_PAIR = {"fwd": (8, 21), "adj": (7, 16)}
N_SM = 152
SM_MAX_MHZ = 2070.0
L2_BYTES = 129 * 2 ** 20


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", type=int, default=4)
    ap.add_argument("--small", action="store_true",
                    help="config 2 at 128x128 pixels (a small case for ncu captures)")
    ap.add_argument("--n-side", type=int, default=0, help="override: pixel grid side")
    ap.add_argument("--n-ant", type=int, default=0, help="override: antennas")
    ap.add_argument("--n-times", type=int, default=0, help="override: snapshots")
    ap.add_argument("--no-gains", action="store_true", help="the workload without its gains")
    ap.add_argument("--iters", type=int, default=0,
                    help="FISTA steps per bench step (default 5; 200 with --full-solve)")
    ap.add_argument("--full-solve", action="store_true",
                    help="a step is one whole solve: power iteration for L, then --iters FISTA steps")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="skip the (untimed) tile-shape autotuner")
    ap.add_argument("--shape", default="",
                    help="set the tile shapes instead of autotuning: 'nst,ctas_per_sm,npoly' of the "
                         "forward, ':', the same of the adjoint (e.g. 8,3,1:4,3,1); profiler runs use "
                         "this so the captured kernels are the ones a plain run's autotuner picks")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--ops-only", action="store_true",
                    help="a step is one forward + one adjoint through the C ABI (device pointers)")
    ap.add_argument("--serve", action="store_true",
                    help="serving workload alone: Poisson stream of independent solves through the server")
    ap.add_argument("--requests", type=int, default=0,
                    help="serving requests (default 256 with --serve, 48 in the default line)")
    ap.add_argument("--rate", type=float, default=0.0,
                    help="serving arrival rate, 1/s (default 20 with --serve, 2 in the default line)")
    ap.add_argument("--no-serve", action="store_true", help="leave the serving object out of the line")
    ap.add_argument("--fp64-sample", type=int, default=3)
    ap.add_argument("--table1", action="store_true",
                    help="the noise-free lambda sweep of Table 1 at its sizes (1024^2 px x 37,800 vis)")
    ap.add_argument("--table1-cap", type=int, default=1000, help="--table1: FISTA steps at most per lambda")
    ap.add_argument("--ticks", type=int, default=4, help="serving: ticks per round")
    ap.add_argument("--max-pairs", type=float, default=4e9, help="serving: work in flight per tick")
    ap.add_argument("--admission", default="two_lanes", choices=["two_lanes", "arrival"],
                    help="serving: admission policy of the server")
    args = ap.parse_args(argv)
    if not args.iters:
        args.iters = 200 if args.full_solve else 5
    return args


def step_text(args) -> str:
    """What one timed step is (the config's `step`)."""
    if args.ops_only:
        return "one forward + one adjoint (device pointers)"
    if args.full_solve:
        return f"one solve: power iteration (<=50) + {args.iters} FISTA steps"
    return (f"{args.iters} FISTA steps at a fixed L (power iteration once, untimed), each one "
            "forward + one adjoint, plus the forward of I_0, through sl1m_solve")


def bench_config(args, w) -> dict:
    """The line's `config`, the same for both arms."""
    return {"workload": w.name, "n_pix": w.n_pix, "n_vis": w.n_vis, "step": step_text(args),
            "precision": args.precision, "l2": "flushed between steps (268 MB write)",
            "parallelism": f"replicas{args.gpus}" if args.gpus > 1 else "1 GPU"}


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        import torch
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return ws, rank, local


def job_totals(seconds: float, units: float, ws: int, device="cpu"):
    """(slowest rank's seconds, all ranks' units): the whole job's time and
    work.  Every rank calls it (two all-reduces over the process group);
    with one rank it returns its arguments."""
    if ws <= 1:
        return float(seconds), float(units)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t[0]), float(u[0])


def workload(cfg: int, rank: int = 0, small: bool = False, args=None):
    from paper_1310_2078_gb300 import synth
    kw = {}
    if args is not None and cfg in (2, 3, 4):
        for k in ("n_side", "n_ant", "n_times"):
            if getattr(args, k, 0):
                kw[k] = getattr(args, k)
    w = synth.config2(n_side=128) if small else synth.CONFIGS[cfg](**kw)
    if args is not None and getattr(args, "no_gains", False) and w.gains is not None:
        w.gains = None
        w.name += "-no-gains"
    if rank:
        # weak scaling: every rank solves its own independent problem of the same shape
        rng = synth.rng_for(synth.BASE_SEED + 100 * rank + cfg)
        w.noise = synth.complex_noise(rng, w.n_vis, float(np.std(w.noise.real)) or 0.01)
    return w


def smi_id(index: int) -> str:
    """nvidia-smi's name for CUDA device `index`: CUDA numbers only the devices
    CUDA_VISIBLE_DEVICES lists (by index or UUID), nvidia-smi numbers them all."""
    vis = [v.strip() for v in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if v.strip()]
    return vis[index] if index < len(vis) else str(index)


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={smi_id(self.index)}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                pw.append(float(r[3]))
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        load = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": float(np.median(load)), "sm_max_mhz": max(mx),
                "power_w_max": max(pw) if pw else None, "samples": len(sm),
                "reasons": sorted(reasons)}


KERNEL_SOURCES = ("sl1m_mixed.cu", "sl1m_fp64.cu", "sl1m_devfn.cuh", "sl1m_dev.h", "sl1m_sincos_poly.h")


def kernel_source_hash(csrc=None):
    """First 12 hex digits of the SHA-1 of the operator kernels' sources with
    comments removed and whitespace collapsed: a profile summary records it,
    so counters taken on other kernel code are not reported as this code's
    (an edit of a comment leaves the code, and the hash, unchanged).  csrc:
    the source directory (default: the package's)."""
    import hashlib
    csrc = csrc or os.path.join(ROOT, "paper_1310_2078_gb300", "csrc")
    h = hashlib.sha1()
    for f in KERNEL_SOURCES:
        with open(os.path.join(csrc, f), encoding="utf-8") as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)     # block comments
        src = re.sub(r"//[^\n]*", " ", src)                  # line comments
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:12]


def ncu_traffic(kernel, nst, npoly, ctas, workload):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summaries, or None when no summary matches this kernel, tile shape, grid,
    workload and kernel source (the counters belong to the kernel as it was
    captured)."""
    src = kernel_source_hash()
    pdir = os.path.join(ROOT, "profiles")
    try:
        names = sorted(os.listdir(pdir))
    except OSError:
        return None
    pat = (r"^traffic: kernel=(\S+) nst=(\d+) npoly=(\d+) ctas=(\d+) workload=(\S+) "
           r"src=([0-9a-f]+) dram_bytes_per_launch=(\d+)$")
    for name in names:
        try:
            with open(os.path.join(pdir, name)) as f:
                text = f.read()
        except OSError:
            continue
        for m in re.finditer(pat, text, re.M):
            key = (m.group(1), int(m.group(2)), int(m.group(3)), int(m.group(4)), m.group(5), m.group(6))
            if key == (kernel, nst, npoly, ctas, workload, src):
                return int(m.group(7))
    return None


def sfu_peak(w, op="fwd"):
    """SFU issue bound of operator op ("fwd" or "adj") on workload w (Gpairs/s).

    Per pair the SFU runs the trigonometry (forward: sin and cos, adjoint:
    cos) plus exp2 for a Gaussian pixel; the bound is N_SM x 16 MUFU/clk x
    max clock over the MUFU ops per pair, weighted by the share of pairs of
    each kind (time per pair adds up).  For all-Dirac work a second figure is
    returned: the bound when a share of the pairs takes its trigonometry on
    the FMA pipe, a linear program over two limits per SM sub-partition --
    one warp instruction issued per clock and one MUFU warp instruction per 8
    clocks -- with the fewest instructions a pair can take on either path
    (INSTR_PER_PAIR)."""
    per_sm_clk = N_SM * SM_MAX_MHZ * 1e6 / 1e9
    kinds = np.zeros(w.n_pix, np.int32) if w.kind is None else np.asarray(w.kind)
    f_gauss = float(np.mean(kinds != 0))
    ops = SFU_OPS_PER_PAIR[op]
    mufu = (1 - f_gauss) * ops["dirac"] + f_gauss * ops["gauss"]
    peak = per_sm_clk * MUFU_PER_SM_CLK / mufu
    basis = (f"SFU issue: {N_SM} SM x {MUFU_PER_SM_CLK} MUFU/clk x {SM_MAX_MHZ:.0f} MHz / "
             f"{mufu:.3g} MUFU per pair ({100 * (1 - f_gauss):.0f}% Dirac pairs at {ops['dirac']}, "
             f"{100 * f_gauss:.0f}% Gaussian at {ops['gauss']})")
    alt = None
    if f_gauss == 0.0:
        # per sub-partition and clock: x SFU-path and y FMA-path warp-pairs,
        # m x <= 1/8 (MUFU), a x + b y <= 1 (issue); maximise x + y
        a, b = INSTR_PER_PAIR[op]
        x = min(1.0 / (8.0 * ops["dirac"]), 1.0 / a)
        y = max(0.0, (1.0 - a * x) / b)
        pairs_per_sm_clk = 4 * 32 * (x + y)
        alt = {"peak": per_sm_clk * pairs_per_sm_clk,
               "basis": "LP over issue (1 warp instr/clk/SMSP) and MUFU (1/8 per clk/SMSP): "
                        f"{a} instr/pair on the SFU path, {b} with the trigonometry on the FMA pipe; "
                        f"{pairs_per_sm_clk:.2f} pairs/clk/SM at {100 * y / (x + y):.0f}% FMA-path pairs"}
    return peak, basis, alt


def sfu_peak_measured(w, sfu, op="fwd"):
    """The SFU bound of operator op on workload w from the measured MUFU rates
    (Gpairs/s): a pair takes a sin and a cos (forward) or a cos (adjoint), and
    an exp2 when its pixel is Gaussian, so its time on the unit is m / (sin-
    or-cos rate) + f_gauss / (exp2 rate)."""
    kinds = np.zeros(w.n_pix, np.int32) if w.kind is None else np.asarray(w.kind)
    f_gauss = float(np.mean(kinds != 0))
    m = SFU_OPS_PER_PAIR[op]["dirac"]
    t_pair = m / sfu["sincos_per_s"] + f_gauss / sfu["ex2_per_s"]
    per_clk_sm = {k: v / (N_SM * SM_MAX_MHZ * 1e6) for k, v in sfu.items()}
    return {"peak": 1.0 / t_pair / 1e9,
            "basis": "sl1m_measure_sfu: sin/cos and exp2 results per second on this GPU; "
                     f"{m} sin/cos + {f_gauss:.3g} exp2 per pair",
            "measured_per_s": sfu,
            "per_clk_per_sm_at_max_clock": per_clk_sm}


def baseline_inputs(w):
    """The seeded x [n_pix] and r [n_vis] the CPU-baseline sample runs on."""
    rng = np.random.default_rng(0)
    x = np.abs(rng.normal(size=w.n_pix))
    r = rng.normal(size=w.n_vis) + 1j * rng.normal(size=w.n_vis)
    return x, r


def cpu_baseline(w, gpu_fwd=None, gpu_adj=None, budget_s: float = 12.0, threaded: bool = True):
    """The FP64 oracle as it stands, single-threaded, on a bounded sample of
    the same workload: forward rows and adjoint columns; pairs/s.  Given the
    library's forward A x and adjoint Re A^H r of the same inputs, the sampled
    oracle outputs also give their error (max |diff| / max |oracle| over the
    sample)."""
    import oracle
    O = oracle.Problem(w.uvw, w.lm, w.sigma, w.kind, w.weights, w.ant_pair, w.gains)
    x, r = baseline_inputs(w)
    # calibrate: 8 rows
    t0 = time.perf_counter()
    oracle.forward(O, x, rows=np.arange(8))
    per_row = (time.perf_counter() - t0) / 8
    n_rows = max(8, int(0.5 * budget_s / per_row))
    n_cols = max(8, int(0.5 * budget_s / (per_row * w.n_vis / w.n_pix)))
    # prefixes of fixed permutations: a run that samples more rows or columns
    # keeps every row and column of a smaller sample, so errors compare across
    # runs.  The rows also hold the 8 shortest baselines: for the positive x
    # below |V_k| peaks there, so the sample's max |V| is the vector's and the
    # error is normwise over the whole output, as defined.
    short = np.argsort(np.sum(np.asarray(w.uvw)[:, :2] ** 2, axis=1))[:8]
    perm = np.random.default_rng(1).permutation(w.n_vis)
    rows = np.concatenate([short, perm[~np.isin(perm, short)][:max(0, min(n_rows, w.n_vis) - 8)]])
    cols = np.random.default_rng(2).permutation(w.n_pix)[:min(n_cols, w.n_pix)]
    t0 = time.perf_counter()
    fo = oracle.forward(O, x, rows=rows)
    ao = oracle.adjoint(O, r, cols=cols)
    dt = time.perf_counter() - t0
    pairs = len(rows) * w.n_pix + len(cols) * w.n_vis
    out = {"value": pairs / dt, "unit": "pairs/s", "cores": 1, "kind": "oracle",
           "sample": f"{len(rows)} forward rows (the 8 shortest baselines + a random sample) x {w.n_pix} px "
                     f"+ {len(cols)} adjoint columns x {w.n_vis} vis of {w.name}, FP64, single thread, {dt:.1f} s",
           "pairs": float(pairs), "seconds": dt}
    if threaded:
        out["threaded"] = cpu_threaded(O, x, r, rows, cols, fo, ao, pairs)
    if gpu_fwd is not None and gpu_adj is not None:
        out["gpu_error_vs_oracle"] = {
            "forward": float(np.max(np.abs(gpu_fwd[rows] - fo)) / np.max(np.abs(fo))),
            "adjoint": float(np.max(np.abs(gpu_adj[cols] - ao)) / np.max(np.abs(ao))),
            "measure": "max |gpu - oracle| / max |oracle| over the sampled rows / columns"}
    return out


def oracle_stream_estimate(reqs, picks, stream_pairs, budget_s: float = 6.0):
    """The FP64 oracle, single-threaded, timed on bounded samples of the
    requests `picks` of a serving stream; their total pairs over their total
    time, applied to the pairs the whole stream evaluated, estimates a serial
    oracle run of every request (solves/s)."""
    samples = [dict(request=int(i), **cpu_baseline(reqs[i], budget_s=budget_s, threaded=False))
               for i in picks]
    rate = sum(smp["pairs"] for smp in samples) / sum(smp["seconds"] for smp in samples)
    wall = stream_pairs / rate
    return {"value": len(reqs) / wall, "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": f"FP64 oracle forward rows + adjoint columns of requests {[int(i) for i in picks]}, "
                      "single thread; their pair rate (total pairs / total time) applied to all "
                      "requests' pairs (serial)",
            "pairs_per_s": rate, "est_wall_s": wall, "samples": samples}


def cpu_threaded(O, x, r, rows, cols, fo, ao, pairs):
    """The same oracle sample with the outer loop (forward rows, adjoint
    columns) split over every host core: each output is still one
    single-threaded sum in the oracle's order, so the results must equal the
    single-threaded ones bit for bit (checked).  The oracle is a C library
    called through ctypes, which releases the GIL, so threads run in
    parallel."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    n = os.cpu_count() or 1
    rch = np.array_split(rows, n)
    cch = np.array_split(cols, n)
    with ThreadPoolExecutor(max_workers=n) as ex:
        t0 = time.perf_counter()
        fparts = list(ex.map(lambda c: oracle.forward(O, x, rows=c) if len(c) else np.zeros(0, complex), rch))
        aparts = list(ex.map(lambda c: oracle.adjoint(O, r, cols=c) if len(c) else np.zeros(0), cch))
        dt = time.perf_counter() - t0
    same = bool(np.array_equal(np.concatenate(fparts), fo) and np.array_equal(np.concatenate(aparts), ao))
    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    import platform
    return {"value": pairs / dt, "unit": "pairs/s", "cores": n, "seconds": dt,
            "bitwise_identical_to_single_thread": same, "cpu": f"{platform.machine()} {model}".strip()}


def run_reference(args):
    """--impl reference: the FP64 oracle on the host cores (bounded samples).
    Under torchrun only rank 0 runs it (no process group is needed); the
    other ranks exit at once."""
    if int(os.environ.get("RANK", "0")) != 0:
        return
    import oracle
    w = workload(args.config, 0, args.small, args)
    O = oracle.Problem(w.uvw, w.lm, w.sigma, w.kind, w.weights, w.ant_pair, w.gains)
    rng = np.random.default_rng(0)
    x = np.abs(rng.normal(size=w.n_pix))
    r = rng.normal(size=w.n_vis) + 1j * rng.normal(size=w.n_vis)
    t0 = time.perf_counter()
    oracle.forward(O, x, rows=np.arange(4))
    per_row = (time.perf_counter() - t0) / 4
    n_rows = max(4, int(2.0 / per_row))            # ~2 s forward + ~2 s adjoint per step
    n_cols = max(4, int(2.0 / (per_row * w.n_vis / w.n_pix)))
    times, pairs = [], 0
    for s in range(args.warmup + args.steps):
        rows = rng.choice(w.n_vis, min(n_rows, w.n_vis), replace=False)
        cols = rng.choice(w.n_pix, min(n_cols, w.n_pix), replace=False)
        t0 = time.perf_counter()
        oracle.forward(O, x, rows=rows)
        oracle.adjoint(O, r, cols=cols)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
            pairs += len(rows) * w.n_pix + len(cols) * w.n_vis
    T = sum(times)
    val = pairs / T
    sample = (f"per step {min(n_rows, w.n_vis)} forward rows + {min(n_cols, w.n_pix)} adjoint "
              f"columns of {w.name} (FP64 oracle, single thread)")
    out = {"impl": "reference", "metric": "pixel-visibility pairs/s (fwd+adj)", "value": val,
           "unit": "pairs/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * T / len(times), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": bench_config(args, w),
           "cpu_baseline": {"value": val, "unit": "pairs/s", "cores": 1, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": val, "unit": "pairs/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def serving_measure(n_requests, rate, ticks=4, max_pairs=4e9, fp64_sample=3, with_cpu=True, dev=0,
                    admission="two_lanes"):
    """Continuous batching: `n_requests` independent solves arriving as a
    Poisson stream (`rate` per second), each an independently generated
    array/sky with 4k-256k pixels and 2k-100k visibilities, Dirac or wide
    Gaussian pixels, gains on half of them; 200 FISTA steps or relative change
    of E below 1e-6, L by power iteration.  Returns solves/s, latency
    percentiles (submit to result), pairs/s, and the FP64 plain single-solve
    path on a sample of the same requests (same L and iterations, serial):
    its time, its final objective against the mixed path's, and its pair
    rate applied to the whole stream."""
    import torch
    from paper_1310_2078_gb300 import sl1m, synth
    sl1m.load()
    torch.cuda.set_device(dev)
    reqs = [synth.serving_request(i) for i in range(n_requests)]
    arrive = synth.arrivals(n_requests, rate)
    ctx = sl1m.Context(dev)
    # data: V = A x_true + noise through the library's forward (mixed), lambda from the dirty image
    probs, lams = [], []
    for w in reqs:
        P = sl1m.problem_from(ctx, w)
        V = P.forward(w.x_true, sl1m.MIXED) + w.noise
        P.set_vis_data(V)
        lams.append(w.lambda_frac * P.adjoint(V, sl1m.MIXED).max())
        probs.append((P, V))
    torch.cuda.synchronize()
    ctx.counters_reset()
    ctx.server_start(max_slots=64, ticks_per_round=ticks, max_pairs_per_tick=max_pairs,
                     admission=sl1m.ADMIT_TWO_LANES if admission == "two_lanes" else sl1m.ADMIT_ARRIVAL)
    clocks = ClockSampler(dev)
    clocks.start()
    t0 = time.perf_counter()
    tickets = []
    for i, (P, V) in enumerate(probs):
        dt = t0 + arrive[i] - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        tickets.append(ctx.server_submit(P, lams[i], L=0.0, max_iter=200, rel_tol=1e-6))
    results = [ctx.server_wait(t, probs[i][0], timeout_s=-1.0) for i, t in enumerate(tickets)]
    T = time.perf_counter() - t0
    clk = clocks.stop()
    info = ctx.server_info()
    ctx.server_stop()
    launches = ctx.counters()["launches"]
    lat = np.array([st["seconds"] for _, st in results])
    req_pairs = [(2 * st["power_iters"] + 2 * st["iters"] + 2) * float(w.n_vis) * w.n_pix
                 for (_, st), w in zip(results, reqs)]
    pairs = sum(req_pairs)
    # the slowest requests: their size and their work at the stream's pair rate
    slowest = [{"request": int(i), "n_pix": reqs[i].n_pix, "n_vis": reqs[i].n_vis,
                "iters": results[i][1]["iters"], "latency_s": float(lat[i]),
                "own_work_s_at_stream_rate": req_pairs[i] / (pairs / T)}
               for i in np.argsort(-lat)[:5]]
    # FP64 plain single-solve path: requests spread over the lower half of the
    # work distribution, each solved alone with the served solve's L and
    # iterations, and the mixed path alone on the same request beside it
    by_work = np.argsort([w.pairs for w in reqs])
    ranks = np.unique(np.linspace(0, len(reqs) // 2, fp64_sample).astype(int)) if fp64_sample > 0 else []
    cmp = []
    for i in by_work[ranks]:
        P, V = probs[i]
        st_m = results[i][1]
        t1 = time.perf_counter()
        img64, st64 = P.solve(lams[i], L=st_m["L"], max_iter=st_m["iters"], precision=sl1m.FP64)
        t64 = time.perf_counter() - t1
        t1 = time.perf_counter()
        imgm, stm = P.solve(lams[i], L=st_m["L"], max_iter=st_m["iters"], precision=sl1m.MIXED)
        tm = time.perf_counter() - t1
        cmp.append({"request": int(i), "n_pix": reqs[i].n_pix, "n_vis": reqs[i].n_vis,
                    "iters": st_m["iters"], "fp64_s": t64, "mixed_alone_s": tm,
                    "E_rel_diff": abs(stm["E"] - st64["E"]) / st64["E"],
                    "served_E_rel_diff": abs(st_m["E"] - st64["E"]) / st64["E"],
                    "img_err_of_peak": float(np.max(np.abs(imgm - img64)) / max(img64.max(), 1e-300))})
    fp64_solves_per_s = len(cmp) / sum(c["fp64_s"] for c in cmp) if cmp else None
    # the FP64 plain path solving every request serially: its pair rate on the
    # sample (same iterations, L given) applied to the whole stream's pairs
    fp64_pairs = sum((2 * c["iters"] + 1) * float(c["n_vis"]) * c["n_pix"] for c in cmp)
    fp64_rate = fp64_pairs / sum(c["fp64_s"] for c in cmp) if cmp else None
    fp64_serial = None
    if fp64_rate:
        est = n_requests / (pairs / fp64_rate)
        fp64_serial = {"pairs_per_s": fp64_rate, "est_wall_s": pairs / fp64_rate, "est_solves_per_s": est,
                       "served_over_fp64": (n_requests / T) / est,
                       "method": "FP64 single solves, pair rate measured on the sample, "
                                 "applied to all requests' pairs (serial, no overlap)"}
    cpu = None
    if with_cpu:
        cpu = oracle_stream_estimate(reqs, [by_work[0], by_work[len(by_work) // 2]], pairs)
    out = {"metric": "solves/s (continuous batching, mixed precision)", "value": n_requests / T,
           "unit": "solves/s", "n_gpus": 1, "higher_is_better": True, "dtype": "f32+f64",
           "data": "synthetic",
           "config": {"workload": f"serving: {n_requests} requests, Poisson {rate:g}/s, "
                                  "pixels logU(4k,256k), visibilities logU(2k,100k), "
                                  "Dirac/wide-Gaussian 50/50, gains on 50%",
                      "max_slots": 64, "ticks_per_round": ticks, "max_pairs_per_tick": max_pairs,
                      "admission": admission},
           "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                         "mean": float(lat.mean()), "max": float(lat.max())},
           "pairs_per_s": pairs / T, "wall_s": T, "slowest": slowest,
           "iters_mean": float(np.mean([st["iters"] for _, st in results])),
           "server": info, "clocks": clk, "gpu_launches": launches,
           "fp64_plain_single_solve": {"sample": cmp, "solves_per_s_on_sample": fp64_solves_per_s,
                                       "serial_whole_stream": fp64_serial},
           "cpu_baseline": cpu}
    ctx.close()
    return out


def run_table1(args):
    """--table1: the noise-free lambda sweep of Sect. 4.1 (Table 1) at the
    paper's sizes -- 1024^2 Dirac pixels of 30 arcsec, 37,800 visibilities, 50
    point sources, no noise -- with lambda from 1e-6 to 1e-1 of lambda_max
    (the paper's lambda = 1e-2 ... 1e3 span the same decades below its
    lambda_max).  Each solve starts from zero and stops when the relative
    change of E falls below 1e-6, or after --table1-cap steps; L by power
    iteration once.  Reports per lambda the steps taken, the recovered total
    flux against the true one, the residual, and the largest error on the
    sources."""
    import torch
    from paper_1310_2078_gb300 import sl1m, synth
    sl1m.load()
    torch.cuda.set_device(0)
    w = synth.table1()
    ctx = sl1m.Context(0)
    P = sl1m.problem_from(ctx, w)
    V = P.forward(w.x_true, sl1m.FP64)                    # noise-free data, FP64 forward
    P.set_vis_data(V)
    _, lmax = P.dirty_image(sl1m.MIXED)
    L, pit = P.max_eig(50, 1e-6, sl1m.MIXED)
    on = w.x_true > 0
    true_l1 = float(w.x_true.sum())
    rows = []
    t_all = time.perf_counter()
    for f in (1e-6, 1e-5, 1e-4, 1e-3, 1e-2, 1e-1):
        t0 = time.perf_counter()
        img, st = P.solve(f * lmax, L=L, max_iter=args.table1_cap, rel_tol=1e-6, precision=sl1m.MIXED)
        dt = time.perf_counter() - t0
        rows.append({"lambda_over_lambda_max": f, "lambda": f * lmax, "iters": st["iters"],
                     "converged": bool(st["converged"]), "l1": st["l1"], "l1_over_true": st["l1"] / true_l1,
                     "resid2": st["resid2"], "E": st["E"], "nnz": st["nnz"],
                     "max_err_on_sources_of_peak": float(np.max(np.abs(img[on] - w.x_true[on])) / w.x_true.max()),
                     "off_source_flux": float(img[~on].sum()), "seconds": dt})
    T = time.perf_counter() - t_all
    iters = sum(r["iters"] for r in rows)
    out = {"mode": "table1 lambda sweep", "data": "synthetic, noise-free",
           "config": {"workload": w.name, "n_pix": w.n_pix, "n_vis": w.n_vis, "sources": int(on.sum()),
                      "precision": "mixed", "rel_tol": 1e-6, "max_iter": args.table1_cap},
           "true_l1": true_l1, "lambda_max": lmax, "L": L, "power_iters": pit, "rows": rows,
           "wall_s": T, "pairs_per_s": (2 * iters + len(rows)) * float(w.n_pix) * w.n_vis / T}
    print(json.dumps(out))
    ctx.close()


def run_serve(args):
    """--serve: the serving stream alone, as its own line."""
    out = serving_measure(args.requests or 256, args.rate or 20.0, args.ticks, args.max_pairs,
                          args.fp64_sample, not args.no_cpu, admission=args.admission)
    print(json.dumps(out))


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.serve:
        return run_serve(args)
    if args.table1:
        return run_table1(args)
    import torch
    ws, rank, local = dist_init()
    from paper_1310_2078_gb300 import sl1m
    sl1m.load()
    dev = local
    torch.cuda.set_device(dev)
    prec = sl1m.MIXED if args.precision == "mixed" else sl1m.FP64
    w = workload(args.config, rank, args.small, args)
    stream = torch.cuda.Stream(device=dev)
    ctx = sl1m.Context(dev, stream=stream)
    # synthetic visibilities: V = A x_true + noise, formed by the library's own forward
    P = ctx.problem()
    P.set_visibilities(w.uvw, None, w.weights, w.ant_pair)
    P.set_pixels(w.lm, w.sigma, w.kind)
    if w.gains is not None:
        P.set_gains(w.gains)
    V = P.forward(w.x_true, sl1m.FP64 if w.n_vis * w.n_pix < 5e9 else sl1m.MIXED) + w.noise
    P.set_vis_data(V)
    lam = w.lambda_frac * P.adjoint(V * (1 if w.weights is None else w.weights), prec).max()
    if args.shape:                                              # untimed set-up
        sh = [[int(v) for v in part.split(",")] for part in args.shape.split(":")]
        for op in (0, 1):
            P.set_tile_shape(op, sh[op][0], sh[op][1], sh[op][2], precision=prec)
        tuned = {"nst": [sh[0][0], sh[1][0]], "ctas_per_sm": [sh[0][1], sh[1][1]],
                 "npoly": [sh[0][2], sh[1][2]], "source": "--shape"}
    else:
        tuned = None if args.no_autotune else P.autotune(prec)
    sfu = ctx.measure_sfu()                                      # untimed: the measured MUFU rate
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=f"cuda:{dev}")

    if args.ops_only:
        xs = torch.tensor(np.abs(w.x_true) + 0.01, dtype=torch.float64, device=f"cuda:{dev}")
        vs = torch.zeros((w.n_vis, 2), dtype=torch.float64, device=f"cuda:{dev}")
        img_d = torch.zeros(w.n_pix, dtype=torch.float64, device=f"cuda:{dev}")

        def one_step():
            P.forward_dev(xs, vs, prec)
            P.adjoint_dev(vs, img_d, prec)
            return None, {"iters": 0, "power_iters": 0, "E": 0.0, "resid2": 0.0, "nnz": 0, "L": 0.0}
    elif args.full_solve:
        def one_step():
            return P.solve(lam, L=0.0, max_iter=args.iters, precision=prec)
    else:
        L_fixed, _ = P.max_eig(50, 1e-6, prec)                 # once, untimed

        def one_step():
            return P.solve(lam, L=L_fixed, max_iter=args.iters, precision=prec)

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    ctx.profile_reset()
    ctx.counters_reset()
    ctx.profile_enable(True)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev = []
    stats = []
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)                     # L2 flush between steps (outside the events)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        img, st = one_step()
        with torch.cuda.stream(stream):
            e1.record(stream)
        ev.append((e0, e1))
        stats.append(st)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    ctx.profile_enable(False)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    T = sum(step_ms) / 1e3
    counters = ctx.counters()
    prof = {k: ctx.profile_read(k) for k in sl1m.KERNEL_IDS}
    op_pairs = sum(prof[k]["pairs"] for k in ("fwd_fp64", "adj_fp64", "fwd_mixed", "adj_mixed"))
    T_job, pairs_job = job_totals(T, op_pairs, ws, f"cuda:{dev}")
    value = pairs_job / T_job
    rate_key, rate_val = (("solves_per_s", ws * args.steps / T_job) if args.full_solve else
                          ("fista_steps_per_s", ws * args.steps * args.iters / T_job))

    # roofline of the dominant kernel
    keys = ("fwd_mixed", "adj_mixed") if prec == sl1m.MIXED else ("fwd_fp64", "adj_fp64")
    dom = max(keys, key=lambda k: prof[k]["ms"])
    pd = prof[dom]
    achieved = pd["pairs"] / (pd["ms"] / 1e3) / 1e9 if pd["ms"] > 0 else 0.0
    op_of = lambda k: "fwd" if k.startswith("fwd") else "adj"   # noqa: E731
    peak, peak_basis, alt = sfu_peak(w, op_of(dom))
    traffic = None
    if tuned is not None:
        op = 0 if dom.startswith("fwd") else 1
        traffic = ncu_traffic(dom, tuned["nst"][op], tuned["npoly"][op],
                              tuned["ctas_per_sm"][op] * N_SM, w.name)
    # launches that did work: a solver tick launches every operator kernel, but a
    # problem whose phase gives it no role in one skips its units
    worked = {k: max(1, round(prof[k]["pairs"] / (float(w.n_vis) * w.n_pix))) for k in keys}
    roofline = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak,
                "unit": "Gpairs/s", "frac": achieved / peak, "peak_basis": peak_basis,
                "launches": pd["launches"], "launches_with_work": worked[dom],
                "avg_launch_ms": pd["ms"] / worked[dom], "traffic": traffic}
    if alt:
        roofline["peak_sfu_plus_fma_sincos"] = alt
        roofline["frac_of_sfu_plus_fma_sincos"] = achieved / alt["peak"]
    meas = sfu_peak_measured(w, sfu, op_of(dom))
    roofline["peak_measured_sfu"] = meas
    roofline["frac_of_measured_sfu"] = achieved / meas["peak"]
    per_kernel = {}
    for k in keys:
        if prof[k]["ms"] <= 0:
            continue
        rate = prof[k]["pairs"] / (prof[k]["ms"] / 1e3) / 1e9
        pk, _, pk_alt = sfu_peak(w, op_of(k))
        per_kernel[k] = {"launches": prof[k]["launches"], "launches_with_work": worked[k],
                         "avg_launch_ms": prof[k]["ms"] / worked[k], "Gpairs_per_s": rate,
                         "sfu_peak": pk, "frac_of_peak": rate / pk,
                         "frac_of_measured_sfu": rate / sfu_peak_measured(w, sfu, op_of(k))["peak"]}
        if pk_alt:
            per_kernel[k]["frac_of_sfu_plus_fma"] = rate / pk_alt["peak"]
    fin_ms = prof["fwd_finish"]["ms"] + prof["adj_finish"]["ms"]
    fin_bytes = prof["fwd_finish"]["bytes"] + prof["adj_finish"]["bytes"]
    vec = {"kernels": "fwd_finish+adj_finish (residual, threshold, momentum)",
           "achieved_GBps": fin_bytes / (fin_ms / 1e3) / 1e9 if fin_ms else None,
           "share_of_step": fin_ms / (T * 1e3)}

    e2e = None
    if not args.no_e2e and not args.ops_only:
        e2e = run_e2e(ctx, w, V, lam, 0.0 if args.full_solve else L_fixed, prec, args, sl1m, stream, ws)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        xb, rb = baseline_inputs(w)
        cpu = cpu_baseline(w, P.forward(xb, prec), P.adjoint(rb, prec))
    ctx.close()
    serving = None
    if rank == 0 and ws == 1 and not args.no_serve and not args.ops_only:
        del flush
        torch.cuda.empty_cache()
        serving = serving_measure(args.requests or 48, args.rate or 2.0, args.ticks, args.max_pairs,
                                  args.fp64_sample, not args.no_cpu, dev, args.admission)
    if rank == 0:
        out = {"metric": "pixel-visibility pairs/s (fwd+adj)", "value": value, "unit": "pairs/s",
               "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": 1e3 * T_job / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None,
               "dtype": "f32+f64" if prec == sl1m.MIXED else "f64", "data": "synthetic",
               "config": bench_config(args, w), "lambda": lam, "tile_shape": tuned,
               rate_key: rate_val,
               "iters": [s["iters"] for s in stats], "power_iters": stats[-1]["power_iters"],
               "final": {"E": stats[-1]["E"], "resid2": stats[-1]["resid2"],
                         "nnz": stats[-1]["nnz"], "L": stats[-1]["L"]},
               "roofline": roofline, "operator_kernels": per_kernel, "vector_updates": vec,
               "clocks": clk, "gpu_launches": counters["launches"],
               "e2e": e2e, "cpu_baseline": cpu, "serving": serving}
        print(json.dumps(out))
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_e2e(ctx, w, V, lam, L, prec, args, sl1m, stream, ws=1):
    """The same steps from host buffers through the C ABI, every step: set the
    inputs (host layout + H2D), solve (L given, or computed when 0), read the
    image back (D2H) -- all timed, over as many steps as the device-timed
    figure.  With several ranks, each solves its own problem between two
    barriers and the value is all ranks' pairs over the slowest rank's time."""
    import torch
    steps = max(1, args.steps)
    ctx.counters_reset()
    ctx.profile_reset()
    ctx.profile_enable(True)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        Q = ctx.problem()
        Q.set_visibilities(w.uvw, V, w.weights, w.ant_pair)
        Q.set_pixels(w.lm, w.sigma, w.kind)
        if w.gains is not None:
            Q.set_gains(w.gains)
        img, st = Q.solve(lam, L=L, max_iter=args.iters, precision=prec)
        Q.close()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    ctx.profile_enable(False)
    pairs = sum(ctx.profile_read(k)["pairs"] for k in ("fwd_fp64", "adj_fp64", "fwd_mixed", "adj_mixed"))
    dt, pairs = job_totals(dt, pairs, ws, f"cuda:{torch.cuda.current_device()}")
    c = ctx.counters()
    return {"value": pairs / dt, "unit": "pairs/s", "steps": steps,
            "h2d_bytes_per_step": c["h2d_bytes"] // steps, "d2h_bytes_per_step": c["d2h_bytes"] // steps,
            "ms_per_step": 1e3 * dt / steps,
            "timed": "host wall clock around every step (layout, H2D, solve, image D2H), "
                     "device synchronised on both sides"}


if __name__ == "__main__":
    main()
