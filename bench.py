#!/usr/bin/env python
"""Throughput of the mechanical-interaction step (grid + force +
displacement) on GB300: agent-updates/s, with the force kernel's HBM
roofline fraction, an end-to-end figure through the C ABI with host
buffers, and the CPU oracle timed on the host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl own|reference]
                    [--workload clustered_8M|plain_fp64_4096|uniform_200M|batched_sweep_256|
                                growth_division_65536|clustered_1M]
                    [--precision 1|0] [--static 0|1] [--static-leg 0|1]

One step = one iteration of every simulation of the workload.  The timed
region replays the library's CUDA graphs (the production path); a profiled
pass of as many iterations right after it brackets every stage with CUDA
events on the library's stream, which gives the stage times and the force
kernel's launch duration of the roofline.  Under torchrun (N > 1) every rank
steps its own replica of the workload (the single-domain workloads do not
shard) or, for the parameter sweep, its share of the simulations; the value
is the whole-job aggregate over ranks and timing is the maximum over ranks.

The clustered 8M workload keeps its stated re-sort settings (Morton order
every 10 iterations); the autotuner picks only the force kernel, the box
length and the iterations per graph there.  Its line also carries a static-
skip leg: static detection on and off from the same input, settled until
the static fraction changes by less than 0.5% over 10 iterations (at most
500), then 100 timed iterations each.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import platform
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "agent-updates/s (grid+force+displace)"
UNIT = "agent-updates/s"
# Algorithmic bytes of the force kernel (FP32-force path): per agent the
# FP64 position (24 B), an FP32 diameter (4 B), the static flag (1 B), the
# FP32 force (12 B) and the nnz count (1 B); per occupied box 8 B.  FP64
# path: FP64 diameter (8 B) and FP64 force (24 B).
ALG_BYTES_AGENT = {1: 42.0, 0: 58.0}
ALG_BYTES_BOX = 8.0
# DRAM bytes (read + write) per agent of a force kernel, from an ncu capture
# of the 1M-agent clustered case (the per-cluster shape of the 8M case),
# scaled by the agents of a launch for the clustered workloads and null
# elsewhere.  Keyed by force variant; an entry holds only while the
# variant's kernel is the one captured.
FORCE_TRAFFIC_B_PER_AGENT = {5: 104.9}
FORCE_KERNEL = {0: "k_force32s", 1: "k_force32d", 2: "k_force", 3: "k_force32d", 4: "k_force32s (direct)",
                5: "k_force32w", 6: "k_static + k_force32w"}
# Workloads whose configuration fixes the re-sort (interval, curve): the
# autotuner leaves those two knobs alone there.
FIXED_SORT = {"clustered_8M": (10, 0), "clustered_1M": (10, 0)}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="own", choices=["own", "reference"])
    ap.add_argument("--workload", default="clustered_8M")
    ap.add_argument("--precision", type=int, default=1)
    ap.add_argument("--static", type=int, default=0)
    ap.add_argument("--settle", type=int, default=-1,
                    help="untimed iterations before warm-up; -1: 65 for the growth workload (its capacity "
                         "holds from the 65th iteration on), else 50")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--force-variant", type=int, default=-1, help="-1: autotune; else the variant")
    ap.add_argument("--sort-interval", type=int, default=-2, help="-2: autotune/workload default")
    ap.add_argument("--static-leg", type=int, default=-1,
                    help="static detection on/off leg; -1: on for the clustered 8M workload")
    ap.add_argument("--static-steps", type=int, default=100)
    ap.add_argument("--execution-context", type=int, default=0, choices=(0, 1),
                    help="1: the in-place execution context (FP64 path, no static detection)")
    ap.add_argument("--reuse-leg", type=int, default=-1,
                    help="incremental-grid leg; -1: on for the clustered 8M workload")
    ap.add_argument("--iter-batch", type=int, default=-1, help="iterations per graph; -1: autotune")
    ap.add_argument("--box-scale", type=int, default=-1, help="box length in %% of the largest diameter; -1: autotune")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the library's default tuning (with the fixed settings), e.g. for a profiler capture")
    args = ap.parse_args()
    if args.settle < 0:
        args.settle = 65 if args.workload == "growth_division_65536" else 50
    return args


def make_workload(name: str, precision: int, static: int, build: bool = True, exec_ctx: int = 0):
    """(populations, description); build=False describes the 200M-agent
    workload without generating it (populations None)."""
    from paper_2503_10796_gb300 import workloads as W
    if name == "clustered_8M":
        pops = [W.clustered(precision=precision, detect_static=static, sort_interval=10)]
        desc = dict(workload="clustered_8M", agents=8388608, clusters=64, sigma=200.0, side=1.0e4,
                    diameters="U[8,12]", sort_interval=10)
    elif name == "clustered_1M":
        # profiling case: 8 clusters of the same shape in a 5,000 cube
        pops = [W.clustered(n_clusters=8, side=5000.0, precision=precision, detect_static=static,
                            sort_interval=10)]
        desc = dict(workload="clustered_1M", agents=1048576, clusters=8, sigma=200.0, side=5.0e3,
                    diameters="U[8,12]", sort_interval=10)
    elif name == "growth_division_65536":
        pops = [W.growth_division(precision=precision)]
        desc = dict(workload="growth_division_65536", agents_start=65536, agents_cap=2097152,
                    lattice=[32, 32, 64], spacing=10.0, diameter=9.0, divide_diameter=12.0,
                    growth_rate=4000.0, dt=0.01)
    elif name == "plain_fp64_4096":
        pops = [W.plain_fp64(precision=precision)]
        desc = dict(workload="plain_4096", agents=4096, side=160.0, diameters="U[8,12]")
    elif name == "uniform_200M":
        pops = [W.uniform_fraction(200_000_000, precision=precision, sort_interval=10)] if build else None
        desc = dict(workload="uniform_200M", agents=200_000_000, volume_fraction=0.3)
    elif name == "batched_sweep_256":
        pops = W.batched_sweep(precision=precision)
        desc = dict(workload="batched_sweep_256", sims=256, agents=int(sum(p.n for p in pops)))
    else:
        raise SystemExit(f"unknown workload {name}")
    for p in pops or []:
        p.params.detect_static = static
        p.params.execution_context = exec_ctx
    if exec_ctx:
        desc.update(execution_context="in-place")
    slots = sum(max(p.n, p.params.capacity) for p in pops) if pops is not None else desc["agents"]
    desc.update(static_skip=bool(static),
                l2="inputs larger than L2 (no flush needed)" if slots > 1_000_000 else "working set inside L2")
    return pops, desc


def host_info() -> dict:
    """Host cores and CPU model (the oracle runs on one of them)."""
    model = platform.processor() or platform.machine()
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model"):
                model = line.split(":", 1)[1].strip()
                if model:
                    break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model, "machine": platform.machine()}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        return self.summarize(self.lines)

    @staticmethod
    def summarize(lines) -> dict:
        """Median SM clock, the largest maximum clock and the throttle reasons
        seen active in the sampled CSV lines (FIELDS order)."""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def cpu_baseline(name: str, exec_ctx: int = 0):
    """The oracle, as it stands, on a bounded sample of the workload (in the
    execution context of the GPU run)."""
    import oracle
    from paper_2503_10796_gb300 import workloads as W
    oracle.build()
    if name == "clustered_8M":
        pop = W.clustered(n_clusters=8)
        iters, sample = 3, "3 iterations of 8 of the 64 clusters (1,048,576 agents), same per-cluster shape"
    elif name == "plain_fp64_4096":
        pop = W.plain_fp64()
        iters, sample = 10, "the full workload, 10 iterations"
    elif name == "uniform_200M":
        pop = W.uniform_fraction(1_000_000)
        iters, sample = 2, "2 iterations of 1,000,000 agents at the same volume fraction"
    else:
        pops = W.batched_sweep()
        pop = pops[int(np.argsort([p.n for p in pops])[len(pops) // 2])]
        iters, sample = 5, f"5 iterations of the median simulation ({pop.n} agents)"
    s = oracle.Sim(pop.xyz, pop.diameter, pop.params, execution_context=exec_ctx)
    t0 = time.perf_counter()
    s.step(iters)
    dt = time.perf_counter() - t0
    return {"value": pop.n * iters / dt, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
            "seconds": dt, **host_info()}


def parallelism_of(workload: str, world: int) -> str:
    if world > 1 and workload == "batched_sweep_256":
        return f"{world} ranks, simulations sharded (longest-processing-time)"
    return f"{world} independent replicas" if world > 1 else "1 GPU"


def arm_config(desc: dict, parallelism: str, precision: str, args) -> dict:
    """The `config` of a JSON line: the workload (the same for both arms),
    the arm's parallelism and the precision it computes in."""
    return dict(desc, parallelism=parallelism, precision=precision, settle_iterations=args.settle)


def precision_of(p: int) -> str:
    return "fp32-force/fp64-position" if p == 1 else "fp64"


def reference_arm(args):
    """--impl reference: the oracle on the host cores, one bounded sample per step."""
    import oracle
    from paper_2503_10796_gb300 import workloads as W
    oracle.build()
    if args.workload == "clustered_8M":
        pop = W.clustered(n_clusters=2)
        sample = "each step: 1 iteration of 2 of the 64 clusters (262,144 agents)"
    elif args.workload == "plain_fp64_4096":
        pop = W.plain_fp64()
        sample = "each step: 1 iteration of the full workload"
    elif args.workload == "uniform_200M":
        pop = W.uniform_fraction(250_000)
        sample = "each step: 1 iteration of 250,000 agents at the same volume fraction"
    else:
        pops = W.batched_sweep()
        pop = pops[int(np.argsort([p.n for p in pops])[len(pops) // 2])]
        sample = f"each step: 1 iteration of the median simulation ({pop.n} agents)"
    s = oracle.Sim(pop.xyz, pop.diameter, pop.params, execution_context=args.execution_context)
    for _ in range(args.warmup):
        s.step(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s.step(1)
    dt = time.perf_counter() - t0
    v = pop.n * args.steps / dt
    _, desc = make_workload(args.workload, args.precision, args.static, build=False,
                            exec_ctx=args.execution_context)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": arm_config(desc, "1 host core (the oracle, single-threaded)", "fp64 (the oracle)", args),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                             **host_info()},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def settle_static(ctx, n_agents: int, limit: int = 500, window: int = 10, tol: float = 0.005):
    """Step until the static fraction changes by less than `tol` over
    `window` iterations (at most `limit` iterations); returns the iterations
    stepped and the fraction trace."""
    trace = []
    done = 0
    prev = None
    while done < limit:
        ctx.step(window)
        done += window
        f = ctx.stats(0)["static_agents"] / max(n_agents, 1)
        trace.append(round(f, 5))
        if prev is not None and abs(f - prev) < tol:
            break
        prev = f
    return done, trace


def timed_steps(ctx, stream, steps: int):
    """CUDA-event time (ms) of `steps` iterations on the library's stream."""
    import torch
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ctx.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def static_leg(args, local: int, tune_knobs: int, fixed: dict):
    """Static detection on and off on the same input: settle by the rule with
    detection on, step the detection-off context as many iterations, then
    time `--static-steps` iterations of each."""
    import torch
    from paper_2503_10796_gb300 import binding
    out = {}
    ctxs = {}
    stream = torch.cuda.Stream(device=local)
    for on in (1, 0):
        pops, _ = make_workload(args.workload, args.precision, on)
        p = pops[0]
        ctxs[on] = (binding.Context([binding.make_params(p.params)], p.n + 1024, device=local,
                                    stream=stream.cuda_stream), p.n)
        ctxs[on][0].set_agents(0, p.xyz, p.diameter)
    ctx_on, n = ctxs[1]
    settled, trace = settle_static(ctx_on, n)
    ctx_off, _ = ctxs[0]
    ctx_off.step(settled)
    for on in (1, 0):
        ctx = ctxs[on][0]
        if fixed:
            t = ctx.get_tuning()
            t.update(fixed)
            ctx.set_tuning(**t)
        tuning = ctx.autotune(3, tune_knobs) if tune_knobs else None
        ctx.step(args.warmup)
        ctx.sync()
        ms = timed_steps(ctx, stream, args.static_steps)
        st = ctx.stats(0)
        out["on" if on else "off"] = {"value": n * args.static_steps / (ms * 1e-3), "ms_per_step": ms / args.static_steps,
                                      "static_fraction_last_iter": st["static_agents"] / n,
                                      "tuning": ctx.get_tuning() if tuning is None else tuning}
    for on in (1, 0):
        ctxs[on][0].close()
    return {"settle_rule": "until the static fraction changes by < 0.5% over 10 iterations, at most 500",
            "settle_iterations": settled, "static_fraction_trace_every_10": trace,
            "timed_iterations": args.static_steps, "unit": UNIT, **out,
            "speedup": out["on"]["value"] / out["off"]["value"]}


def reuse_leg(args, local: int, tuning: dict):
    """The incremental grid (tuning grid_reuse) on the same workload and
    settings as the timed run: iterations keep the last build's grid while
    every agent stays within the skin of its box.  Times as many iterations
    and reports the grid builds among them."""
    import torch
    from paper_2503_10796_gb300 import binding
    pops, _ = make_workload(args.workload, args.precision, 0)
    p = pops[0]
    stream = torch.cuda.Stream(device=local)
    ctx = binding.Context([binding.make_params(p.params)], p.n + 1024, device=local, stream=stream.cuda_stream)
    ctx.set_agents(0, p.xyz, p.diameter)
    ctx.step(args.settle)
    t = ctx.get_tuning()
    t.update(tuning)
    t.update(grid_reuse=1, box_scale_pct=max(int(t.get("box_scale_pct") or 100), 125))
    ctx.set_tuning(**t)
    ctx.step(args.warmup)
    ctx.sync()
    b0 = ctx.counters()["grid_builds"]
    ms = timed_steps(ctx, stream, args.steps)
    builds = ctx.counters()["grid_builds"] - b0
    ctx.close()
    return {"what": "incremental grid: the last build kept while every agent stays within (L - largest "
                    "diameter) / 2 of its box; rebuilt on re-sorts and when an agent leaves its skin",
            "value": p.n * args.steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / args.steps,
            "timed_iterations": args.steps, "grid_builds": builds, "tuning": ctx_tuning_dict(t)}


def ctx_tuning_dict(t: dict) -> dict:
    return {k: int(v) for k, v in t.items()}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            reference_arm(args)
        return
    import torch
    import torch.distributed as dist
    from paper_2503_10796_gb300 import binding
    torch.cuda.set_device(local)
    if world > 1:
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    pops, desc = make_workload(args.workload, args.precision, args.static, exec_ctx=args.execution_context)
    if world > 1 and args.workload == "batched_sweep_256":
        # independent simulations: shard them, no exchange on the data path
        from paper_2503_10796_gb300 import sharding
        _, pops = sharding.shard(pops, [p.n for p in pops], rank, world)
    parallelism = parallelism_of(args.workload, world)
    total_agents = sum(max(p.n, p.params.capacity) for p in pops)
    # a dedicated stream: the library captures CUDA graphs on it, which the
    # legacy default stream does not allow
    stream = torch.cuda.Stream(device=local)
    ctx = binding.Context([binding.make_params(p.params) for p in pops], total_agents + 1024, device=local,
                          stream=stream.cuda_stream)
    for s, p in enumerate(pops):
        ctx.set_agents(s, p.xyz, p.diameter)
    if args.settle > 0:
        ctx.step(args.settle)
    # tuning: the workload's own re-sort settings where its configuration
    # states them, the autotuner for the rest
    fixed = {}
    knobs = binding.TUNE_ALL
    if args.workload in FIXED_SORT:
        iv, cv = FIXED_SORT[args.workload]
        fixed = {"sort_interval": iv, "sort_curve": cv}
        knobs &= ~(binding.TUNE_INTERVAL | binding.TUNE_CURVE)
    if args.sort_interval >= -1:
        fixed["sort_interval"] = args.sort_interval
        knobs &= ~binding.TUNE_INTERVAL
    if args.force_variant >= 0:
        fixed["force_variant"] = args.force_variant
        knobs &= ~binding.TUNE_FORCE
    if args.iter_batch >= 0:
        fixed["iter_batch"] = args.iter_batch
        knobs &= ~binding.TUNE_BATCH
    if args.box_scale >= 0:
        fixed["box_scale_pct"] = args.box_scale
        knobs &= ~binding.TUNE_BOX
    if fixed:
        t = ctx.get_tuning()
        t.update(fixed)
        ctx.set_tuning(**t)
    tuning = ctx.autotune(3, knobs) if knobs and not args.no_autotune else ctx.get_tuning()
    ctx.step(args.warmup)
    ctx.sync()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier()
    upd0 = sum(ctx.stats(s)["agent_updates"] for s in range(len(pops)))
    c0 = ctx.counters()
    ms = timed_steps(ctx, stream, args.steps)
    barrier()
    clk = clocks.stop()
    ctx.sync()
    c1 = ctx.counters()
    upd1 = sum(ctx.stats(s)["agent_updates"] for s in range(len(pops)))
    updates = float(upd1 - upd0)
    if world > 1:
        t = torch.tensor([ms, updates], device="cuda", dtype=torch.float64)
        tm = t[:1].clone()
        dist.all_reduce(tm, op=dist.ReduceOp.MAX)
        tu = t[1:].clone()
        dist.all_reduce(tu, op=dist.ReduceOp.SUM)
        ms, updates = float(tm.item()), float(tu.item())
    value = updates / (ms * 1e-3)

    # profiled pass of as many iterations: CUDA events around every stage on
    # the library's stream (stage times, the force kernel's launch duration)
    n_agents = sum(ctx.count(s) for s in range(len(pops)))
    st_static = sum(ctx.stats(s)["static_agents"] for s in range(len(pops)))
    ctx.profile(True)
    prof_ms = timed_steps(ctx, stream, args.steps)
    ctx.sync()
    prof = ctx.get_profile()
    ctx.profile(False)

    # roofline of the force kernel
    f = prof["force"]
    force_ms = f["ms"] / max(f["launches"], 1)
    occupied = 0
    for s in range(len(pops)):
        box, _, _ = ctx.grid(s)
        occupied += int(np.unique(box).size)
    prec = args.precision
    alg = ALG_BYTES_AGENT[prec] * (n_agents - st_static) + ALG_BYTES_BOX * occupied
    peak, peak_kind = peaks()
    variant = (tuning or {}).get("force_variant", 5) if prec == 1 else 2
    if args.static and variant in (0, 4):
        variant = 1  # the symmetric walks do not run with static detection
    kernel = FORCE_KERNEL.get(variant, "k_force") if prec == 1 else "k_force64r"
    if prec == 1 and not args.static and variant == 6:
        kernel = "k_force32w"  # no static flags to compute first
    traffic = None
    if prec == 1 and variant in FORCE_TRAFFIC_B_PER_AGENT and args.workload.startswith("clustered"):
        traffic = FORCE_TRAFFIC_B_PER_AGENT[variant] * (n_agents - st_static)
    achieved = alg / (force_ms * 1e-3) / 1e9

    # end to end through the public API with host buffers: every step moves
    # the current population's positions from pinned host memory to the
    # device (bdm_update_agents; diameters too where agents grow), steps
    # once and reads the new positions back into pinned host memory
    e2e = None
    if args.e2e_steps > 0:
        grows = [p.params.growth_rate > 0 for p in pops]
        bufs = []
        for s in range(len(pops)):
            room = max(pops[s].params.capacity, ctx.count(s), 1)
            xp = torch.empty((room, 3), dtype=torch.float64, pin_memory=True).numpy()
            dp = torch.empty((room,), dtype=torch.float64, pin_memory=True).numpy()
            x, _ = ctx.get_agents(s, out=(xp, dp))
            bufs.append([xp, dp, x.shape[0]])
        def e2e_step():
            up = dn = 0
            for s in range(len(pops)):
                xp, dp, k = bufs[s]
                ctx.update_agents(s, xp[:k], dp[:k] if grows[s] else None)
                up += (32 if grows[s] else 24) * k
            ctx.step(1)
            for s in range(len(pops)):
                xp, dp, _ = bufs[s]
                x, _ = ctx.get_agents(s, out=(xp, dp if grows[s] else None))
                bufs[s][2] = x.shape[0]
                dn += (32 if grows[s] else 24) * x.shape[0]
            return up, dn

        e2e_step()  # untimed: the first host-fed step runs a few percent slower
        h2d = d2h = 0
        stepped = 0
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            stepped += sum(bufs[s][2] for s in range(len(pops)))
            up, dn = e2e_step()
            h2d += up
            d2h += dn
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        e2e_updates = float(stepped)
        if world > 1:
            t = torch.tensor([dt, e2e_updates], device="cuda", dtype=torch.float64)
            tm = t[:1].clone()
            dist.all_reduce(tm, op=dist.ReduceOp.MAX)
            tu = t[1:].clone()
            dist.all_reduce(tu, op=dist.ReduceOp.SUM)
            dt, e2e_updates = float(tm.item()), float(tu.item())
        e2e = {"value": e2e_updates / dt, "unit": UNIT,
               "h2d_bytes_per_step": int(h2d // args.e2e_steps), "d2h_bytes_per_step": int(d2h // args.e2e_steps),
               "steps": args.e2e_steps, "warmup_steps": 1, "host_memory": "pinned",
               "per_step": "bdm_update_agents (positions; diameters where agents grow) + bdm_step(1) + "
                           "bdm_get_agents"}
    ctx.close()

    leg = None
    want_leg = args.static_leg if args.static_leg >= 0 else int(args.workload == "clustered_8M" and world == 1)
    want_leg = want_leg and not args.execution_context  # static detection runs in the copy context only
    if want_leg and len(pops) == 1:
        leg = static_leg(args, local, knobs, {k: v for k, v in fixed.items() if k != "force_variant"})
    rleg = None
    want_reuse = args.reuse_leg if args.reuse_leg >= 0 else int(args.workload == "clustered_8M" and world == 1)
    if want_reuse and len(pops) == 1 and prec == 1:
        rleg = reuse_leg(args, local, tuning or {})
        rleg["speedup_vs_rebuild"] = rleg["value"] / value

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.workload, args.execution_context)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32-force/f64-position" if prec == 1 else "f64", "data": "synthetic",
            "config": arm_config(desc, parallelism, precision_of(prec), args),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "kernel": kernel,
                         "peak_source": f"{peak_kind} hbm_gbs", "force_ms_per_launch": force_ms,
                         "alg_bytes_per_launch": alg,
                         "timing": "CUDA events around the force stage on the library's stream, profiled "
                                   "pass of as many iterations right after the timed region"},
            "stages_ms_per_iter": {k: v["ms"] / max(v["launches"], 1) for k, v in prof.items() if v["launches"]},
            "profiled_ms_per_step": prof_ms / args.steps,
            "static_agents_last_iter": st_static,
            "tuning": tuning,
            "clocks": clk,
            "e2e": e2e,
            "gpu_launches": c1["kernels"] - c0["kernels"],
            "graph_launches": c1["graph_launches"] - c0["graph_launches"],
            "static_skip_leg": leg,
            "incremental_grid_leg": rleg,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
