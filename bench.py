#!/usr/bin/env python
"""Throughput of the asynchrony-tolerant (AT) forward step on GB300: grid-point updates/s in FP64.

Workload (default): 1D u_t + u_x = 0.1 u_xx on [0, 2 pi), N = 2^24 points in 4096 emulated PEs,
4th-order central differences inside, (1,4,2)/(2,4,2) AT stencils at PE edges, L = 4 uniform delays,
10-mode multi-sine initial condition, 1000 forward-Euler steps.  One bench step = one whole run:
initial condition, 1000 fused steps (delay draw + halo extrapolation + stencil + Euler update in one
kernel per step) and the error statistics against the analytic solution.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 runs one independent replica per rank (the emulated PEs live on one GPU; there is no data
exchange between GPUs), so scaling is weak.  --impl reference times the FP64 CPU oracle on the host
cores instead (rank 0 only).  One JSON line is printed by rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "grid-point updates/s (FP64)"
PEAK_FP64_FLOPS = 152 * 2 * 2 * 2.07e9  # 152 SMs x 2 FP64 FMA lanes/clk x 2 flop x 2.07 GHz max clock
# DRAM bytes (read + write) per launch of the step kernel, the mean of two launches of one ncu capture of the current
# kernel source; None where no capture of the current source exists.
MEASURED_TRAFFIC = {
    ("1d_n16m", "forward_group_kernel<1,2,false>"): 136.95e6 + 80.50e6,
    ("1d_n16m_case2", "forward_group_kernel<1,1,false>"): None,
    ("1d_n16m_case3", "forward_group_kernel<1,1,false>"): 135.27e6 + 80.13e6,
    ("1d_n16m_case4", "forward_group_kernel<1,2,true>"): 271.91e6 + 209.17e6,
    ("1d_n16m_case5", "forward_group_kernel<1,3,true>"): 409.85e6 + 221.76e6,
    ("1d_n16m_case6", "forward_group_kernel<1,2,true>"): 271.83e6 + 209.14e6,
}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def replica_seed(seed: int, rank: int, stride: int = 1) -> int:
    """Seed of this rank's independent replica (ranks share no data; each runs its own delay realization)."""
    return int(seed) + stride * int(rank)


def max_over_ranks(value: float, world: int, device=None) -> float:
    """The job's time is the slowest rank's: all-reduce MAX (NCCL on GPUs, gloo on CPU in the tests)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time (weak scaling)."""
    return world * units_per_rank / seconds


def time_levels(spec) -> int:
    return max(1, int(spec.get("tsteps", 1)))


def flops_per_update(spec) -> int:
    """FP64 flops per interior point: the merged stencil, 1 multiply + 2*h*dim FMAs (2 flops each); with
    Adams-Bashforth (ts levels) also the ts FMAs that add the weighted right-hand sides to U^n.  Burgers' equation
    keeps its two derivatives apart (below)."""
    h = spec["order"] // 2
    ts = time_levels(spec)
    if spec.get("burgers", 0):
        # Burgers: dt D1 u (1 multiply + 2h-1 FMAs), dt alpha D2 u (1 multiply + 2h FMAs), -u_i * D1 + D2 (1 FMA),
        # then U^n + that (1 add) or the ts Adams-Bashforth FMAs
        f = 1 + 2 * (2 * h - 1) + 1 + 2 * (2 * h) + 2
        return f + (2 * ts if ts > 1 else 1)
    f = 1 + 2 * (2 * h * spec["dim"])
    if ts > 1:
        f += 2 * ts
    return f


def fp64_ops_per_update(spec) -> int:
    """FP64 instructions per interior point, what the FP64 pipe executes: the flops above are FMAs but the leading
    multiplies (issued as FMAs onto zero) and Burgers' final add."""
    h, ts = spec["order"] // 2, time_levels(spec)
    if spec.get("burgers", 0):
        return 4 * h + 2 + (ts if ts > 1 else 1)
    return (flops_per_update(spec) + 1) // 2


def bytes_per_update(spec) -> int:
    """Algorithmic HBM bytes per point and step: read U^n, write U^{n+1}; with Adams-Bashforth also read the ts-1
    stored right-hand sides and write dt f^n (halo reads of delayed levels are not counted)."""
    ts = time_levels(spec)
    return 16 + (8 * ts if ts > 1 else 0)


def launches_per_run(spec, T: int) -> int:
    """Kernels of this library one timed run launches: the reset (initial field, Adams-Bashforth pre-history and
    its history counter, the first delay draw), T forward steps (one counter update before the captured graphs,
    each 50-step graph holding 50 step kernels and a counter kernel; the remainder launched one by one) and the
    error statistics."""
    dim, ts = spec["dim"], time_levels(spec)
    wave = 1 if dim == 1 else 2
    if spec.get("burgers", 0):  # no analytic pre-history: the history counter only
        reset = wave + 1 + (1 if ts > 1 else 0)
    else:
        reset = wave + 1 + (((ts - 1) * (wave + 1) + 1) if ts > 1 else 0)
    chunks = T // 50
    step = (1 + 51 * chunks if chunks else 0) + (T - 50 * chunks)
    stats = 2 if dim == 1 else 3
    return reset + step + stats


def cpu_sample(spec, nsteps: int, threads: int) -> float:
    """Oracle updates/s on `nsteps` steps of the full-size grid, initial condition excluded."""
    import oracle
    cfg = oracle.Config(spec)
    t0 = time.perf_counter()
    oracle.run(cfg, 0, want_log=False, threads=threads)
    t_ic = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.run(cfg, nsteps, want_log=False, threads=threads)
    t = time.perf_counter() - t0 - t_ic
    return cfg.ntot * nsteps / max(t, 1e-9)


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    spec, total_steps = W.workload(args.workload)
    cores = os.cpu_count() or 1
    sample_steps = args.ref_sample_steps
    for _ in range(args.warmup):
        cpu_sample(spec, 1, cores)
    vals = [cpu_sample(spec, sample_steps, cores) for _ in range(args.steps)]
    v = statistics.median(vals)
    ntot = 1
    for x in spec["n"]:
        ntot *= x
    ms = ntot * total_steps / v * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "points": ntot, "time_steps": total_steps},
            "cpu_baseline": {"value": v, "unit": "updates/s", "cores": cores, "kind": "oracle",
                             "sample": f"{sample_steps} steps of the full {ntot}-point grid per bench step, "
                                       f"initial condition excluded, OpenMP over points"},
            "e2e": {"value": v, "unit": "updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


SWEEPS = ("sweep_scaling", "sweep_kmom")


def sweep_members(name: str):
    """Member lists of the paper's sweeps (Sec. 5.2) with synchronous twins: (specs, steps, groups, twins).
    sweep_scaling: Fig. "at-ord2-procs", Case 1 with p_k = {0.2, 0.5, 0.3}, P in {2..32} at N = 512, strong
    (P = 16) and weak (P/N = 1/16) series over N in {128..1024}, 32 realizations each, every member to t = 0.1.
    sweep_kmom: Fig. "at-kmom", Case 4 at N = 512, P = 16, L in {2, 3, 4} with p_k = 1/L, 64 realizations each."""
    if name == "sweep_scaling":
        ns = (128, 256, 512, 1024)
        grids = [(512, P) for P in (2, 4, 8, 16, 32)] + [(n, 16) for n in ns] + [(n, n // 16) for n in ns]
        return W.scaling_members(1, grids, range(800, 832))
    return W.moment_members(4, (2, 3, 4), range(900, 964))


def run_ensemble(args, rank: int, world: int, local: int):
    """1024 1D realizations (N_r in 2^10..2^16, L_r in 2..4, 5000 steps) in one persistent graph launch, against
    the same realizations run one problem at a time through the single-problem path (graph-captured steps)."""
    import torch
    import torch.distributed as dist
    from paper_1702_00496_gb300 import Ensemble, Solver

    groups_in = twins = None
    if args.workload == "ensemble":
        specs, T = W.ensemble_members()
        if args.time_steps is not None:
            T = args.time_steps
        steps = [T] * len(specs)
    else:
        specs, steps, groups_in, twins = sweep_members(args.workload)
        T = None
    for s in specs:
        s["seed"] = replica_seed(s["seed"], rank, 100000)
    updates = sum(s["n"][0] * st for s, st in zip(specs, steps))
    stream = torch.cuda.current_stream()
    threads, ctas = args.threads, args.ctas_per_sm
    if threads == 0:
        from paper_1702_00496_gb300 import autotune
        threads, ctas = autotune.tune_ensemble(specs, steps, device=f"cuda:{local}", use_cache=not args.retune)
    ens = Ensemble(specs, steps, threads=threads, ctas_per_sm=ctas, device=f"cuda:{local}", stream=stream,
                   groups=groups_in, twins=twins)
    for _ in range(args.warmup):
        ens.run()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        ens.run()
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    per, groups = ens.stats()
    ms = max_over_ranks(ms, world, f"cuda:{local}")
    # the same realizations one problem at a time: reset, T steps, statistics, in sequence
    one = None
    if not args.skip_one_at_a_time and T is not None:
        solvers = [Solver(s, device=f"cuda:{local}", stream=stream) for s in specs]
        for sv in solvers:  # builds each solver's captured step graph outside the timed region
            sv.step(50)
            sv.reset()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for sv in solvers:
            sv.reset()
            sv.step(T)
            sv.error_stats()
        torch.cuda.synchronize()
        one = (time.perf_counter() - t0) * 1e3
        for sv in solvers:
            sv.close()
    ens.close()
    if rank == 0:
        line = {"metric": METRIC + " -- batched ensemble", "value": world * updates / (ms / 1e3), "unit": "updates/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": args.workload, "members": len(specs),
                           "time_steps": T if T is not None else [min(steps), max(steps)],
                           "total_points": sum(s["n"][0] for s in specs), "point_updates": updates,
                           "launch": {"threads": threads, "ctas_per_sm": ctas}},
                "one_at_a_time_ms": one, "speedup_vs_one_at_a_time": (one / ms) if one else None,
                "groups": groups, "clocks": clocks, "gpu_launches": args.steps * 4}
        print(json.dumps(line), flush=True)


def run_adjoint(args, rank: int, world: int, local: int):
    """Gradient of 1/2 ||U^T - u_target||^2 (256^3, order 4, 2000 steps) by the hand-written adjoint with
    sqrt(T) checkpointing, against the forward run alone: reports the adjoint/forward time ratio."""
    import torch
    from paper_1702_00496_gb300 import Solver

    spec, T = W.workload("adjoint_256")
    if args.time_steps is not None:
        T = args.time_steps
    spec["seed"] = replica_seed(spec["seed"], rank)
    ntot = spec["n"][0] * spec["n"][1] * spec["n"][2]
    stream = torch.cuda.current_stream()
    s = Solver(spec, device=f"cuda:{local}", stream=stream)
    target = torch.zeros(ntot, dtype=torch.float64, device=f"cuda:{local}")
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    fwd, adj, adj_u0, bwd = [], [], [], []
    sampler = ClockSampler(local)
    for it in range(args.warmup + args.steps):
        if it == args.warmup:
            sampler.start()
        s.reset()
        a, b = ev(), ev()
        a.record(stream)
        s.step(T)
        b.record(stream)
        s.reset()
        c, m, d = ev(), ev(), ev()
        c.record(stream)
        s.adjoint_forward(T, args.adjoint_every)
        m.record(stream)
        lam = s.field().reshape(-1) - target
        g, ga = s.adjoint_backward(lam)
        d.record(stream)
        s.reset()
        e, f = ev(), ev()
        e.record(stream)
        s.adjoint_forward(T, args.adjoint_every)
        g0, _ = s.adjoint_backward(s.field().reshape(-1) - target, want_alpha=False)
        f.record(stream)
        torch.cuda.synchronize()
        if it >= args.warmup:
            fwd.append(a.elapsed_time(b))
            adj.append(c.elapsed_time(d))
            bwd.append(m.elapsed_time(d))
            adj_u0.append(e.elapsed_time(f))
    clocks = sampler.stop()
    s.close()
    f_ms, a_ms = statistics.median(fwd), statistics.median(adj)
    if rank == 0:
        line = {"metric": METRIC + " -- adjoint", "value": world * ntot * T / (a_ms / 1e3), "unit": "updates/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": a_ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": "adjoint_256", "points": ntot, "time_steps": T,
                           "checkpoint_every": args.adjoint_every or "sqrt(T)",
                           "levels_resident": args.adjoint_every >= T},
                "forward_ms": f_ms, "adjoint_ms": a_ms, "adjoint_forward_ratio": a_ms / f_ms,
                "backward_ms": statistics.median(bwd),
                "backward_step_forward_step_ratio": statistics.median(bwd) / f_ms,
                "adjoint_u0_only_ms": statistics.median(adj_u0),
                "adjoint_u0_only_forward_ratio": statistics.median(adj_u0) / f_ms,
                "note": "adjoint_ms = forward pass with checkpoints + backward sweep (restore, recompute, transposed "
                        "steps) for dJ/du0 and dJ/dalpha; backward_ms = the sweep alone, T backward steps against "
                        "forward_ms's T forward steps; the u0-only sweep needs no recompute; with every level "
                        "resident (--adjoint-every >= T) the forward pass keeps all levels and nothing is recomputed",
                "grad_alpha": ga, "clocks": clocks}
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="1d_n16m")
    ap.add_argument("--ref-sample-steps", type=int, default=10)
    ap.add_argument("--cpu-sample-steps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--time-steps", type=int, default=None, help="override the steps per run (profiling only)")
    ap.add_argument("--threads", type=int, default=0, help="ensemble: threads per CTA (0: library default)")
    ap.add_argument("--ctas-per-sm", type=int, default=0, help="ensemble: CTAs per SM (0: occupancy limit)")
    ap.add_argument("--skip-one-at-a-time", action="store_true")
    ap.add_argument("--retune", action="store_true", help="ignore the autotuner cache")
    ap.add_argument("--launch", default="", help="forward step: fixed launch shape THREADS,BLOCKS_PER_SM (no tuning)")
    ap.add_argument("--adjoint-every", type=int, default=0,
                    help="adjoint: checkpoint interval (0: sqrt(T); >= T: every level resident, no recompute)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if args.workload == "ensemble" or args.workload in SWEEPS:
        return run_ensemble(args, rank, world, local)
    if args.workload == "adjoint_256":
        return run_adjoint(args, rank, world, local)

    from paper_1702_00496_gb300 import Solver

    spec, T = W.workload(args.workload)
    if args.time_steps is not None:
        T = args.time_steps
    spec["seed"] = replica_seed(spec["seed"], rank)  # independent replica per rank
    ntot = 1
    for x in spec["n"]:
        ntot *= x
    stream = torch.cuda.current_stream()
    solver = Solver(spec, log_steps=0, device=f"cuda:{local}", stream=stream)
    from paper_1702_00496_gb300 import autotune
    if args.launch:
        launch = tuple(int(v) for v in args.launch.split(","))
        from paper_1702_00496_gb300 import at_set_launch
        at_set_launch(solver.h, *launch)
        solver.reset()
    else:
        launch = autotune.tune_forward(solver, spec, use_cache=not args.retune)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float64, device=f"cuda:{local}")  # 512 MiB > L2
    kern_ev = []
    burgers = bool(spec.get("burgers", 0))
    # Burgers' equation has no analytic solution: its run reports the statistics of U^T - U^0 (the RMS change)
    u_ic = solver.field().clone() if burgers else None

    def stats():
        return solver.error_stats_ref(u_ic, 1) if burgers else solver.error_stats()

    def one_step(record=False):
        flush.zero_()
        solver.reset()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        solver.step(T)
        e1.record(stream)
        st = stats()  # blocks
        if record:
            kern_ev.append((e0, e1))
        return st

    for _ in range(args.warmup):
        one_step()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    sampler = ClockSampler(local)
    barrier()
    sampler.start()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    last = None
    for _ in range(args.steps):
        last = one_step(record=True)
    t_end.record(stream)
    barrier()
    clocks = sampler.stop()
    ms = t_start.elapsed_time(t_end) / args.steps
    kern_ms = sum(a.elapsed_time(b) for a, b in kern_ev) / (args.steps * T)
    ms = max_over_ranks(ms, world, f"cuda:{local}")
    value = aggregate_rate(ntot * T, world, ms / 1e3)

    # end to end through the public API: pinned host field in, final field and statistics out
    solver.reset()
    torch.cuda.synchronize()
    u0_host = torch.empty(ntot, dtype=torch.float64, pin_memory=True)
    u0_host.copy_(solver.field().reshape(-1))
    out_host = torch.empty(ntot, dtype=torch.float64, pin_memory=True)
    u0_dev = torch.empty(ntot, dtype=torch.float64, device=f"cuda:{local}")
    e2e_steps = max(1, min(args.steps, 3))

    def e2e_step():
        flush.zero_()
        u0_dev.copy_(u0_host, non_blocking=True)
        solver.reset(u0_dev)
        solver.step(T)
        st = stats()
        out_host.copy_(solver.field().reshape(-1), non_blocking=True)
        torch.cuda.synchronize()
        return st

    e2e_step()
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    barrier()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e_s = max_over_ranks(e2e_s, world, f"cuda:{local}")
    e2e_value = aggregate_rate(ntot * T, world, e2e_s)

    peaks = measured_peaks()
    flops_launch = flops_per_update(spec) * ntot
    achieved = flops_launch / (kern_ms / 1e3)
    bytes_launch = bytes_per_update(spec) * ntot
    hbm = peaks.get("hbm_gbs")
    kname = f"forward_group_kernel<{spec['dim']},{spec['order'] // 2},{'true' if time_levels(spec) > 1 else 'false'}>"
    roofline = {"bound": "alu", "achieved": achieved / 1e12, "peak": PEAK_FP64_FLOPS / 1e12, "unit": "TFLOP/s",
                "frac": achieved / PEAK_FP64_FLOPS, "traffic": MEASURED_TRAFFIC.get((args.workload, kname)),
                "traffic_unit": "bytes per launch (DRAM read + write, ncu)",
                "algorithmic_bytes_per_launch": bytes_launch,
                "kernel": kname, "launch_ms": kern_ms,
                "peak_source": "152 SMs x 2 FP64 FMA/clk x 2 flop x 2070 MHz",
                "fp64_lanes_per_clk_sm": fp64_ops_per_update(spec) * ntot / (kern_ms / 1e3) / 152 / 2.07e9,
                "hbm_gbs": bytes_launch / (kern_ms / 1e3) / 1e9,
                "hbm_frac_of_measured": (bytes_launch / (kern_ms / 1e3) / 1e9 / hbm) if hbm else None}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        v = cpu_sample(spec, args.cpu_sample_steps, cores)
        cpu = {"value": v, "unit": "updates/s", "cores": cores, "kind": "oracle",
               "sample": f"{args.cpu_sample_steps} steps of the full {ntot}-point grid, initial condition excluded, "
                         f"OpenMP over points"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "updates/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": args.workload, "points": ntot, "pes": spec["pe"], "order": spec["order"],
                           "L": spec["L"], "time_levels": time_levels(spec), "time_steps_per_step": T, "l2": "flushed (512 MiB write) each step",
                           "replicas": world, "launch": {"threads": launch[0], "blocks_per_sm": launch[1]}},
                "e2e": {"value": e2e_value, "unit": "updates/s", "h2d_bytes_per_step": 8 * ntot,
                        "d2h_bytes_per_step": 8 * ntot + 8 * 9},
                "roofline": roofline, "cpu_baseline": cpu, "clocks": clocks,
                "gpu_launches": args.steps * launches_per_run(spec, T),
                ("final_rms_change" if burgers else "final_rms_error"): last["rms"]}
        print(json.dumps(line), flush=True)
    solver.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
