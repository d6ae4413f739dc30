#!/usr/bin/env python
"""Throughput of the asynchrony-tolerant (AT) forward step on GB300: grid-point updates/s in FP64.

Headline workload: 1D u_t + u_x = 0.1 u_xx on [0, 2 pi), N = 2^24 points in 4096 emulated PEs, 4th-order central
differences inside, (1,4,2)/(2,4,2) AT stencils at PE edges, L = 4 uniform delays, 10-mode multi-sine initial
condition, 1000 forward-Euler steps.  One bench step = one whole run: initial condition, 1000 fused steps (delay
draw + halo extrapolation + stencil + Euler update in one kernel per step) and the error statistics against the
analytic solution.

At N = 1 the same JSON line also carries a record per other workload ("configs"), each timed on the device with
its own warm-up, clock samples, roofline and CPU-oracle sample: the 1D N = 256 run (2000 steps), the 3D 512^3 runs
of orders 2 and 4 (500 steps), the batched ensemble of 1024 realizations (5000 steps) against the same
realizations one problem at a time, and the gradient workload (256^3, 2000 steps) with sqrt(T) checkpoints and
with every level resident, against its forward run.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--no-configs]

N > 1 runs one independent replica per rank (the emulated PEs live on one GPU; there is no data
exchange between GPUs), so scaling is weak.  --impl reference times the FP64 CPU oracle on the host
cores instead (rank 0 only).  One JSON line is printed by rank 0.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "grid-point updates/s (FP64)"
FP64_FMA_LANES_PER_SM = 2  # FP64 FMA lanes per SM per clock on GB300 (nominal)
# DRAM bytes (read + write) per launch of the step kernel, the mean of two launches of one ncu capture of the current
# kernel source; None where no capture of the current source exists.
MEASURED_TRAFFIC = {
    ("1d_n16m", "forward_group_kernel<1,2,0>"): 136.95e6 + 80.50e6,
    # blocks of 4 steps: one block launch (137.4 MB read, 79.2 MB written) and one zone launch (4.6 MB read) per
    # block, per step
    ("1d_n16m", "blocks of 4"): (137.4e6 + 79.2e6 + 4.6e6) / 4,
    ("1d_n16m_case2", "forward_group_kernel<1,1,0>"): None,
    ("1d_n16m_case3", "forward_group_kernel<1,1,0>"): 135.27e6 + 80.13e6,
    ("1d_n16m_case4", "forward_group_kernel<1,2,2>"): 271.86e6 + 208.75e6,
    ("1d_n16m_case5", "forward_group_kernel<1,3,1>"): 409.85e6 + 221.76e6,
    ("1d_n16m_case6", "forward_group_kernel<1,2,1>"): 271.83e6 + 209.14e6,
    # 3D: captured at 256^3 (the same 64^3 PEs; a 512^3 ring is 5-6 GB) over launches 5 and 6 of a 10-step run,
    # scaled to 512^3 by the 8x points
    ("3d_512_o2", "forward_group_kernel<3,1,0>"): 8 * (370.01e6 + 116.13e6),
    ("3d_512_o4", "forward_group_kernel<3,2,0>"): 8 * (475.21e6 + 122.36e6),
}
TRAFFIC_NOTES = {
    "3d_512_o2": "DRAM read + write per launch from ncu at 256^3 in 4^3 PEs of 64^3, scaled by points to 512^3",
    "3d_512_o4": "DRAM read + write per launch from ncu at 256^3 in 4^3 PEs of 64^3, scaled by points to 512^3",
}


# The ensemble kernel's DRAM read + write per point update: ncu on a 100-step launch of the 1024 members (21.16 GB
# read, 13.72 GB written, 1.794e9 updates); the full 5000-step launch scales with its updates.
ENSEMBLE_DRAM_BYTES_PER_UPDATE = (21.16e9 + 13.72e9) / 1.7944576e9


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


def launches_per_run(spec, T: int, K: int = 1) -> int:
    """Kernels of this library one timed run launches: the reset (initial field, Adams-Bashforth pre-history and
    its history counter, the first delay draw), T forward steps (one counter update before the captured graphs,
    each graph of G = 50 steps -- 48 in blocks of K = 4 or 3: whole blocks -- holding its step kernels, a block
    being one zone launch and one block launch, and a counter kernel; the remainder launched one by one) and the
    error statistics."""
    dim, ts = spec["dim"], time_levels(spec)
    wave = 1 if dim == 1 else 2
    if spec.get("burgers", 0):  # no analytic pre-history: the history counter only
        reset = wave + 1 + (1 if ts > 1 else 0)
    else:
        reset = wave + 1 + (((ts - 1) * (wave + 1) + 1) if ts > 1 else 0)
    G = 50 // K * K if K > 1 else 50

    def launches(steps):
        return (steps // K) * 2 + steps % K if K > 1 else steps

    chunks = T // G
    step = (1 + (launches(G) + 1) * chunks if chunks else 0) + launches(T - G * chunks)
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


def cpu_model() -> str:
    """The host CPU's model string (lscpu, else /proc/cpuinfo, else the platform module)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def cpu_forward_baseline(spec, steps_all: int, steps_single: int = 0, what: str = "") -> dict:
    """The oracle (as it stands) on the host cores: `steps_all` steps of the full grid with OpenMP over points on
    every core and, when steps_single > 0, `steps_single` steps on one thread; initial condition excluded."""
    cores = os.cpu_count() or 1
    ntot = 1
    for x in spec["n"]:
        ntot *= x
    out = {"value": cpu_sample(spec, steps_all, cores), "unit": "updates/s", "cores": cores, "kind": "oracle",
           "sample": f"{steps_all} steps of the full {ntot}-point grid{what}, initial condition excluded, "
                     f"OpenMP over points", "cpu_model": cpu_model()}
    if steps_single > 0:
        out["single_thread"] = {"value": cpu_sample(spec, steps_single, 1), "unit": "updates/s", "cores": 1,
                                "sample": f"{steps_single} steps of the full grid on one thread, initial condition "
                                          f"excluded"}
    return out


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
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "ms_per_step_extrapolated": True,
            "ms_per_step_note": f"each bench step times {sample_steps} of the workload's {total_steps} steps; "
                                f"ms_per_step scales that sample to the whole run",
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "points": ntot, "time_steps": total_steps},
            "cpu_baseline": {"value": v, "unit": "updates/s", "cores": cores, "kind": "oracle",
                             "cpu_model": cpu_model(),
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


# --------------------------------------------------------------------------------------------- device peaks
def fp64_peak(local: int):
    """Nominal FP64 rate of this device: SMs x 2 FMA lanes x 2 flop x the maximum SM clock (MEASURED_PEAKS.json's
    sm_max_mhz, else nvidia-smi's clocks.max.sm, else 2070 MHz).  Returns (sms, mhz, flop/s)."""
    import torch
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    mhz = measured_peaks().get("sm_max_mhz")
    if not mhz:
        try:
            out = subprocess.run(["nvidia-smi", f"--id={local}", "--query-gpu=clocks.max.sm",
                                  "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=10)
            mhz = float(out.stdout.strip().splitlines()[0])
        except (OSError, ValueError, IndexError, subprocess.SubprocessError):
            mhz = 2070.0
    return sms, float(mhz), sms * FP64_FMA_LANES_PER_SM * 2 * float(mhz) * 1e6


def measure_dgemm(local: int, n: int = 8192, reps: int = 3):
    """cuBLAS FP64 GEMM rate on this device (torch.matmul, n^3, 2 n^3 flop, best of `reps` after one warm-up):
    a measured FP64 ceiling beside the nominal one."""
    import torch
    try:
        a = torch.randn(n, n, dtype=torch.float64, device=f"cuda:{local}")
        b = torch.randn(n, n, dtype=torch.float64, device=f"cuda:{local}")
        c = torch.matmul(a, b)
        best = None
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b, out=c)
            e1.record()
            e1.synchronize()
            t = e0.elapsed_time(e1) / 1e3
            best = t if best is None else min(best, t)
        del a, b, c
        torch.cuda.empty_cache()
        return 2.0 * n ** 3 / best / 1e12
    except RuntimeError:
        return None


def roofline_alu(flop_per_launch, bytes_per_launch, launch_ms, ops_per_launch, kernel, local, clocks, traffic=None,
                 dgemm=None):
    """FP64-pipe roofline of one kernel: achieved flop/s of its algorithmic work against the device's nominal FP64
    rate; the FP64 lanes it issues per clock and SM (at the median SM clock sampled during the timed region); the
    achieved HBM rate of its algorithmic bytes against the measured copy rate."""
    sms, mhz, peak = fp64_peak(local)
    achieved = flop_per_launch / (launch_ms / 1e3)
    mhz_run = (clocks or {}).get("sm_mhz") or mhz
    hbm = measured_peaks().get("hbm_gbs")
    gbs = bytes_per_launch / (launch_ms / 1e3) / 1e9
    out = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
           "frac": achieved / peak, "traffic": traffic,
           "traffic_unit": "bytes per launch (DRAM read + write, ncu)",
           "algorithmic_bytes_per_launch": bytes_per_launch, "kernel": kernel, "launch_ms": launch_ms,
           "peak_source": f"nominal: {sms} SMs x {FP64_FMA_LANES_PER_SM} FP64 FMA lanes/clk x 2 flop x {mhz:.0f} MHz",
           "fp64_lanes_per_clk_sm": ops_per_launch / (launch_ms / 1e3) / sms / (mhz_run * 1e6),
           "fp64_lanes_clock_mhz": mhz_run,
           "hbm_gbs": gbs, "hbm_frac_of_measured": (gbs / hbm) if hbm else None}
    if dgemm:
        out["dgemm_fp64_tflops"] = dgemm
        out["frac_of_dgemm"] = achieved / 1e12 / dgemm
    return out


def _free():
    import gc
    import torch
    gc.collect()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


# --------------------------------------------------------------------------------------------- forward runs
def measure_forward(spec, T, args, local, warmup, steps, world=1, e2e=False, flush_l2=True, workload="",
                    launch_shape=None, dgemm=None):
    """Time `steps` whole runs (reset, T fused steps, statistics) after `warmup` runs, CUDA events on the launching
    stream, clocks sampled meanwhile; optionally the same end to end through the public API with host buffers."""
    import torch
    import torch.distributed as dist
    from paper_1702_00496_gb300 import Solver, autotune, at_set_launch

    ntot = 1
    for x in spec["n"]:
        ntot *= x
    stream = torch.cuda.current_stream()
    solver = Solver(spec, log_steps=0, device=f"cuda:{local}", stream=stream)
    if launch_shape:
        launch = tuple(launch_shape)
        at_set_launch(solver.h, *launch)
        solver.reset()
    else:
        launch = autotune.tune_forward(solver, spec, use_cache=not args.retune)
    from paper_1702_00496_gb300 import at_set_fusion
    kblock = at_set_fusion(solver.h, args.block_steps)  # 1D Euler: K-step blocks where the shape admits them
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float64, device=f"cuda:{local}") if flush_l2 else None
    kern_ev = []
    burgers = bool(spec.get("burgers", 0))
    # Burgers' equation has no analytic solution: its run reports the statistics of U^T - U^0 (the RMS change)
    u_ic = solver.field().clone() if burgers else None

    def stats():
        return solver.error_stats_ref(u_ic, 1) if burgers else solver.error_stats()

    def one_step(record=False):
        if flush is not None:
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

    for _ in range(warmup):
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
    for _ in range(steps):
        last = one_step(record=True)
    t_end.record(stream)
    barrier()
    clocks = sampler.stop()
    ms = t_start.elapsed_time(t_end) / steps
    kern_ms = sum(a.elapsed_time(b) for a, b in kern_ev) / (steps * T)
    ms = max_over_ranks(ms, world, f"cuda:{local}")
    out = {"value": aggregate_rate(ntot * T, world, ms / 1e3), "ms_per_step": ms, "launch": launch,
           "clocks": clocks, "last": last, "ntot": ntot, "T": T, "block_steps": kblock}

    if e2e:
        # end to end through the public API: pinned host field in, final field and statistics out
        solver.reset()
        torch.cuda.synchronize()
        u0_host = torch.empty(ntot, dtype=torch.float64, pin_memory=True)
        u0_host.copy_(solver.field().reshape(-1))
        out_host = torch.empty(ntot, dtype=torch.float64, pin_memory=True)
        u0_dev = torch.empty(ntot, dtype=torch.float64, device=f"cuda:{local}")
        e2e_steps = max(1, min(steps, 3))

        def e2e_step():
            if flush is not None:
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
        out["e2e"] = {"value": aggregate_rate(ntot * T, world, e2e_s), "unit": "updates/s",
                      "h2d_bytes_per_step": 8 * ntot, "d2h_bytes_per_step": 8 * ntot + 8 * 9}

    # the step kernel's first template arguments: dimension, h, and 0 forward Euler / 1 Adams-Bashforth / 2 AB2 in
    # its steady form (1D, linear)
    ab = 0 if time_levels(spec) == 1 else (2 if time_levels(spec) == 2 and spec["dim"] == 1 and not spec.get("burgers")
                                           else 1)
    kname = f"forward_group_kernel<{spec['dim']},{spec['order'] // 2},{ab}>"
    ops = fp64_ops_per_update(spec)
    bytes_update = bytes_per_update(spec)
    traffic = MEASURED_TRAFFIC.get((workload, kname))
    if kblock > 1:
        # blocks of K steps: 2 h K + 1 FP64 operations per point and block away from PE boundaries; U^n is read and
        # U^{n+K} written once per block
        traffic = MEASURED_TRAFFIC.get((workload, f"blocks of {kblock}"))
        kname = (f"forward_block_kernel<{spec['order'] // 2},{kblock}> + forward_zones_kernel<{spec['order'] // 2},"
                 f"{kblock}> (blocks of {kblock} steps)")
        ops = (spec["order"] * kblock + 1) / kblock
        bytes_update = 16 / kblock
    out["roofline"] = roofline_alu(flops_per_update(spec) * ntot, bytes_update * ntot, kern_ms,
                                   ops * ntot, kname, local, clocks, traffic, dgemm)
    if kblock > 1:
        out["roofline"]["traffic_note"] = "DRAM read + write per step (a block launch and a zone launch per K steps, ncu)"
    out["roofline"]["fp64_ops_per_update_executed"] = ops
    if kblock > 1:
        out["roofline"]["note"] = ("achieved counts the single step's algorithmic flop per update (1 multiply and "
                                   "2 h FMAs); blocks of K steps execute 2 h K + 1 FP64 operations per point and "
                                   "block away from PE boundaries (fp64_ops_per_update_executed), so the FP64 "
                                   "lanes per clock use that count")
    if workload in TRAFFIC_NOTES:
        out["roofline"]["traffic_note"] = TRAFFIC_NOTES[workload]
    out["gpu_launches"] = steps * launches_per_run(spec, T, kblock)
    solver.close()
    del flush
    return out


def forward_record(name, spec, T, args, local, warmup, steps, cpu_steps, note="", dgemm=None):
    """A per-workload record of the default line: device throughput, roofline, clocks, CPU-oracle sample."""
    r = measure_forward(spec, T, args, local, warmup, steps, flush_l2=False, workload=name, dgemm=dgemm)
    cpu = cpu_forward_baseline(spec, cpu_steps) if cpu_steps > 0 else None
    ntot = r["ntot"]
    rec = {"metric": METRIC, "value": r["value"], "unit": "updates/s", "ms_per_step": r["ms_per_step"],
           "steps": steps, "warmup": warmup,
           "config": {"workload": name, "points": ntot, "pes": spec["pe"], "order": spec["order"], "L": spec["L"],
                      "time_steps_per_step": T, "block_steps": r["block_steps"],
                      "launch": {"threads": r["launch"][0], "blocks_per_sm": r["launch"][1]},
                      "l2": ("inputs larger than L2 (ring of " + f"{8 * ntot * (spec['L'] + spec['order'] // 2 + 1) / 2**30:.1f} GiB)"
                             if 8 * ntot > 256 * 2**20 else "on-chip: the whole ring fits in L2")},
           "roofline": r["roofline"], "clocks": r["clocks"], "cpu_baseline": cpu,
           "final_rms_error": r["last"]["rms"], "gpu_launches": r["gpu_launches"]}
    if note:
        rec["note"] = note
    return rec


# --------------------------------------------------------------------------------------------- ensemble
def measure_ensemble(args, local, specs, steps_list, T, groups_in, twins, warmup, steps, one_at_a_time, world=1,
                     rank=0):
    """One persistent graph launch over all members per bench step; optionally the same members one problem at
    a time through the single-problem path (reset, T graph-captured steps, statistics, in sequence)."""
    import torch
    import torch.distributed as dist
    from paper_1702_00496_gb300 import Ensemble, Solver

    updates = sum(s["n"][0] * st for s, st in zip(specs, steps_list))
    stream = torch.cuda.current_stream()
    threads, ctas = args.threads, args.ctas_per_sm
    if threads == 0:
        from paper_1702_00496_gb300 import autotune
        threads, ctas = autotune.tune_ensemble(specs, steps_list, device=f"cuda:{local}", use_cache=not args.retune)
    ens = Ensemble(specs, steps_list, threads=threads, ctas_per_sm=ctas, device=f"cuda:{local}", stream=stream,
                   groups=groups_in, twins=twins)
    for _ in range(warmup):
        ens.run()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        ens.run()
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / steps
    per, groups = ens.stats()
    ms = max_over_ranks(ms, world, f"cuda:{local}")
    ens.close()
    del ens
    _free()
    one = None
    one_clocks = None
    if one_at_a_time and T is not None:
        solvers = [Solver(s, device=f"cuda:{local}", stream=stream) for s in specs]
        for sv in solvers:  # builds each solver's captured step graph outside the timed region
            sv.step(50)
            sv.reset()
        torch.cuda.synchronize()
        sampler = ClockSampler(local)
        sampler.start()
        t0 = time.perf_counter()
        for sv in solvers:
            sv.reset()
            sv.step(T)
            sv.error_stats()
        torch.cuda.synchronize()
        one = (time.perf_counter() - t0) * 1e3
        one_clocks = sampler.stop()
        for sv in solvers:
            sv.close()
        del solvers
        _free()
    flop = 9 * updates  # order 4, forward Euler: 1 multiply + 4 FMAs per update
    rec = {"metric": METRIC + " -- batched ensemble", "value": world * updates / (ms / 1e3), "unit": "updates/s",
           "ms_per_step": ms, "steps": steps, "warmup": warmup,
           "config": {"workload": args.workload if args.workload in SWEEPS else "ensemble", "members": len(specs),
                      "time_steps": T if T is not None else [min(steps_list), max(steps_list)],
                      "total_points": sum(s["n"][0] for s in specs), "point_updates": updates,
                      "launch": {"threads": threads, "ctas_per_sm": ctas},
                      "l2": "not flushed: the rings of the members running at once (152, up to 3.5 MiB each) "
                            "exceed the L2, so every step streams them from HBM"},
           "one_at_a_time_ms": one, "speedup_vs_one_at_a_time": (one / ms) if one else None,
           "one_at_a_time_clocks": one_clocks, "groups": groups, "clocks": clocks, "gpu_launches": steps * 4}
    if T is not None:
        rec["roofline"] = roofline_alu(flop, 16 * updates, ms, 5 * updates, "ensemble_kernel (whole graph launch)",
                                       local, clocks, ENSEMBLE_DRAM_BYTES_PER_UPDATE * updates)
        rec["roofline"]["traffic_note"] = ("DRAM read + write per update from one ncu capture of a 100-step launch of "
                                           "the same members, scaled to this launch's updates")
    return rec


def persistent_single(spec, T, local, warmup, steps) -> dict:
    """One small problem as a single member of the persistent engine (initial condition, all T steps in one CTA,
    statistics; one graph launch per run), timed with CUDA events like the other records."""
    import torch
    from paper_1702_00496_gb300 import Ensemble
    stream = torch.cuda.current_stream()
    ens = Ensemble([spec], [T], threads=128, ctas_per_sm=1, device=f"cuda:{local}", stream=stream)
    for _ in range(warmup):
        ens.run()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        ens.run()
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / steps
    per, _ = ens.stats()
    ens.close()
    return {"value": spec["n"][0] * T / (ms / 1e3), "unit": "updates/s", "ms_per_step": ms, "steps": steps,
            "warmup": warmup, "threads": 128, "final_rms_error": per[0]["rms"], "clocks": clocks}


def ensemble_cpu_baseline(specs, T, members: int = 16, steps: int = 200) -> dict:
    """The oracle on the first `members` realizations for `steps` steps each (all cores, OpenMP over points)."""
    cores = os.cpu_count() or 1
    upd, t = 0, 0.0
    for s in specs[:members]:
        v = cpu_sample(s, steps, cores)
        upd += s["n"][0] * steps
        t += s["n"][0] * steps / v
    return {"value": upd / t, "unit": "updates/s", "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
            "sample": f"the first {members} of the {len(specs)} realizations, {steps} of their {T} steps each, one "
                      f"after another, OpenMP over points, initial conditions excluded"}


def run_ensemble(args, rank: int, world: int, local: int):
    """1024 1D realizations (N_r in 2^10..2^16, L_r in 2..4, 5000 steps) in one persistent graph launch, against
    the same realizations run one problem at a time through the single-problem path (graph-captured steps)."""
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
    rec = measure_ensemble(args, local, specs, steps, T, groups_in, twins, args.warmup, args.steps,
                           not args.skip_one_at_a_time, world, rank)
    if rank == 0:
        rec.update({"n_gpus": world, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                    "dtype": "f64", "data": "synthetic"})
        print(json.dumps(rec), flush=True)


# --------------------------------------------------------------------------------------------- adjoint
ADJ_FLOP_PER_CELL = 54  # 3D order 4, transposed step with the alpha term: 13 + 13 + 1 FMAs per cell
ADJ_DRAM_BYTES_PER_LAUNCH = 1.67e9 + 0.32e9  # ncu, one backward step with the alpha term at 256^3


def measure_adjoint(args, local, T, every, warmup, steps, rank=0, world=1, forward=True):
    """The gradient of 1/2 ||U^T - u_target||^2 (256^3, order 4) by the hand-written adjoint: forward run alone,
    checkpointed forward pass + backward sweep for dJ/du0 and dJ/dalpha, and the dJ/du0-only sweep."""
    import torch
    from paper_1702_00496_gb300 import Solver

    spec, _ = W.workload("adjoint_256")
    spec["seed"] = replica_seed(spec["seed"], rank)
    ntot = spec["n"][0] * spec["n"][1] * spec["n"][2]
    stream = torch.cuda.current_stream()
    s = Solver(spec, device=f"cuda:{local}", stream=stream)
    target = torch.zeros(ntot, dtype=torch.float64, device=f"cuda:{local}")
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    fwd, adj, adj_u0, bwd = [], [], [], []
    sampler = ClockSampler(local)
    ga = None
    for it in range(warmup + steps):
        if it == warmup:
            torch.cuda.synchronize()
            sampler.start()
        if forward:
            s.reset()
            a, b = ev(), ev()
            a.record(stream)
            s.step(T)
            b.record(stream)
        s.reset()
        c, m, d = ev(), ev(), ev()
        c.record(stream)
        s.adjoint_forward(T, every)
        m.record(stream)
        lam = s.field().reshape(-1) - target
        g, ga = s.adjoint_backward(lam)
        d.record(stream)
        s.reset()
        e, f = ev(), ev()
        e.record(stream)
        s.adjoint_forward(T, every)
        g0, _ = s.adjoint_backward(s.field().reshape(-1) - target, want_alpha=False)
        f.record(stream)
        torch.cuda.synchronize()
        if it >= warmup:
            if forward:
                fwd.append(a.elapsed_time(b))
            adj.append(c.elapsed_time(d))
            bwd.append(m.elapsed_time(d))
            adj_u0.append(e.elapsed_time(f))
    clocks = sampler.stop()
    work_bytes = 8 * s.work.numel()
    s.close()
    del s, target, g, g0, lam
    _free()
    out = {"adjoint_ms": statistics.median(adj), "backward_ms": statistics.median(bwd),
           "adjoint_u0_only_ms": statistics.median(adj_u0), "workspace_bytes": work_bytes, "grad_alpha": ga,
           "clocks": clocks, "ntot": ntot}
    if forward:
        out["forward_ms"] = statistics.median(fwd)
    return out


def adjoint_cpu_baseline(n: int = 64, P: int = 2, steps: int = 20) -> dict:
    """The oracle's literal adjoint (full history kept, no checkpoints; one thread) on a small problem of the
    gradient workload's kind (order 4, L = 3): updates/s of the whole gradient (forward + backward) and the oracle's
    own gradient/forward time ratio (its forward run on one thread too)."""
    import numpy as np
    import oracle
    spec, _ = W.adjoint_spec(n, P, steps)
    cfg = oracle.Config(spec)
    target = np.zeros(cfg.shape)
    t0 = time.perf_counter()
    oracle.run(cfg, steps, want_log=False, threads=1)
    t_fwd = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.adjoint(cfg, steps, target)
    t_adj = time.perf_counter() - t0
    ntot = cfg.ntot
    return {"value": ntot * steps / t_adj, "unit": "updates/s", "cores": 1, "kind": "oracle",
            "cpu_model": cpu_model(), "oracle_adjoint_forward_ratio": t_adj / t_fwd,
            "sample": f"{n}^3 in {P}^3 PEs, order 4, L = 3, {steps} steps on one thread: the oracle's whole gradient "
                      f"(forward run with every level kept, then the literal transposed steps) against its forward "
                      f"run"}


def adjoint_record(args, local, T, warmup, steps) -> dict:
    """Config-5 record: the forward run, the gradient with sqrt(T) checkpoints and with every level resident."""
    import torch
    sq = measure_adjoint(args, local, T, 0, warmup, steps)
    f_ms = sq["forward_ms"]
    ntot = sq["ntot"]
    R = 6  # L + T levels of the order-4, L = 3 problem
    rec = {"metric": "adjoint/forward time ratio (FP64)", "value": sq["adjoint_ms"] / f_ms, "unit": "ratio",
           "higher_is_better": False, "steps": steps, "warmup": warmup,
           "config": {"workload": "adjoint_256", "points": ntot, "pes": [4, 4, 4], "order": 4, "L": 3,
                      "time_steps": T, "l2": "inputs larger than L2 (128 MiB per level, ring of 6 levels)"},
           "forward_ms": f_ms,
           "sqrt_t": {"checkpoint_every": math.ceil(math.sqrt(T)), "workspace_bytes": sq["workspace_bytes"],
                      "adjoint_ms": sq["adjoint_ms"], "adjoint_forward_ratio": sq["adjoint_ms"] / f_ms,
                      "backward_ms": sq["backward_ms"], "backward_forward_ratio": sq["backward_ms"] / f_ms,
                      "u0_only_ms": sq["adjoint_u0_only_ms"],
                      "u0_only_forward_ratio": sq["adjoint_u0_only_ms"] / f_ms, "clocks": sq["clocks"]},
           "grad_alpha": sq["grad_alpha"],
           "fma_floor": {"alpha_resident": (13 + 27) / 13, "alpha_sqrt_t": (13 + 13 + 27) / 13,
                         "u0_only": (13 + 13) / 13,
                         "note": "FP64 FMAs per cell: forward step 13, transposed step 13 (27 with the alpha term "
                                 "<lambda, dt D2_AT U>), recompute of a checkpointed segment 13; the whole "
                                 "gradient in dJ/dalpha cannot cost less than these multiples of the forward run on "
                                 "the FP64 pipe, so <= 3x for dJ/dalpha is below what the pipe allows; dJ/du0 alone "
                                 "needs no forward level and no recompute"}}
    free = torch.cuda.mem_get_info(local)[0]
    need = 8 * ntot * (T + 3 * R + 8)  # every level, the adjoint ring, the solver's ring and small fields
    if free > need:
        rs = measure_adjoint(args, local, T, T, warmup, steps, forward=False)
        rec["resident"] = {"checkpoint_every": T, "workspace_bytes": rs["workspace_bytes"],
                           "adjoint_ms": rs["adjoint_ms"], "adjoint_forward_ratio": rs["adjoint_ms"] / f_ms,
                           "backward_ms": rs["backward_ms"], "backward_forward_ratio": rs["backward_ms"] / f_ms,
                           "u0_only_ms": rs["adjoint_u0_only_ms"],
                           "u0_only_forward_ratio": rs["adjoint_u0_only_ms"] / f_ms, "clocks": rs["clocks"]}
        rec["roofline"] = roofline_alu(ADJ_FLOP_PER_CELL * ntot, 8 * 8 * ntot, rs["backward_ms"] / T, 27 * ntot,
                                       "adjoint_step_kernel (transposed step with the alpha term, every level "
                                       "resident)", local, rs["clocks"], ADJ_DRAM_BYTES_PER_LAUNCH)
        rec["roofline"]["traffic_note"] = ("DRAM read + write of one backward step at 256^3 from one ncu capture "
                                           "(1.67 GB read, 0.32 GB written)")
    else:
        rec["resident"] = {"skipped": f"needs {need / 1e9:.0f} GB free, {free / 1e9:.0f} GB free"}
        rec["roofline"] = None
    rec["cpu_baseline"] = adjoint_cpu_baseline()
    return rec


def run_adjoint(args, rank: int, world: int, local: int):
    """Gradient of 1/2 ||U^T - u_target||^2 (256^3, order 4, 2000 steps) by the hand-written adjoint with
    sqrt(T) checkpointing (or every level resident), against the forward run alone."""
    spec, T = W.workload("adjoint_256")
    if args.time_steps is not None:
        T = args.time_steps
    r = measure_adjoint(args, local, T, args.adjoint_every, args.warmup, args.steps, rank, world)
    ntot, f_ms, a_ms = r["ntot"], r["forward_ms"], r["adjoint_ms"]
    if rank == 0:
        line = {"metric": METRIC + " -- adjoint", "value": world * ntot * T / (a_ms / 1e3), "unit": "updates/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": a_ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": "adjoint_256", "points": ntot, "time_steps": T,
                           "checkpoint_every": args.adjoint_every or "sqrt(T)",
                           "levels_resident": args.adjoint_every >= T},
                "forward_ms": f_ms, "adjoint_ms": a_ms, "adjoint_forward_ratio": a_ms / f_ms,
                "backward_ms": r["backward_ms"], "backward_step_forward_step_ratio": r["backward_ms"] / f_ms,
                "adjoint_u0_only_ms": r["adjoint_u0_only_ms"],
                "adjoint_u0_only_forward_ratio": r["adjoint_u0_only_ms"] / f_ms,
                "workspace_bytes": r["workspace_bytes"],
                "note": "adjoint_ms = forward pass with checkpoints + backward sweep (restore, recompute, transposed "
                        "steps) for dJ/du0 and dJ/dalpha; backward_ms = the sweep alone, T backward steps against "
                        "forward_ms's T forward steps; the u0-only sweep needs no recompute; with every level "
                        "resident (--adjoint-every >= T) the forward pass keeps all levels and nothing is recomputed",
                "grad_alpha": r["grad_alpha"], "clocks": r["clocks"]}
        print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------------------------- default line
def config_records(args, local, dgemm) -> dict:
    """The other workloads, each measured on the device with its own warm-up (3 runs), timed runs, clocks,
    roofline and CPU-oracle sample.  Run at N = 1 only.  A record that fails carries its error instead."""
    recs = {}
    sub_w, sub_k = 3, max(1, min(args.steps, 3))

    def guarded(name, fn):
        try:
            recs[name] = fn()
        except Exception as e:  # one failed record must not lose the headline line
            recs[name] = {"error": f"{type(e).__name__}: {e}"}
        _free()

    def n256():
        # 1D N = 256 (2000 steps): the whole ring is on chip, so one launch per step is bound by launch latency;
        # the persistent engine runs the same problem (same delays, same field) inside one CTA without launches
        spec, T = W.workload("1d_n256")
        r = forward_record("1d_n256", spec, T, args, local, sub_w, sub_k, 0,
                           note="2 KB field: latency-bound, no HBM or FP64-pipe bound applies; value = one launch "
                                "per step (Solver), persistent = the whole run in one CTA of the ensemble engine")
        r["persistent"] = persistent_single(spec, T, local, sub_w, sub_k)
        r["cpu_baseline"] = {"value": cpu_sample(spec, T, 1), "unit": "updates/s", "cores": 1, "kind": "oracle",
                             "cpu_model": cpu_model(), "sample": f"the whole {T}-step run on one thread"}
        return r

    def three_d(name):
        spec, T = W.workload(name)
        return forward_record(name, spec, T, args, local, sub_w, sub_k, 2, dgemm=dgemm)

    def ensemble():
        # batched ensemble (1024 realizations x 5000 steps) against one problem at a time
        specs, T = W.ensemble_members()
        r = measure_ensemble(args, local, specs, [T] * len(specs), T, None, None, sub_w, sub_k, True)
        r.pop("groups", None)
        r["cpu_baseline"] = ensemble_cpu_baseline(specs, T)
        return r

    def adjoint():
        # gradient workload: adjoint/forward time ratio with sqrt(T) checkpoints and with every level resident
        _, T = W.workload("adjoint_256")
        return adjoint_record(args, local, T, sub_w, max(1, min(args.steps, 2)))

    guarded("1d_n256", n256)
    for name in ("3d_512_o2", "3d_512_o4"):  # 3D 512^3, orders 2 and 4 (500 steps)
        guarded(name, lambda: three_d(name))
    guarded("ensemble", ensemble)
    guarded("adjoint_256", adjoint)
    return recs


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="1d_n16m")
    ap.add_argument("--ref-sample-steps", type=int, default=10)
    ap.add_argument("--cpu-sample-steps", type=int, default=20)
    ap.add_argument("--cpu-single-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-configs", action="store_true", help="headline workload only (no per-workload records)")
    ap.add_argument("--time-steps", type=int, default=None, help="override the steps per run (profiling only)")
    ap.add_argument("--threads", type=int, default=0, help="ensemble: threads per CTA (0: library default)")
    ap.add_argument("--ctas-per-sm", type=int, default=0, help="ensemble: CTAs per SM (0: occupancy limit)")
    ap.add_argument("--skip-one-at-a-time", action="store_true")
    ap.add_argument("--retune", action="store_true", help="ignore the autotuner cache")
    ap.add_argument("--launch", default="", help="forward step: fixed launch shape THREADS,BLOCKS_PER_SM (no tuning)")
    ap.add_argument("--block-steps", type=int, default=4,
                    help="1D forward Euler: steps per block of at_step (at_set_fusion; 1 = single steps)")
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

    spec, T = W.workload(args.workload)
    if args.time_steps is not None:
        T = args.time_steps
    spec["seed"] = replica_seed(spec["seed"], rank)  # independent replica per rank
    headline_default = args.workload == "1d_n16m" and args.time_steps is None
    dgemm = measure_dgemm(local) if (rank == 0 and world == 1 and headline_default and not args.no_configs) else None
    launch_shape = tuple(int(v) for v in args.launch.split(",")) if args.launch else None
    r = measure_forward(spec, T, args, local, args.warmup, args.steps, world, e2e=True, workload=args.workload,
                        launch_shape=launch_shape, dgemm=dgemm)
    ntot, launch, burgers = r["ntot"], r["launch"], bool(spec.get("burgers", 0))

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_forward_baseline(spec, args.cpu_sample_steps, args.cpu_single_steps)
    configs = None
    if rank == 0 and world == 1 and headline_default and not args.no_configs:
        _free()
        configs = config_records(args, local, dgemm)

    if rank == 0:
        line = {"metric": METRIC, "value": r["value"], "unit": "updates/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": args.workload, "points": ntot, "pes": spec["pe"], "order": spec["order"],
                           "L": spec["L"], "time_levels": time_levels(spec), "time_steps_per_step": T,
                           "block_steps": r["block_steps"],
                           "l2": "flushed (512 MiB write) each step",
                           "replicas": world, "launch": {"threads": launch[0], "blocks_per_sm": launch[1]}},
                "e2e": r["e2e"], "roofline": r["roofline"], "cpu_baseline": cpu, "clocks": r["clocks"],
                "gpu_launches": r["gpu_launches"],
                ("final_rms_change" if burgers else "final_rms_error"): r["last"]["rms"]}
        if configs is not None:
            line["configs"] = configs
            line["configs_note"] = ("per-workload records, N = 1 only; each has its own warm-up, timed runs, clocks, "
                                    "roofline and CPU-oracle sample; gpu_launches counts the headline runs only")
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
