"""Launch-shape autotuner.

Two searches, each timed with CUDA events on the problem itself and cached per device in a JSON file:
  - per-step forward kernel: threads per block x cap of blocks per SM (the tile of its grid-stride loop),
    timed over a sample of steps;
  - persistent ensemble: threads per CTA x CTAs per SM, timed on a temporal sample of the run (the same
    members for fewer steps; every member has the same step count, so the load balance is preserved).
"""
from __future__ import annotations

import json
import os

import torch

from . import binding as B

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "autotune.json")
FORWARD_CANDIDATES = [(t, b) for t in (128, 256, 512) for b in (4, 8, 16, 32)]
ENSEMBLE_CANDIDATES = [(1024, 1), (512, 2), (512, 1), (256, 4), (256, 2)]


def _load_cache() -> dict:
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(key: str, value) -> None:
    cache = _load_cache()
    cache[key] = value
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def _device_key() -> str:
    return torch.cuda.get_device_name().replace(" ", "_")


def forward_signature(spec: dict) -> str:
    return (f"{_device_key()}|fwd|dim{spec['dim']}|n{'x'.join(map(str, spec['n']))}|pe{'x'.join(map(str, spec['pe']))}"
            f"|o{spec['order']}|L{spec['L']}|s{spec['scheme']}|t{max(1, int(spec.get('tsteps', 1)))}")


def tune_forward(solver, spec: dict, sample_steps: int = 50, use_cache: bool = True):
    """Pick (threads, blocks_per_sm) for a Solver; leaves the solver at step 0 with the best shape set."""
    key = forward_signature(spec)
    if use_cache and key in _load_cache():
        t, b = _load_cache()[key]["best"]
        B.at_set_launch(solver.h, t, b)
        solver.reset()
        return t, b
    stream = torch.cuda.current_stream()
    times = {}
    for t, b in FORWARD_CANDIDATES:
        B.at_set_launch(solver.h, t, b)
        solver.reset()
        solver.step(sample_steps)  # builds the captured graph for this shape
        solver.reset()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        solver.step(sample_steps)
        e1.record(stream)
        e1.synchronize()
        times[f"{t}x{b}"] = e0.elapsed_time(e1) / sample_steps
    best = min(times, key=times.get)
    t, b = (int(v) for v in best.split("x"))
    B.at_set_launch(solver.h, t, b)
    solver.reset()
    _store(key, {"best": [t, b], "ms_per_step": times})
    return t, b


def ensemble_signature(specs, nsteps) -> str:
    steps = [int(nsteps)] * len(specs) if not hasattr(nsteps, "__len__") else [int(v) for v in nsteps]
    sizes = sorted(s["n"][0] for s in specs)
    work = sum(s["n"][0] * st for s, st in zip(specs, steps))
    return (f"{_device_key()}|ens|count{len(specs)}|n{sizes[0]}-{sizes[-1]}|sum{sum(sizes)}|steps{max(steps)}"
            f"|work{work}|o{max(s['order'] for s in specs)}|t{max(int(s.get('tsteps', 1)) for s in specs)}")


def tune_ensemble(specs, nsteps, sample_steps: int = 200, device="cuda", use_cache: bool = True):
    """Pick (threads, ctas_per_sm) for an ensemble by timing candidates on a temporal sample: every member runs
    the same fraction of its steps (at most sample_steps for the longest), so the load balance is preserved."""
    from .solver import Ensemble
    key = ensemble_signature(specs, nsteps)
    if use_cache and key in _load_cache():
        return tuple(_load_cache()[key]["best"])
    steps = [int(nsteps)] * len(specs) if not hasattr(nsteps, "__len__") else [int(v) for v in nsteps]
    frac = min(1.0, sample_steps / max(1, max(steps)))
    sample = [max(1, int(round(st * frac))) if st > 0 else 0 for st in steps]
    stream = torch.cuda.current_stream()
    times = {}
    for t, c in ENSEMBLE_CANDIDATES:
        ens = Ensemble(specs, sample, threads=t, ctas_per_sm=c, device=device, stream=stream)
        ens.run()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ens.run()
        e1.record(stream)
        e1.synchronize()
        times[f"{t}x{c}"] = e0.elapsed_time(e1)
        ens.close()
    best = min(times, key=times.get)
    t, c = (int(v) for v in best.split("x"))
    _store(key, {"best": [t, c], "ms_sample": times, "sample_steps": sample_steps})
    return t, c
