"""Seeded synthetic inputs for the asynchrony-tolerant finite-difference workloads.

This module holds no arithmetic of the method: it only draws the random initial-condition
parameters (amplitudes A ~ U(0.5, 1), phases phi ~ U(0, 2 pi), Sec. 5.1 Eq. "IC"), encodes a delay
probability vector {p_0..p_{L-1}} (Sec. 5.1) as integer bin thresholds, and names the workloads.
Both the CUDA path and the oracle receive these values as inputs.

Workloads (the paper's experiments use synthetic multi-sine fields only, so these are the inputs
themselves, not stand-ins for a dataset):
  1d_n256      1D, N=256,  8 PEs,    CD2 + (1,2,2)b/(2,2,2)b, L=3, 2000 steps
  1d_n16m      1D, N=2^24, 4096 PEs, CD4 + (1,4,2)/(2,4,2),   L=4, 1000 steps
  3d_512_o2/4  3D, 512^3, 8x8x8 PEs,  order 2 or 4, L=3, dt = dx^2, 500 steps
  3d_256_o2/4  the same PE shape (64^3) at 256^3 in 4x4x4 PEs (profiling captures that fit a few GB)
  ensemble     1024 1D realizations, N_r in {2^10..2^16}, P_r=N_r/64, L_r in {2,3,4}, 5000 steps
  adjoint_256  3D 256^3, 4x4x4 PEs, order 4, L=3, 2000 steps
  1d_n16m_case2  the paper's Case 2 scaled to N=2^24, 4096 PEs: CD2 + (2,1,2), Euler, diffusion, L=3, 1000 steps
  1d_n16m_case3  the paper's Case 3 scaled to N=2^24, 4096 PEs: CD2 + (1,2,2)a/(2,2,2)a, Euler, L=3, 1000 steps
  1d_n16m_case4  the paper's Case 4 scaled to N=2^24, 4096 PEs: CD4 + (1,4,2)/(2,4,2), AB2, L=3, 1000 steps
  1d_n16m_case5  the paper's Case 5 scaled to N=2^24, 4096 PEs: CD6 + (2,6,2), AB3, L=3, 1000 steps
  1d_n16m_case6  the paper's Case 6 (viscous Burgers) at N=2^24, 4096 PEs: CD4 + (1,4,2)/(2,4,2), AB2, L=3
"""
from __future__ import annotations

import math
import numpy as np

SYNC, ASYNC_STD, AT, AT_SPACE2, AT_SPACE1 = 0, 1, 2, 3, 4
TWO_PI = 2.0 * math.pi


def ic_params(seed: int, dim: int, kappas) -> dict:
    """Amplitudes and phases for Eq. "IC" on every axis (same wavenumbers per axis)."""
    rng = np.random.default_rng(np.random.SeedSequence([int(seed), 0x1C]))
    kap = np.asarray(list(kappas), dtype=np.int32)
    m = kap.size
    amp = rng.uniform(0.5, 1.0, size=(dim, m))
    phase = rng.uniform(0.0, TWO_PI, size=(dim, m))
    return {"nmodes": int(m), "amp": amp, "phase": phase, "kappa": np.tile(kap, (dim, 1))}


def thresholds_from_probs(p) -> np.ndarray:
    """Cumulative bin edges of {p_0..p_{L-1}} on the 32-bit uniform word: t_m = round(2^32 sum_{i<=m} p_i),
    m = 0..L-2 (the last edge is 2^32 and is implicit)."""
    p = np.asarray(p, dtype=np.float64)
    if p.ndim != 1 or p.size < 1 or np.any(p < 0) or abs(p.sum() - 1.0) > 1e-12:
        raise ValueError("probabilities must be non-negative and sum to 1")
    cum = np.cumsum(p)[:-1]
    return np.array([min(int(round(v * 2.0 ** 32)), 2 ** 32) for v in cum], dtype=np.uint64)


def make(dim, n, pe, order, L, scheme, c, alpha, dt, seed, kappas, probs=None, ic_seed=None, tsteps=1) -> dict:
    spec = {"dim": dim, "n": list(n), "pe": list(pe), "order": order, "L": L, "scheme": scheme,
            "c": list(c), "alpha": float(alpha), "dt": float(dt), "seed": int(seed), "tsteps": int(tsteps),
            "thresholds": None if probs is None else thresholds_from_probs(probs)}
    spec.update(ic_params(seed if ic_seed is None else ic_seed, dim, kappas))
    return spec


def dx_of(n: int) -> float:
    return TWO_PI / n


def wl_1d(n, P, order, L, steps, seed, kappas, scheme=AT, c=1.0, alpha=0.1, r_alpha=0.1, probs=None, tsteps=1):
    dt = r_alpha * dx_of(n) ** 2 / alpha
    return make(1, [n], [P], order, L, scheme, [c], alpha, dt, seed, kappas, probs, tsteps=tsteps), steps


def wl_3d(n, P, order, L, steps, seed, scheme=AT, c=(1.0, 1.0, 1.0), alpha=0.05, dt=None, kappas=(1, 2, 3),
          tsteps=1):
    nn = list(n) if hasattr(n, "__len__") else [n, n, n]
    pp = list(P) if hasattr(P, "__len__") else [P, P, P]
    if dt is None:
        # dt = dx^2 as in the 1D workloads: r_alpha = alpha dt / dx^2 = 0.05 per axis at alpha = 0.05.  With
        # forward Euler the order-4 AT stencils in 3D need r_alpha <= 1/16 per axis: their halo extrapolates
        # old levels, which amplifies the modes whose per-step factor 1 - 3 r_alpha 64/12 turns negative.
        dt = dx_of(max(nn)) ** 2
    return make(3, nn, pp, order, L, scheme, list(c), alpha, dt, seed, kappas, tsteps=tsteps), steps


def workload(name: str, scheme: int = AT):
    """(spec, nsteps) of a named workload."""
    if name == "1d_n256":
        return wl_1d(256, 8, 2, 3, 2000, 1, range(1, 5), scheme)
    if name == "1d_n16m":
        return wl_1d(1 << 24, 4096, 4, 4, 1000, 2, range(1, 11), scheme)
    if name == "3d_512_o2":
        return wl_3d(512, 8, 2, 3, 500, 3, scheme)
    if name == "3d_512_o4":
        return wl_3d(512, 8, 4, 3, 500, 3, scheme)
    if name == "3d_256_o2":
        return wl_3d(256, 4, 2, 3, 500, 3, scheme)
    if name == "3d_256_o4":
        return wl_3d(256, 4, 4, 3, 500, 3, scheme)
    if name == "adjoint_256":
        return adjoint_spec(256, 4, 2000)
    if name in ("1d_n16m_case2", "1d_n16m_case3", "1d_n16m_case4", "1d_n16m_case5", "1d_n16m_case6"):
        spec = paper_case(int(name[-1]), 1 << 24, 2, (1 / 3, 1 / 3, 1 / 3), P=4096)
        if scheme != AT:
            spec["scheme"] = scheme
        return spec, 1000
    raise KeyError(name)


def paper_case(case: int, n: int, seed: int, p0_probs=(1.0, 0.0, 0.0), P: int = 16):
    """Cases 1 to 5 of the paper's case table: kappa = {3,4,5}, A = {2, 0.5, 1.5} (as in Fig. "at-prob-all"),
    L = len(p0_probs), alpha = 0.1, phases random per seed.  Case 1: advection-diffusion, forward Euler, CD2 with
    (1,2,2)b/(2,2,2)b, r_alpha = 0.1 (Fig. "at-ord2-procs").  Case 2: diffusion, forward Euler, CD2 with (2,1,2);
    Case 3: advection-diffusion, forward Euler, CD2 with (1,2,2)a/(2,2,2)a; both at r_alpha = 0.1 (not given for
    Fig. "at-prob-all"; Case 1's value).  Case 6: the viscous Burgers' equation u_t + u u_x = alpha u_xx, AB2, CD4
    with (1,4,2)/(2,4,2), r_alpha = 0.05 (Case 4's), the same initial condition.  Case 4: advection-diffusion, AB2,
    CD4 with
    (1,4,2)/(2,4,2); Case 5: diffusion, AB3, CD6 with (2,6,2).  The paper does not give c or r_alpha for Cases 4
    and 5: c = 1 (Case 4) or 0 (Case 5), r_alpha = 0.05 (Case 4) or 0.01 (Case 5): with the time-extrapolated
    halos, AB2 and AB3 stay stable at every delay mix only at these smaller steps (the oracle diverges at
    r_alpha = 0.1 / 0.02 when p_0 <= 0.3)."""
    order, tsteps, c, r, scheme = {1: (2, 1, 1.0, 0.1, AT), 2: (2, 1, 0.0, 0.1, AT_SPACE1),
                                   3: (2, 1, 1.0, 0.1, AT_SPACE2), 4: (4, 2, 1.0, 0.05, AT),
                                   5: (6, 3, 0.0, 0.01, AT), 6: (4, 2, 0.0, 0.05, AT)}[case]
    probs = list(p0_probs)
    spec, _ = wl_1d(n, P, order, len(probs), 0, seed, (3, 4, 5), scheme=scheme, c=c, alpha=0.1, r_alpha=r,
                    probs=probs if len(probs) > 1 else None, tsteps=tsteps)
    spec["amp"] = np.array([[2.0, 0.5, 1.5]])
    if case == 6:
        spec["burgers"] = 1  # Case 6: the viscous Burgers' equation, AB2, CD4 with (1,4,2)/(2,4,2)
    return spec


def steps_to(spec, t_final: float) -> int:
    return int(round(t_final / spec["dt"]))


def _with_sync_twins(specs, steps, groups, sync_group):
    """Append a synchronous twin after each member: the same scheme, initial condition and steps with every delay
    0 (L = 1; for the time-expanded rows this is the central scheme, the stencils expanded in space keep their
    edge form at k = 0).  Returns the lists with the twin index of every member (-1 for the twins themselves)."""
    k = len(specs)
    twins = [k + i for i in range(k)] + [-1] * k
    sync = []
    for sp in specs:
        t = dict(sp)
        t["L"] = 1
        t["thresholds"] = None
        sync.append(t)
    return specs + sync, steps + steps, groups + [sync_group(g) for g in groups], twins


def moment_members(case: int, Ls, seeds, n: int = 512, P: int = 16, t_final: float = 0.1):
    """Members of the delay-moment sweep of Fig. "at-kmom" (N = 512, P = 16): for each L, uniform delays p_k = 1/L
    (Eq. "aveE_scaling_gen_L"), one member per seed, each with a synchronous twin.  Group of an asynchronous
    member: L; of its twin: 100 + L.  Returns (specs, steps, groups, twins)."""
    specs, steps, groups = [], [], []
    for L in Ls:
        for sd in seeds:
            sp = paper_case(case, n, sd, [1.0 / L] * L, P)
            specs.append(sp)
            steps.append(steps_to(sp, t_final))
            groups.append(L)
    return _with_sync_twins(specs, steps, groups, lambda g: 100 + g)


def scaling_members(case: int, grids, seeds, probs=(0.2, 0.5, 0.3), t_final: float = 0.1):
    """Members of the strong/weak scaling sweep of Fig. "at-ord2-procs": one member per (N, P) in `grids` and seed,
    with p_k = {0.2, 0.5, 0.3}, each with a synchronous twin.  Group of grid i: i; of the twins: 1000 + i.  Each
    member runs to t_final at its own dt (r_alpha fixed), so the step counts differ.  Returns (specs, steps,
    groups, twins)."""
    specs, steps, groups = [], [], []
    for i, (n, P) in enumerate(grids):
        for sd in seeds:
            sp = paper_case(case, n, sd, list(probs), P)
            specs.append(sp)
            steps.append(steps_to(sp, t_final))
            groups.append(i)
    return _with_sync_twins(specs, steps, groups, lambda g: 1000 + g)


def adjoint_spec(n=256, P=4, steps=2000, alpha=0.05, alpha_target=0.06, seed=5):
    """3D order-4 AT problem of the adjoint workload; dt is fixed by r_alpha = 0.05 at alpha_target (the 3D
    order-4 AT limit is 1/16 per axis), so both alpha values share one dt."""
    dt = 0.05 * dx_of(n) ** 2 / alpha_target
    spec, _ = wl_3d(n, P, 4, 3, steps, seed, AT, alpha=alpha, dt=dt)
    return spec, steps


def ensemble_members(count=1024, base_seed=1000, log2n=(10, 16), P_width=64, Ls=(2, 3, 4), order=4,
                     steps=5000, kappas=range(1, 5), draw_seed=4):
    """The realizations of the batched ensemble: N_r drawn from {2^lo..2^hi}, L_r from Ls,
    seed_r = base_seed + r, each with its own initial-condition phases."""
    rng = np.random.default_rng(np.random.SeedSequence([draw_seed, 0xE5]))
    lo, hi = log2n
    out = []
    for r in range(count):
        n = 1 << int(rng.integers(lo, hi + 1))
        L = int(rng.choice(np.asarray(Ls)))
        spec, _ = wl_1d(n, n // P_width, order, L, steps, base_seed + r, kappas)
        out.append(spec)
    return out, steps
