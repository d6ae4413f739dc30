"""GPU parity over a seeded random sweep of problem shapes, against the oracle.

Each case draws a dimension (1 or 3), points and PEs per axis (PE widths from the minimum 2h up, multiples of 4
and not, axes left unsplit, point counts that are not a multiple of 4 so the per-point kernel runs), an order
(2, 4, 6), a scheme (synchronous, the standard scheme read at delayed levels, the time-expanded AT rows, the rows
expanded in space), a delay range L from 1 to 8 with uniform or binned delays (Sec. 5.1), an integrator (forward
Euler or Adams-Bashforth with two or three levels, Sec. 4.1) and, in 1D, the viscous Burgers' equation.  Bars as
in the other parity tests: the delay log bit-exact, the field within 1e-12 relative L2 and elementwise within
1e-12 of its max norm after the whole run.
"""
import os

import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

THREADS = os.cpu_count() or 1
TOL = 1e-12
CASES = 48


def _axis(rng, order, ragged):
    """(points, PEs) of one axis: PE width from 2h = order up, some widths not multiples of 4."""
    pe = int(rng.choice([1, 2, 3, 4, 5]))
    width = int(rng.choice([order, order + 1, 4, 6, 8, 12, 16]))
    width = max(width, order)
    if not ragged and width % 4:
        width += 4 - width % 4
    return pe * width, pe


def draw_case(i: int) -> tuple:
    rng = np.random.default_rng(np.random.SeedSequence([int(i), 0x5EED]))
    dim = 1 if rng.random() < 0.6 else 3
    order = int(rng.choice([2, 4, 6]))
    scheme = int(rng.choice([W.SYNC, W.ASYNC_STD, W.AT, W.AT, W.AT_SPACE2, W.AT_SPACE1]))
    if scheme >= W.AT_SPACE2:
        order = 2
    tsteps = 1 if scheme >= W.AT_SPACE2 else int(rng.choice([1, 1, 2, 3]))
    L = int(rng.integers(1, 9))
    burgers = dim == 1 and scheme <= W.AT and rng.random() < 0.25
    ragged = rng.random() < 0.3
    probs = None
    if L > 1 and rng.random() < 0.4:
        p = rng.random(L) + 0.05
        probs = list(p / p.sum())
    r_alpha = 0.004 if order == 6 or L > 4 or tsteps == 3 else 0.01
    alpha = 0.1
    if dim == 1:
        width = max(order, int(rng.choice([order, order + 1, 4, 6, 8, 12, 16, 32, 64])))
        if not ragged and width % 4:
            width += 4 - width % 4
        P = int(rng.choice([1, 2, 3, 5, 8, 16, 32]))
        n = P * width
        c = 0.0 if (scheme == W.AT_SPACE1 or burgers) else float(rng.uniform(-1.0, 1.0))
        spec, _ = W.wl_1d(n, P, order, L, 0, 7000 + i, range(1, 4), scheme=scheme, c=c, alpha=alpha,
                          r_alpha=r_alpha, probs=probs, tsteps=tsteps)
        if burgers:
            spec["burgers"] = 1
    else:
        axes = [_axis(rng, order, ragged and a == 0) for a in range(3)]
        n = [v[0] for v in axes]
        P = [v[1] for v in axes]
        c = (0.0, 0.0, 0.0) if scheme == W.AT_SPACE1 else tuple(float(v) for v in rng.uniform(-0.4, 0.4, 3))
        dt = r_alpha * W.dx_of(max(n)) ** 2 / alpha
        spec, _ = W.wl_3d(n, P, order, L, 0, 7000 + i, scheme=scheme, c=c, alpha=alpha, dt=dt, kappas=(1, 2),
                          tsteps=tsteps)
        if probs is not None:
            spec["thresholds"] = W.thresholds_from_probs(probs)
    nsteps = int(rng.integers(12, 41))
    return spec, nsteps


@pytest.mark.parametrize("i", range(CASES))
def test_random_shape_matches_oracle(i):
    from paper_1702_00496_gb300 import Solver
    spec, nsteps = draw_case(i)
    s = Solver(spec, log_steps=nsteps)
    s.step(nsteps)
    s.sync()
    u = s.field().cpu().numpy().copy()
    d = s.delays().cpu().numpy().copy()
    s.close()
    ref, dref, _ = oracle.run(oracle.Config(spec), nsteps, threads=THREADS)
    assert np.array_equal(d, dref), "delay logs differ"
    assert np.isfinite(ref).all()
    rel = np.linalg.norm(u - ref) / np.linalg.norm(ref)
    assert rel <= TOL, rel
    assert np.abs(u - ref).max() <= TOL * np.abs(ref).max()
