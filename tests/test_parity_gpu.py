"""GPU parity: the sm_103a forward path against the FP64 CPU oracle on the same seeded inputs.

Bars: delay logs bit-exact; fields within 1e-12 relative L2 (and elementwise within 1e-12 of the
field's max norm) after the full run; statistics within round-off of the oracle's on the same field.
"""
import os

import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

TOL = 1e-12
THREADS = os.cpu_count() or 1


def _gpu_run(spec, nsteps, log=True, single_steps=False):
    from paper_1702_00496_gb300 import Solver, at_set_fusion
    s = Solver(spec, log_steps=nsteps if log else 0)
    if single_steps:
        at_set_fusion(s.h, 1)
    s.step(nsteps)
    s.sync()
    u = s.field().cpu().numpy().copy()
    d = s.delays().cpu().numpy().copy() if log else None
    st = s.error_stats()
    s.close()
    return u, d, st


def _compare(spec, nsteps, stats=True):
    u, d, st = _gpu_run(spec, nsteps)
    cfg = oracle.Config(spec)
    ref, dref, _ = oracle.run(cfg, nsteps, threads=THREADS)
    assert np.array_equal(d, dref), "delay logs differ"
    rel = np.linalg.norm(u - ref) / np.linalg.norm(ref)
    assert rel <= TOL, rel
    assert np.abs(u - ref).max() <= TOL * np.abs(ref).max()
    if stats:
        # Both sides evaluate u_a with their own sin/exp (a few ulp of |u_a| apart), so E = U - u_a agrees to
        # ~1e-15 |u_a| absolutely; relative agreement of tiny errors is not expected.
        so = oracle.error_stats(cfg, u, nsteps)
        atol = 1e-13 * so["ua_rms"]
        for key in ("rms", "max_abs", "mean_abs", "mean", "rms_I", "rms_B"):
            assert abs(st[key] - so[key]) <= 1e-9 * abs(so[key]) + atol, key
        assert st["ua_rms"] == pytest.approx(so["ua_rms"], rel=1e-13)
        assert (st["n_I"], st["n_B"], st["step"]) == (so["n_I"], so["n_B"], nsteps)
    return u, ref


def test_1d_n256_order2_full_run():
    spec, steps = W.workload("1d_n256")
    _compare(spec, steps)


@pytest.mark.parametrize("scheme", [W.SYNC, W.ASYNC_STD, W.AT])
@pytest.mark.parametrize("order", [2, 4])
def test_1d_schemes_ragged_tiles(order, scheme):
    # 12000 points in 30 PEs of 400: several thread blocks and a ragged last block
    spec, _ = W.wl_1d(12000, 30, order, 4, 0, 77, range(1, 11), scheme=scheme)
    _compare(spec, 300)


def test_1d_binned_delays_fig_at_sol1():
    spec, _ = W.wl_1d(128, 4, 2, 3, 0, 9, (2, 3, 5), probs=[0.5, 0.3, 0.2])
    _compare(spec, 1500)


@pytest.mark.parametrize("order", [2, 4])
def test_1d_minimum_pe_width(order):
    spec, _ = W.wl_1d(64 * order, 64, order, 3, 0, 5, (1, 3))  # S = order = 2h
    _compare(spec, 200)


def test_single_delay_level_equals_synchronous_run():
    """L = 1: every delay is 0, so the AT scheme is the synchronous one, bit for bit in single steps, and to
    rounding in at_step's blocks wherever the shape admits them."""
    spec, _ = W.wl_1d(512, 8, 4, 1, 0, 6, (1, 2))
    u_at, d, _ = _gpu_run(spec, 100, single_steps=True)
    u_blk, _, _ = _gpu_run(spec, 100)
    assert not d.any()
    spec["scheme"] = W.SYNC
    u_sync, _, _ = _gpu_run(spec, 100)
    assert np.array_equal(u_at, u_sync)
    assert np.linalg.norm(u_blk - u_sync) / np.linalg.norm(u_sync) <= 1e-13


@pytest.mark.parametrize("modes", [range(1, 17), range(9, 25)], ids=["k_to_16", "k_9_to_24"])
def test_initial_condition_at_high_wavenumbers(modes):
    """The mode sums over k by the three-term recurrences (largest k at most 16) and by the rotation (above), against
    the oracle's libm sines: an error made at wavenumber j reaches k at most (k - j)-fold, under 16^2/2 ulp of the
    amplitude sum for the first, a few ulp per rotation for the second."""
    spec, _ = W.wl_1d(1000, 10, 4, 3, 0, 9, modes)
    u, _, _ = _gpu_run(spec, 0, log=False)
    ref = oracle.initial(oracle.Config(spec))
    bound = 128 * np.finfo(float).eps * np.abs(spec["amp"]).sum()
    assert np.abs(u - ref).max() <= bound


def test_zero_steps_is_the_initial_condition():
    spec, _ = W.wl_1d(1000, 10, 4, 3, 0, 8, range(1, 5))
    u, _, st = _gpu_run(spec, 0, log=False)
    ref = oracle.initial(oracle.Config(spec))
    assert np.abs(u - ref).max() <= 4e-15 * np.abs(ref).max()
    assert st["rms"] <= 1e-14 * st["ua_rms"] and st["step"] == 0


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("scheme", [W.SYNC, W.ASYNC_STD, W.AT])
def test_3d_small(order, scheme):
    # |c|^2 dt stays below 2 alpha, the forward-Euler limit of central advection
    spec, _ = W.wl_3d([24, 20, 16], [3, 2, 4], order, 3, 0, 31, scheme=scheme, c=(0.5, -0.35, 0.2))
    _compare(spec, 40)


def test_3d_unsplit_axis_and_binned_delays():
    spec, _ = W.wl_3d([16, 12, 20], [2, 1, 5], 4, 3, 0, 32, c=(0.3, 0.3, 0.3))
    spec["thresholds"] = W.thresholds_from_probs([0.2, 0.5, 0.3])
    _compare(spec, 30)


# ------------------------------------------------------------ full-size workloads
def _closed_form_sync_1d(spec, nsteps, idx):
    n = spec["n"][0]
    dx = 2 * np.pi / n
    x = idx * dx
    u = np.zeros(len(idx))
    for A, ph, kap in zip(spec["amp"][0], spec["phase"][0], spec["kappa"][0]):
        th = kap * dx
        s1 = (8 * np.sin(th) - np.sin(2 * th)) / (6 * dx)
        s2 = (-2 * np.cos(2 * th) + 32 * np.cos(th) - 30) / (12 * dx ** 2)
        G = 1 + spec["dt"] * (-spec["c"][0] * 1j * s1 + spec["alpha"] * s2)
        u += A * np.imag(G ** nsteps * np.exp(1j * (kap * x + ph)))
    return u


def test_full_size_1d_n16m_delays_and_field():
    """N = 2^24, 4096 PEs, order 4, L = 4: the whole 1000-step delay log bit-exact, the field after a
    100-step prefix against the oracle, and the 1000-step synchronous field against its closed form."""
    spec, steps = W.workload("1d_n16m")
    cfg = oracle.Config(spec)
    from paper_1702_00496_gb300 import Solver
    s = Solver(spec, log_steps=steps)
    s.step(100)
    s.sync()
    u100 = s.field().cpu().numpy().copy()
    s.step(steps - 100)
    s.sync()
    assert np.array_equal(s.delays().cpu().numpy(), oracle.delay_log(cfg, steps))
    s.close()
    ref, _, _ = oracle.run(cfg, 100, want_log=False, threads=THREADS)
    assert np.linalg.norm(u100 - ref) / np.linalg.norm(ref) <= TOL
    spec["scheme"] = W.SYNC
    u, _, _ = _gpu_run(spec, steps, log=False)
    idx = np.random.default_rng(0).choice(spec["n"][0], 4096, replace=False)
    want = _closed_form_sync_1d(spec, steps, idx)
    assert np.abs(u[idx] - want).max() <= TOL * np.abs(want).max()


def test_full_size_1d_n16m_sampled_after_the_whole_run():
    """N = 2^24, 4096 PEs, order 4, L = 4, all 1000 asynchronous steps in the launch shape bench.py picks: cells on
    PE edges and inside PEs against the oracle, which steps each sampled cell inside its domain of dependence
    only (the same values as a whole oracle run, bit for bit)."""
    from paper_1702_00496_gb300 import Solver, autotune
    spec, steps = W.workload("1d_n16m")
    s = Solver(spec)
    autotune.tune_forward(s, spec)
    s.reset()
    s.step(steps)
    s.sync()
    u = s.field().cpu().numpy().copy()
    s.close()
    S = spec["n"][0] // spec["pe"][0]
    rng = np.random.default_rng(1)
    pes = rng.choice(spec["pe"][0], 6, replace=False)
    pos = sorted({int(p * S + o) for p in pes for o in (0, 1, S // 2, S - 2, S - 1)})
    ref = oracle.run_samples(oracle.Config(spec), steps, pos)
    assert np.abs(u[pos] - ref).max() <= TOL * np.abs(u).max()


@pytest.mark.parametrize("order", [2, 4])
def test_full_size_3d_512_prefix(order):
    """512^3 in 8^3 PEs: delay log of the 500-step run bit-exact; field after a 6-step prefix vs oracle."""
    spec, steps = W.workload(f"3d_512_o{order}")
    cfg = oracle.Config(spec)
    from paper_1702_00496_gb300 import Solver
    s = Solver(spec, log_steps=steps)
    s.step(6)
    s.sync()
    u = s.field().cpu().numpy().copy()
    s.step(steps - 6)
    s.sync()
    assert np.array_equal(s.delays().cpu().numpy(), oracle.delay_log(cfg, steps))
    st = s.error_stats()
    s.close()
    ref, _, _ = oracle.run(cfg, 6, want_log=False, threads=THREADS)
    assert np.linalg.norm(u - ref) / np.linalg.norm(ref) <= TOL
    assert np.isfinite(st["rms"]) and st["rms"] < 1e-2 * st["ua_rms"]


def test_launch_shapes_do_not_change_results():
    """Every launch shape the autotuner may pick gives the same bits (the arithmetic per point is fixed)."""
    from paper_1702_00496_gb300 import Solver, at_set_launch
    for spec in (W.wl_1d(4096, 16, 4, 4, 0, 12, range(1, 6))[0], W.wl_3d([32, 24, 16], [4, 3, 2], 4, 3, 0, 13,
                                                                         c=(0.3, 0.2, 0.1))[0]):
        ref = None
        for threads, bps in ((256, 32), (128, 4), (512, 16), (256, 1)):
            s = Solver(spec)
            at_set_launch(s.h, threads, bps)
            s.step(120)
            s.sync()
            u = s.field().clone()
            s.close()
            if ref is None:
                ref = u
            assert torch.equal(u, ref), (threads, bps)


# ------------------------------------------------------------ maximum sizes of the delay process
@pytest.mark.parametrize("order,r_alpha", [(2, 0.05), (4, 0.02), (6, 0.005)])
def test_largest_delay_range(order, r_alpha):
    """L = 8, the largest delay range: delays 0..7, the deepest halo reach (ring of L + T = 8 + 4 levels at order 6)."""
    spec, _ = W.wl_1d(4096, 16, order, 8, 0, 501, range(1, 6), r_alpha=r_alpha)
    _compare(spec, 100)


def test_largest_delay_range_3d_with_binned_delays():
    spec, _ = W.wl_3d([16, 16, 12], [2, 2, 3], 4, 8, 0, 502, c=(0.2, 0.2, 0.2), dt=0.02 * W.dx_of(16) ** 2 / 0.05)
    spec["thresholds"] = W.thresholds_from_probs([0.05, 0.05, 0.1, 0.1, 0.2, 0.2, 0.15, 0.15])
    _compare(spec, 30)
