"""GPU parity of the sixth-order stencils (CD6 with the (2,6,2) AT rows) and of Adams-Bashforth time stepping
(two and three levels, Sec. 4.1 Eq. "time_disc") against the oracle, and the paper's Cases 4 and 5 (Fig.
"at-prob-all" (c), (d)) run on the GPU.

Bars as for the forward-Euler path: delay logs bit-exact, fields within 1e-12 relative L2 and elementwise
within 1e-12 of the field's max norm.
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


def _solver(spec, log_steps=0):
    from paper_1702_00496_gb300 import Solver
    return Solver(spec, log_steps=log_steps)


def _compare(spec, nsteps, u0=None):
    s = _solver(spec, nsteps)
    if u0 is not None:
        s.reset(torch.as_tensor(u0, device="cuda"))
    s.step(nsteps)
    s.sync()
    u = s.field().cpu().numpy().copy()
    d = s.delays().cpu().numpy().copy()
    st = s.error_stats()
    s.close()
    cfg = oracle.Config(spec)
    ref, dref, _ = oracle.run(cfg, nsteps, threads=THREADS, u0=u0)
    assert np.array_equal(d, dref), "delay logs differ"
    rel = np.linalg.norm(u - ref) / np.linalg.norm(ref)
    assert rel <= TOL, rel
    assert np.abs(u - ref).max() <= TOL * np.abs(ref).max()
    so = oracle.error_stats(cfg, u, nsteps)
    for key in ("rms", "max_abs", "rms_I", "rms_B"):
        assert abs(st[key] - so[key]) <= 1e-9 * abs(so[key]) + 1e-13 * so["ua_rms"], key
    return u, ref


# 12000 points in 30 PEs of 400: several thread blocks, a ragged last block, 300 steps (six captured graphs)
CASES_1D = [
    ("o6_at_euler", dict(order=6, r_alpha=0.02)),
    ("o6_std_euler", dict(order=6, r_alpha=0.1, scheme=W.ASYNC_STD)),
    ("o6_sync_euler", dict(order=6, r_alpha=0.1, scheme=W.SYNC)),
    ("o4_at_ab2", dict(order=4, r_alpha=0.05, tsteps=2)),
    ("o6_at_ab3", dict(order=6, r_alpha=0.01, tsteps=3)),
    ("o2_at_ab2", dict(order=2, r_alpha=0.05, tsteps=2)),
    ("o4_std_ab3", dict(order=4, r_alpha=0.02, tsteps=3, scheme=W.ASYNC_STD)),
    ("o6_sync_ab2", dict(order=6, r_alpha=0.02, tsteps=2, scheme=W.SYNC)),
]


@pytest.mark.parametrize("name,kw", CASES_1D, ids=[c[0] for c in CASES_1D])
def test_1d_order6_and_multistep(name, kw):
    kw = dict(kw)
    order = kw.pop("order")
    spec, _ = W.wl_1d(12000, 30, order, 4, 0, 81 + len(name), range(1, 11), **kw)
    _compare(spec, 300)


@pytest.mark.parametrize("tsteps", [1, 2, 3])
def test_1d_point_path_order6(tsteps):
    # N = 250 is not a multiple of 4: the per-point kernel (and per-point Adams-Bashforth update)
    spec, _ = W.wl_1d(250, 5, 6, 3, 0, 86, (1, 2, 3), r_alpha=0.01, tsteps=tsteps)
    _compare(spec, 300)


@pytest.mark.parametrize("S", [6, 8])
def test_1d_minimum_pe_width_order6(S):
    # S = 6 = 2h takes the per-point kernel (S not a multiple of 4), S = 8 the grouped one
    spec, _ = W.wl_1d(48 * S, 48, 6, 3, 0, 87, (1, 3), r_alpha=0.01, tsteps=3)
    _compare(spec, 200)


@pytest.mark.parametrize("order,tsteps,r", [(6, 1, 0.05), (4, 2, 0.05), (6, 3, 0.02), (2, 3, 0.02)])
def test_3d_order6_and_multistep(order, tsteps, r):
    dt = r * W.dx_of(24) ** 2 / 0.05
    spec, _ = W.wl_3d([24, 20, 16], [3, 2, 2], order, 3, 0, 88 + order + tsteps, c=(0.5, -0.35, 0.2), dt=dt,
                      tsteps=tsteps)
    _compare(spec, 60)


@pytest.mark.parametrize("tsteps", [2, 3])
def test_multistep_from_a_callers_field_starts_with_euler(tsteps):
    """at_reset with a field: no analytic pre-history, so the run starts with forward Euler, then AB2 (the
    oracle's start from u0)."""
    spec, _ = W.wl_1d(4096, 16, 4, 3, 0, 90, (1, 2, 5), r_alpha=0.02, tsteps=tsteps)
    rng = np.random.default_rng(5)
    u0 = oracle.initial(oracle.Config(spec)) + 0.01 * rng.standard_normal(4096)
    _compare(spec, 120, u0=u0)


def test_reset_restores_the_analytic_prehistory():
    spec, _ = W.wl_1d(4096, 16, 6, 3, 0, 91, (1, 2, 5), r_alpha=0.01, tsteps=3)
    s = _solver(spec)
    s.step(77)
    first = s.field().clone()
    s.reset(torch.zeros(4096, dtype=torch.float64, device="cuda"))
    s.step(13)
    s.reset()
    s.step(77)
    assert torch.equal(s.field(), first)
    s.close()


@pytest.mark.parametrize("tsteps,order", [(3, 6), (2, 4)])
def test_graph_chunks_and_single_launches_agree(tsteps, order):
    """300 steps in one call (six captured 50-step graphs) and in calls of 7 and 293 (single launches, then
    graphs starting mid-history) give the same bits: the integrator reads its history level from the device (AB3),
    or every step has both levels and takes the steady form in graphs and single launches alike (AB2)."""
    spec, _ = W.wl_1d(8192, 32, order, 4, 0, 92, range(1, 6), r_alpha=0.01, tsteps=tsteps)
    a = _solver(spec)
    a.step(300)
    b = _solver(spec)
    b.step(7)
    b.step(293)
    assert torch.equal(a.field(), b.field())
    a.close()
    b.close()


def test_ab2_from_a_callers_field_across_call_splits():
    """From a caller's field the first AB2 step has one stored level (the general form, a single launch); the rest
    take the steady form.  One call of 300 steps against calls of 1, 1, 49 and 249 (the start-up step alone, then
    graphs from mid-run): the same bits; and against the oracle."""
    spec, _ = W.wl_1d(8192, 32, 4, 3, 0, 95, range(1, 6), r_alpha=0.02, tsteps=2)
    rng = np.random.default_rng(6)
    u0 = oracle.initial(oracle.Config(spec)) + 0.01 * rng.standard_normal(8192)
    u0_dev = torch.as_tensor(u0, device="cuda")
    a = _solver(spec)
    a.reset(u0_dev)
    a.step(300)
    b = _solver(spec)
    b.reset(u0_dev)
    for n in (1, 1, 49, 249):
        b.step(n)
    assert torch.equal(a.field(), b.field())
    u = a.field().cpu().numpy().copy()
    a.close()
    b.close()
    ref, _, _ = oracle.run(oracle.Config(spec), 300, threads=THREADS, u0=u0, want_log=False)
    assert np.linalg.norm(u - ref) / np.linalg.norm(ref) <= TOL


@pytest.mark.parametrize("tsteps", [2, 3])
def test_steady_form_is_bitwise_the_general_combination(tsteps):
    """Once both levels are stored, a single problem's AB2 steps take the combination's steady form (the weights
    read as kernel parameters); the ensemble engine takes the general form, which looks the number of stored
    levels up at every step.  The operations are the same, so the bits are: members against single problems, 130
    steps (graphs and single launches); AB3 takes the general form on both sides."""
    from paper_1702_00496_gb300 import Ensemble
    specs = [W.wl_1d(n, n // 16, order, L, 0, 950 + r, range(1, 5), r_alpha=0.02, tsteps=tsteps)[0]
             for r, (n, order, L) in enumerate([(256, 4, 3), (1024, 6, 4), (512, 2, 3)])]
    ens = Ensemble(specs, 130)
    ens.run()
    for r, spec in enumerate(specs):
        s = _solver(spec)
        s.step(130)
        s.sync()
        assert torch.equal(ens.field(r), s.field().reshape(-1)), r
        s.close()
    ens.close()


def test_launch_shapes_do_not_change_multistep_results():
    from paper_1702_00496_gb300 import at_set_launch
    for spec in (W.wl_1d(4096, 16, 6, 4, 0, 93, range(1, 6), r_alpha=0.01, tsteps=3)[0],
                 W.wl_1d(4096, 16, 4, 4, 0, 96, range(1, 6), r_alpha=0.02, tsteps=2)[0],
                 W.wl_3d([32, 24, 16], [4, 3, 2], 4, 3, 0, 94, c=(0.3, 0.2, 0.1), tsteps=2)[0]):
        ref = None
        for threads, bps in ((256, 32), (128, 4), (512, 16)):
            s = _solver(spec)
            at_set_launch(s.h, threads, bps)
            s.step(120)
            u = s.field().clone()
            s.close()
            if ref is None:
                ref = u
            assert torch.equal(u, ref), (threads, bps)


@pytest.mark.parametrize("name", ["1d_n16m_case4", "1d_n16m_case5"])
def test_full_size_cases_4_and_5_sampled_after_the_whole_run(name):
    """N = 2^24, 4096 PEs, AB2 with CD4 / AB3 with CD6, all 1000 asynchronous steps in the launch shape bench.py
    picks: PE-edge and interior cells against the oracle stepped inside their domain of dependence."""
    from paper_1702_00496_gb300 import autotune
    spec, steps = W.workload(name)
    s = _solver(spec)
    autotune.tune_forward(s, spec)
    s.reset()
    s.step(steps)
    s.sync()
    u = s.field().cpu().numpy().copy()
    s.close()
    S = spec["n"][0] // spec["pe"][0]
    pes = np.random.default_rng(2).choice(spec["pe"][0], 4, replace=False)
    pos = sorted({int(p * S + o) for p in pes for o in (0, 1, 2, S // 2, S - 3, S - 1)})
    ref = oracle.run_samples(oracle.Config(spec), steps, pos)
    assert np.abs(u[pos] - ref).max() <= TOL * np.abs(u).max()


# ------------------------------------------------------------ the paper's Cases 4 and 5 on the GPU
def _slope(ns, errs):
    return np.polyfit(np.log(np.asarray(ns, float)), np.log(np.asarray(errs)), 1)[0]


@pytest.mark.parametrize("case,ns,slope", [(4, (64, 128, 256), -4.0), (5, (128, 192, 256), -6.0)])
def test_paper_cases_4_and_5_on_the_gpu(case, ns, slope):
    """Fig. "at-prob-all" (c), (d): RMS error against the analytic solution at t = 0.1 falls at the design
    slope for every delay mix; at the smallest grid the GPU field matches the oracle's."""
    for probs in ((1.0, 0.0, 0.0), (0.7, 0.2, 0.1), (0.0, 0.5, 0.5)):
        errs = []
        for n in ns:
            spec = W.paper_case(case, n, 300, probs)
            steps = int(round(0.1 / spec["dt"]))
            s = _solver(spec)
            s.step(steps)
            errs.append(s.error_stats()["rms"])
            if n == ns[0]:
                u = s.field().cpu().numpy()
                ref, _, _ = oracle.run(oracle.Config(spec), steps, want_log=False, threads=THREADS)
                assert np.linalg.norm(u - ref) / np.linalg.norm(ref) <= TOL
            s.close()
        assert abs(_slope(ns, errs) - slope) < 0.25, (probs, errs)


# ------------------------------------------------------------ the ensemble engine with the new schemes
def test_ensemble_with_order6_and_multistep_members():
    from paper_1702_00496_gb300 import Ensemble
    specs = []
    for r, (case, n) in enumerate([(4, 64), (4, 128), (5, 128), (5, 192), (4, 256), (5, 256)]):
        specs.append(W.paper_case(case, n, 400 + r, (0.0, 0.5, 0.5)))
    specs.append(W.wl_1d(512, 8, 6, 4, 0, 410, range(1, 5), r_alpha=0.02)[0])  # order 6, forward Euler
    specs.append(W.wl_1d(512, 8, 4, 3, 0, 411, range(1, 5))[0])                # order 4, forward Euler
    nsteps = 500
    ens = Ensemble(specs, nsteps, log=True)
    ens.run()
    per, _ = ens.stats()
    for r, spec in enumerate(specs):
        cfg = oracle.Config(spec)
        ref, dref, _ = oracle.run(cfg, nsteps, threads=THREADS)
        u = ens.field(r).cpu().numpy()
        assert np.array_equal(ens.delays(r).cpu().numpy(), dref), r
        assert np.linalg.norm(u - ref) / np.linalg.norm(ref) <= TOL, r
        so = oracle.error_stats(cfg, u, nsteps)
        assert abs(per[r]["rms"] - so["rms"]) <= 1e-9 * so["rms"] + 1e-13 * so["ua_rms"], r
    ens.close()


def test_adjoint_rejects_a_multistep_run_with_the_analytic_prehistory():
    from paper_1702_00496_gb300 import binding as B
    for spec in (W.wl_1d(256, 8, 4, 3, 0, 95, (1, 2), tsteps=2)[0],):
        s = _solver(spec)
        with pytest.raises(RuntimeError):
            B.at_adjoint_workspace(s.h, 10, 0)
        s.close()
