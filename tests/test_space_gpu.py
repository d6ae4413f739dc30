"""GPU parity of the AT stencils expanded in space -- (1,2,2)a, (2,2,2)a (Case 3) and (2,1,2) (Case 2) -- against
the oracle, in the per-step kernels (grouped and per-point, 1D and 3D) and the ensemble engine, and the paper's
Sec. 5.2 behaviour of Cases 2 and 3 run on the GPU.  Bars: delay logs bit-exact, fields within 1e-12."""
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


def _compare(spec, nsteps):
    from paper_1702_00496_gb300 import Solver
    s = Solver(spec, log_steps=nsteps)
    s.step(nsteps)
    s.sync()
    u = s.field().cpu().numpy().copy()
    d = s.delays().cpu().numpy().copy()
    st = s.error_stats()
    s.close()
    cfg = oracle.Config(spec)
    ref, dref, _ = oracle.run(cfg, nsteps, threads=THREADS)
    assert np.array_equal(d, dref), "delay logs differ"
    assert np.linalg.norm(u - ref) / np.linalg.norm(ref) <= TOL
    assert np.abs(u - ref).max() <= TOL * np.abs(ref).max()
    so = oracle.error_stats(cfg, u, nsteps)
    for key in ("rms", "max_abs", "rms_I", "rms_B"):
        assert abs(st[key] - so[key]) <= 1e-9 * abs(so[key]) + 1e-13 * so["ua_rms"], key
    return u


@pytest.mark.parametrize("scheme,c", [(W.AT_SPACE2, 1.0), (W.AT_SPACE1, 0.0)])
@pytest.mark.parametrize("probs", [None, (0.3, 0.3, 0.2, 0.2)])
def test_1d_space_expanded_rows(scheme, c, probs):
    spec, _ = W.wl_1d(12000, 30, 2, 4, 0, 120, range(1, 11), scheme=scheme, c=c, probs=probs)
    _compare(spec, 300)


@pytest.mark.parametrize("scheme,c", [(W.AT_SPACE2, 1.0), (W.AT_SPACE1, 0.0)])
def test_1d_point_path_and_minimum_pe_width(scheme, c):
    # N = 250 (not a multiple of 4) and S = 2 (the rows reach three cells into the neighbouring PEs)
    for n, P in ((250, 5), (64, 32)):
        spec, _ = W.wl_1d(n, P, 2, 3, 0, 121, (1, 2, 3), scheme=scheme, c=c)
        _compare(spec, 200)


@pytest.mark.parametrize("scheme,c", [(W.AT_SPACE2, (0.5, -0.35, 0.2)), (W.AT_SPACE1, (0.0, 0.0, 0.0))])
def test_3d_space_expanded_rows(scheme, c):
    spec, _ = W.wl_3d([24, 20, 16], [3, 2, 4], 2, 3, 0, 122, scheme=scheme, c=c)
    _compare(spec, 40)


def test_launch_shapes_do_not_change_space_expanded_results():
    from paper_1702_00496_gb300 import Solver, at_set_launch
    spec, _ = W.wl_1d(4096, 16, 2, 4, 0, 123, range(1, 6), scheme=W.AT_SPACE2)
    ref = None
    for threads, bps in ((256, 32), (128, 4), (512, 16)):
        s = Solver(spec)
        at_set_launch(s.h, threads, bps)
        s.step(120)
        u = s.field().clone()
        s.close()
        if ref is None:
            ref = u
        assert torch.equal(u, ref), (threads, bps)


def test_ensemble_members_with_space_expanded_rows():
    from paper_1702_00496_gb300 import Ensemble
    specs = [W.paper_case(case, n, 130 + i, (0.4, 0.3, 0.3)) for i, (case, n) in
             enumerate([(2, 64), (2, 256), (3, 128), (3, 512), (1, 256), (4, 128)])]
    steps = [W.steps_to(s, 0.05) for s in specs]
    ens = Ensemble(specs, steps, log=True)
    ens.run()
    per, _ = ens.stats()
    for r, spec in enumerate(specs):
        cfg = oracle.Config(spec)
        ref, dref, _ = oracle.run(cfg, steps[r], threads=THREADS)
        u = ens.field(r).cpu().numpy()
        assert np.array_equal(ens.delays(r).cpu().numpy(), dref), r
        assert np.linalg.norm(u - ref) / np.linalg.norm(ref) <= TOL, r
        so = oracle.error_stats(cfg, u, steps[r])
        assert abs(per[r]["rms"] - so["rms"]) <= 1e-9 * so["rms"] + 1e-13 * so["ua_rms"], r
    ens.close()


def _slope(ns, errs):
    return float(np.polyfit(np.log(ns), np.log(errs), 1)[0])


@pytest.mark.parametrize("case", [2, 3])
def test_cases_2_and_3_on_the_gpu(case):
    """Fig. "at-prob-all" (a), (b): slope -2 at p_0 = 1 and asymptotically at p_0 = 0.7; Fig. "at-kmom": the
    asynchronous part of the error proportional to E[k] (the rows' leading asynchronous terms are linear in k)."""
    from paper_1702_00496_gb300 import Ensemble
    ns = (64, 128, 256, 512)
    for probs, lo in (((1.0, 0.0, 0.0), 0), ((0.7, 0.2, 0.1), 2)):
        specs = [W.paper_case(case, n, 300, probs) for n in ns]
        steps = [W.steps_to(s, 0.1) for s in specs]
        ens = Ensemble(specs, steps)
        ens.run()
        per, _ = ens.stats()
        errs = [per[r]["rms"] for r in range(len(ns))]
        assert abs(_slope(ns[lo:], errs[lo:]) + 2.0) < (0.1 if lo == 0 else 0.3), (probs, errs)
        ens.close()
    Ls = (2, 3, 4, 5)
    specs, steps, groups, twins = W.moment_members(case, Ls, range(900, 948))
    ens = Ensemble(specs, steps, groups=groups, twins=twins)
    ens.run()
    _, grp = ens.stats()
    g = {x["key"]: x for x in grp}
    ratio = np.array([(g[L]["mean"] - g[100 + L]["mean"]) / g[100 + L]["mean"] / ((L - 1) / 2.0) for L in Ls])
    assert np.all(ratio > 0) and np.ptp(ratio) <= 0.15 * ratio.max(), ratio
    ens.close()


SPACE_ADJ = [
    ("1d_case3", lambda: W.wl_1d(256, 8, 2, 4, 0, 160, (1, 2, 3), scheme=W.AT_SPACE2, c=1.0)[0], 80),
    ("1d_case2", lambda: W.wl_1d(256, 8, 2, 3, 0, 161, (1, 2, 3), scheme=W.AT_SPACE1, c=0.0)[0], 80),
    ("1d_min_width", lambda: W.wl_1d(64, 32, 2, 3, 0, 162, (1, 3), scheme=W.AT_SPACE2, c=1.0)[0], 60),
    ("3d_space2", lambda: W.wl_3d([16, 12, 8], [2, 3, 2], 2, 3, 0, 163, scheme=W.AT_SPACE2, c=(0.3, 0.2, 0.1))[0], 20),
    ("3d_space1", lambda: W.wl_3d([16, 12, 8], [2, 3, 2], 2, 3, 0, 164, scheme=W.AT_SPACE1, c=(0.0, 0.0, 0.0))[0], 20),
]


@pytest.mark.parametrize("name,make,nsteps", SPACE_ADJ, ids=[c[0] for c in SPACE_ADJ])
def test_adjoint_of_space_expanded_rows(name, make, nsteps):
    """The transposed step through the edge rows (in-PE taps to level n, buffer taps to n - k) against the
    oracle's literal transpose."""
    from paper_1702_00496_gb300 import Solver
    spec = make()
    cfg = oracle.Config(spec)
    rng = np.random.default_rng(8)
    target = 0.5 * oracle.initial(cfg) + 0.1 * rng.standard_normal(cfg.shape)
    s = Solver(spec)
    s.adjoint_forward(nsteps, 9)
    lam = s.field() - torch.as_tensor(target, device="cuda")
    J = 0.5 * float((lam * lam).sum())
    g, ga = s.adjoint_backward(lam.clone())
    s.close()
    Jo, go, gao = oracle.adjoint(cfg, nsteps, target)
    assert J == pytest.approx(Jo, rel=1e-11)
    assert np.linalg.norm(g.cpu().numpy() - go) / np.linalg.norm(go) <= 1e-12
    assert ga == pytest.approx(gao, rel=1e-10)
