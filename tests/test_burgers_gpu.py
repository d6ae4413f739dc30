"""GPU parity of the viscous Burgers' equation (Case 6) against the oracle, the reference-field statistics
(at_error_stats_ref) against their definition, and the paper's Fig. "at-ord4-nl" convergence run on the GPU.
Bars: delay logs bit-exact, fields within 1e-12 relative L2."""
import os

import numpy as np
import pytest

import oracle
import workloads as W
from burgers_exact import cole_hopf

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

TOL = 1e-12
THREADS = os.cpu_count() or 1


def _gpu(spec, nsteps, u0=None, log=True):
    from paper_1702_00496_gb300 import Solver
    s = Solver(spec, log_steps=nsteps if log else 0)
    if u0 is not None:
        s.reset(torch.as_tensor(u0, device="cuda"))
    s.step(nsteps)
    s.sync()
    u = s.field().cpu().numpy().copy()
    d = s.delays().cpu().numpy().copy() if log else None
    s.close()
    return u, d


def _compare(spec, nsteps, u0=None):
    u, d = _gpu(spec, nsteps, u0)
    ref, dref, _ = oracle.run(oracle.Config(spec), nsteps, threads=THREADS, u0=u0)
    assert np.array_equal(d, dref)
    assert np.linalg.norm(u - ref) / np.linalg.norm(ref) <= TOL
    assert np.abs(u - ref).max() <= TOL * np.abs(ref).max()


def _burgers(n, P, order, L, seed, tsteps, scheme=W.AT, probs=None, r_alpha=0.05):
    spec, _ = W.wl_1d(n, P, order, L, 0, seed, (3, 4, 5), scheme=scheme, c=0.0, alpha=0.1, r_alpha=r_alpha,
                      probs=probs, tsteps=tsteps)
    spec["burgers"] = 1
    return spec


@pytest.mark.parametrize("order,tsteps,scheme", [(4, 2, W.AT), (2, 1, W.AT), (6, 3, W.AT), (4, 2, W.ASYNC_STD),
                                                 (4, 1, W.SYNC)])
def test_burgers_parity(order, tsteps, scheme):
    spec = _burgers(12000, 30, order, 4, 140 + order + tsteps, tsteps, scheme,
                    r_alpha=0.01 if order == 6 else 0.05)
    _compare(spec, 300)


def test_burgers_point_path_and_callers_field():
    spec = _burgers(250, 5, 4, 3, 141, 2)
    _compare(spec, 200)
    spec = _burgers(4096, 16, 4, 3, 142, 2)
    _compare(spec, 200, u0=cole_hopf(4096, 0.0, 0.1))


def test_burgers_converges_to_cole_hopf_on_the_gpu():
    errs = {W.AT: [], W.ASYNC_STD: []}
    ns = (64, 128, 256)
    for scheme in errs:
        for n in ns:
            spec = _burgers(n, 16, 4, 3, 7, 2, scheme, probs=(0.3, 0.5, 0.2))
            steps = W.steps_to(spec, 0.2)
            u, _ = _gpu(spec, steps, u0=cole_hopf(n, 0.0, 0.1), log=False)
            errs[scheme].append(np.sqrt(np.mean((u - cole_hopf(n, steps * spec["dt"], 0.1)) ** 2)))
    assert abs(np.polyfit(np.log(ns), np.log(errs[W.AT]), 1)[0] + 4.0) < 0.15, errs
    assert abs(np.polyfit(np.log(ns), np.log(errs[W.ASYNC_STD]), 1)[0] + 1.0) < 0.15, errs


def test_case6_against_a_finer_run_with_reference_statistics():
    """Fig. "at-ord4-nl" measured the paper's way: each coarse run against a synchronous run four times finer that
    ends at the same time, through at_error_stats_ref; the statistics equal their definition on the fields."""
    from paper_1702_00496_gb300 import Solver
    nf, ns = 1024, (64, 128, 256)
    errs = {}
    for probs in ((1.0, 0.0, 0.0), (0.3, 0.5, 0.2)):
        errs[probs] = []
        for n in ns:
            spec = W.paper_case(6, n, 300, probs)
            steps = W.steps_to(spec, 0.1)
            fine = Solver(W.paper_case(6, nf, 300))
            fine.step(steps * (nf // n) ** 2)
            ref = fine.field().clone()
            fine.close()
            s = Solver(spec)
            s.step(steps)
            st = s.error_stats_ref(ref, nf // n)
            u = s.field().cpu().numpy()
            s.close()
            e = u - ref.cpu().numpy()[::nf // n]
            assert st["rms"] == pytest.approx(np.sqrt(np.mean(e * e)), rel=1e-12)
            assert st["max_abs"] == pytest.approx(np.abs(e).max(), rel=1e-15)
            assert st["ua_rms"] == pytest.approx(np.sqrt(np.mean(ref.cpu().numpy()[::nf // n] ** 2)), rel=1e-12)
            errs[probs].append(st["rms"])
        e = errs[probs]
        assert abs(np.log(e[2] / e[1]) / np.log(2) + 4.0) < 0.25, e
    assert np.all(np.abs(np.array(errs[(0.3, 0.5, 0.2)]) / np.array(errs[(1.0, 0.0, 0.0)]) - 1) < 0.01)


def test_reference_statistics_in_3d():
    from paper_1702_00496_gb300 import Solver
    spec, _ = W.wl_3d([8, 6, 4], [2, 2, 2], 2, 3, 0, 143, c=(0.2, 0.1, 0.3))
    fine_spec, _ = W.wl_3d([16, 12, 8], [2, 2, 2], 2, 3, 0, 143, c=(0.2, 0.1, 0.3), dt=spec["dt"])
    f = Solver(fine_spec)
    f.step(10)
    ref = f.field().clone()
    f.close()
    s = Solver(spec)
    s.step(10)
    st = s.error_stats_ref(ref, 2)
    e = s.field().cpu().numpy() - ref.cpu().numpy()[::2, ::2, ::2]
    s.close()
    assert st["rms"] == pytest.approx(np.sqrt(np.mean(e * e)), rel=1e-12)
    assert st["mean"] == pytest.approx(np.mean(e), rel=1e-9, abs=1e-15)


def test_burgers_rejections():
    from paper_1702_00496_gb300 import Ensemble, Solver, binding as B
    spec = _burgers(256, 8, 4, 3, 144, 2)
    s = Solver(spec)
    with pytest.raises(B.ATError):
        s.error_stats()  # no analytic solution
    s.close()
    with pytest.raises(B.ATError):
        Ensemble([spec], 10)


BURGERS_ADJ = [(4, 2, W.AT, 256, 8), (2, 1, W.AT, 256, 8), (4, 1, W.ASYNC_STD, 256, 8), (6, 3, W.AT, 256, 8),
               (4, 2, W.AT, 250, 5)]


@pytest.mark.parametrize("order,tsteps,scheme,n,P", BURGERS_ADJ)
def test_burgers_adjoint_matches_cpu_adjoint(order, tsteps, scheme, n, P):
    """The transposed Burgers step (state-dependent: the D1 taps carry -U_i^n, U_i^n receives -D1 U) against the
    oracle's literal transpose; the u0-only sweep (which still recomputes the forward levels) gives the same bits."""
    from paper_1702_00496_gb300 import Solver
    spec = _burgers(n, P, order, 3, 150 + order + tsteps, tsteps, scheme, r_alpha=0.01 if order == 6 else 0.02)
    cfg = oracle.Config(spec)
    rng = np.random.default_rng(6)
    target = 0.5 * oracle.initial(cfg) + 0.1 * rng.standard_normal(cfg.shape)
    nsteps = 60
    grads = []
    for want_alpha, every in ((True, 7), (False, 7), (True, nsteps)):  # every = nsteps: all levels resident
        s = Solver(spec)
        s.adjoint_forward(nsteps, every)
        u = s.field().clone()
        lam = u - torch.as_tensor(target, device="cuda")
        J = 0.5 * float((lam * lam).sum())
        g, ga = s.adjoint_backward(lam.clone(), want_alpha)
        grads.append(g.clone())
        s.close()
        if want_alpha and every == 7:
            Jo, go, gao = oracle.adjoint(cfg, nsteps, target)
            assert J == pytest.approx(Jo, rel=1e-11)
            assert np.linalg.norm(g.cpu().numpy() - go) / np.linalg.norm(go) <= 1e-12
            assert ga == pytest.approx(gao, rel=1e-10)
    assert torch.equal(grads[0], grads[1]) and torch.equal(grads[0], grads[2])
