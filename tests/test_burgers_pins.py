"""The oracle's viscous Burgers' equation (Sec. 5.1, Eq. "general" with beta_1 = u, beta_2 = alpha; Case 6)
against exact Cole-Hopf solutions: the reference is pinned to the PDE, and the runs converge at the design order of
their stencils and time integrator -- with the time-expanded AT rows also under delays (Fig. "at-ord4-nl"), while
the standard scheme read at delayed levels drops to first order.  CPU only."""
import numpy as np
import pytest

import oracle
import workloads as W
from burgers_exact import cole_hopf

ALPHA = 0.1


def test_cole_hopf_reference_solves_burgers():
    n, t, dt = 256, 0.3, 1e-5
    k = np.fft.fftfreq(n, 1.0 / n)
    u = cole_hopf(n, t, ALPHA)
    ut = (cole_hopf(n, t + dt, ALPHA) - cole_hopf(n, t - dt, ALPHA)) / (2 * dt)
    uh = np.fft.fft(u)
    ux = np.fft.ifft(1j * k * uh).real
    uxx = np.fft.ifft(-(k ** 2) * uh).real
    assert np.abs(ut + u * ux - ALPHA * uxx).max() < 1e-7 * np.abs(ut).max()


def _error(order, tsteps, scheme, probs, n, t_final=0.2):
    spec, _ = W.wl_1d(n, 16, order, 3, 0, 7, (1,), scheme=scheme, c=0.0, alpha=ALPHA, r_alpha=0.05, probs=probs,
                      tsteps=tsteps)
    spec["burgers"] = 1
    steps = W.steps_to(spec, t_final)
    u, _, _ = oracle.run(oracle.Config(spec), steps, want_log=False, threads=4, u0=cole_hopf(n, 0.0, ALPHA))
    return np.sqrt(np.mean((u - cole_hopf(n, steps * spec["dt"], ALPHA)) ** 2))


@pytest.mark.parametrize("order,tsteps,scheme,probs,slope,tol", [
    (2, 1, W.SYNC, None, -2.0, 0.1),
    (4, 2, W.SYNC, None, -4.0, 0.15),
    (4, 2, W.AT, (0.7, 0.2, 0.1), -4.0, 0.15),
    (4, 2, W.AT, (0.3, 0.5, 0.2), -4.0, 0.15),
    (4, 2, W.ASYNC_STD, (0.3, 0.5, 0.2), -1.0, 0.15),
])
def test_burgers_converges_at_the_design_order(order, tsteps, scheme, probs, slope, tol):
    ns = (64, 128, 256)
    errs = [_error(order, tsteps, scheme, probs, n) for n in ns]
    assert abs(np.polyfit(np.log(ns), np.log(errs), 1)[0] - slope) < tol, errs


def test_burgers_is_rejected_where_it_is_not_defined():
    spec, _ = W.wl_1d(64, 4, 4, 3, 0, 1, (1,), c=1.0)
    spec["burgers"] = 1  # c must be 0: the advecting speed is u
    with pytest.raises(ValueError):
        oracle.Config(spec)
    spec, _ = W.wl_3d([8, 8, 8], [2, 2, 2], 2, 3, 0, 2, c=(0.0, 0.0, 0.0))
    spec["burgers"] = 1  # one-dimensional only
    with pytest.raises(ValueError):
        oracle.Config(spec)


def test_case6_converges_at_fourth_order_against_a_finer_run():
    """Fig. "at-ord4-nl": Case 6 (Eq. "IC" with kappa = {3,4,5}, A = {2, 0.5, 1.5}) converges at fourth order
    against a synchronous run four times finer, at every delay mix, and the delays hardly change the error."""
    nf, ns = 1024, (64, 128, 256)
    ref = {}
    errs = {}
    for probs in ((1.0, 0.0, 0.0), (0.7, 0.2, 0.1), (0.3, 0.5, 0.2)):
        errs[probs] = []
        for n in ns:
            spec = W.paper_case(6, n, 300, probs)
            steps = W.steps_to(spec, 0.1)
            if n not in ref:  # the fine run ends at the same time: its dt is (n/nf)^2 of the coarse one
                ref[n], _, _ = oracle.run(oracle.Config(W.paper_case(6, nf, 300)), steps * (nf // n) ** 2,
                                          want_log=False, threads=4)
            u, _, _ = oracle.run(oracle.Config(spec), steps, want_log=False, threads=4)
            errs[probs].append(np.sqrt(np.mean((u - ref[n][::nf // n]) ** 2)))
        e = errs[probs]
        assert abs(np.log(e[2] / e[1]) / np.log(2) + 4.0) < 0.25, e
    sync = np.array(errs[(1.0, 0.0, 0.0)])
    for probs in ((0.7, 0.2, 0.1), (0.3, 0.5, 0.2)):
        assert np.all(np.abs(np.array(errs[probs]) / sync - 1) < 0.01)


@pytest.mark.parametrize("order,tsteps,scheme", [(4, 2, W.AT), (2, 1, W.AT), (4, 1, W.ASYNC_STD), (6, 3, W.AT)])
def test_burgers_adjoint_matches_central_differences(order, tsteps, scheme):
    """The literal transpose of the Burgers step: the D1 taps carry -U_i^n and U_i^n receives -D1 U.  J is no longer
    quadratic in u0, so both directions use Richardson-extrapolated central differences."""
    spec, _ = W.wl_1d(128, 8, order, 3, 0, 71, (3, 4, 5), scheme=scheme, c=0.0, r_alpha=0.02 if order < 6 else 0.01,
                      tsteps=tsteps)
    spec["burgers"] = 1
    cfg = oracle.Config(spec)
    rng = np.random.default_rng(3)
    u0 = oracle.initial(cfg)
    tgt = 0.5 * u0 + 0.1 * rng.standard_normal(cfg.shape)
    nsteps = 40
    J, g, ga = oracle.adjoint(cfg, nsteps, tgt)

    def Jf(u, alpha=spec["alpha"]):
        sp = dict(spec)
        sp["alpha"] = alpha
        uu, _, _ = oracle.run(oracle.Config(sp), nsteps, want_log=False, u0=u)
        return 0.5 * float(np.sum((uu - tgt) ** 2))

    assert J == pytest.approx(Jf(u0), rel=1e-14)

    def rich(f, h):
        d1 = (f(h) - f(-h)) / (2 * h)
        d2 = (f(h / 2) - f(-h / 2)) / h
        return (4 * d2 - d1) / 3

    v = rng.standard_normal(cfg.shape)
    assert float(np.sum(g * v)) == pytest.approx(rich(lambda e: Jf(u0 + e * v), 1e-3), rel=1e-8)
    a0 = spec["alpha"]
    assert ga == pytest.approx(rich(lambda e: Jf(u0, a0 + e), 1e-3 * a0), rel=1e-7)
