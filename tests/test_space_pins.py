"""The oracle's stencils expanded in space -- (1,2,2)a, (2,2,2)a and (2,1,2) of the tables "atschemes-left/right",
the paper's Cases 3 and 2 -- against what the paper fixes independently of the typed rows: the Taylor conditions of
Eq. "cond", the printed leading-order terms, the mirror symmetry of the left and right tables, Example 1's
uniform-delay scheme (Eq. "ex1-1"), and the convergence and delay-moment behaviour of Sec. 5.2.  CPU only."""
from fractions import Fraction
from math import factorial

import numpy as np
import pytest

import oracle
import workloads as W

S = 16


def _taps(scheme, deriv, side, k):
    """Exact taps (j, l, c) of the edge row (dx = 1) on side 0 (buffer points on the left) or 1 (right)."""
    pos = 0 if side == 0 else S - 1
    kL, kR = (k, 0) if side == 0 else (0, k)
    return [(j, l, Fraction(c).limit_denominator(1000)) for j, l, c in oracle.taps(2, scheme, deriv, pos, S, 1, kL,
                                                                                     kR, 1.0)]


def _moment(taps, p, q):
    return sum(c * Fraction(j) ** p * Fraction(-l) ** q for j, l, c in taps) / (factorial(p) * factorial(q))


ROWS = [  # scheme, d, a (order of the row), printed leading terms {(p, q): |coefficient| / k^q}
    (W.AT_SPACE2, 1, 2, {(1, 1): Fraction(1, 4), (3, 0): Fraction(5, 12)}),
    (W.AT_SPACE2, 2, 2, {(2, 1): Fraction(1, 3), (4, 0): Fraction(13, 12)}),
    (W.AT_SPACE1, 2, 1, {(1, 1): Fraction(1, 2), (3, 0): Fraction(1, 2)}),
]


@pytest.mark.parametrize("scheme,d,a,lead", ROWS)
@pytest.mark.parametrize("side", [0, 1])
@pytest.mark.parametrize("k", [1, 2, 3])
def test_rows_satisfy_eq_cond_and_have_the_printed_leading_terms(scheme, d, a, lead, side, k):
    taps = _taps(scheme, d, side, k)
    for p in range(d + a + 1):
        for q in range((d + a - p + 1) // 2 + 1):
            if p + 2 * q >= d + a:
                continue
            assert _moment(taps, p, q) == (1 if (p, q) == (d, 0) else 0), (p, q)
    for (p, q), c in lead.items():
        assert abs(_moment(taps, p, q)) == c * k ** q, (p, q)
    # the asynchronous row (0, 1) cancels: the coefficients on each side of the PE boundary sum to zero, so the
    # edge row does not see a jump across the boundary
    assert sum(c for j, l, c in taps if l == 0) == 0 and sum(c for j, l, c in taps if l > 0) == 0


@pytest.mark.parametrize("scheme,d", [(W.AT_SPACE2, 1), (W.AT_SPACE2, 2), (W.AT_SPACE1, 2)])
def test_right_rows_mirror_the_left_rows(scheme, d):
    left = {(j, l): c for j, l, c in _taps(scheme, d, 0, 2)}
    right = {(-j, l): c * (-1) ** d for j, l, c in _taps(scheme, d, 1, 2)}
    assert left == right


def test_uniform_delay_example1_is_the_right_122a_row():
    """Eq. "ex1-1": (-3 U_{i-1} + 3 U_i - U_{i+1}^{n-k} + U_{i+2}^{n-k}) / (4 dx)."""
    want = {(-1, 0): Fraction(-3, 4), (0, 0): Fraction(3, 4), (1, 2): Fraction(-1, 4), (2, 2): Fraction(1, 4)}
    assert {(j, l): c for j, l, c in _taps(W.AT_SPACE2, 1, 1, 2)} == want


def test_rows_are_used_only_for_delayed_sides():
    for scheme, d in ((W.AT_SPACE2, 1), (W.AT_SPACE2, 2), (W.AT_SPACE1, 2)):
        cd = {(1, 0): Fraction(1, 2), (-1, 0): Fraction(-1, 2)} if d == 1 else \
             {(1, 0): Fraction(1), (0, 0): Fraction(-2), (-1, 0): Fraction(1)}
        assert {(j, l): c for j, l, c in _taps(scheme, d, 0, 0)} == cd


def _slope(ns, errs):
    return float(np.polyfit(np.log(ns), np.log(errs), 1)[0])


@pytest.mark.parametrize("case", [2, 3])
def test_cases_2_and_3_converge_at_second_order(case):
    """Fig. "at-prob-all" (a), (b): slope -2 without delays (p_0 = 1) and, asymptotically, with p_0 = 0.7."""
    ns = (64, 128, 256, 512)
    for probs, lo in (((1.0, 0.0, 0.0), 0), ((0.7, 0.2, 0.1), 2)):
        errs = []
        for n in ns:
            spec = W.paper_case(case, n, 300, probs)
            steps = W.steps_to(spec, 0.1)
            cfg = oracle.Config(spec)
            u, _, _ = oracle.run(cfg, steps, want_log=False, threads=4)
            errs.append(oracle.error_stats(cfg, u, steps)["rms"])
        assert abs(_slope(ns[lo:], errs[lo:]) + 2.0) < (0.1 if lo == 0 else 0.3), (probs, errs)


@pytest.mark.parametrize("case", [2, 3])
def test_cases_2_and_3_asynchronous_error_is_linear_in_the_mean_delay(case):
    """The leading asynchronous terms of (2,1,2), (1,2,2)a and (2,2,2)a are linear in k (tables'
    leading-term column), so (E - E_s)/E_s is proportional to E[k] = (L - 1)/2 for p_k = 1/L."""
    from test_sweep_pins import _sweep
    Ls = (2, 3, 4, 5)
    res = _sweep(*W.moment_members(case, Ls, range(300, 312)))
    ratio = np.array([(res[L][0] - res[L][1]) / res[L][1] / ((L - 1) / 2.0) for L in Ls])
    assert np.all(ratio > 0) and np.ptp(ratio) <= 0.15 * ratio.max(), ratio


@pytest.mark.parametrize("scheme,c", [(W.AT_SPACE2, 1.0), (W.AT_SPACE1, 0.0)])
def test_adjoint_of_the_space_expanded_rows_matches_central_differences(scheme, c):
    spec, _ = W.wl_1d(64, 8, 2, 3, 0, 44, (1, 2, 3), scheme=scheme, c=c)
    cfg = oracle.Config(spec)
    rng = np.random.default_rng(9)
    u0 = oracle.initial(cfg)
    tgt = 0.5 * u0 + 0.1 * rng.standard_normal(cfg.shape)
    nsteps = 50

    def J(u, alpha=spec["alpha"]):
        sp = dict(spec)
        sp["alpha"] = alpha
        uu, _, _ = oracle.run(oracle.Config(sp), nsteps, want_log=False, u0=u)
        return 0.5 * float(np.sum((uu - tgt) ** 2))

    Jo, g, ga = oracle.adjoint(cfg, nsteps, tgt)
    assert Jo == pytest.approx(J(u0), rel=1e-14)
    v = rng.standard_normal(cfg.shape)
    assert float(np.sum(g * v)) == pytest.approx((J(u0 + 1e-3 * v) - J(u0 - 1e-3 * v)) / 2e-3, rel=1e-8)
    a0, h = spec["alpha"], 1e-3 * spec["alpha"]
    d1 = (J(u0, a0 + h) - J(u0, a0 - h)) / (2 * h)
    d2 = (J(u0, a0 + h / 2) - J(u0, a0 - h / 2)) / h
    assert ga == pytest.approx((4 * d2 - d1) / 3, rel=1e-6)
