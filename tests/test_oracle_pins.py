"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU needed).

Each test checks the oracle against something other than itself: an independent implementation
(numpy's Philox), the Taylor-moment conditions of Eq. "cond", printed leading truncation terms,
closed-form discrete solutions, the PDE itself, finite differences, and the convergence slopes
reported in Sec. 5.2.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import workloads as W


# ----------------------------------------------------------------------------- Philox
def _philox_generic(ctr, key, w, M, Wc, rounds=10):
    """Philox round function (Salmon et al., SC'11) for any word width w."""
    mask = (1 << w) - 1
    c, k = list(ctr), list(key)
    for _ in range(rounds):
        p0, p1 = M[0] * c[0], M[1] * c[2]
        hi0, lo0, hi1, lo1 = p0 >> w, p0 & mask, p1 >> w, p1 & mask
        c = [hi1 ^ c[1] ^ k[0], lo1, hi0 ^ c[3] ^ k[1], lo0]
        k = [(k[0] + Wc[0]) & mask, (k[1] + Wc[1]) & mask]
    return c


M64 = (0xD2E7470EE14C6C93, 0xCA5A826395121157)
W64 = (0x9E3779B97F4A7C15, 0xBB67AE8584CAA73B)
M32 = (0xD2511F53, 0xCD9E8D57)
W32 = (0x9E3779B9, 0xBB67AE85)


def test_generic_philox_matches_numpy_4x64():
    # numpy's Philox is an independent implementation of Philox4x64-10; it increments the counter
    # before producing a block, so counter c yields the block of c + 1.
    for ctr, key in [([0, 0, 0, 0], [0, 0]), ([5, 7, 9, 11], [123, 456]),
                     ([2 ** 64 - 3, 1, 2, 3], [2 ** 63 + 5, 77])]:
        bg = np.random.Philox(counter=np.array(ctr, dtype=np.uint64), key=np.array(key, dtype=np.uint64))
        got = [int(v) for v in bg.random_raw(4)]
        nxt = list(ctr)
        nxt[0] = (nxt[0] + 1) % 2 ** 64
        assert got == _philox_generic(nxt, key, 64, M64, W64)


@pytest.mark.parametrize("ctr,key", [([0, 0, 0, 0], [0, 0]), ([1, 2, 3, 4], [5, 6]),
                                     ([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2), ([999, 3071, 0, 0], [3, 0])])
def test_oracle_philox4x32_matches_generic(ctr, key):
    assert oracle.philox4x32_10(ctr, key) == _philox_generic(ctr, key, 32, M32, W32)


def _kat_rows():
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "philox4x32_10_kat.txt")
    rows = []
    for line in open(path):
        line = line.strip()
        if line and not line.startswith("#"):
            v = [int(t, 16) for t in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_oracle_philox4x32_reproduces_the_published_known_answers():
    """The authors' known-answer vectors of Philox4x32-10 (tests/golden/philox4x32_10_kat.txt): this pins the
    oracle's 32-bit multipliers and key increments against values computed outside this repository."""
    rows = _kat_rows()
    assert len(rows) == 3
    for ctr, key, want in rows:
        assert oracle.philox4x32_10(ctr, key) == want
        assert _philox_generic(ctr, key, 32, M32, W32) == want


def test_delay_word_is_counter_keyed():
    seed, n, b = 0x1234_5678_9ABC_DEF0, 17, 42
    x0 = _philox_generic([n, b, 0, 0], [seed & 0xFFFFFFFF, seed >> 32], 32, M32, W32)[0]
    for L in (2, 3, 4):
        assert oracle.delay_raw(seed, n, b, L) == (x0 * L) >> 32


# ------------------------------------------------------------------------- delay bins
def _draws(L, count, thresholds=None, seed=7):
    return np.array([oracle.delay_raw(seed, n // 64, n % 64, L, thresholds) for n in range(count)])


@pytest.mark.parametrize("L", [2, 3, 4])
def test_uniform_delays_chi2(L):
    k = _draws(L, 30000)
    assert k.min() >= 0 and k.max() <= L - 1
    obs = np.bincount(k, minlength=L)
    exp = len(k) / L
    chi2 = float(((obs - exp) ** 2 / exp).sum())
    # chi-square with L-1 dof: P(chi2 > 25) < 1e-4 for dof <= 3
    assert chi2 < 25.0, (obs, chi2)


def test_binned_delays_follow_probabilities():
    p = [0.5, 0.3, 0.2]  # the bins of Fig. "at-sol1"
    thr = W.thresholds_from_probs(p)
    k = _draws(3, 30000, thr)
    freq = np.bincount(k, minlength=3) / len(k)
    for m in range(3):
        sigma = math.sqrt(p[m] * (1 - p[m]) / len(k))
        assert abs(freq[m] - p[m]) < 5 * sigma
    assert set(_draws(3, 2000, W.thresholds_from_probs([1.0, 0.0, 0.0]))) == {0}
    assert set(_draws(3, 2000, W.thresholds_from_probs([0.0, 0.0, 1.0]))) == {2}


def test_delay_clamp_before_level_zero():
    # levels n-k .. n-k-(T-1) must exist
    assert oracle.delay_effective(2, 0, 3) == 0
    assert oracle.delay_effective(2, 2, 3) == 0
    assert oracle.delay_effective(2, 3, 3) == 1
    assert oracle.delay_effective(2, 4, 3) == 2
    assert oracle.delay_effective(3, 1, 1) == 1
    assert oracle.delay_effective(0, 100, 3) == 0


# ------------------------------------------------------------------- stencil moments
def _frac(c):
    return Fraction(c).limit_denominator(10 ** 7)


def _moment(taps, p, q):
    return sum(_frac(c) * Fraction(j) ** p * Fraction(-l) ** q for j, l, c in taps)


def _cond_rows(d, a, r=2):
    return [(p, q) for p in range(d + a + 1) for q in range(d + a + 1) if p + r * q < d + a]


CASES = []
for order in (2, 4, 6):
    h = order // 2
    S = 8
    for pos in list(range(h)) + list(range(S - h, S)):
        for k in range(4):
            CASES.append((order, pos, S, k))


@pytest.mark.parametrize("order,pos,S,k", CASES)
@pytest.mark.parametrize("deriv", [1, 2])
def test_at_taps_satisfy_taylor_conditions(order, pos, S, k, deriv):
    """Eq. "cond" with dt ~ dx^2 (r = 2): every (p,q) with p + 2q < d + a has zero moment except the
    (d,0) row, which equals d!.  dx = 1 here; each row's dx^p dt^q factor is common to the row."""
    left, right = (k, 0) if pos < order // 2 else (0, k)
    taps = oracle.taps(order, oracle.AT, deriv, pos, S, 1, left, right, 1.0)
    assert any(l > 0 for _, l, _ in taps) == (k > 0)
    for p, q in _cond_rows(deriv, order):
        want = math.factorial(deriv) if (p, q) == (deriv, 0) else 0
        assert _moment(taps, p, q) == want, (p, q)


@pytest.mark.parametrize("order", [2, 4, 6])
@pytest.mark.parametrize("deriv", [1, 2])
def test_at_taps_reduce_to_central_difference_at_k0(order, deriv):
    sync = oracle.taps(order, oracle.SYNC, deriv, 0, 8, 1, 0, 0, 1.0)
    at0 = oracle.taps(order, oracle.AT, deriv, 0, 8, 1, 0, 0, 1.0)
    assert sync == at0
    assert all(l == 0 for _, l, _ in sync)
    # the central differences themselves: exact up to order a on polynomials
    for p in range(order + deriv):
        want = math.factorial(deriv) if p == deriv else 0
        assert _moment(sync, p, 0) == want


@pytest.mark.parametrize("order", [2, 4, 6])
def test_standard_scheme_read_asynchronously_breaks_a_condition(order):
    """Eq. "general_deriv_async": the standard stencil at delayed levels violates the (0,1) row for d=2,
    which is why its accuracy drops (Sec. 2)."""
    taps = oracle.taps(order, oracle.ASYNC_STD, 2, 0, 8, 1, 2, 0, 1.0)
    assert _moment(taps, 0, 1) != 0


# ------------------------------------------------------------- printed truncation terms
def _history_value(x, t, omega=1.3, kap=1.0):
    return np.sin(kap * x - omega * t + 0.4)


@pytest.mark.parametrize("side", ["left", "right"])
@pytest.mark.parametrize("k", [1, 2, 3])
def test_printed_leading_async_terms(side, k):
    """Async minus sync derivative at an edge point, on exact smooth data, against the leading terms
    of the tables: (2,2,2)b: (1/2) k(k+1) u_tt dt^2/dx^2; (2,4,2): (5/24) k(k+1)(k+2) u_ttt dt^3/dx^2
    (signs from the extrapolation remainder: the delayed halo is low by u^(T) prod(k+m) dt^T / T!)."""
    dx, dt, omega = 1e-3, 2e-4, 1.3
    S = 16
    utt = lambda: -omega ** 2 * _history_value(0.0, 0.0)  # d2/dt2 at x_i, t_n
    uttt = lambda: omega ** 3 * np.cos(0.4)                # d3/dt3 at x_i, t_n
    cases = [(2, 0 if side == "left" else S - 1, 0.5 * k * (k + 1) * utt() * dt ** 2 / dx ** 2),
             (4, 0 if side == "left" else S - 1, (5.0 / 24.0) * k * (k + 1) * (k + 2) * uttt() * dt ** 3 / dx ** 2),
             (4, 1 if side == "left" else S - 2, -(1.0 / 72.0) * k * (k + 1) * (k + 2) * uttt() * dt ** 3 / dx ** 2)]
    for order, pos, lead in cases:
        kL, kR = (k, 0) if side == "left" else (0, k)
        def evaluate(scheme):
            taps = oracle.taps(order, scheme, 2, pos, S, 1, kL, kR, dx)
            return sum(c * _history_value(j * dx, -l * dt, omega) for j, l, c in taps)
        diff = evaluate(oracle.AT) - evaluate(oracle.SYNC)
        # the halo is extrapolated low by the remainder, so the D2 error has sign -sign(tap weight)
        assert diff == pytest.approx(-lead, rel=1e-2), (order, pos)


# ------------------------------------------------------------------- step wiring
def _smooth_history(cfg, nlev, dt):
    return [oracle.analytic(cfg, -m * dt) for m in range(nlev)]


def test_step_applies_each_side_delay_to_its_own_buffer_points_1d():
    spec, _ = W.wl_1d(96, 4, 4, 3, 0, 5, (1, 2))
    cfg = oracle.Config(spec)
    S, h = 24, 2
    lev = _smooth_history(cfg, 6, spec["dt"])
    base = oracle.step(cfg, lev, np.zeros(8, np.int32))
    for side in range(8):
        keff = np.zeros(8, np.int32)
        keff[side] = 2
        moved = np.nonzero(oracle.step(cfg, lev, keff) != base)[0]
        p, s = divmod(side, 2)
        want = np.arange(p * S, p * S + h) if s == 0 else np.arange((p + 1) * S - h, (p + 1) * S)
        assert np.array_equal(moved, want), (side, moved)


def test_step_applies_each_face_delay_to_its_own_layer_3d():
    spec, _ = W.wl_3d([8, 12, 16], [2, 3, 4], 2, 3, 0, 6)
    cfg = oracle.Config(spec)
    lev = _smooth_history(cfg, 5, spec["dt"])
    nb = cfg.num_sides
    assert nb == 6 * 24
    base = oracle.step(cfg, lev, np.zeros(nb, np.int32))
    rng = np.random.default_rng(0)
    for side in rng.choice(nb, 12, replace=False):
        keff = np.zeros(nb, np.int32)
        keff[side] = 1
        moved = oracle.step(cfg, lev, keff) != base
        pe, face = divmod(int(side), 6)
        a, s = divmod(face, 2)
        Sx, Sy, Sz = 4, 4, 4
        px, py, pz = pe % 2, (pe // 2) % 3, pe // 6
        want = np.zeros(cfg.shape, bool)  # shape (z, y, x)
        zs, ys, xs = slice(pz * Sz, (pz + 1) * Sz), slice(py * Sy, (py + 1) * Sy), slice(px * Sx, (px + 1) * Sx)
        lo = [px * Sx, py * Sy, pz * Sz][a]
        hi = lo + 4 - 1
        layer = lo if s == 0 else hi
        sl = [xs, ys, zs]
        sl[a] = slice(layer, layer + 1)
        want[sl[2], sl[1], sl[0]] = True
        assert np.array_equal(moved, want), side


# ------------------------------------------------------- synchronous run: closed forms
def _symbols(order, kap, dx):
    th = kap * dx
    if order == 2:
        return np.sin(th) / dx, (2 * np.cos(th) - 2) / dx ** 2
    return (8 * np.sin(th) - np.sin(2 * th)) / (6 * dx), (-2 * np.cos(2 * th) + 32 * np.cos(th) - 30) / (12 * dx ** 2)


def _exact_discrete_1d(spec, nsteps):
    n = spec["n"][0]
    dx = 2 * np.pi / n
    x = np.arange(n) * dx
    u = np.zeros(n)
    for A, ph, kap in zip(spec["amp"][0], spec["phase"][0], spec["kappa"][0]):
        s1, s2 = _symbols(spec["order"], kap, dx)
        G = 1 + spec["dt"] * (-spec["c"][0] * 1j * s1 + spec["alpha"] * s2)
        u += A * np.imag(G ** nsteps * np.exp(1j * (kap * x + ph)))
    return u


@pytest.mark.parametrize("order", [2, 4])
def test_sync_run_matches_exact_discrete_solution_1d(order):
    spec, _ = W.wl_1d(120, 5, order, 3, 0, 11, (1, 2, 5, 9), scheme=W.SYNC)
    u, log, _ = oracle.run(oracle.Config(spec), 300)
    ref = _exact_discrete_1d(spec, 300)
    assert np.abs(u - ref).max() < 1e-12 * np.abs(ref).max()
    assert not log.any()


def _exact_discrete_3d(spec, nsteps):
    n = spec["n"]
    axes = [np.arange(n[a]) * 2 * np.pi / n[a] for a in range(3)]
    terms = []  # per axis: list of (coef, wavenumber, phase-field)
    for a in range(3):
        lst = []
        for A, ph, kap in zip(spec["amp"][a], spec["phase"][a], spec["kappa"][a]):
            for s in (1, -1):
                lst.append((s * A / 2j, s * kap, np.exp(1j * s * (kap * axes[a] + ph))))
        terms.append(lst)
    out = np.zeros((n[2], n[1], n[0]), complex)
    for cx, kx, ex in terms[0]:
        for cy, ky, ey in terms[1]:
            for cz, kz, ez in terms[2]:
                lam = 0
                for a, kk in enumerate((kx, ky, kz)):
                    s1, s2 = _symbols(spec["order"], kk, 2 * np.pi / n[a])
                    lam = lam + (-spec["c"][a] * 1j * s1 + spec["alpha"] * s2)
                G = 1 + spec["dt"] * lam
                out += cx * cy * cz * G ** nsteps * ez[:, None, None] * ey[None, :, None] * ex[None, None, :]
    return out.real


@pytest.mark.parametrize("order", [2, 4])
def test_sync_run_matches_exact_discrete_solution_3d(order):
    spec, _ = W.wl_3d([12, 16, 20], [2, 2, 2], order, 3, 0, 12, scheme=W.SYNC, c=(1.0, -0.5, 0.25))
    u, _, _ = oracle.run(oracle.Config(spec), 40)
    ref = _exact_discrete_3d(spec, 40)
    assert np.abs(u - ref).max() < 1e-12 * np.abs(ref).max()


def test_initial_condition_and_analytic_solution_satisfy_the_pde():
    spec, _ = W.wl_1d(256, 8, 2, 3, 0, 13, (1, 2, 3, 4))
    spec["c"] = [0.7]
    cfg = oracle.Config(spec)
    assert np.array_equal(oracle.initial(cfg), oracle.analytic(cfg, 0.0))
    t, h = 0.3, 1e-4
    u = oracle.analytic(cfg, t)
    ut = (oracle.analytic(cfg, t + h) - oracle.analytic(cfg, t - h)) / (2 * h)
    k = np.fft.fftfreq(256, d=1.0 / 256)
    uh = np.fft.fft(u)
    ux = np.fft.ifft(1j * k * uh).real
    uxx = np.fft.ifft(-(k ** 2) * uh).real
    resid = ut + 0.7 * ux - spec["alpha"] * uxx
    assert np.abs(resid).max() < 1e-6 * np.abs(uxx).max()


def test_analytic_3d_is_product_of_1d_solutions_and_satisfies_pde():
    spec, _ = W.wl_3d([16, 20, 24], [2, 2, 2], 2, 3, 0, 14, c=(0.3, -0.2, 0.9))
    cfg = oracle.Config(spec)
    t, h = 0.2, 1e-4
    u = oracle.analytic(cfg, t)
    ut = (oracle.analytic(cfg, t + h) - oracle.analytic(cfg, t - h)) / (2 * h)
    rhs = np.zeros_like(u)
    for a, ax in zip(range(3), (2, 1, 0)):
        n = spec["n"][a]
        k = np.fft.fftfreq(n, d=1.0 / n)
        shape = [1, 1, 1]
        shape[ax] = n
        kk = k.reshape(shape)
        uh = np.fft.fft(u, axis=ax)
        rhs += -spec["c"][a] * np.fft.ifft(1j * kk * uh, axis=ax).real + spec["alpha"] * np.fft.ifft(-(kk ** 2) * uh, axis=ax).real
    assert np.abs(ut - rhs).max() < 1e-6 * np.abs(rhs).max()


def test_sync_run_converges_to_analytic_at_second_order():
    errs = []
    for n in (64, 128, 256):
        spec, _ = W.wl_1d(n, 4, 2, 3, 0, 21, (1, 2, 3), scheme=W.SYNC)
        steps = int(round(0.25 / spec["dt"]))
        cfg = oracle.Config(spec)
        u, _, _ = oracle.run(cfg, steps, want_log=False)
        errs.append(oracle.error_stats(cfg, u, steps)["rms"])
    slopes = np.diff(np.log(errs)) / np.log(2)
    assert np.all(np.abs(slopes + 2) < 0.15), slopes


# -------------------------------------------------------- statistical order gates
def _async_minus_sync(n, P, order, scheme, seeds, tfinal=0.2):
    out = []
    for seed in seeds:
        spec, _ = W.wl_1d(n, P, order, 3, 0, seed, (3, 4, 5), scheme=scheme)
        steps = int(round(tfinal / spec["dt"]))
        ua, _, _ = oracle.run(oracle.Config(spec), steps, want_log=False)
        spec["scheme"] = W.SYNC
        us, _, _ = oracle.run(oracle.Config(spec), steps, want_log=False)
        out.append(np.sqrt(np.mean((ua - us) ** 2)))
    return float(np.mean(out))  # ensemble mean over delay realizations


def _slope(ns, errs):
    return float(np.polyfit(np.log(ns), np.log(errs), 1)[0])


@pytest.mark.parametrize("order,weak,strong", [(2, -2.0, -3.0), (4, -4.0, -5.0)])
def test_at_schemes_keep_design_order(order, weak, strong):
    """Eq. "aveE_scaling": the asynchronous error of an order-a AT scheme scales as dx^a at fixed P/N
    (weak scaling) and as dx^(a+1) at fixed P (strong scaling); Sec. 5.2 reports -2 and -3 for
    Case 1."""
    ns, seeds = (64, 128, 256), (101, 102, 103)
    e_weak = [_async_minus_sync(n, n // 16, order, W.AT, seeds) for n in ns]
    e_strong = [_async_minus_sync(n, 4, order, W.AT, seeds) for n in ns]
    assert abs(_slope(ns, e_weak) - weak) < 0.6, e_weak
    assert abs(_slope(ns, e_strong) - strong) < 0.4, e_strong


@pytest.mark.parametrize("order", [2, 4])
def test_standard_scheme_degrades_to_first_order(order):
    """Sec. 5.2, Fig. "at-ord4-async": the standard scheme run asynchronously converges at slope -1."""
    ns = (64, 128, 256, 512)
    e = [_async_minus_sync(n, 4, order, W.ASYNC_STD, (101, 102, 103)) for n in ns]
    assert abs(_slope(ns, e) + 1.0) < 0.25, e


# ------------------------------------------------------------------------ statistics
def test_error_stats_definitions():
    spec, _ = W.wl_1d(64, 4, 4, 3, 0, 31, (1, 2))
    cfg = oracle.Config(spec)
    rng = np.random.default_rng(3)
    u = rng.standard_normal(64)
    st = oracle.error_stats(cfg, u, 7)
    e = u - oracle.analytic(cfg, 7 * spec["dt"])
    pos = np.arange(64) % 16
    edge = (pos < 2) | (pos >= 14)
    assert st["rms"] == pytest.approx(np.sqrt(np.mean(e ** 2)), rel=1e-14)
    assert st["max_abs"] == pytest.approx(np.abs(e).max(), rel=1e-15)
    assert st["mean_abs"] == pytest.approx(np.abs(e).mean(), rel=1e-14)
    assert st["mean"] == pytest.approx(e.mean(), rel=1e-12, abs=1e-15)
    assert st["rms_B"] == pytest.approx(np.sqrt(np.mean(e[edge] ** 2)), rel=1e-14)
    assert st["rms_I"] == pytest.approx(np.sqrt(np.mean(e[~edge] ** 2)), rel=1e-14)
    assert (st["n_I"], st["n_B"]) == (48, 16)


@pytest.mark.parametrize("dim", [1, 3])
def test_error_stats_closed_forms(dim):
    """Sec. 4's averages on fields whose answers are closed forms: the analytic solution plus a constant delta
    (every average |delta|, the mean delta), plus delta on I_B only (rms_I = 0, rms = |delta| sqrt(|I_B|/|I|)),
    and the sizes of I_I and I_B from the PE geometry: prod over split axes of P (S - 2h) interior points."""
    if dim == 1:
        spec, _ = W.wl_1d(96, 6, 4, 3, 0, 33, (1, 2))
    else:
        spec, _ = W.wl_3d([24, 16, 16], [2, 2, 2], 4, 3, 0, 34)
    cfg = oracle.Config(spec)
    h = spec["order"] // 2
    n_int = 1
    for n, P in zip(spec["n"], spec["pe"]):
        n_int *= P * (n // P - 2 * h) if P > 1 else n
    N = int(np.prod(spec["n"]))
    t = 5 * spec["dt"]
    ua = oracle.analytic(cfg, t)
    delta = -3.0e-3
    st = oracle.error_stats(cfg, ua + delta, 5)
    assert (st["n_I"], st["n_B"]) == (n_int, N - n_int)
    for key in ("rms", "max_abs", "mean_abs", "rms_I", "rms_B"):
        assert st[key] == pytest.approx(abs(delta), rel=1e-12), key
    assert st["mean"] == pytest.approx(delta, rel=1e-12)
    assert st["ua_rms"] == pytest.approx(np.sqrt(np.mean(ua ** 2)), rel=1e-14)
    # delta on the boundary points only: find them as the points a forced delay can reach (within h of a face)
    edge = np.zeros(cfg.shape, dtype=bool)
    for a, (n, P) in enumerate(zip(spec["n"], spec["pe"])):
        if P < 2:
            continue
        pos = np.arange(n) % (n // P)
        e1 = (pos < h) | (pos >= n // P - h)
        edge |= e1.reshape([-1 if b == a else 1 for b in range(dim)][::-1])
    st = oracle.error_stats(cfg, ua + delta * edge, 5)
    assert st["rms_I"] <= 1e-15 and st["max_abs"] == pytest.approx(abs(delta), rel=1e-12)
    assert st["rms_B"] == pytest.approx(abs(delta), rel=1e-12)
    assert st["rms"] == pytest.approx(abs(delta) * np.sqrt((N - n_int) / N), rel=1e-12)


@pytest.mark.parametrize("case", ["at_o4", "at_o6", "std_o4", "space2_o2", "space1_o2", "burgers_o4", "burgers_ab2",
                                  "case4_ab2", "case5_ab3"])
def test_sampled_run_equals_the_full_run(case):
    """run_samples steps each sampled cell only inside its domain of dependence (reach max(h, 3) per step); it must
    give the full run's values bit for bit, including cells on PE edges and next to the periodic wrap, for forward
    Euler and for Adams-Bashforth (analytic pre-history, and Burgers' Euler start)."""
    if case.startswith("burgers"):
        spec = W.paper_case(6, 256, 13, (0.4, 0.3, 0.3))
        if case == "burgers_o4":
            spec["tsteps"] = 1
    elif case.startswith("case"):
        spec = W.paper_case(int(case[4]), 384, 15, (0.4, 0.3, 0.3))
    else:
        order = int(case[-1])
        scheme = {"at": W.AT, "std": W.ASYNC_STD, "space2": W.AT_SPACE2, "space1": W.AT_SPACE1}[case.split("_")[0]]
        c = 0.0 if scheme == W.AT_SPACE1 else 1.0
        spec, _ = W.wl_1d(768, 12, order, 4, 0, 14, range(1, 6), scheme=scheme, c=c,
                          r_alpha=0.02 if order == 6 else 0.1)
    cfg = oracle.Config(spec)
    n = spec["n"][0]
    S = n // spec["pe"][0]
    steps = 120
    full, _, _ = oracle.run(cfg, steps, want_log=False)
    pos = [0, 1, S - 1, S, 2 * S + 3, n // 2, n - 2, n - 1]
    assert np.array_equal(oracle.run_samples(cfg, steps, pos), full.reshape(-1)[pos])


# ----------------------------------------------------------------------------- adjoint
def _J(cfg, nsteps, tgt, u0):
    u, _, _ = oracle.run(cfg, nsteps, want_log=False, u0=u0)
    return 0.5 * float(np.sum((u - tgt) ** 2))


@pytest.mark.parametrize("dim", [1, 3])
def test_adjoint_matches_central_differences(dim):
    if dim == 1:
        spec, _ = W.wl_1d(64, 4, 4, 3, 0, 41, (1, 2, 3))
        nsteps = 60
    else:
        spec, _ = W.wl_3d([8, 8, 12], [2, 2, 3], 4, 3, 0, 42)
        nsteps = 12
    cfg = oracle.Config(spec)
    rng = np.random.default_rng(5)
    u0 = oracle.initial(cfg)
    tgt = u0 * 0.5 + 0.1 * rng.standard_normal(cfg.shape)
    J, g, ga = oracle.adjoint(cfg, nsteps, tgt)
    assert J == pytest.approx(_J(cfg, nsteps, tgt, u0), rel=1e-14)
    for _ in range(3):
        v = rng.standard_normal(cfg.shape)
        eps = 1e-3  # J is quadratic in u0: the central difference is exact up to rounding
        fd = (_J(cfg, nsteps, tgt, u0 + eps * v) - _J(cfg, nsteps, tgt, u0 - eps * v)) / (2 * eps)
        assert np.sum(g * v) == pytest.approx(fd, rel=1e-8)
    # alpha: Richardson-extrapolated central differences
    a0 = spec["alpha"]
    def Ja(a):
        s = dict(spec)
        s["alpha"] = a
        return _J(oracle.Config(s), nsteps, tgt, u0)
    h = 1e-3 * a0
    d1 = (Ja(a0 + h) - Ja(a0 - h)) / (2 * h)
    d2 = (Ja(a0 + h / 2) - Ja(a0 - h / 2)) / h
    fd = (4 * d2 - d1) / 3
    assert ga == pytest.approx(fd, rel=1e-6)


@pytest.mark.parametrize("order,tsteps", [(4, 2), (6, 3), (2, 3)])
def test_multistep_adjoint_matches_central_differences(order, tsteps):
    """The transposed Adams-Bashforth run (from a caller's field: Euler, AB2, then AB3) against central
    differences of the forward map in u0 (exact for the quadratic misfit) and in alpha (Richardson)."""
    spec, _ = W.wl_1d(128, 8, order, 3, 0, 71, (1, 2, 3), r_alpha=0.02, tsteps=tsteps)
    cfg = oracle.Config(spec)
    rng = np.random.default_rng(7)
    u0 = oracle.initial(cfg) + 0.01 * rng.standard_normal(cfg.shape)
    tgt = 0.5 * u0 + 0.1 * rng.standard_normal(cfg.shape)
    nsteps = 40
    J, g, ga = oracle.adjoint(cfg, nsteps, tgt, u0=u0)
    assert J == pytest.approx(_J(cfg, nsteps, tgt, u0), rel=1e-14)
    for _ in range(3):
        v = rng.standard_normal(cfg.shape)
        fd = (_J(cfg, nsteps, tgt, u0 + 1e-3 * v) - _J(cfg, nsteps, tgt, u0 - 1e-3 * v)) / 2e-3
        assert np.sum(g * v) == pytest.approx(fd, rel=1e-8)
    a0 = spec["alpha"]

    def Ja(a):
        s = dict(spec)
        s["alpha"] = a
        return _J(oracle.Config(s), nsteps, tgt, u0)
    h = 1e-3 * a0
    d1 = (Ja(a0 + h) - Ja(a0 - h)) / (2 * h)
    d2 = (Ja(a0 + h / 2) - Ja(a0 - h / 2)) / h
    assert ga == pytest.approx((4 * d2 - d1) / 3, rel=1e-6)
    with pytest.raises(RuntimeError):  # from Eq. "IC" the pre-history depends on alpha: not covered
        oracle.adjoint(cfg, nsteps, tgt)


def test_printed_leading_async_term_of_the_sixth_order_row():
    """(2,6,2): (49/864) k(k+1)(k+2)(k+3) u^(0,4) dt^4/dx^2 (the left row read with U_{i-3}); sign from the
    four-level extrapolation remainder, which leaves the halo low by u_tttt prod(k+m) dt^4 / 4!."""
    dx, dt, omega = 3e-3, 1e-3, 1.3
    u4 = omega ** 4 * np.sin(0.4)  # d4/dt4 of sin(x - omega t + 0.4) at (0, 0)
    for k in (1, 2, 3):
        for side, pos, kl, kr in (("left", 0, k, 0), ("right", 15, 0, k)):
            def evaluate(scheme):
                taps = oracle.taps(6, scheme, 2, pos, 16, 1, kl, kr, dx)
                return sum(c * _history_value(j * dx, -l * dt, omega) for j, l, c in taps)
            lead = (49.0 / 864.0) * k * (k + 1) * (k + 2) * (k + 3) * u4 * dt ** 4 / dx ** 2
            # next term: the buffer cells sit 1..3 dx from x_i, a relative O(dx cot 0.4) ~ 2 % shift
            assert evaluate(oracle.AT) - evaluate(oracle.SYNC) == pytest.approx(-lead, rel=5e-2), (k, side)


@pytest.mark.parametrize("tsteps,order", [(2, 4), (3, 6), (2, 2)])
def test_multistep_sync_run_matches_its_fourier_recurrence(tsteps, order):
    """Adams-Bashforth (Eq. "time_ab2"; three levels: 23/12, -16/12, 5/12) on one Fourier mode: the amplitude obeys
    a_{n+1} = a_n + dt sum_m beta_m lam a_{n-m}, lam the symbol of the central stencils, with the levels before
    t = 0 taken from the analytic solution a(t) = exp((-alpha kappa^2 - i c kappa) t) a_0."""
    spec, _ = W.wl_1d(60, 5, order, 3, 0, 15, (2, 5), scheme=W.SYNC, tsteps=tsteps, r_alpha=0.05)
    u, _, _ = oracle.run(oracle.Config(spec), 150)
    n = spec["n"][0]
    dx, dt, c, al = 2 * np.pi / n, spec["dt"], spec["c"][0], spec["alpha"]
    beta = {2: [1.5, -0.5], 3: [23 / 12, -16 / 12, 5 / 12]}[tsteps]
    x = np.arange(n) * dx
    ref = np.zeros(n)
    for A, ph, kap in zip(spec["amp"][0], spec["phase"][0], spec["kappa"][0]):
        th = kap * dx
        if order == 2:
            s1, s2 = np.sin(th) / dx, (2 * np.cos(th) - 2) / dx ** 2
        elif order == 4:
            s1, s2 = _symbols(4, kap, dx)
        else:
            s1 = (45 * 2 * np.sin(th) - 9 * 2 * np.sin(2 * th) + 2 * np.sin(3 * th)) / (60 * dx)
            s2 = (2 * 2 * np.cos(3 * th) - 27 * 2 * np.cos(2 * th) + 270 * 2 * np.cos(th) - 490) / (180 * dx ** 2)
        lam = -c * 1j * s1 + al * s2
        mu = -al * kap ** 2 - 1j * c * kap
        f_hist = [lam * np.exp(mu * (-m * dt)) for m in range(1, tsteps)]  # f^{-1}, f^{-2}
        a = 1.0 + 0j
        hist = [lam * a] + f_hist
        for _ in range(150):
            a = a + dt * sum(b * fm for b, fm in zip(beta, hist))
            hist = [lam * a] + hist[:-1]
        ref += A * np.imag(a * np.exp(1j * (kap * x + ph)))
    assert np.abs(u - ref).max() < 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("case,ns,slope", [(4, (64, 128, 256), -4.0), (5, (96, 128, 192), -6.0)])
def test_paper_cases_4_and_5_keep_their_design_order(case, ns, slope):
    """Fig. "at-prob-all" (c), (d): with the time-expanded AT stencils and AB2 / AB3 the error against the
    analytic solution falls at slope -4 (Case 4) and -6 (Case 5) whether the PEs run synchronously
    (p_0 = 1) or with delays (p_0 = 0.7, 0)."""
    for probs in ((1.0, 0.0, 0.0), (0.7, 0.2, 0.1), (0.0, 0.5, 0.5)):
        errs = []
        for n in ns:
            spec = W.paper_case(case, n, 300, probs)
            steps = int(round(0.1 / spec["dt"]))
            cfg = oracle.Config(spec)
            u, _, _ = oracle.run(cfg, steps, want_log=False, threads=4)
            errs.append(oracle.error_stats(cfg, u, steps)["rms"])
        assert abs(_slope(ns, errs) - slope) < 0.25, (probs, errs)
