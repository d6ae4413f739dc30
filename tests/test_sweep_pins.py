"""The oracle against the paper's scaling and delay-moment laws (Sec. 5.2, Eq. "aveE_scaling_gen2",
Eq. "aveE_scaling_gen_kmom", Eq. "aveE_scaling_gen_L", Figs. "at-ord2-procs" and "at-kmom"), on the member lists
the GPU sweeps run (workloads.scaling_members / moment_members).  CPU only.

Measures, per group of realizations (delay seeds): E and E_s, the ensemble means of the RMS error of the
asynchronous members and of their synchronous twins, and D, the mean over members of the mean |U - U_sync|
(the asynchronous part of the error on the same initial condition).
"""
import multiprocessing as mp
from concurrent.futures import ProcessPoolExecutor

import numpy as np
import pytest

import oracle
import workloads as W


def _run_one(args):
    spec, steps = args
    cfg = oracle.Config(spec)
    u, _, _ = oracle.run(cfg, steps, want_log=False, threads=1)
    return u, oracle.error_stats(cfg, u, steps)["rms"]


def _sweep(specs, steps, groups, twins):
    with ProcessPoolExecutor(8, mp_context=mp.get_context("spawn")) as ex:
        res = list(ex.map(_run_one, zip(specs, steps)))
    out = {}
    for g in sorted({groups[r] for r in range(len(specs)) if twins[r] >= 0}):
        idx = [r for r in range(len(specs)) if groups[r] == g and twins[r] >= 0]
        E = np.mean([res[r][1] for r in idx])
        Es = np.mean([res[twins[r]][1] for r in idx])
        D = np.mean([np.mean(np.abs(res[r][0] - res[twins[r]][0])) for r in idx])
        out[g] = (E, Es, D)
    return out


def _slope(x, y):
    return float(np.polyfit(np.log(x), np.log(y), 1)[0])


def test_case1_asynchronous_error_scales_with_p_and_n():
    """Eq. "aveE_scaling_gen2" for Case 1 ((1,2,2)b/(2,2,2)b, p_k = {0.2, 0.5, 0.3}): the asynchronous part of
    the error grows linearly with P at fixed N (Fig. "at-ord2-procs" (a), inset), falls as dx^3 at fixed P
    (strong scaling) and as dx^2 at fixed P/N (weak scaling)."""
    seeds = range(500, 506)
    Ps = (2, 4, 8, 16, 32)
    res = _sweep(*W.scaling_members(1, [(512, P) for P in Ps], seeds))
    assert abs(_slope(Ps, [res[i][2] for i in range(len(Ps))]) - 1.0) < 0.1
    ns = (128, 256, 512)
    res = _sweep(*W.scaling_members(1, [(n, 16) for n in ns], seeds))
    assert abs(_slope(ns, [res[i][2] for i in range(len(ns))]) + 3.0) < 0.3
    res = _sweep(*W.scaling_members(1, [(n, n // 16) for n in ns], seeds))
    assert abs(_slope(ns, [res[i][2] for i in range(len(ns))]) + 2.0) < 0.3


@pytest.mark.parametrize("case,Ls,law,spread", [
    (1, (2, 3, 4, 5), lambda L: (L * L - 1) / 3.0, 0.15),                        # <k^2> + <k>
    (4, (2, 3, 4), lambda L: (L ** 3 + 2 * L * L - L - 2) / 4.0, 0.05),          # <k^3> + 3<k^2> + 2<k>
])
def test_asynchronous_error_follows_the_delay_moments(case, Ls, law, spread):
    """Eq. "aveE_scaling_gen_L" (Fig. "at-kmom", N = 512, P = 16, p_k = 1/L): (E - E_s)/E_s is proportional to
    the delay-moment polynomial of the scheme -- (L^2 - 1)/3 = E[k(k+1)] for the second-order b rows, and
    (L^3 + 2L^2 - L - 2)/4 = E[k(k+1)(k+2)] for (1,4,2)/(2,4,2) (the printed polynomial repeats L^3; this is the
    moment it stands for).  Checked as a constant ratio across L, up to the next-order terms."""
    res = _sweep(*W.moment_members(case, Ls, range(300, 312)))
    ratio = np.array([(res[L][0] - res[L][1]) / res[L][1] / law(L) for L in Ls])
    assert np.all(np.sign(ratio) == np.sign(ratio[0]))
    assert np.ptp(ratio) <= spread * np.abs(ratio).max(), ratio
