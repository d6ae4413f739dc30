"""The paper's scaling and delay-moment sweeps (Sec. 5.2, Figs. "at-ord2-procs" and "at-kmom") on the GPU ensemble
engine: members with their own step counts, summary groups and synchronous twins in one persistent launch.

Checks: sampled members against the oracle (delays bit-exact, fields within 1e-12), the per-member twin
differences and the per-group summaries against their definitions on the GPU's own fields, and the laws the
oracle pins (tests/test_sweep_pins.py) measured from the device summaries with more realizations.
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


def _ensemble(specs, steps, groups, twins, log=False):
    from paper_1702_00496_gb300 import Ensemble
    ens = Ensemble(specs, steps, log=log, groups=groups, twins=twins)
    ens.run()
    per, grp = ens.stats()
    return ens, per, {g["key"]: g for g in grp}


def _slope(x, y):
    return float(np.polyfit(np.log(x), np.log(y), 1)[0])


def test_sweep_members_match_the_oracle_and_their_summaries():
    specs, steps, groups, twins = W.scaling_members(1, [(128, 8), (256, 16), (512, 16)], range(700, 704))
    ens, per, grp = _ensemble(specs, steps, groups, twins, log=True)
    fields = [ens.field(r).cpu().numpy() for r in range(len(specs))]
    # sampled members (asynchronous and synchronous, each grid) against the oracle
    for r in (0, 5, 10, len(specs) - 1):
        cfg = oracle.Config(specs[r])
        ref, dref, _ = oracle.run(cfg, steps[r], threads=THREADS)
        assert np.array_equal(ens.delays(r).cpu().numpy(), dref), r
        assert np.linalg.norm(fields[r] - ref) / np.linalg.norm(ref) <= 1e-12, r
        assert per[r]["step"] == steps[r]
    # twin differences and group summaries from the GPU's own fields
    for r in range(len(specs)):
        if twins[r] < 0:
            assert per[r]["diff"] == 0.0 and per[r]["dabs"] == 0.0
            continue
        d = fields[r] - fields[twins[r]]
        assert per[r]["diff"] == pytest.approx(np.sqrt(np.mean(d * d)), rel=1e-12)
        assert per[r]["dabs"] == pytest.approx(np.mean(np.abs(d)), rel=1e-12)
    for key, g in grp.items():
        idx = [r for r in range(len(specs)) if groups[r] == key]
        rms = np.array([per[r]["rms"] for r in idx])
        assert g["count"] == len(idx) and g["ntwin"] == sum(twins[r] >= 0 for r in idx)
        assert g["mean"] == pytest.approx(rms.mean(), rel=1e-12)
        assert g["var"] == pytest.approx(rms.var(ddof=1), rel=1e-9)
        assert g["abs_mean"] == pytest.approx(np.mean([per[r]["mean_abs"] for r in idx]), rel=1e-12)
        if g["ntwin"]:
            assert g["dabs_mean"] == pytest.approx(np.mean([per[r]["dabs"] for r in idx]), rel=1e-12)
            assert g["diff_mean"] == pytest.approx(np.mean([per[r]["diff"] for r in idx]), rel=1e-12)
    ens.close()


def test_case1_scaling_laws_on_the_gpu():
    """Fig. "at-ord2-procs": asynchronous part of the error (mean |U - U_sync|) linear in P at N = 512, slope -3
    at fixed P (strong), -2 at fixed P/N (weak); 32 realizations per point."""
    seeds = range(800, 832)
    Ps = (2, 4, 8, 16, 32)
    ns = (128, 256, 512, 1024)
    grids = [(512, P) for P in Ps] + [(n, 16) for n in ns] + [(n, n // 16) for n in ns]
    ens, per, grp = _ensemble(*W.scaling_members(1, grids, seeds))
    D = [grp[i]["dabs_mean"] for i in range(len(grids))]
    assert abs(_slope(Ps, D[:5]) - 1.0) < 0.1, D[:5]
    assert abs(_slope(ns, D[5:9]) + 3.0) < 0.3, D[5:9]
    assert abs(_slope(ns, D[9:]) + 2.0) < 0.3, D[9:]
    ens.close()


@pytest.mark.parametrize("case,Ls,law,spread", [
    (1, (2, 3, 4, 5), lambda L: (L * L - 1) / 3.0, 0.15),
    (4, (2, 3, 4), lambda L: (L ** 3 + 2 * L * L - L - 2) / 4.0, 0.05),
])
def test_delay_moment_laws_on_the_gpu(case, Ls, law, spread):
    """Fig. "at-kmom": (E - E_s)/E_s proportional to the delay-moment polynomial across L (N = 512, P = 16,
    p_k = 1/L); 48 realizations per L, E and E_s from the device group means."""
    ens, per, grp = _ensemble(*W.moment_members(case, Ls, range(900, 948)))
    ratio = np.array([(grp[L]["mean"] - grp[100 + L]["mean"]) / grp[100 + L]["mean"] / law(L) for L in Ls])
    assert np.all(np.sign(ratio) == np.sign(ratio[0]))
    assert np.ptp(ratio) <= spread * np.abs(ratio).max(), ratio
    ens.close()
