"""GPU parity of the persistent ensemble engine: every realization against the oracle (delays bit-exact,
fields within 1e-12 relative L2), its statistics and the per-grid-size ensemble mean and variance."""
import os

import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

THREADS = os.cpu_count() or 1


def _members(count, sizes, Ls, orders, seed0=500):
    rng = np.random.default_rng(seed0)
    out = []
    for r in range(count):
        n = int(rng.choice(sizes))
        order = int(rng.choice(orders))
        spec, _ = W.wl_1d(n, n // 16, order, int(rng.choice(Ls)), 0, seed0 + r, range(1, 5))
        out.append(spec)
    return out


def _check_members(ens, specs, nsteps, idx):
    per, groups = ens.stats()
    for r in idx:
        cfg = oracle.Config(specs[r])
        ref, dref, _ = oracle.run(cfg, nsteps, threads=THREADS)
        u = ens.field(r).cpu().numpy()
        assert np.array_equal(ens.delays(r).cpu().numpy(), dref), r
        assert np.linalg.norm(u - ref) / np.linalg.norm(ref) <= 1e-12, r
        so = oracle.error_stats(cfg, u, nsteps)
        atol = 1e-13 * so["ua_rms"]
        for key in ("rms", "max_abs", "mean_abs", "rms_I", "rms_B"):
            assert abs(per[r][key] - so[key]) <= 1e-9 * so[key] + atol, (r, key)
    return per, groups


@pytest.mark.parametrize("threads,ctas", [(1024, 0), (512, 2), (256, 0), (128, 1)])
def test_mixed_ensemble_matches_oracle(threads, ctas):
    from paper_1702_00496_gb300 import Ensemble
    specs = _members(14, [128, 256, 512, 1024], [2, 3, 4], [2, 4])
    nsteps = 400
    ens = Ensemble(specs, nsteps, log=True, threads=threads, ctas_per_sm=ctas)
    ens.run()
    per, groups = _check_members(ens, specs, nsteps, range(len(specs)))
    # per grid size: mean and unbiased variance of the RMS errors
    for g in groups:
        rms = np.array([per[r]["rms"] for r in range(len(specs)) if specs[r]["n"][0] == g["key"]])
        assert g["count"] == len(rms)
        assert g["mean"] == pytest.approx(rms.mean(), rel=1e-12)
        if len(rms) > 1:
            assert g["var"] == pytest.approx(rms.var(ddof=1), rel=1e-9, abs=1e-30)
    ens.close()


def test_ensemble_is_bitwise_the_single_problem_path():
    """Each member equals the single-problem path run in single steps (the engine steps one step at a time)."""
    from paper_1702_00496_gb300 import Ensemble, Solver, at_set_fusion
    specs = _members(5, [256, 1024], [3, 4], [4], seed0=900)
    ens = Ensemble(specs, 250)
    ens.run()
    for r, spec in enumerate(specs):
        s = Solver(spec)
        at_set_fusion(s.h, 1)
        s.step(250)
        s.sync()
        assert torch.equal(ens.field(r), s.field().reshape(-1)), r
        s.close()
    ens.close()


def test_single_member_and_repeated_runs():
    from paper_1702_00496_gb300 import Ensemble
    specs = _members(1, [512], [3], [4], seed0=77)
    ens = Ensemble(specs, 100, log=True)
    ens.run()
    a = ens.field(0).clone()
    ens.run()
    assert torch.equal(a, ens.field(0))
    _check_members(ens, specs, 100, [0])
    ens.close()


def test_full_ensemble_workload_sampled():
    """1024 realizations, N_r in {2^10..2^16}, P_r = N_r/64, L_r in {2,3,4}, 5000 steps, one launch in the launch
    shape the autotuner picks for the bench: the first member of every (N_r, L_r) pair (21 members: every grid
    size with every delay range) against the oracle over the full run, all statistics finite."""
    from paper_1702_00496_gb300 import Ensemble, autotune
    specs, nsteps = W.ensemble_members()
    threads, ctas = autotune.tune_ensemble(specs, [nsteps] * len(specs))
    ens = Ensemble(specs, nsteps, log=True, threads=threads, ctas_per_sm=ctas)
    ens.run()
    first = {}
    for r, s in enumerate(specs):
        first.setdefault((s["n"][0], s["L"]), r)
    pick = sorted(first.values())
    assert len(pick) == 21
    per, groups = _check_members(ens, specs, nsteps, pick)
    assert len(groups) == 7 and sum(g["count"] for g in groups) == 1024
    assert all(np.isfinite(g["mean"]) and g["mean"] > 0 for g in groups)
    ens.close()
