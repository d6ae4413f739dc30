"""K-step blocks of the 1D forward-Euler step (at_set_fusion) against single steps and the oracle.

Inside a PE, away from its boundaries, K steps of the constant interior stencil are one stencil of half-width hK
(the K-fold composition of its taps, exact in exact arithmetic); the cells near PE boundaries are stepped one step
at a time with the delayed halos of Tables "atschemes-left/right".  Bars: the same delay log bit for bit, fields
within 1e-13 of single steps and within 1e-12 of the oracle after the whole run."""
import os

import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

THREADS = os.cpu_count() or 1


def _k_used(spec, k=4):
    from paper_1702_00496_gb300 import Solver, at_set_fusion
    s = Solver(spec)
    used = at_set_fusion(s.h, k)
    s.close()
    return used


def test_block_length_follows_the_shape():
    assert _k_used(W.wl_1d(1 << 14, 16, 4, 4, 0, 1, (1, 2))[0]) == 4
    assert _k_used(W.wl_1d(1 << 14, 16, 4, 4, 0, 1, (1, 2))[0], 2) == 2
    assert _k_used(W.wl_1d(1 << 14, 16, 4, 1, 0, 1, (1, 2))[0]) == 3          # R = L + T = 4: K < R
    assert _k_used(W.wl_1d(1 << 14, 16, 4, 1, 0, 1, (1, 2), scheme=W.SYNC)[0]) == 1  # R = 2
    assert _k_used(W.wl_1d(256, 16, 4, 4, 0, 1, (1, 2))[0]) == 1               # PEs of 16 cells: zones cost more
    assert _k_used(W.wl_1d(64 * 16, 16, 4, 4, 0, 1, (1, 2))[0]) == 1           # PEs of 64: blocks would save < 5 %
    assert _k_used(W.wl_1d(144 * 16, 16, 4, 4, 0, 1, (1, 2))[0]) == 4          # PEs of 144: they save 5 %
    assert _k_used(W.wl_1d(128 * 16, 16, 4, 4, 0, 1, (1, 2))[0]) == 3
    assert _k_used(W.wl_1d(1 << 14, 16, 4, 3, 0, 1, (1, 2), tsteps=2, r_alpha=0.05)[0]) == 1  # Adams-Bashforth
    assert _k_used(W.wl_1d(1 << 14, 16, 2, 3, 0, 1, (1, 2), scheme=W.AT_SPACE2)[0]) == 1      # rows in space
    assert _k_used(W.wl_1d(1002, 6, 4, 4, 0, 1, (1, 2))[0]) == 1               # not groups of four
    assert _k_used(W.wl_3d([32, 24, 16], [2, 2, 2], 4, 3, 0, 1)[0]) == 1


def _run(spec, nsteps, k, log=True):
    from paper_1702_00496_gb300 import Solver, at_set_fusion
    s = Solver(spec, log_steps=nsteps if log else 0)
    used = at_set_fusion(s.h, k)
    s.step(nsteps)
    s.sync()
    u = s.field().cpu().numpy().copy()
    d = s.delays().cpu().numpy().copy() if log else None
    s.close()
    return u, d, used


BLOCK_CASES = [
    ("o2_at", lambda: W.wl_1d(4096, 16, 2, 3, 0, 31, range(1, 5))[0]),
    ("o4_at_L8_binned", lambda: W.wl_1d(4096, 16, 4, 8, 0, 32, range(1, 5), r_alpha=0.02,
                                        probs=[0.3, 0.1, 0.1, 0.1, 0.1, 0.1, 0.1, 0.1])[0]),
    ("o6_at", lambda: W.wl_1d(6144, 16, 6, 3, 0, 33, range(1, 5), r_alpha=0.02)[0]),
    ("o4_std", lambda: W.wl_1d(4096, 16, 4, 4, 0, 34, range(1, 5), scheme=W.ASYNC_STD)[0]),
    ("o4_sync_L5", lambda: W.wl_1d(4096, 16, 4, 5, 0, 35, range(1, 5), scheme=W.SYNC)[0]),
    ("o4_unsplit", lambda: W.wl_1d(2048, 1, 4, 4, 0, 36, range(1, 5))[0]),
    ("o4_narrowest", lambda: W.wl_1d(144 * 16, 16, 4, 4, 0, 37, range(1, 5))[0]),   # narrowest PEs with K = 4
    ("o2_narrowest", lambda: W.wl_1d(72 * 8, 8, 2, 3, 0, 38, range(1, 5))[0]),
    ("o4_k3", lambda: W.wl_1d(128 * 16, 16, 4, 4, 0, 40, range(1, 5))[0]),
]


@pytest.mark.parametrize("name,make", BLOCK_CASES, ids=[c[0] for c in BLOCK_CASES])
def test_blocks_match_single_steps_and_the_oracle(name, make):
    """Blocks of K = 4 (or less where the shape demands) against single steps: 103 steps = two 48-step graphs
    of 12 blocks, one more block and 3 single steps (K = 4); and against the oracle."""
    spec = make()
    nsteps = 103
    u1, d1, k1 = _run(spec, nsteps, 1)
    uk, dk, kk = _run(spec, nsteps, 4)
    assert k1 == 1 and kk > 1
    assert np.array_equal(d1, dk), "blocks changed the delay log"
    assert np.linalg.norm(uk - u1) / np.linalg.norm(u1) <= 1e-13
    ref, dref, _ = oracle.run(oracle.Config(spec), nsteps, threads=THREADS)
    assert np.array_equal(dk, dref)
    assert np.linalg.norm(uk - ref) / np.linalg.norm(ref) <= 1e-12
    assert np.abs(uk - ref).max() <= 1e-12 * np.abs(ref).max()


def test_remainder_blocks_and_call_splits():
    """Steps split into calls of 7, 45 and 51 (blocks start at each call, remainders run as blocks and single
    steps) against one call: equal up to rounding; the delays and the levels later steps read stay exact."""
    from paper_1702_00496_gb300 import Solver
    spec, _ = W.wl_1d(8192, 32, 4, 4, 0, 39, range(1, 5))
    a = Solver(spec, log_steps=103)
    for n in (7, 45, 51):
        a.step(n)
    b = Solver(spec, log_steps=103)
    b.step(103)
    a.sync()
    b.sync()
    assert torch.equal(a.delays(), b.delays())
    ua, ub = a.field().cpu().numpy(), b.field().cpu().numpy()
    assert np.linalg.norm(ua - ub) / np.linalg.norm(ub) <= 1e-13
    a.close()
    b.close()


def test_full_size_1d_workload_in_blocks_against_single_steps():
    """The 1D N = 2^24, 4096-PE, order-4, L = 4 workload for all 1000 steps in blocks of 4 against single steps."""
    spec, steps = W.workload("1d_n16m")
    u1, _, _ = _run(spec, steps, 1, log=False)
    uk, _, kk = _run(spec, steps, 4, log=False)
    assert kk == 4
    assert np.linalg.norm(uk - u1) / np.linalg.norm(u1) <= 1e-13
