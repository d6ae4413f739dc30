"""CPU tests of the C-ABI library: it loads, exports what include/at.h declares, and its host-side
code (coefficient derivation, delay generator, argument checks) matches the paper and the oracle.
No kernel is launched here."""
import os
import re
from fractions import Fraction

import numpy as np
import pytest

import oracle
import paper_1702_00496_gb300 as P
from paper_1702_00496_gb300 import binding as B
import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden")


def _golden(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append(line.split())
    return rows


def test_library_exports_every_declared_entry_point():
    header = open(os.path.join(ROOT, "include", "at.h")).read()
    declared = set(re.findall(r"^\s*(?:int|const char \*)\s*(at_\w+)\s*\(", header, re.M))
    assert declared == set(B.EXPORTS), declared ^ set(B.EXPORTS)
    lib = B.load()
    for name in declared:
        assert hasattr(lib, name), name
    assert B.at_last_error() == "" or isinstance(B.at_last_error(), str)


# --------------------------------------------------------------------- coefficients
def test_example3_two_stage_coefficients():
    rows = _golden("example3_cd4-at.txt")
    cd = [int(v) for v in rows[0][1:6]]
    den = int(rows[0][6])
    c = P.at_coeffs(2, 4, 4)
    assert (c.h, c.T) == (2, 3)
    assert [Fraction(c.cd_num[j], c.cd_den) for j in range(5)] == [Fraction(v, den) for v in cd]
    for r in rows[1:]:
        k = int(r[1])
        want = [Fraction(int(v)) for v in r[2:5]]
        assert [Fraction(c.w_num[k][m], c.w_den[k]) for m in range(3)] == want
        # the printed polynomials
        assert want == [Fraction(k * k + 3 * k + 2, 2), -Fraction(k * k + 2 * k), Fraction(k * k + k, 2)]


@pytest.mark.parametrize("deriv,order,cd,den", [(1, 2, [-1, 0, 1], 2), (2, 2, [1, -2, 1], 1),
                                                 (1, 4, [1, -8, 0, 8, -1], 12), (2, 4, [-1, 16, -30, 16, -1], 12),
                                                 (1, 6, [-1, 9, -45, 0, 45, -9, 1], 60),
                                                 (2, 6, [2, -27, 270, -490, 270, -27, 2], 180)])
def test_central_weights_and_time_width(deriv, order, cd, den):
    c = P.at_coeffs(deriv, order, 3)
    got = [Fraction(c.cd_num[j], c.cd_den) for j in range(2 * c.h + 1)]
    assert got == [Fraction(v, den) for v in cd]
    assert c.T == order // 2 + 1
    for k in range(3):  # (1,2,2)b / (2,2,2)b weights (k+1, -k); order 4: the Example 3 polynomials
        w = [Fraction(c.w_num[k][m], c.w_den[k]) for m in range(c.T)]
        if order == 2:
            assert w == [k + 1, -k]
        if order == 6:  # the weights of the (2,6,2) rows: a cubic in k per delayed level
            assert w == [Fraction(k ** 3 + 6 * k ** 2 + 11 * k + 6, 6), -Fraction(k ** 3 + 5 * k ** 2 + 6 * k, 2),
                         Fraction(k ** 3 + 4 * k ** 2 + 3 * k, 2), -Fraction(k ** 3 + 3 * k ** 2 + 2 * k, 6)]


def _merge(taps):
    out = {}
    for j, l, c in taps:
        out[(j, l)] = out.get((j, l), 0.0) + c
    return {key: v for key, v in out.items() if v != 0.0}


@pytest.mark.parametrize("order", [2, 4, 6])
@pytest.mark.parametrize("deriv", [1, 2])
@pytest.mark.parametrize("scheme", [P.AT_SYNC, P.AT_ASYNC_STD, P.AT_AT])
def test_derived_taps_equal_the_oracle_tables(order, deriv, scheme):
    """The library derives its stencils by solving Eq. "cond"; the oracle types them from the tables."""
    _compare_taps(order, deriv, scheme)


@pytest.mark.parametrize("deriv,scheme", [(1, P.AT_AT_SPACE2), (2, P.AT_AT_SPACE2), (2, P.AT_AT_SPACE1)])
def test_derived_space_expanded_rows_equal_the_oracle_tables(deriv, scheme):
    """(1,2,2)a, (2,2,2)a, (2,1,2): the library solves the single system on each row's shape."""
    _compare_taps(2, deriv, scheme)


def test_space_expanded_schemes_reject_what_they_do_not_define():
    with pytest.raises(B.ATError):
        P.at_stencil_taps(1, 2, P.AT_AT_SPACE1, 1, 0, 0)  # (2,1,2) has no first derivative
    with pytest.raises(B.ATError):
        P.at_stencil_taps(2, 4, P.AT_AT_SPACE2, 1, 0, 0)  # the rows are second order
    for field, value in (("order", 4), ("tsteps", 2)):
        spec, _ = W.wl_1d(256, 8, 2, 3, 0, 1, (1, 2), scheme=W.AT_SPACE2)
        spec[field] = value
        with pytest.raises(B.ATError):
            P.at_ring_slots(B.Config(spec))
    spec, _ = W.wl_1d(256, 8, 2, 3, 0, 1, (1, 2), scheme=W.AT_SPACE1)  # c = 1: (2,1,2) is for diffusion
    with pytest.raises(B.ATError):
        P.at_ring_slots(B.Config(spec))
    spec["c"] = [0.0]
    assert P.at_ring_slots(B.Config(spec)) == 3 + 1


def _compare_taps(order, deriv, scheme):
    S = 10
    for k in range(4):
        for pos in range(order // 2):
            for side in (0, 1):
                lib = _merge(P.at_stencil_taps(deriv, order, scheme, k, pos, side))
                opos = pos if side == 0 else S - 1 - pos
                kL, kR = (k, 0) if side == 0 else (0, k)
                orc = _merge(oracle.taps(order, scheme, deriv, opos, S, 1, kL, kR, 1.0))
                assert lib.keys() == orc.keys(), (k, pos, side)
                for key in lib:
                    assert lib[key] == pytest.approx(orc[key], rel=1e-14, abs=1e-14)


def test_example2_single_system():
    rows = _golden("example2_ex2-1.txt")
    js = [int(r[0]) for r in rows]
    for k in (1, 2, 3):
        ls = [0 if r[1] == "0" else k for r in rows]
        rc, frac, c, rank = P.at_solve_stencil(2, 4, 1, js, ls)
        assert rc == B.AT_OK and rank == 11
        assert [Fraction(n, d) for n, d in frac] == [Fraction(int(r[2]), int(r[3])) for r in rows]


def test_example1_closed_form_and_degenerate_cases():
    for r in _golden("example1_ex1.txt"):
        k1, k2, status = int(r[0]), int(r[1]), r[2]
        rc, frac, _, rank = P.at_solve_stencil(1, 2, 2, [-1, 0, 1, 2], [0, 0, k1, k2])
        if status == "ok":
            assert rc == B.AT_OK
            den = 2 * (3 * k1 - k2)
            want = [Fraction(-4 * k1 + k2, den), Fraction(3 * k1, den), Fraction(-k2, den), Fraction(k1, den)]
            assert [Fraction(n, d) for n, d in frac] == want
            if k1 == k2:
                assert want == [Fraction(-3, 4), Fraction(3, 4), Fraction(-1, 4), Fraction(1, 4)]
        elif status == "inconsistent":
            assert rc == B.AT_ERR_INCONSISTENT and rank == 3
        else:
            assert rc == B.AT_ERR_SINGULAR and rank == 3


def test_artificial_delay_on_both_sides():
    """Sec. 3.2 with the single system: imposing the buffer point's delay k on the opposite point as well (an
    artificial delay at an interior point) leaves the central difference itself second-order accurate for
    dt ~ dx^2 (Eq. "deriv22": the (0,1) row and every even power of dx drop out), while the delay on one side alone
    is inconsistent; and no such both-sides central stencil reaches fourth order, since the u^(1,1) dx dt row then
    asks the same sum to be 1 and 0."""
    for k in (1, 2, 3):
        rc, frac, _, rank = P.at_solve_stencil(1, 2, 2, [-1, 1], [k, k])
        assert rc == B.AT_OK and rank == 2
        assert [Fraction(n, d) for n, d in frac] == [Fraction(-1, 2), Fraction(1, 2)]
        rc, _, _, rank = P.at_solve_stencil(1, 2, 2, [-1, 1], [0, k])
        assert rc == B.AT_ERR_INCONSISTENT and rank == 2
        rc, _, _, _ = P.at_solve_stencil(1, 4, 2, [-2, -1, 1, 2], [k, k, k, k])
        assert rc == B.AT_ERR_INCONSISTENT
    rc, frac, _, _ = P.at_solve_stencil(1, 4, 2, [-2, -1, 1, 2], [0, 0, 0, 0])
    assert rc == B.AT_OK
    assert [Fraction(n, d) for n, d in frac] == [Fraction(1, 12), Fraction(-2, 3), Fraction(2, 3), Fraction(-1, 12)]


def test_coeffs_argument_errors():
    for args in [(3, 2, 3), (1, 3, 3), (1, 8, 3), (1, 2, 0), (1, 2, 9)]:
        with pytest.raises(B.ATError) as e:
            P.at_coeffs(*args)
        assert e.value.code == B.AT_ERR_ARG


# ------------------------------------------------------------------------- delays
@pytest.mark.parametrize("L", [1, 2, 3, 4, 8])
def test_host_delay_generator_is_bit_exact_with_the_oracle(L):
    rng = np.random.default_rng(L)
    thr = None if L < 3 else W.thresholds_from_probs(np.full(L, 1.0 / L))
    for _ in range(300):
        seed = int(rng.integers(0, 2 ** 63))
        n, b = int(rng.integers(0, 10 ** 6)), int(rng.integers(0, 10 ** 5))
        assert P.at_delay(seed, n, b, L) == oracle.delay_raw(seed, n, b, L)
        if thr is not None:
            assert P.at_delay(seed, n, b, L, thr) == oracle.delay_raw(seed, n, b, L, thr)


# -------------------------------------------------------------------- config checks
def test_ring_depth_and_side_count():
    spec, _ = W.workload("1d_n16m")
    cfg = B.Config(spec)
    assert P.at_ring_slots(cfg) == 4 + 3 and P.at_num_sides(cfg) == 2 * 4096
    spec, _ = W.workload("3d_512_o2")
    cfg = B.Config(spec)
    assert P.at_ring_slots(cfg) == 3 + 2 and P.at_num_sides(cfg) == 6 * 512
    spec["scheme"] = W.ASYNC_STD
    assert P.at_ring_slots(B.Config(spec)) == 3 + 1
    # Adams-Bashforth: tsteps - 1 stored right-hand sides after the L + T levels
    for tsteps, extra in ((0, 0), (1, 0), (2, 1), (3, 2)):
        spec, _ = W.wl_1d(256, 8, 6, 3, 0, 1, (1, 2), tsteps=tsteps)
        assert P.at_ring_slots(B.Config(spec)) == 3 + 4 + extra


@pytest.mark.parametrize("field,value", [("n", [100]), ("pe", [3]), ("order", 8), ("order", 3), ("L", 0), ("L", 9),
                                         ("scheme", 5), ("dim", 2), ("dt", -1.0), ("pe", [128]), ("tsteps", 4),
                                         ("tsteps", -1)])
def test_invalid_configs_are_rejected_on_the_host(field, value):
    spec, _ = W.wl_1d(256, 8, 4, 3, 0, 1, (1, 2))
    spec[field] = value
    with pytest.raises(B.ATError) as e:
        P.at_ring_slots(B.Config(spec))
    assert e.value.code == B.AT_ERR_ARG


def test_descending_thresholds_are_rejected():
    spec, _ = W.wl_1d(256, 8, 2, 3, 0, 1, (1, 2))
    spec["thresholds"] = np.array([3 << 30, 1 << 30], dtype=np.uint64)
    with pytest.raises(B.ATError):
        P.at_num_sides(B.Config(spec))


def test_ensemble_members_must_be_1d_with_aligned_sizes():
    from paper_1702_00496_gb300.binding import at_ensemble_sizes
    ok, _ = W.wl_1d(1024, 16, 4, 3, 0, 1, (1, 2))
    bad_dim, _ = W.wl_3d([16, 16, 16], [2, 2, 2], 2, 3, 0, 2)
    bad_n, _ = W.wl_1d(1022, 2, 4, 3, 0, 3, (1, 2))
    bad_s, _ = W.wl_1d(1020, 170, 4, 3, 0, 4, (1, 2))  # PE width 6
    assert at_ensemble_sizes([B.Config(ok)], 10)[0] == (3 + 3) * 1024  # R = L + T
    for spec in (bad_dim, bad_n, bad_s):
        with pytest.raises(B.ATError) as e:
            at_ensemble_sizes([B.Config(ok), B.Config(spec)], 10)
        assert e.value.code == B.AT_ERR_ARG


def test_ensemble_runs_are_validated_and_sized_per_member():
    from paper_1702_00496_gb300.binding import at_ensemble_sizes
    a, _ = W.wl_1d(1024, 16, 4, 3, 0, 1, (1, 2))                # R = 6, 32 sides
    b, _ = W.wl_1d(512, 8, 6, 3, 0, 2, (1, 2), tsteps=3)        # R = 3 + 4 + 2, 16 sides
    c, _ = W.wl_1d(1024, 16, 2, 3, 0, 3, (1, 2), scheme=W.SYNC)  # R = 3 + 1, 32 sides
    cfgs = [B.Config(s) for s in (a, b, c)]
    ring, log = at_ensemble_sizes(cfgs, [10, 20, 30], twins=[2, -1, 0])
    assert ring == 6 * 1024 + 9 * 512 + 4 * 1024 and log == 10 * 32 + 20 * 16 + 30 * 32
    bad = [dict(nsteps=[10, -1, 5]), dict(nsteps=[10, 1, 1], twins=[0, -1, -1]), dict(nsteps=5, twins=[1, -1, -1]),
           dict(nsteps=5, twins=[3, -1, -1]), dict(nsteps=5, groups=[-2, 0, 0]), dict(nsteps=[1 << 32, 1, 1])]
    for kw in bad:
        with pytest.raises(B.ATError) as e:
            at_ensemble_sizes(cfgs, kw.pop("nsteps"), **kw)
        assert e.value.code == B.AT_ERR_ARG
    with pytest.raises(ValueError):
        at_ensemble_sizes(cfgs, [1, 2])


def test_noalloc_binding_refuses_a_host_field():
    """at_error_stats_noalloc takes no length: the binding checks the tensor (CUDA, float64, contiguous, long
    enough) before the call, so a host tensor never reaches the library."""
    import torch
    spec, _ = W.wl_1d(4096, 16, 4, 4, 0, 81, range(1, 6))
    for bad in (torch.zeros(4096, dtype=torch.float64), np.zeros(4096)):
        with pytest.raises(B.ATError) as e:
            B.at_error_stats_noalloc(B.Config(spec), bad, 0)
        assert e.value.code == B.AT_ERR_ARG


def test_library_delay_word_reproduces_the_published_known_answer():
    """The library's host copy of the delay generator (at_delay) against the first word of the all-zero
    Philox4x32-10 known-answer vector (counter (0,0,0,0), key (0,0): step 0, side 0, seed 0; the other published
    vectors have counter words that at_delay keeps at zero).  Two-bin thresholds at x0 and x0 + 1 fix the word
    exactly."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    x0 = int(rows[0][6], 16)
    assert [int(v, 16) for v in rows[0][:6]] == [0] * 6
    assert P.at_delay(0, 0, 0, 2, np.array([x0], dtype=np.uint64)) == 1
    assert P.at_delay(0, 0, 0, 2, np.array([x0 + 1], dtype=np.uint64)) == 0
    for L in (2, 3, 4, 8):
        assert P.at_delay(0, 0, 0, L) == (x0 * L) >> 32
