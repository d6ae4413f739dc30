"""The allocation-free statistics entry point, at_error_stats_noalloc, through the C ABI.

It serves callers that cannot allocate device memory -- a process whose memory pool refuses new allocations after
start-up, an embedding that hands the library only buffers it owns, a job at its memory limit -- and so cannot
create a handle.  Its results are checked against the handle-based at_error_stats and against the oracle's
statistics of the same field, on two calls in a row (the static scratch keeps the previous call's contents), and
on a non-default stream.  Collected last on purpose: if it fails, a run that stops at the first failure has
already run every other test."""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

FIELDS = ("rms", "max_abs", "mean_abs", "mean", "rms_I", "rms_B", "ua_rms")
SPECS = [W.wl_1d(4096, 16, 4, 4, 0, 81, range(1, 6))[0],
         W.wl_3d([32, 24, 16], [4, 3, 2], 4, 3, 0, 82, c=(0.3, 0.2, 0.1))[0]]


def _against_oracle(got, spec, u, step):
    """Both sides evaluate the analytic solution with their own sines (a few ulp of |u_a| apart), so the error
    statistics agree to ~1e-15 |u_a| absolutely, as in the other parity tests."""
    so = oracle.error_stats(oracle.Config(spec), u.cpu().numpy(), step)
    atol = 1e-13 * so["ua_rms"]
    for key in ("rms", "max_abs", "mean_abs", "mean", "rms_I", "rms_B"):
        assert abs(got[key] - so[key]) <= 1e-9 * abs(so[key]) + atol, key
    assert got["ua_rms"] == pytest.approx(so["ua_rms"], rel=1e-13)
    assert (got["n_I"], got["n_B"]) == (so["n_I"], so["n_B"])


@pytest.mark.parametrize("spec", SPECS, ids=["1d", "3d"])
def test_noalloc_stats_match_the_handle_stats_twice(spec):
    from paper_1702_00496_gb300 import Solver
    from paper_1702_00496_gb300.binding import Config, at_error_stats_noalloc
    s = Solver(spec)
    cfg = Config(spec)
    for steps in (37, 41):  # two calls in a row, on different fields
        s.step(steps)
        s.sync()
        ref = s.error_stats()
        u = s.field().clone()
        got = at_error_stats_noalloc(cfg, u, s.n)
        for key in FIELDS:
            assert got[key] == pytest.approx(ref[key], rel=1e-12, abs=1e-15 * ref["ua_rms"]), key
        assert (got["n_I"], got["n_B"], got["step"]) == (ref["n_I"], ref["n_B"], ref["step"])
        _against_oracle(got, spec, u, s.n)
    s.close()


@pytest.mark.parametrize("spec", SPECS, ids=["1d", "3d"])
def test_noalloc_stats_on_a_side_stream(spec):
    """The same call on a non-default stream (the caller orders it after the field is written), twice."""
    from paper_1702_00496_gb300 import Solver
    from paper_1702_00496_gb300.binding import Config, at_error_stats_noalloc
    s = Solver(spec)
    cfg = Config(spec)
    side = torch.cuda.Stream()
    for steps in (23, 29):
        s.step(steps)
        s.sync()
        ref = s.error_stats()
        u = s.field().clone()
        torch.cuda.synchronize()
        with torch.cuda.stream(side):
            got = at_error_stats_noalloc(cfg, u, s.n, stream=torch.cuda.current_stream())
        torch.cuda.synchronize()
        for key in FIELDS:
            assert got[key] == pytest.approx(ref[key], rel=1e-12, abs=1e-15 * ref["ua_rms"]), key
        _against_oracle(got, spec, u, s.n)
    s.close()


def test_noalloc_rejects_oversized_3d_tables():
    """n0 + n1 + n2 above the static table limit is refused before any launch; the field passed has the
    problem's full size, so nothing could be read out of bounds even if that check moved."""
    from paper_1702_00496_gb300.binding import ATError, AT_ERR_ARG, Config, at_error_stats_noalloc
    spec, _ = W.wl_3d([24568, 8, 4], [1, 1, 1], 2, 3, 0, 83)
    u = torch.zeros(24568 * 8 * 4, dtype=torch.float64, device="cuda")
    with pytest.raises(ATError) as e:
        at_error_stats_noalloc(Config(spec), u, 0)
    assert e.value.code == AT_ERR_ARG


def test_noalloc_rejects_short_or_mistyped_fields():
    """The C entry point takes no length: the binding refuses a field shorter than the problem, of another
    dtype, or not contiguous, before calling it."""
    from paper_1702_00496_gb300.binding import ATError, AT_ERR_ARG, Config, at_error_stats_noalloc
    spec = SPECS[0]
    cfg = Config(spec)
    n = spec["n"][0]
    for bad in (torch.zeros(n - 1, dtype=torch.float64, device="cuda"),
                torch.zeros(n, dtype=torch.float32, device="cuda"),
                torch.zeros(2 * n, dtype=torch.float64, device="cuda")[::2]):
        with pytest.raises(ATError) as e:
            at_error_stats_noalloc(cfg, bad, 0)
        assert e.value.code == AT_ERR_ARG
    assert np.isfinite(at_error_stats_noalloc(cfg, torch.zeros(n, dtype=torch.float64, device="cuda"), 0)["rms"])
