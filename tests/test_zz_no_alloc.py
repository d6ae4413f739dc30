"""The allocation-free statistics entry point (for callers that cannot allocate device memory) against the
handle-based at_error_stats, through the C ABI, on two calls in a row.  Collected last on purpose."""
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

FIELDS = ("rms", "max_abs", "mean_abs", "mean", "rms_I", "rms_B", "ua_rms")


@pytest.mark.parametrize("spec", [W.wl_1d(4096, 16, 4, 4, 0, 81, range(1, 6))[0],
                                  W.wl_3d([32, 24, 16], [4, 3, 2], 4, 3, 0, 82, c=(0.3, 0.2, 0.1))[0]],
                         ids=["1d", "3d"])
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
    s.close()


def test_noalloc_rejects_oversized_3d_tables():
    from paper_1702_00496_gb300.binding import ATError, AT_ERR_ARG, Config, at_error_stats_noalloc
    spec, _ = W.wl_3d([16384, 8192, 8], [1, 1, 1], 2, 3, 0, 83)
    u = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(ATError) as e:
        at_error_stats_noalloc(Config(spec), u, 0)
    assert e.value.code == AT_ERR_ARG
