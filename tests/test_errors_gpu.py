"""Failure detection without a GPU fault: invalid calls and broken runs come back as status codes from the
host-side checks (the library never traps, aborts or hangs the device)."""
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def test_stepping_past_the_delay_log_is_refused():
    from paper_1702_00496_gb300 import Solver
    from paper_1702_00496_gb300.binding import ATError, AT_ERR_STATE
    spec, _ = W.wl_1d(256, 8, 4, 3, 0, 91, (1, 2))
    s = Solver(spec, log_steps=10)
    s.step(10)
    with pytest.raises(ATError) as e:
        s.step(1)
    assert e.value.code == AT_ERR_STATE and s.n == 10
    s.sync()
    s.close()


def test_adjoint_calls_out_of_order_are_refused():
    from paper_1702_00496_gb300 import Solver
    from paper_1702_00496_gb300.binding import ATError, AT_ERR_STATE
    spec, _ = W.wl_1d(256, 8, 4, 3, 0, 92, (1, 2))
    s = Solver(spec)
    lam = torch.zeros(256, dtype=torch.float64, device="cuda")
    with pytest.raises(ATError) as e:
        s.adjoint_backward(lam)
    assert e.value.code == AT_ERR_STATE
    s.step(3)
    with pytest.raises(ATError) as e:
        s.adjoint_forward(5)
    assert e.value.code == AT_ERR_STATE
    s.reset()
    s.adjoint_forward(5)
    s.step(1)  # any stepping after the checkpointed pass invalidates it
    with pytest.raises(ATError) as e:
        s.adjoint_backward(lam)
    assert e.value.code == AT_ERR_STATE
    s.close()


def test_adjoint_forward_past_the_delay_log_is_refused():
    """Both forward-pass forms (checkpoints, and one segment holding every level) keep at_step's log limit."""
    from paper_1702_00496_gb300 import Solver
    from paper_1702_00496_gb300.binding import ATError, AT_ERR_STATE
    spec, _ = W.wl_1d(256, 8, 4, 3, 0, 95, (1, 2))
    for every in (0, 12):
        s = Solver(spec, log_steps=10)
        with pytest.raises(ATError) as e:
            s.adjoint_forward(12, every)
        assert e.value.code == AT_ERR_STATE and s.n == 0
        s.adjoint_forward(10, every)
        assert s.n == 10
        s.sync()
        s.close()


def test_diverging_run_reports_non_finite_statistics():
    from paper_1702_00496_gb300 import Solver
    from paper_1702_00496_gb300.binding import ATError, AT_ERR_NONFINITE
    spec, _ = W.wl_1d(256, 8, 2, 3, 0, 93, (1, 2), r_alpha=10.0)  # far beyond the Euler limit
    s = Solver(spec)
    s.step(2000)
    with pytest.raises(ATError) as e:
        s.error_stats()
    assert e.value.code == AT_ERR_NONFINITE
    s.sync()  # the context is still usable
    s.close()


def test_undersized_buffers_and_bad_launch_shapes_are_rejected():
    from paper_1702_00496_gb300.binding import (ATError, AT_ERR_ARG, Config, at_init, at_ring_slots,
                                               at_set_launch)
    from paper_1702_00496_gb300 import Solver
    spec, _ = W.wl_1d(256, 8, 4, 3, 0, 94, (1, 2))
    cfg = Config(spec)
    ring = torch.empty(at_ring_slots(cfg) * 256 - 1, dtype=torch.float64, device="cuda")
    with pytest.raises(ATError) as e:
        at_init(cfg, ring)
    assert e.value.code == AT_ERR_ARG
    s = Solver(spec)
    with pytest.raises(ATError) as e:
        at_set_launch(s.h, 100, 4)
    assert e.value.code == AT_ERR_ARG
    s.step(5)
    s.sync()
    s.close()
