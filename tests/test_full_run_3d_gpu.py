"""GPU parity of the 3D workloads after their whole runs, against the FP64 oracle, element by element.

The 3D workloads split the box into PEs of 64^3 points (Sec. 2; 512^3 in 8^3 PEs for the 500-step advection-
diffusion runs of orders 2 and 4, 256^3 in 4^3 PEs for the 2000-step order-4 run of the gradient workload).  By
default these tests keep that PE shape, the delay process (L = 3, one draw per PE face and step, Sec. 5.1), the
time-step rule and the step counts, on 128^3 points in 2^3 PEs, where a whole oracle run takes seconds: every
code path of the 3D step (interior groups, edge groups of every face kind, the lagged levels of every delay)
runs for the full number of steps, and rounding accumulates over all of them.  With ATFD_FULL_SIZE=1 they also
run the workloads at their full sizes (512^3 x 500 steps, 256^3 x 2000 steps; the oracle then needs minutes on
all host cores).

Bars: delay logs bit-exact; fields within 1e-12 relative L2 and elementwise within 1e-12 of the max norm.
"""
import os

import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

TOL = 1e-12
THREADS = os.cpu_count() or 1
FULL = os.environ.get("ATFD_FULL_SIZE", "") == "1"
full_size = pytest.mark.skipif(not FULL, reason="full-size oracle runs take minutes: set ATFD_FULL_SIZE=1")


def _check_field(u, ref):
    rel = np.linalg.norm(u - ref) / np.linalg.norm(ref)
    assert rel <= TOL, rel
    assert np.abs(u - ref).max() <= TOL * np.abs(ref).max()
    return rel


def _forward_vs_oracle(spec, nsteps, tuned=True):
    """The whole run on the GPU (in the launch shape the autotuner picks, as the bench runs it) and in the oracle."""
    from paper_1702_00496_gb300 import Solver, autotune
    s = Solver(spec, log_steps=nsteps)
    if tuned:
        autotune.tune_forward(s, spec)
        s.reset()
    s.step(nsteps)
    s.sync()
    u = s.field().cpu().numpy().copy()
    d = s.delays().cpu().numpy().copy()
    st = s.error_stats()
    s.close()
    cfg = oracle.Config(spec)
    ref, dref, _ = oracle.run(cfg, nsteps, threads=THREADS)
    assert np.array_equal(d, dref), "delay logs differ"
    _check_field(u, ref)
    so = oracle.error_stats(cfg, u, nsteps)
    atol = 1e-13 * so["ua_rms"]
    for key in ("rms", "max_abs", "mean_abs", "rms_I", "rms_B"):
        assert abs(st[key] - so[key]) <= 1e-9 * abs(so[key]) + atol, key
    assert (st["n_I"], st["n_B"]) == (so["n_I"], so["n_B"])


def _adjoint_forward_vs_oracle(spec, nsteps, every=0):
    """The forward pass of the gradient (at_adjoint_forward: the same steps as at_step, with checkpoints every
    `every` steps, 0 = ceil(sqrt(T))) over the whole run, against the oracle's run."""
    from paper_1702_00496_gb300 import Solver
    s = Solver(spec, log_steps=nsteps)
    s.adjoint_forward(nsteps, every)
    s.sync()
    u = s.field().cpu().numpy().copy()
    d = s.delays().cpu().numpy().copy()
    s.close()
    ref, dref, _ = oracle.run(oracle.Config(spec), nsteps, threads=THREADS)
    assert np.array_equal(d, dref), "delay logs differ"
    _check_field(u, ref)


@pytest.mark.parametrize("order", [2, 4])
def test_advection_diffusion_pe_shape_of_512_run_all_500_steps(order):
    """128^3 in 2^3 PEs of 64^3 (the PE shape of the 512^3 workload), c = (1, 1, 1), alpha = 0.05, dt = dx^2,
    L = 3, all 500 steps."""
    spec, steps = W.wl_3d(128, 2, order, 3, 500, 3)
    _forward_vs_oracle(spec, steps)


def test_gradient_workload_pe_shape_forward_field_all_2000_steps():
    """The forward field of the gradient workload's PE shape (64^3 PEs, order 4, L = 3, alpha = 0.05, its dt)
    on 128^3 in 2^3 PEs, after all 2000 steps of the checkpointed forward pass."""
    spec, steps = W.adjoint_spec(128, 2, 2000)
    _adjoint_forward_vs_oracle(spec, steps)


@full_size
@pytest.mark.parametrize("order", [2, 4])
def test_full_size_512_all_500_steps(order):
    spec, steps = W.workload(f"3d_512_o{order}")
    _forward_vs_oracle(spec, steps)


@full_size
def test_full_size_gradient_workload_forward_field_all_2000_steps():
    spec, steps = W.workload("adjoint_256")
    _adjoint_forward_vs_oracle(spec, steps)
