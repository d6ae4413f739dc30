"""GPU adjoint: the hand-written transposed AT step against the CPU adjoint (oracle) and against central finite
differences of the GPU forward run; checkpoint intervals and the autograd wrapper."""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def _gpu_grad(spec, nsteps, target, every=0, u0=None):
    from paper_1702_00496_gb300 import Solver
    s = Solver(spec)
    if u0 is not None:
        s.reset(torch.as_tensor(u0, device="cuda"))
    s.adjoint_forward(nsteps, every)
    u = s.field().clone()
    tgt = torch.as_tensor(target, device="cuda").reshape(u.shape)
    lam = u - tgt
    J = 0.5 * float((lam * lam).sum())
    g, ga = s.adjoint_backward(lam)
    out = (J, g.cpu().numpy(), ga, u.cpu().numpy())
    s.close()
    return out


CASES = [
    ("1d_o4_L3", lambda: W.wl_1d(256, 8, 4, 3, 0, 61, (1, 2, 3))[0], 80),
    ("1d_o2_L4", lambda: W.wl_1d(192, 6, 2, 4, 0, 62, (1, 4))[0], 90),
    ("1d_o4_std", lambda: W.wl_1d(256, 8, 4, 3, 0, 63, (1, 2), scheme=W.ASYNC_STD)[0], 60),
    ("1d_o4_sync", lambda: W.wl_1d(256, 8, 4, 3, 0, 64, (1, 2), scheme=W.SYNC)[0], 60),
    ("1d_point_path", lambda: W.wl_1d(250, 5, 4, 3, 0, 65, (1, 2))[0], 50),
    ("3d_o4", lambda: W.wl_3d([16, 12, 8], [2, 2, 2], 4, 3, 0, 66, c=(0.3, 0.2, 0.1))[0], 20),
    ("3d_o2_unsplit", lambda: W.wl_3d([12, 16, 8], [3, 1, 2], 2, 4, 0, 67, c=(0.2, 0.2, 0.2))[0], 25),
    ("1d_o6_L3", lambda: W.wl_1d(256, 8, 6, 3, 0, 68, (1, 2, 3), r_alpha=0.02)[0], 60),
    ("1d_o6_point_path", lambda: W.wl_1d(250, 5, 6, 4, 0, 69, (1, 2), r_alpha=0.02)[0], 50),
    ("3d_o6", lambda: W.wl_3d([24, 16, 16], [2, 2, 2], 6, 3, 0, 70, c=(0.3, 0.2, 0.1), dt=0.02 * W.dx_of(24) ** 2 / 0.05)[0],
     20),
    # PEs of 4 = 2h cells: each group starts and ends its PE, so its x taps reach both neighbour PEs
    ("1d_o4_pe_width_4", lambda: W.wl_1d(64, 16, 4, 3, 0, 75, (1, 2, 3))[0], 60),
    ("3d_o4_pe_width_4", lambda: W.wl_3d([8, 8, 12], [2, 2, 3], 4, 3, 0, 76, c=(0.3, 0.2, 0.1))[0], 20),
]


@pytest.mark.parametrize("name,make,nsteps", CASES, ids=[c[0] for c in CASES])
def test_adjoint_matches_cpu_adjoint(name, make, nsteps):
    spec = make()
    cfg = oracle.Config(spec)
    rng = np.random.default_rng(3)
    target = 0.5 * oracle.initial(cfg) + 0.1 * rng.standard_normal(cfg.shape)
    J, g, ga, _ = _gpu_grad(spec, nsteps, target)
    Jo, go, gao = oracle.adjoint(cfg, nsteps, target)
    assert J == pytest.approx(Jo, rel=1e-11)
    assert np.linalg.norm(g - go) / np.linalg.norm(go) <= 1e-12
    assert ga == pytest.approx(gao, rel=1e-10)


CKPT_CASES = [
    ("1d_o4", lambda: W.wl_1d(512, 8, 4, 4, 0, 71, (1, 2, 3))[0], 97, False),
    # PEs of 16 x 12 x 8: the checkpoints keep the older levels on 4 of every S cells per axis only
    ("3d_o4", lambda: W.wl_3d([32, 24, 16], [2, 2, 2], 4, 3, 0, 79, c=(0.3, 0.2, 0.1))[0], 31, False),
    # Adams-Bashforth from a caller's field: the checkpoints also hold the stored right-hand sides
    ("1d_ab2", lambda: W.wl_1d(512, 8, 4, 3, 0, 78, (1, 2, 3), r_alpha=0.05, tsteps=2)[0], 61, True),
]


@pytest.mark.parametrize("name,make,nsteps,callers_field", CKPT_CASES, ids=[c[0] for c in CKPT_CASES])
def test_checkpoint_interval_does_not_change_the_gradient(name, make, nsteps, callers_field):
    """Every checkpoint interval -- each step, sqrt(T), uneven segments, one segment with every level resident --
    gives the same bits: a checkpoint restores U^{n0} and, of the older levels, the cells the steps read at delayed
    levels (those within the buffer reach of a PE face), so the recomputed levels are the forward pass's."""
    spec = make()
    cfg = oracle.Config(spec)
    target = np.zeros(cfg.shape)
    u0 = oracle.initial(cfg) if callers_field else None
    ref = None
    for every in (0, 1, 5, 13, nsteps):
        J, g, ga, _ = _gpu_grad(spec, nsteps, target, every, u0=u0)
        if ref is None:
            ref = (J, g, ga)
        assert J == ref[0] and ga == ref[2] and np.array_equal(g, ref[1]), every


def test_zero_steps_gradient_is_the_seed():
    spec, _ = W.wl_1d(128, 4, 4, 3, 0, 72, (1, 2))
    target = np.ones(128)
    J, g, ga, u = _gpu_grad(spec, 0, target)
    assert np.array_equal(g, u - target) and ga == 0.0


def test_autograd_function():
    from paper_1702_00496_gb300 import at_forward
    spec, _ = W.wl_3d([16, 12, 8], [2, 2, 2], 4, 3, 0, 73, c=(0.3, 0.2, 0.1))
    cfg = oracle.Config(spec)
    u0 = torch.as_tensor(oracle.initial(cfg), device="cuda").requires_grad_(True)
    alpha = torch.tensor(spec["alpha"], dtype=torch.float64, device="cuda", requires_grad=True)
    target = torch.zeros_like(u0)
    u = at_forward(u0, alpha, spec, 15)
    loss = 0.5 * ((u - target) ** 2).sum()
    loss.backward()
    Jo, go, gao = oracle.adjoint(cfg, 15, np.zeros(cfg.shape))
    assert float(loss) == pytest.approx(Jo, rel=1e-11)
    assert np.linalg.norm(u0.grad.cpu().numpy() - go) / np.linalg.norm(go) <= 1e-12
    assert float(alpha.grad) == pytest.approx(gao, rel=1e-10)


def test_full_size_adjoint_against_finite_differences():
    """256^3, 4^3 PEs, order 4, L = 3, 2000 steps; u_target from a forward run at alpha = 0.06 with the same
    delays; the gradient in u0 against central differences on 16 random directions (exact for the quadratic
    misfit up to rounding) and the alpha derivative against Richardson-extrapolated differences."""
    from paper_1702_00496_gb300 import Solver
    spec, nsteps = W.workload("adjoint_256")
    t_spec = dict(spec)
    t_spec["alpha"] = 0.06
    s = Solver(t_spec)
    s.step(nsteps)
    target = s.field().clone()
    s.close()
    s = Solver(spec)
    u0 = s.field().clone()
    s.adjoint_forward(nsteps)
    lam = s.field() - target
    g, ga = s.adjoint_backward(lam.clone())
    s.close()

    def J(u_init, alpha=spec["alpha"]):
        sp = dict(spec)
        sp["alpha"] = alpha
        sv = Solver(sp)
        sv.reset(u_init)
        sv.step(nsteps)
        r = sv.field() - target
        val = 0.5 * float(torch.dot(r.reshape(-1), r.reshape(-1)))
        sv.close()
        return val

    gen = torch.Generator(device="cuda").manual_seed(11)
    for _ in range(16):
        v = torch.randn(u0.shape, dtype=torch.float64, device="cuda", generator=gen)
        eps = 1e-2
        fd = (J(u0 + eps * v) - J(u0 - eps * v)) / (2 * eps)
        assert float(torch.dot(g.reshape(-1), v.reshape(-1))) == pytest.approx(fd, rel=1e-6)
    a0 = spec["alpha"]
    h = 1e-3 * a0
    d1 = (J(u0, a0 + h) - J(u0, a0 - h)) / (2 * h)
    d2 = (J(u0, a0 + h / 2) - J(u0, a0 - h / 2)) / h
    assert ga == pytest.approx((4 * d2 - d1) / 3, rel=1e-6)


def test_u0_only_sweep_gives_the_same_u0_gradient():
    from paper_1702_00496_gb300 import Solver
    spec, _ = W.wl_3d([16, 12, 8], [2, 2, 2], 4, 3, 0, 74, c=(0.3, 0.2, 0.1))
    grads = []
    for want_alpha in (True, False):
        s = Solver(spec)
        s.adjoint_forward(30, 7)
        g, ga = s.adjoint_backward(s.field().clone(), want_alpha)
        grads.append(g.clone())
        assert (ga is None) == (not want_alpha)
        s.close()
    assert torch.equal(grads[0], grads[1])


# ------------------------------------------------------------ Adams-Bashforth runs (from a caller's field)
AB_CASES = [
    ("1d_o4_ab2", lambda: W.wl_1d(256, 8, 4, 3, 0, 81, (1, 2, 3), r_alpha=0.02, tsteps=2)[0], 80),
    ("1d_o6_ab3", lambda: W.wl_1d(256, 8, 6, 4, 0, 82, (1, 2, 3), r_alpha=0.01, tsteps=3)[0], 60),
    ("1d_o2_ab3_point", lambda: W.wl_1d(250, 5, 2, 3, 0, 83, (1, 2), r_alpha=0.02, tsteps=3)[0], 70),
    ("1d_o4_std_ab2", lambda: W.wl_1d(256, 8, 4, 3, 0, 84, (1, 2), r_alpha=0.02, tsteps=2, scheme=W.ASYNC_STD)[0], 60),
    ("1d_o2_sync_ab2", lambda: W.wl_1d(128, 4, 2, 1, 0, 85, (1, 2), r_alpha=0.02, tsteps=2, scheme=W.SYNC)[0], 40),
    ("3d_o4_ab2", lambda: W.wl_3d([16, 12, 8], [2, 2, 2], 4, 3, 0, 86, c=(0.3, 0.2, 0.1), tsteps=2)[0], 20),
]


@pytest.mark.parametrize("name,make,nsteps", AB_CASES, ids=[c[0] for c in AB_CASES])
def test_multistep_adjoint_matches_cpu_adjoint(name, make, nsteps):
    spec = make()
    cfg = oracle.Config(spec)
    rng = np.random.default_rng(4)
    u0 = oracle.initial(cfg) + 0.01 * rng.standard_normal(cfg.shape)
    target = 0.5 * u0 + 0.1 * rng.standard_normal(cfg.shape)
    J, g, ga, _ = _gpu_grad(spec, nsteps, target, u0=u0)
    Jo, go, gao = oracle.adjoint(cfg, nsteps, target, u0=u0)
    assert J == pytest.approx(Jo, rel=1e-11)
    assert np.linalg.norm(g - go) / np.linalg.norm(go) <= 1e-12
    assert ga == pytest.approx(gao, rel=1e-10)


def test_multistep_adjoint_checkpoints_and_start():
    """The checkpoint interval does not change the bits; a run from Eq. "IC" (analytic pre-history, which depends
    on alpha) is refused with AT_ERR_STATE."""
    from paper_1702_00496_gb300 import Solver, binding as B
    spec, _ = W.wl_1d(512, 8, 6, 4, 0, 87, (1, 2, 3), r_alpha=0.01, tsteps=3)
    cfg = oracle.Config(spec)
    u0 = oracle.initial(cfg) + 0.01
    target = np.zeros(512)
    ref = None
    for every in (0, 1, 7, 97):
        J, g, ga, _ = _gpu_grad(spec, 97, target, every, u0=u0)
        if ref is None:
            ref = (J, g, ga)
        assert J == ref[0] and ga == ref[2] and np.array_equal(g, ref[1]), every
    s = Solver(spec)
    with pytest.raises(B.ATError) as e:
        s.adjoint_forward(10)
    assert e.value.code == B.AT_ERR_STATE
    s.close()


def test_multistep_autograd_function():
    from paper_1702_00496_gb300 import at_forward
    spec, _ = W.wl_1d(256, 8, 4, 3, 0, 88, (1, 2, 3), r_alpha=0.02, tsteps=2)
    cfg = oracle.Config(spec)
    u0n = oracle.initial(cfg) + 0.02
    u0 = torch.as_tensor(u0n, device="cuda").requires_grad_(True)
    alpha = torch.tensor(spec["alpha"], dtype=torch.float64, device="cuda", requires_grad=True)
    u = at_forward(u0, alpha, spec, 50)
    loss = 0.5 * (u ** 2).sum()
    loss.backward()
    Jo, go, gao = oracle.adjoint(cfg, 50, np.zeros(cfg.shape), u0=u0n)
    assert float(loss.detach()) == pytest.approx(Jo, rel=1e-11)
    assert np.linalg.norm(u0.grad.cpu().numpy() - go) / np.linalg.norm(go) <= 1e-12
    assert float(alpha.grad) == pytest.approx(gao, rel=1e-10)
