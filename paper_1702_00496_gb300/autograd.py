"""torch.autograd.Function over the AT forward run, differentiated by the hand-written adjoint kernels."""
from __future__ import annotations

import torch

from .solver import Solver


class ATForward(torch.autograd.Function):
    """U^nsteps = AT forward run of `nsteps` steps of the problem `spec` from u0, with diffusivity alpha.

    backward() returns dJ/du0 and dJ/dalpha through the same delays (replayed from the counter-based generator),
    using checkpoints every ckpt_every steps (0: ceil(sqrt(nsteps)); ckpt_every >= nsteps keeps every level in the
    workspace, about nsteps fields, and recomputes nothing).
    """

    @staticmethod
    def forward(ctx, u0: torch.Tensor, alpha: torch.Tensor, spec: dict, nsteps: int, ckpt_every: int = 0):
        s = dict(spec)
        s["alpha"] = float(alpha)
        solver = Solver(s, device=u0.device)
        solver.reset(u0.detach())
        solver.adjoint_forward(int(nsteps), int(ckpt_every))
        ctx.solver = solver
        ctx.alpha_meta = (alpha.dtype, alpha.device, alpha.shape)
        return solver.field().clone().view_as(u0)

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        solver = ctx.solver
        want_alpha = ctx.needs_input_grad[1]
        g0, ga = solver.adjoint_backward(grad_out.detach(), want_alpha)
        solver.close()
        ctx.solver = None
        dtype, device, shape = ctx.alpha_meta
        galpha = torch.full(shape, ga, dtype=dtype, device=device) if want_alpha else None
        return g0.view_as(grad_out), galpha, None, None, None


def at_forward(u0: torch.Tensor, alpha: torch.Tensor, spec: dict, nsteps: int, ckpt_every: int = 0) -> torch.Tensor:
    return ATForward.apply(u0, alpha, spec, nsteps, ckpt_every)
