"""Device-memory plumbing around the C ABI: a solver whose ring buffer and delay log are torch tensors."""
from __future__ import annotations

import torch

from . import binding as B


class Solver:
    """One AT problem on the GPU.

    The ring buffer holds the L + T time levels (level m in slot m mod (L + T)) and, for Adams-Bashforth, the
    stored right-hand sides after them; the delay log holds the raw delay of every PE side at every step, so
    the run can be replayed.  All arithmetic happens in
    libatfd's kernels; this class only allocates memory and forwards calls.
    """

    def __init__(self, spec: dict, log_steps: int = 0, device: str | torch.device = "cuda", stream=None):
        B.load()
        self.cfg = B.Config(spec)
        self.R = B.at_ring_slots(self.cfg)
        self.sides = B.at_num_sides(self.cfg)
        self.device = torch.device(device)
        self.ring = torch.empty(self.R * self.cfg.ntot, dtype=torch.float64, device=self.device)
        self.log_steps = int(log_steps)
        self.log = (torch.zeros(self.log_steps * self.sides, dtype=torch.uint8, device=self.device)
                    if self.log_steps > 0 else None)
        self.stream = stream
        self.h = B.at_init(self.cfg, self.ring, self.log, self.log_steps, stream)

    def reset(self, u0: torch.Tensor | None = None) -> None:
        """Back to step 0 with U^0 = Eq. "IC" (u0 None) or the given device field."""
        if u0 is not None:
            u0 = u0.reshape(-1).to(device=self.device, dtype=torch.float64).contiguous()
        B.at_reset(self.h, u0)

    def step(self, nsteps: int) -> None:
        B.at_step(self.h, nsteps)

    def sync(self) -> None:
        B.at_sync(self.h)

    @property
    def n(self) -> int:
        return B.at_state(self.h)[0]

    def field(self) -> torch.Tensor:
        """View of U^n inside the ring (shape (nx,) or (nz, ny, nx))."""
        _, ptr = B.at_state(self.h)
        off = (ptr - self.ring.data_ptr()) // self.ring.element_size()
        return self.ring[off:off + self.cfg.ntot].view(self.cfg.shape)

    def delays(self) -> torch.Tensor:
        """Raw delays logged so far, [steps, sides] uint8."""
        if self.log is None:
            raise RuntimeError("solver was created without a delay log")
        return self.log.view(self.log_steps, self.sides)[: self.n]

    def error_stats(self) -> dict:
        return B.at_error_stats(self.h)

    def error_stats_ref(self, ref: torch.Tensor, refine: int) -> dict:
        """Statistics of U^n - V for a reference field V `refine` times finer on every axis (e.g. a finer run)."""
        ref = ref.reshape(-1).to(device=self.device, dtype=torch.float64).contiguous()
        return B.at_error_stats_ref(self.h, ref, refine)

    def adjoint_forward(self, nsteps: int, ckpt_every: int = 0) -> None:
        """Run nsteps from step 0 keeping checkpoints every ckpt_every steps (0: ceil(sqrt(nsteps)); ckpt_every >=
        nsteps: every level stays in the workspace and the backward sweep recomputes nothing)."""
        n = B.at_adjoint_workspace(self.h, nsteps, ckpt_every)
        if getattr(self, "work", None) is None or self.work.numel() < n:
            self.work = None
            self.work = torch.empty(n, dtype=torch.float64, device=self.device)
        B.at_adjoint_forward(self.h, nsteps, ckpt_every, self.work)

    def adjoint_backward(self, lam: torch.Tensor, want_alpha: bool = True):
        """dJ/dU^0 (shaped like the field) and dJ/dalpha (None if not wanted) for lam = dJ/dU^nsteps."""
        lam = lam.reshape(-1).to(device=self.device, dtype=torch.float64).contiguous()
        g = torch.empty(self.cfg.ntot, dtype=torch.float64, device=self.device)
        ga = B.at_adjoint_backward(self.h, lam, g, want_alpha)
        return g.view(self.cfg.shape), ga

    def close(self) -> None:
        if self.h is not None:
            B.at_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Ensemble:
    """Many independent 1D realizations advanced in one persistent, graph-captured launch.

    nsteps: one step count for every member, or one per member.  groups: optional summary-group labels (default:
    group by grid size).  twins: optional index per member of the member whose final field it is compared with
    (-1: none), e.g. its synchronous twin.
    """

    def __init__(self, specs, nsteps, log: bool = False, threads: int = 0, ctas_per_sm: int = 0,
                 device: str | torch.device = "cuda", stream=None, groups=None, twins=None):
        B.load()
        self.cfgs = [B.Config(s) for s in specs]
        count = len(self.cfgs)
        self.steps = ([int(nsteps)] * count if not hasattr(nsteps, "__len__") else [int(v) for v in nsteps])
        self.nsteps = max(self.steps)
        self.device = torch.device(device)
        ring_len, log_len = B.at_ensemble_sizes(self.cfgs, self.steps, groups, twins)
        self.ring = torch.empty(ring_len, dtype=torch.float64, device=self.device)
        self.log = torch.zeros(log_len, dtype=torch.uint8, device=self.device) if log else None
        self.R = [B.at_ring_slots(c) for c in self.cfgs]
        self.sides = [B.at_num_sides(c) for c in self.cfgs]
        self.ring_off, self.log_off = [], []
        ro = lo = 0
        for c, R, nb, st in zip(self.cfgs, self.R, self.sides, self.steps):
            self.ring_off.append(ro)
            self.log_off.append(lo)
            ro += R * c.ntot
            lo += st * nb
        self.h = B.at_ensemble_create(self.cfgs, self.steps, self.ring, self.log, threads, ctas_per_sm, stream,
                                      groups, twins)

    def run(self) -> None:
        B.at_ensemble_run(self.h)

    def stats(self):
        return B.at_ensemble_stats(self.h, len(self.cfgs))

    def field(self, r: int) -> torch.Tensor:
        """Member r's field at its final step (valid after run())."""
        c = self.cfgs[r]
        levels = self.R[r] - (c.tsteps - 1)  # slots after the L + T levels hold Adams-Bashforth right-hand sides
        slot = self.steps[r] % levels
        o = self.ring_off[r] + slot * c.ntot
        return self.ring[o:o + c.ntot]

    def delays(self, r: int) -> torch.Tensor:
        if self.log is None:
            raise RuntimeError("ensemble was created without a delay log")
        o = self.log_off[r]
        return self.log[o:o + self.steps[r] * self.sides[r]].view(self.steps[r], self.sides[r])

    def close(self) -> None:
        if self.h is not None:
            B.at_ensemble_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
