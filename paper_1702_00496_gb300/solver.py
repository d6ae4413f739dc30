"""Device-memory plumbing around the C ABI: a solver whose ring buffer and delay log are torch tensors."""
from __future__ import annotations

import torch

from . import binding as B


class Solver:
    """One AT problem on the GPU.

    The ring buffer holds R = L + T full time levels (level m in slot m mod R); the delay log holds the
    raw delay of every PE side at every step, so the run can be replayed.  All arithmetic happens in
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
        n = self.n
        slot = n % self.R
        return self.ring[slot * self.cfg.ntot:(slot + 1) * self.cfg.ntot].view(self.cfg.shape)

    def delays(self) -> torch.Tensor:
        """Raw delays logged so far, [steps, sides] uint8."""
        if self.log is None:
            raise RuntimeError("solver was created without a delay log")
        return self.log.view(self.log_steps, self.sides)[: self.n]

    def error_stats(self) -> dict:
        return B.at_error_stats(self.h)

    def close(self) -> None:
        if self.h is not None:
            B.at_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
