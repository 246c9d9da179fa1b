"""``torch.autograd.Function`` over the discrete adjoint of the library.

``CdWindow.apply(U, dr, window)`` returns the drag coefficient of one
cylinder averaged over a window of time steps, as a function of the inflow
speed ``U`` (0-d tensor) and the radial offsets ``dr`` of its markers (1-d
tensor, one per marker: marker l sits at centre + (R + dr_l)(cos t_l, sin t_l)).
The forward runs ``btdf_adjoint_forward`` (the window from a fixed start
state, a checkpoint every ``every`` steps); the backward runs
``btdf_adjoint_backward`` (segment recomputation and the hand-written reverse
kernels) and maps dJ/dX, dJ/dY onto the radial directions.  tau, ds and drs
are held fixed (nu fixed as U varies).  All arithmetic runs in the CUDA
library; this module only moves arguments and results.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import torch

from . import btdf as B


@dataclass
class DragWindow:
    """One lattice with a single cylinder, the start state of the window and
    the window's length.  ``theta`` are the markers' polar angles about
    (cx, cy) and ``radius`` their unperturbed distance."""
    lattice: B.Lattice
    start: bytes
    cx: float
    cy: float
    radius: float
    theta: np.ndarray
    nsteps: int
    every: int = 50
    body: int = 0
    dref: float = 1.0
    _tape: tuple = field(default=None, repr=False)

    @classmethod
    def for_lattice(cls, lattice, cx, cy, radius, nsteps, every=50, body=0, dref=None):
        """Takes the lattice's current state as the window start."""
        n = lattice.body_markers[body]
        theta = 2.0 * np.pi * np.arange(n, dtype=np.float64) / n
        return cls(lattice, lattice.save_state(), float(cx), float(cy), float(radius), theta,
                   int(nsteps), int(every), int(body), float(2.0 * radius if dref is None else dref))

    def positions(self, dr):
        r = self.radius + np.asarray(dr, dtype=np.float64)
        return self.cx + r * np.cos(self.theta), self.cy + r * np.sin(self.theta)

    def evaluate(self, U, dr) -> float:
        """J(U, dr); leaves the tape of this evaluation in the lattice."""
        lat = self.lattice
        lat.set_inflow(float(U))
        X, Y = self.positions(dr)
        lat.move_markers(self.body, X, Y)
        lat.load_state(self.start)
        J = lat.adjoint_forward(self.nsteps, self.every, self.body, self.dref)
        self._tape = (float(U), np.array(dr, dtype=np.float64, copy=True))
        return J

    def gradients(self, U, dr):
        """(dJ/dU, dJ/d dr) at (U, dr), re-running the forward window first
        when the lattice holds the tape of another evaluation."""
        if self._tape is None or self._tape[0] != float(U) or not np.array_equal(self._tape[1], dr):
            self.evaluate(U, dr)
        dU, dX, dY = self.lattice.adjoint_backward()
        first = self.lattice.body_first_marker(self.body)
        n = len(self.theta)
        ddr = dX[first:first + n] * np.cos(self.theta) + dY[first:first + n] * np.sin(self.theta)
        return dU, ddr


class CdWindow(torch.autograd.Function):
    """J = window-averaged Cd as a differentiable function of (U, dr)."""

    @staticmethod
    def forward(ctx, U, dr, window: DragWindow):
        u = float(U.detach().cpu())
        d = dr.detach().cpu().double().numpy()
        J = window.evaluate(u, d)
        ctx.window, ctx.u, ctx.d = window, u, d
        ctx.meta = (U.dtype, U.device, dr.dtype, dr.device)
        return torch.tensor(J, dtype=torch.float64, device=U.device)

    @staticmethod
    def backward(ctx, gJ):
        dU, ddr = ctx.window.gradients(ctx.u, ctx.d)
        udt, udev, rdt, rdev = ctx.meta
        g = float(gJ.detach().cpu())
        return (torch.tensor(g * dU, dtype=udt, device=udev),
                torch.from_numpy(g * ddr).to(dtype=rdt, device=rdev), None)
