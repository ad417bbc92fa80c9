"""Differentiable trajectories: x(T) as a torch.autograd.Function of the
body-frame dipoles m~ and the uniform field B, backed by the library's
hand-written adjoint (bpm_adjoint_begin / bpm_adjoint_end).

forward  : sets m~ and B on the handle, resets the starting state and runs
           n_steps steps with a checkpoint every `checkpoint_every` steps;
           returns the final positions [N, 3].
backward : given dL/dx(T), runs the reverse sweep and returns dL/dm~ and
           dL/dB.
"""
from __future__ import annotations

import numpy as np
import torch

from . import bpm as _bpm


class Trajectory(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m_body, B, sim, start, n_steps, checkpoint_every):
        sim.set_dipoles(np.ascontiguousarray(m_body.detach().cpu().numpy(), dtype=np.float64))
        sim.set_field(B=np.ascontiguousarray(B.detach().cpu().numpy(), dtype=np.float64))
        x0, q0, v0, w0, t0 = start
        sim.set_state(x0, q0, v0, w0, t0)
        sim.adjoint_begin(int(n_steps), int(checkpoint_every))
        x, _, _, _, _ = sim.get_state()
        ctx.sim = sim
        ctx.device = m_body.device
        return torch.from_numpy(x).to(m_body.device)

    @staticmethod
    def backward(ctx, grad_x):
        g = np.ascontiguousarray(grad_x.detach().cpu().numpy(), dtype=np.float64)
        gm, gB = ctx.sim.adjoint_end(g)
        return (torch.from_numpy(gm).to(ctx.device), torch.from_numpy(gB).to(ctx.device),
                None, None, None, None)


def final_positions(m_body: torch.Tensor, B: torch.Tensor, sim: "_bpm.Simulation", start, n_steps: int,
                    checkpoint_every: int = 50) -> torch.Tensor:
    """x(T) [N, 3] after n_steps from `start` = (x, q, v, omega, t)."""
    return Trajectory.apply(m_body, B, sim, start, n_steps, checkpoint_every)
