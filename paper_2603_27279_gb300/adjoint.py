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


def _device_f64(t: torch.Tensor, device) -> torch.Tensor:
    return t.detach().to(device=device, dtype=torch.float64).contiguous()


class Trajectory(torch.autograd.Function):
    """m~ [N, 3], dL/dx and dL/dm~ cross the C ABI as device tensors when the
    inputs live on the GPU (the library reads and writes them in place); only
    the three components of B and of dL/dB go through the host, as the ABI
    takes the uniform field on the host."""

    @staticmethod
    def forward(ctx, m_body, B, sim, start, n_steps, checkpoint_every):
        dev = m_body.device
        mb = _device_f64(m_body, dev) if m_body.is_cuda else np.ascontiguousarray(
            m_body.detach().cpu().numpy(), dtype=np.float64)
        sim.set_dipoles(mb)
        sim.set_field(B=np.ascontiguousarray(B.detach().cpu().numpy(), dtype=np.float64))
        x0, q0, v0, w0, t0 = start
        sim.set_state(x0, q0, v0, w0, t0)
        sim.adjoint_begin(int(n_steps), int(checkpoint_every))
        ctx.sim = sim
        ctx.device = dev
        if m_body.is_cuda:
            x = torch.empty((sim.n, 3), dtype=torch.float64, device=dev)
            _bpm.bpm_get_state(sim.h, x=x)
            return x
        x, _, _, _, _ = sim.get_state()
        return torch.from_numpy(x)

    @staticmethod
    def backward(ctx, grad_x):
        sim = ctx.sim
        if grad_x.is_cuda:
            g = _device_f64(grad_x, grad_x.device)
            gm = torch.empty((sim.n, 3), dtype=torch.float64, device=grad_x.device)
            gB = _bpm.bpm_adjoint_end(sim.h, g, gm)
            return gm.to(ctx.device), torch.from_numpy(gB).to(ctx.device), None, None, None, None
        gm, gB = sim.adjoint_end(np.ascontiguousarray(grad_x.detach().cpu().numpy(), dtype=np.float64))
        return (torch.from_numpy(gm).to(ctx.device), torch.from_numpy(gB).to(ctx.device),
                None, None, None, None)


def final_positions(m_body: torch.Tensor, B: torch.Tensor, sim: "_bpm.Simulation", start, n_steps: int,
                    checkpoint_every: int = 50) -> torch.Tensor:
    """x(T) [N, 3] after n_steps from `start` = (x, q, v, omega, t)."""
    return Trajectory.apply(m_body, B, sim, start, n_steps, checkpoint_every)
