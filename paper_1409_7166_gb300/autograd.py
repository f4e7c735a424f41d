"""``torch.autograd.Function`` over pg_adjoint (argument marshalling only).

``IRDropObjective.apply(grid, r_g, c_val, h, nsteps, vref, margin, ckpt_every)``
returns the worst-IR-drop objective J of the RC transient of ``grid`` with
resistor conductances ``r_g`` and capacitances ``c_val`` (netlist order, CUDA
float64 tensors); ``backward`` returns dJ/dr_g and dJ/dc_val computed by the
library's discrete adjoint.  The forward pass pushes the values into the grid
(``pg_update_values``) and runs the adjoint once, keeping the gradients for
the backward pass.
"""
from __future__ import annotations

import torch

from . import binding as B


class IRDropObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, grid, r_g, c_val, h, nsteps, vref=1.0, margin=0.05, ckpt_every=50):
        r_g = r_g.detach().contiguous()
        c_val = c_val.detach().contiguous()
        B.pg_set_stream(grid.handle, torch.cuda.current_stream().cuda_stream)
        B.pg_update_values(grid.handle, r_g=r_g, c_val=c_val)
        gG = torch.empty_like(r_g)
        gC = torch.empty_like(c_val)
        J, st = B.pg_adjoint(grid.handle, h, nsteps, vref, margin, ckpt_every, dJ_dG=gG, dJ_dC=gC)
        ctx.save_for_backward(gG, gC)
        ctx.stats = st
        return torch.tensor(J, dtype=torch.float64, device=r_g.device)

    @staticmethod
    def backward(ctx, grad_out):
        gG, gC = ctx.saved_tensors
        return None, grad_out * gG, grad_out * gC, None, None, None, None, None
