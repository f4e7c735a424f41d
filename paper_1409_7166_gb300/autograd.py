"""``torch.autograd.Function`` over pg_adjoint (argument marshalling only).

``IRDropObjective.apply(grid, r_g, c_val, h, nsteps, vref, margin, ckpt_every, l_val)``
returns the worst-IR-drop objective J of the transient of ``grid`` with
resistor conductances ``r_g``, capacitances ``c_val`` and (RLC grids)
inductances ``l_val`` (netlist order, CUDA float64 tensors; ``l_val`` may be
None for RC grids); ``backward`` returns dJ/dr_g, dJ/dc_val and dJ/dl_val
computed by the library's discrete adjoint.  The forward pass pushes the values into the grid
(``pg_update_values``) and runs the adjoint once, keeping the gradients for
the backward pass.
"""
from __future__ import annotations

import torch

from . import binding as B


class IRDropObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, grid, r_g, c_val, h, nsteps, vref=1.0, margin=0.05, ckpt_every=50, l_val=None):
        r_g = r_g.detach().contiguous()
        c_val = c_val.detach().contiguous()
        l_val = None if l_val is None else l_val.detach().contiguous()
        B.pg_set_stream(grid.handle, torch.cuda.current_stream().cuda_stream)
        B.pg_update_values(grid.handle, r_g=r_g, c_val=c_val, l_val=l_val)
        gG = torch.empty_like(r_g)
        gC = torch.empty_like(c_val)
        gL = None if l_val is None else torch.empty_like(l_val)
        J, st = B.pg_adjoint(grid.handle, h, nsteps, vref, margin, ckpt_every, dJ_dG=gG, dJ_dC=gC, dJ_dL=gL)
        ctx.save_for_backward(gG, gC, *(() if gL is None else (gL,)))
        ctx.has_l = gL is not None
        ctx.stats = st
        return torch.tensor(J, dtype=torch.float64, device=r_g.device)

    @staticmethod
    def backward(ctx, grad_out):
        saved = ctx.saved_tensors
        gG, gC = saved[0], saved[1]
        gL = grad_out * saved[2] if ctx.has_l else None
        return None, grad_out * gG, grad_out * gC, None, None, None, None, None, gL
