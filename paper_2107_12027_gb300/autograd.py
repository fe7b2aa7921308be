"""torch.autograd wrapper of the adjoint (gradients with respect to initial data).

``RKSteps.apply(prim0, grid, x0, nsteps, dt)`` advances the initial primitive
state ``prim0`` ([m, ny, nx] FP64 CUDA tensor; m = 4 on RHD grids, 8 on RMHD
grids) on the grid's mesh ``x0`` by
``nsteps`` SSP-RK3 steps and returns the final conserved state J U; its
backward pass runs the library's adjoint (recorded mesh velocities and steps,
per-step checkpoints) and returns the gradient with respect to ``prim0``.
"""
from __future__ import annotations

import torch

from . import esmm


class RKSteps(torch.autograd.Function):
    @staticmethod
    def forward(ctx, prim0, grid, x0, nsteps, dt=0.0):
        prim0 = prim0.detach().contiguous()
        grid.state_set(prim0, x0.contiguous())
        grid.adjoint_record(int(nsteps), float(dt))
        out = torch.empty_like(prim0)
        grid.state_get(esmm.GET_CONS, out)
        ctx.grid = grid
        return out

    @staticmethod
    def backward(ctx, grad_cons):
        lam_prim = torch.empty_like(grad_cons)
        ctx.grid.adjoint_vjp(grad_cons.contiguous(), None, lam_prim)
        return lam_prim, None, None, None, None
