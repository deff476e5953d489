"""torch.autograd wrapper of the simulation: gradients of a loss on the final
temperature with respect to needle power, tip position and per-label
conductivity and perfusion, through the library's discrete adjoint
(rfa_backward, sqrt(N) checkpoints and recomputation).

Argument marshalling only: the forward pass is rfa_set_tissue +
rfa_place_needle + rfa_step(record) + rfa_get_temperature, the backward pass
is rfa_backward; every numeric step runs in librfa.so.
"""
from __future__ import annotations

import copy
from typing import Sequence

import torch

from . import Grid, rfa_get_temperature


def pack_params(needle, table: Sequence) -> torch.Tensor:
    """[P, tip_x, tip_y, tip_z, k[0..L-1], w_b[0..L-1]] as float64."""
    vals = [needle.power, *[float(t) for t in needle.tip]]
    vals += [t.k for t in table] + [t.w_b for t in table]
    return torch.tensor(vals, dtype=torch.float64)


class BioheatRun(torch.autograd.Function):
    """T_final = run(params); dL/dparams from the adjoint of every step."""

    @staticmethod
    def forward(ctx, params, grid: Grid, labels, table, needle, nsteps: int):
        L = len(table)
        p = params.detach().cpu().double().tolist()
        tab = [copy.copy(t) for t in table]
        for l in range(L):
            tab[l].k = p[4 + l]
            tab[l].w_b = p[4 + L + l]
        nd = copy.copy(needle)
        nd.power = p[0]
        nd.tip = (p[1], p[2], p[3])
        grid.set_tissue(labels, tab)
        grid.place_needle(nd)
        grid.step(int(nsteps), record=True)
        T = torch.empty(grid.shape, dtype=torch.float32, device="cuda")
        rfa_get_temperature(grid.handle, T, True, False)
        ctx.grid = grid
        ctx.dtype = params.dtype
        return T

    @staticmethod
    def backward(ctx, grad_T):
        g = ctx.grid.backward(grad_T.detach().contiguous().float())
        return torch.from_numpy(g).to(ctx.dtype), None, None, None, None, None


def simulate(grid: Grid, labels, table, needle, params: torch.Tensor, nsteps: int) -> torch.Tensor:
    """Final temperature [nz, ny, nx] (CUDA, float32), differentiable in ``params``
    (see ``pack_params`` for the layout)."""
    return BioheatRun.apply(params, grid, labels, table, needle, nsteps)
