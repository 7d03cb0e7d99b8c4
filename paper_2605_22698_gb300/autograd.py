"""torch.autograd.Function around the library's separate forward and backward.

forward calls mlip_energy_forward: the energy only, no adjoint kernel; the
library keeps its copy of the positions and species, the neighbour list and
the node features of every layer.  backward calls mlip_energy_backward with
the incoming gradient: the library computes the edge geometry, the harmonics
and every layer's radial weights again from the saved positions (nothing per
edge is stored between the two calls) and runs its hand-written adjoint,
returning g dE/dr.  Argument marshalling only; nothing of the model is
computed in Python.

The backward differentiates the model's last forward: another evaluation of
the same model between the two calls makes the backward fail loudly
(MlipError), never return a stale gradient.
"""
from __future__ import annotations

import torch

from . import binding


class _Energy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pos, species, model, cell, pbc, stream):
        e = binding.mlip_energy_forward(model.h, pos.detach().contiguous(), species, cell, pbc, stream=stream)
        ctx.model, ctx.n, ctx.stream = model, int(pos.shape[0]), stream
        return e.reshape(())

    @staticmethod
    def backward(ctx, grad_e):
        g = binding.mlip_energy_backward(ctx.model.h, ctx.n, grad_e.detach(), stream=ctx.stream)
        return g, None, None, None, None, None


def energy(model: binding.Model, pos: torch.Tensor, species: torch.Tensor, cell, pbc, stream=None) -> torch.Tensor:
    """Energy (float64 scalar tensor) of one system whose positions (float64
    [n, 3]) and species (int32 [n]) are CUDA tensors; differentiable in pos:
    torch.autograd.grad(E, pos) is dE/dr = -F from the library's adjoint."""
    if not (pos.is_cuda and species.is_cuda):
        raise ValueError("positions and species must be CUDA tensors")
    if pos.dtype != torch.float64 or species.dtype != torch.int32:
        raise ValueError("positions must be float64 and species int32")
    return _Energy.apply(pos, species, model, cell, pbc, stream)
