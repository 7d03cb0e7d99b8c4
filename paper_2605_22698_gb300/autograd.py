"""torch.autograd.Function around the library's energy call.

The adjoint is the library's hand-written backward (it recomputes the
harmonics and the radial weights per tile instead of storing per-edge
intermediates): one call produces the energy and dE/dr = -F, and the
backward of this Function only scales the stored -F by the incoming gradient.
Argument marshalling only; nothing of the model is computed in Python.
"""
from __future__ import annotations

import torch

from . import binding


class _Energy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pos, species, model, cell, pbc, stream):
        out = binding.mlip_energy_forces(model.h, pos.detach().contiguous(), species, cell, pbc, forces=True,
                                         stress=False, stream=stream)
        ctx.save_for_backward(out["forces"])
        return out["energy"].reshape(())

    @staticmethod
    def backward(ctx, grad_e):
        (forces,) = ctx.saved_tensors
        return -forces * grad_e, None, None, None, None, None


def energy(model: binding.Model, pos: torch.Tensor, species: torch.Tensor, cell, pbc, stream=None) -> torch.Tensor:
    """Energy (float64 scalar tensor) of one system whose positions (float64
    [n, 3]) and species (int32 [n]) are CUDA tensors; differentiable in pos:
    torch.autograd.grad(E, pos) is -F from the library's adjoint."""
    if not (pos.is_cuda and species.is_cuda):
        raise ValueError("positions and species must be CUDA tensors")
    if pos.dtype != torch.float64 or species.dtype != torch.int32:
        raise ValueError("positions must be float64 and species int32")
    return _Energy.apply(pos, species, model, cell, pbc, stream)
