"""torch.autograd glue over the library's hand-written adjoints.

Both functions only marshal tensors: every value and every derivative comes
from the library's kernels (the energy adjoint of Eq. 1, F = -dE/dr, and the
weight adjoint of the loss of Eq. 3).

- ``energy(handle, positions, species, cell)``: E(r) as a 0-dim float64
  tensor.  The forward call already runs the adjoint pair passes (the library
  evaluates E and F together), so backward returns -F times the incoming
  gradient.  Second derivatives are not provided.
- ``batch_loss(handle, weights, batch)``: the training loss L(w) of a built
  batch as a 0-dim float64 tensor, differentiable in the flat FP32 weight
  vector (blob order, ``ALLEGRO_Q_N_PARAMS`` entries).  The forward call
  loads ``weights`` into the context (``allegro_set_weights``, which also
  resets the library's own Adam state) and runs ``allegro_loss_grad``;
  backward returns the saved gradient times the incoming gradient.  With
  it a torch optimizer can drive the library's loss and gradient.
"""
import numpy as np
import torch

from . import (ALLEGRO_FP32, allegro_energy_forces, allegro_loss_grad, allegro_set_weights)


class EnergyFunction(torch.autograd.Function):
    @staticmethod
    def forward(fctx, positions, handle, species, cell, precision):
        pos = positions.detach().to(torch.float64).contiguous()
        forces = torch.empty((pos.shape[0], 3), dtype=torch.float32, device=pos.device)
        e = allegro_energy_forces(handle, pos, species, cell, forces, None, precision)
        fctx.save_for_backward(forces)
        return torch.tensor(e, dtype=torch.float64, device=positions.device)

    @staticmethod
    def backward(fctx, grad_e):
        (forces,) = fctx.saved_tensors
        return -grad_e * forces.to(torch.float64), None, None, None, None


class BatchLossFunction(torch.autograd.Function):
    @staticmethod
    def forward(fctx, weights, handle, batch, w_energy, w_force):
        w = weights.detach().to(torch.float32).contiguous()
        allegro_set_weights(handle, w)
        grad = torch.empty_like(w)
        loss = allegro_loss_grad(handle, batch, w_energy, w_force, grad)
        fctx.save_for_backward(grad)
        return torch.tensor(loss, dtype=torch.float64, device=weights.device)

    @staticmethod
    def backward(fctx, grad_l):
        (grad,) = fctx.saved_tensors
        return (grad_l * grad.to(torch.float64)).to(torch.float32), None, None, None, None


def energy(handle, positions, species, cell, precision=ALLEGRO_FP32):
    """Total energy E(positions) (N x 3 float64 CUDA tensor), differentiable
    in positions through the library's force kernels."""
    return EnergyFunction.apply(positions, handle, species, np.asarray(cell, dtype=np.float64), int(precision))


def batch_loss(handle, weights, batch, w_energy=1.0, w_force=100.0):
    """Loss of the built batch (``make_batch``) at ``weights`` (float32 CUDA
    tensor), differentiable in weights through the library's weight adjoint."""
    return BatchLossFunction.apply(weights, handle, batch, float(w_energy), float(w_force))
