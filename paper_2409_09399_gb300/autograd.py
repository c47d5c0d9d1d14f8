"""Differentiable grid-integration energy (torch.autograd.Function).

E(R, V, D) = sum_g V_g rho_g[D; R] dV = sum_blocks D . H^V[V; R]     (Eq. 2, 3)

Forward and backward each make one call of the hand-written adjoint entry point
gint_energy_grads, which re-evaluates the orbital values (nothing from the
forward pass is stored) and forms, scaled by the upstream gradient on the
device:
  dE/dR_I = -F_I            (the Pulay force, Eq. 4)
  dE/dV_g = rho_g dV        (Eq. 3)
  dE/dD   = H^V             (Eq. 2)
and, through ``energy_and_strain``, dE/d(eps) = sum_I Pi_I = -Omega sigma (Eq. 5).
The handle carries the geometry: when the positions given differ from the
handle's, the handle is moved to them first (gint_update_positions with the
pattern kept, so D stays laid out on it; a displacement that changes the pair
pattern raises GINT_ERR_PATTERN_MISMATCH).
"""
from __future__ import annotations

import numpy as np
import torch

from .gint import Gint


def _move_to(g: Gint, pos):
    """Put the handle at positions ``pos`` (a tensor) if it is not there already."""
    p = pos.detach().to("cpu", torch.float64).numpy().reshape(g.n_atoms, 3)
    if not np.array_equal(p, g.pos):
        g.update_positions(p, keep_pattern=True)


class GintEnergy(torch.autograd.Function):
    """E = gint energy for handle ``g`` at positions ``pos`` (the handle follows ``pos``)."""

    @staticmethod
    def forward(ctx, pos, V, D, g: Gint):
        if not V.is_cuda or not D.is_cuda:
            raise TypeError("V and D must be CUDA tensors")
        _move_to(g, pos)
        ctx.g = g
        ctx.save_for_backward(pos.detach().clone(), V, D)
        out = g.energy_grads(V, D, want=("E",))
        return out["E"].reshape(()).to(pos.device)

    @staticmethod
    def backward(ctx, grad_E):
        pos, V, D = ctx.saved_tensors
        g = ctx.g
        _move_to(g, pos)  # another forward may have moved the handle since
        want = tuple(k for k, need in zip(("R", "V", "D"), ctx.needs_input_grad[:3]) if need)
        if not want:
            return None, None, None, None
        out = g.energy_grads(V, D, grad_E=grad_E.detach(), want=want)
        grad_pos = out["R"].to(pos.device, pos.dtype) if "R" in out else None
        return grad_pos, out.get("V"), out.get("D"), None


def energy(g: Gint, pos, V, D):
    """Differentiable E(pos, V, D) on handle ``g`` (pos: (n, 3) tensor; the handle is moved to it)."""
    return GintEnergy.apply(pos, V, D, g)


def energy_and_strain(g: Gint, V, D):
    """(E, dE/d(eps)) with eps a homogeneous strain of atoms, images and grid at fixed V_g and dV."""
    out = g.energy_grads(V, D, want=("E", "eps"))
    return out["E"].reshape(()), out["eps"]
