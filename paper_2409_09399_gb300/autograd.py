"""Differentiable grid-integration energy (torch.autograd.Function).

E(R, V, D) = sum_g V_g rho_g[D; R] dV = sum_blocks D . H^V[V; R]     (Eq. 2, 3)

Forward runs gint_force_stress for E only.  Backward calls the hand-written
kernels again, re-evaluating the orbital values (nothing from the forward
pass is stored):
  dE/dR_I = -F_I            (gint_force_stress; F is the Pulay force, Eq. 4)
  dE/dV_g = rho_g dV        (gint_rho)
  dE/dD   = H^V             (gint_vlocal)
and, through ``energy_and_strain``, dE/d(eps) = -Omega sigma (Eq. 5).
The geometry is fixed per handle: positions enter the function as a tensor
so that autograd routes dE/dR, while the handle (built by ``gint_setup`` for
those positions) supplies the pattern, the bricks and the tables.
"""
from __future__ import annotations

import torch

from .gint import Gint


class GintEnergy(torch.autograd.Function):
    """E = gint energy for handle ``g`` at positions ``pos`` (must equal the handle's)."""

    @staticmethod
    def forward(ctx, pos, V, D, g: Gint):
        if not V.is_cuda or not D.is_cuda:
            raise TypeError("V and D must be CUDA tensors")
        ctx.g = g
        ctx.save_for_backward(V, D)
        ctx.pos_device = pos.device
        ctx.pos_dtype = pos.dtype
        _, _, _, E = g.force_stress(V, D)
        return E.reshape(()).to(pos.device)

    @staticmethod
    def backward(ctx, grad_E):
        V, D = ctx.saved_tensors
        g = ctx.g
        grad_pos = grad_V = grad_D = None
        ge = grad_E.to(V.device)
        if ctx.needs_input_grad[0]:
            F, _, _, _ = g.force_stress(V, D)
            grad_pos = (-F * ge).to(ctx.pos_device, ctx.pos_dtype)
        if ctx.needs_input_grad[1]:
            rho = g.rho(D)
            grad_V = rho * (g.dV * ge)
        if ctx.needs_input_grad[2]:
            H = g.vlocal(V)
            grad_D = H * ge
        return grad_pos, grad_V, grad_D, None


def energy(g: Gint, pos, V, D):
    """Differentiable E(pos, V, D) on handle ``g`` (pos: (n, 3) tensor equal to the handle's positions)."""
    return GintEnergy.apply(pos, V, D, g)


def energy_and_strain(g: Gint, V, D):
    """(E, dE/d(eps)) with eps a homogeneous strain of atoms, images and grid at fixed V_g and dV."""
    _, sigma, _, E = g.force_stress(V, D)
    return E.reshape(()), -sigma * g.omega
