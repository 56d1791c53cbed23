"""torch.autograd.Function around the matvec and its adjoint kernel.

H(J) = -sum_b J_b s_u.s_v is symmetric and linear in J (Eq. E-2-1), so for a loss L(y)
with y = H(J) x and g = dL/dy:
    dL/dx   = H(J) g                         (the same row kernel, Eq. E-4-b)
    dL/dJ_b = -sum_i g_i [(s_u.s_v) x]_i     (the bond-correlation kernel)
"""
from __future__ import annotations

import numpy as np
import torch

from . import api


class HeisenbergMatvec(torch.autograd.Function):
    """y = HeisenbergMatvec.apply(x, J, basis, u, v): x on the GPU ([dim], float64/float32),
    J a float64 tensor of couplings (any device; its gradient comes back on that device),
    u, v integer site arrays."""

    @staticmethod
    def forward(ctx, x, J, basis, u, v):
        bonds = api.BondList.make(u, v, J.detach().cpu().numpy())
        ctx.basis, ctx.bonds = basis, bonds
        ctx.save_for_backward(x)
        ctx.J_device = J.device
        return api.matvec(basis, bonds, x)

    @staticmethod
    def backward(ctx, g):
        (x,) = ctx.saved_tensors
        g = g.contiguous()
        gx = api.matvec(ctx.basis, ctx.bonds, g) if ctx.needs_input_grad[0] else None
        gJ = None
        if ctx.needs_input_grad[1]:
            gJ = (-api.bond_corr(ctx.basis, ctx.bonds, g, x)).to(ctx.J_device)
        return gx, gJ, None, None, None


def ground_energy_grad(basis, u, v, J: np.ndarray, steps: int, seed: int = 0, v0=None):
    """E0 and dE0/dJ (Hellmann-Feynman) through the library's e0_grad."""
    bonds = api.BondList.make(u, v, J)
    e0, g, _, rc = api.e0_grad(basis, bonds, steps, v0=v0, seed=seed)
    return e0, g, rc
