"""torch.autograd.Function for the spin energy (Methods, "Gradient, HVP, and
Hessian via the autograd engine").

    E = energy(m, ctx)                     # forward: E(m), FP64 scalar
    g, = torch.autograd.grad(E, m, create_graph=True)   # backward: grad E
    Hv, = torch.autograd.grad(g, m, v)     # double backward: hess E v

The forward calls moto_energy (double arithmetic) and each derivative is one
launch of the library: the backward of E calls
moto_energy_euclid_grad, the backward of grad E calls moto_euclid_hvp, and so
does every further backward (E is quadratic in m, so hess E is constant and
symmetric; third derivatives vanish).  The upstream scalar of a backward
scales the field with one torch multiply; no derivative is formed in Python.
"""
from __future__ import annotations

import torch

from . import moto_energy, moto_energy_euclid_grad, moto_euclid_hvp


def _check_field(ctx, x):
    if x.dtype != ctx.dtype or x.device != ctx.device:
        raise TypeError(f"expected a {ctx.dtype} tensor on {ctx.device}")
    if tuple(x.shape) != (3, ctx.L2, ctx.L1):
        raise ValueError(f"expected shape (3, {ctx.L2}, {ctx.L1}), got {tuple(x.shape)}")
    return x.contiguous()


class _HessApply(torch.autograd.Function):
    """v -> hess E v (linear in v, independent of m)."""

    @staticmethod
    def forward(fctx, v, ctx):
        fctx.moto = ctx
        v = _check_field(ctx, v)
        hv = torch.empty_like(v)
        moto_euclid_hvp(ctx.handle, v, 3 * ctx.N, hv, 3 * ctx.N, 1)
        return hv

    @staticmethod
    def backward(fctx, gout):
        return _HessApply.apply(gout.contiguous(), fctx.moto), None


class _Grad(torch.autograd.Function):
    """m -> grad E(m); its Jacobian is hess E."""

    @staticmethod
    def forward(fctx, m, ctx):
        fctx.moto = ctx
        m = _check_field(ctx, m)
        g = torch.empty_like(m)
        out = torch.empty(2, dtype=torch.float64, device=m.device)
        moto_energy_euclid_grad(ctx.handle, m, g, out)
        return g

    @staticmethod
    def backward(fctx, gout):
        return _HessApply.apply(gout.contiguous(), fctx.moto), None


class MotoEnergy(torch.autograd.Function):
    """m (3, L2, L1) -> E (FP64 scalar tensor)."""

    @staticmethod
    def forward(fctx, m, ctx):
        fctx.moto = ctx
        m = _check_field(ctx, m)
        fctx.save_for_backward(m)
        E = torch.empty(1, dtype=torch.float64, device=m.device)
        moto_energy(ctx.handle, m, E)
        return E[0]

    @staticmethod
    def backward(fctx, gE):
        (m,) = fctx.saved_tensors
        g = _Grad.apply(m, fctx.moto)
        return gE.to(g.dtype) * g, None


def energy(m: torch.Tensor, ctx) -> torch.Tensor:
    """E(m) with first and second derivatives through the library (ctx: a
    ``Context`` of the same lattice, dtype and device as m)."""
    return MotoEnergy.apply(m, ctx)
