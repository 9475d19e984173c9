"""torch.autograd bindings for the effective conductivity.

sigma_* is a smooth (holomorphic) function of the conductivities.  The first
variation of the energy <sigma E.E> = sigma_* |e|^2 (Eq. J12, J13 of the paper,
bilinear dot product) gives

    d sigma_* / d sigma(x) = E(x).E(x) / (N |e|^2),

so the backward pass is one more field solve (the field is recomputed rather
than kept between forward and backward) followed by the library's pointwise
gradient kernel.  For complex inputs the returned gradient follows PyTorch's
convention for holomorphic maps: grad_input = grad_output * conj(d sigma_*/d z).

Only argument marshalling happens here: the solves and the gradient run in
liblsfft.so.
"""
from __future__ import annotations

import torch

from . import Grid


def _scalar_out(value: complex, like: torch.Tensor) -> torch.Tensor:
    if like.is_complex():
        return torch.tensor(value, dtype=like.dtype)
    return torch.tensor(value.real, dtype=like.dtype)


class SigmaStarOfSigma1(torch.autograd.Function):
    """sigma_*(sigma_1) on a two-phase grid: forward(sigma1 (0-d tensor), grid, e, opts dict)."""

    @staticmethod
    def forward(ctx, sigma1: torch.Tensor, grid: Grid, e, opts: dict):
        s1 = complex(sigma1.detach().cpu().item())
        r = grid.solve(s1, e, **opts)
        value = r.sigma_star
        r.free()
        ctx.grid, ctx.e, ctx.opts, ctx.s1 = grid, list(e), dict(opts), s1
        ctx.complex_in = sigma1.is_complex()
        return _scalar_out(value, sigma1).to(sigma1.device)

    @staticmethod
    def backward(ctx, grad_out):
        r = ctx.grid.solve(ctx.s1, ctx.e, **ctx.opts)       # recompute the field
        d1, _ = ctx.grid.gradient(r, ctx.e)
        r.free()
        if ctx.complex_in:
            g = grad_out * torch.tensor(d1.conjugate(), dtype=grad_out.dtype, device=grad_out.device)
        else:
            g = grad_out * d1.real
        return g, None, None, None


class SigmaStarOfField(torch.autograd.Function):
    """sigma_* of a per-voxel conductivity field (CUDA tensor of the grid's shape):
    forward(sigma_field, grid, e, opts dict), MS or EM scheme."""

    @staticmethod
    def forward(ctx, sigma: torch.Tensor, grid: Grid, e, opts: dict):
        grid.set_sigma_field(sigma.detach())
        r = grid.solve(1.0, e, **opts)
        value = r.sigma_star
        r.free()
        ctx.grid, ctx.e, ctx.opts = grid, list(e), dict(opts)
        ctx.save_for_backward(sigma.detach())
        return _scalar_out(value, sigma).to(sigma.device)

    @staticmethod
    def backward(ctx, grad_out):
        (sigma,) = ctx.saved_tensors
        ctx.grid.set_sigma_field(sigma)
        r = ctx.grid.solve(1.0, ctx.e, **ctx.opts)          # recompute the field
        dt = torch.complex64 if r.precision == 0 else torch.complex128
        g = torch.empty(sigma.shape, dtype=dt, device=sigma.device)
        ctx.grid.gradient(r, ctx.e, g.data_ptr())
        r.free()
        if sigma.is_complex():
            return grad_out * g.conj().to(sigma.dtype), None, None, None
        return grad_out * g.real.to(sigma.dtype), None, None, None


def sigma_star(sigma1: torch.Tensor, grid: Grid, e, **opts) -> torch.Tensor:
    return SigmaStarOfSigma1.apply(sigma1, grid, e, opts)


def sigma_star_field(sigma: torch.Tensor, grid: Grid, e, **opts) -> torch.Tensor:
    return SigmaStarOfField.apply(sigma, grid, e, opts)
