"""torch.autograd integration: the renderer as a differentiable function of (V, sigma).

forward  -> dm_render (image of the mesh under the PSF, Eq. 1)
backward -> dm_render_adjoint (Eq. 6, 9-10 and the chain rule through the transfer
            function); the mesh spectrum is recomputed inside the adjoint call rather than
            saved from the forward, so the autograd graph holds only V and sigma.
"""

from __future__ import annotations

import torch

from .api import PSF, Renderer


class _Render(torch.autograd.Function):
    @staticmethod
    def forward(ctx, V, sigma, F, renderer: Renderer, grid, band_tau: float, label: str, weights):
        psf = PSF(sigma=tuple(float(s) for s in sigma.detach().cpu().tolist()), band_tau=band_tau)
        img = renderer.render(V.detach(), F, grid, psf, label=label, weights=weights)
        ctx.renderer, ctx.grid, ctx.psf, ctx.label, ctx.weights, ctx.F = renderer, grid, psf, label, weights, F
        ctx.save_for_backward(V, sigma)
        return img

    @staticmethod
    def backward(ctx, dI):
        V, sigma = ctx.saved_tensors
        dV, dpsf = ctx.renderer.render_adjoint(V.detach(), ctx.F, ctx.grid, ctx.psf,
                                               dI.contiguous().to(ctx.renderer.real), label=ctx.label,
                                               weights=ctx.weights)
        dV = dV.to(V.dtype) if ctx.needs_input_grad[0] else None
        ds = dpsf.to(device=sigma.device, dtype=sigma.dtype) if ctx.needs_input_grad[1] else None
        return dV, ds, None, None, None, None, None, None


def render(V: torch.Tensor, sigma: torch.Tensor, F: torch.Tensor, renderer: Renderer, grid, band_tau: float = 0.0,
           label: str = "surface", weights=None) -> torch.Tensor:
    """Differentiable image of the mesh (V [n_v, 3] float64, F [n_t, 3] int32) under a diagonal
    Gaussian PSF with standard deviations `sigma` [3]. Gradients flow to V and sigma."""
    return _Render.apply(V, sigma, F, renderer, grid, band_tau, label, weights)
