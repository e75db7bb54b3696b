"""torch.autograd.Functions over the imaging operator and its adjoint.

Both functions run on an ``Imager`` whose geometry was set by ``Imager.bin``
(uvw, weights); they change only the values gridded through that geometry.
m is the imager's image side (its grid side n unless the grid is padded).

GridFn   vis (complex64 [n_vis]) -> image (float32 [m, m]) = A vis, the
         w-stacked image (grid, inverse FFT per plane, w-correct, stack).
         backward: grad_vis = A^H grad_image -- w-spread, forward FFT,
         degrid, the hand-written adjoint (the oracle pins it).
DegridFn image (float32 [m, m]) -> model visibilities (complex64 [n_vis]) = D x,
         the degridding predictor of Eq. 1 (x / n / taper, forward FFT per plane,
         degrid, no weights).  backward: grad_image = Re(D^H grad_vis) --
         grid with unit weights, inverse FFT, w-correct with the same scaling.

With torch's convention for complex tensors (the gradient of L = sum(y * Re(M z))
with respect to z is M^H y), these backward passes are the exact gradients of
the forward operators, which is what makes chi^2 = sum w |V_obs - D x|^2
differentiable with respect to the image pixels.
"""
from __future__ import annotations

import torch

from .imager import IMAGE_FLAGS, PREDICT_FLAGS, Imager


class GridFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vis: torch.Tensor, imager: Imager, weight: torch.Tensor | None = None,
                flags: int = IMAGE_FLAGS):
        imager.bin_values(vis.detach().contiguous(), weight)
        img = imager.image_from_binned(flags)
        ctx.imager, ctx.weight, ctx.flags = imager, weight, flags
        return img

    @staticmethod
    def backward(ctx, grad_image: torch.Tensor):
        g = ctx.imager.adjoint(grad_image.detach().float().contiguous(), ctx.weight, ctx.flags)
        return g, None, None, None


class DegridFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, image: torch.Tensor, imager: Imager, flags: int = PREDICT_FLAGS):
        v = imager.adjoint(image.detach().float().contiguous(), None, flags)
        ctx.imager, ctx.flags = imager, flags
        return v

    @staticmethod
    def backward(ctx, grad_vis: torch.Tensor):
        im = ctx.imager
        im.bin_values(grad_vis.detach().to(torch.complex64).contiguous(), None)
        g = im.image_from_binned(ctx.flags)
        return g, None, None


def grid_image(vis, imager, weight=None, flags=IMAGE_FLAGS):
    """Differentiable w-stacked image of ``vis`` through ``imager``'s binning."""
    return GridFn.apply(vis, imager, weight, flags)


def predict(image, imager, flags=PREDICT_FLAGS):
    """Differentiable model visibilities of ``image`` through ``imager``'s binning."""
    return DegridFn.apply(image, imager, flags)


def chi2(image, imager, vis_obs, weight):
    """chi^2 = sum_m w_m |V_obs,m - (D x)_m|^2, differentiable in the image x."""
    r = vis_obs - predict(image, imager)
    return (weight * (r.real ** 2 + r.imag ** 2)).sum()
