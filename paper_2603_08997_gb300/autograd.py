"""torch.autograd.Function wrappers of the rasterizer and the loss.

`render(flat, model, renderer)` returns the planar images of the renderer's
views (concatenated, [3*total_pixels]) as a differentiable function of the
flat parameter buffer; its backward is gs_render_bwd (reverse traversal with
per-tile transmittance checkpoints).  `photometric_loss(image, target,
renderer)` is Eq. (loss) per view with gs_loss / gs_loss_backward.

A renderer holds the forward state of one call (pairs, checkpoints): call
backward before the renderer's next forward.
"""
from __future__ import annotations

import torch

from .raster import GaussianModel, Renderer


class RenderFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, flat: torch.Tensor, model: GaussianModel, renderer: Renderer):
        if not flat.is_contiguous() or flat.dtype != torch.float32 or flat.numel() != model.flat.numel():
            raise ValueError("flat must be the model's contiguous float32 parameter buffer layout")
        renderer.forward(model.c_params(flat))
        ctx.model, ctx.renderer = model, renderer
        ctx.save_for_backward(flat)
        return renderer.image.clone()

    @staticmethod
    def backward(ctx, grad_image: torch.Tensor):
        (flat,) = ctx.saved_tensors
        model, renderer = ctx.model, ctx.renderer
        grad = torch.zeros_like(flat)
        renderer.backward(model.c_params(flat), model.c_grads(grad), dL_dimage=grad_image.contiguous(),
                          accumulate=False)
        return grad, None, None


class LossFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, image: torch.Tensor, target: torch.Tensor, renderer: Renderer):
        saved = renderer.image
        renderer.image = image.contiguous()
        try:
            loss = renderer.compute_loss(target, with_grad=True).clone()
        finally:
            renderer.image = saved
        ctx.renderer = renderer
        ctx.grad = renderer.dL_dimage.clone()
        return loss

    @staticmethod
    def backward(ctx, grad_loss: torch.Tensor):
        r = ctx.renderer
        g = ctx.grad
        out = torch.empty_like(g)
        for v in range(r.views.n):
            w, h = r.views.sizes[v]
            o = 3 * r.views.pix_offsets[v]
            out[o:o + 3 * w * h] = g[o:o + 3 * w * h] * grad_loss[v]
        return out, None, None


def render(flat: torch.Tensor, model: GaussianModel, renderer: Renderer) -> torch.Tensor:
    return RenderFunction.apply(flat, model, renderer)


def photometric_loss(image: torch.Tensor, target: torch.Tensor, renderer: Renderer) -> torch.Tensor:
    """Per-view loss vector [n_views] (Eq. loss, lambda from the renderer's settings)."""
    return LossFunction.apply(image, target, renderer)
