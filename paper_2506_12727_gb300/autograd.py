"""torch.autograd.Function around the rasterizer's forward and backward.

`render(rasterizer, params, sh_degree)` returns the packed images of the
rasterizer's views ([sum_v 3 H_v W_v], float32) as a differentiable function of
the Gaussian parameters; the backward runs mvgs_render_views_backward.  The
blend state between the two is what the forward keeps in the rasterizer's
state buffer (sorted lists, final transmittance, last contributor per pixel);
the backward recomputes each pixel's transmittances from it instead of
storing per-pixel lists.  One rasterizer holds one forward's state: call its
backward before the next forward on the same rasterizer (a backward whose
state a later forward has overwritten raises instead of returning wrong
gradients).

Optional per-record outputs for the densification statistics can be requested
with `adc=(g_mean2d, e1)` buffers (see mvgs_render_views_backward).
"""
from __future__ import annotations

import torch

from . import mvgs

PARAMS = ("means", "log_scales", "quats", "opacity_logits", "sh")


class _RenderViews(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rasterizer, sh_degree, adc, means, log_scales, quats, opacity_logits, sh):
        tensors = [t.detach().contiguous() for t in (means, log_scales, quats, opacity_logits, sh)]
        params = dict(zip(PARAMS, tensors))
        img = rasterizer.forward(mvgs.make_scene(params, sh_degree))
        ctx.rasterizer = rasterizer
        ctx.generation = rasterizer.generation
        ctx.sh_degree = sh_degree
        ctx.adc = adc
        ctx.save_for_backward(*tensors)
        return img

    @staticmethod
    def backward(ctx, dimg):
        if ctx.rasterizer.generation != ctx.generation:
            raise RuntimeError("the rasterizer's state belongs to a later forward: call backward before rendering "
                               "again with the same rasterizer, or use one rasterizer per pending backward")
        tensors = ctx.saved_tensors
        params = dict(zip(PARAMS, tensors))
        grads = {k: torch.empty_like(v) for k, v in params.items()}
        g_mean2d, e1 = ctx.adc if ctx.adc is not None else (None, None)
        ctx.rasterizer.backward(mvgs.make_scene(params, ctx.sh_degree), dimg.contiguous(), grads, g_mean2d, e1)
        return (None, None, None) + tuple(grads[k] for k in PARAMS)


def render(rasterizer, params: dict, sh_degree: int, adc=None) -> torch.Tensor:
    """Differentiable render of all the rasterizer's views.  `params` maps the
    five parameter names to CUDA float32 tensors (may require grad)."""
    return _RenderViews.apply(rasterizer, sh_degree, adc, *(params[k] for k in PARAMS))
