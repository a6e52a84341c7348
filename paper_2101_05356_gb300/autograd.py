"""torch.autograd.Function over the library's forward and hand-written adjoint.

The forward returns the rendered image and keeps only references to the
parameter tensors; the backward re-traces with the same Philox counters
(fr_backward) instead of storing hit records."""
from __future__ import annotations

import torch

from .facert import PARAM_NAMES


class RenderFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, renderer, iteration, face_id, *params):
        dp = {n: p.detach().contiguous() for n, p in zip(PARAM_NAMES, params)}
        img = renderer.forward(dp, iteration, face_id)
        ctx.renderer = renderer
        ctx.iteration = iteration
        ctx.face_id = face_id
        ctx.save_for_backward(*params)
        return img

    @staticmethod
    def backward(ctx, grad_image):
        params = ctx.saved_tensors
        dp = {n: p.detach().contiguous() for n, p in zip(PARAM_NAMES, params)}
        g = ctx.renderer.backward(dp, grad_image.contiguous(), ctx.iteration, ctx.face_id)
        return (None, None, None) + tuple(g[n] if ctx.needs_input_grad[3 + k] else None
                                          for k, n in enumerate(PARAM_NAMES))


def render(renderer, params: dict, iteration: int = 0, face_id: int = 0) -> torch.Tensor:
    """Differentiable render: image = F(params); gradients flow to every tensor
    of `params` that requires grad."""
    return RenderFn.apply(renderer, iteration, face_id, *[params[n] for n in PARAM_NAMES])
