"""torch.autograd.Function over the library's forward and hand-written adjoint.

The forward returns the rendered image and keeps only references to the
parameter tensors; the backward re-traces with the same Philox counters
(fr_backward) instead of storing hit records.  The parameters are the groups
of fr_params, including the light-stage geometry (light_d, light_a, light_p)
when it is given."""
from __future__ import annotations

import torch

from .facert import ALL_PARAM_NAMES


class RenderFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, renderer, iteration, face_id, names, *params):
        dp = {n: p.detach().contiguous() for n, p in zip(names, params)}
        img = renderer.forward(dp, iteration, face_id)
        ctx.renderer = renderer
        ctx.iteration = iteration
        ctx.face_id = face_id
        ctx.names = names
        ctx.save_for_backward(*params)
        return img

    @staticmethod
    def backward(ctx, grad_image):
        params = ctx.saved_tensors
        dp = {n: p.detach().contiguous() for n, p in zip(ctx.names, params)}
        g = ctx.renderer.backward(dp, grad_image.contiguous(), ctx.iteration, ctx.face_id)
        return (None, None, None, None) + tuple(g[n] if ctx.needs_input_grad[4 + k] else None
                                                for k, n in enumerate(ctx.names))


def render(renderer, params: dict, iteration: int = 0, face_id: int = 0) -> torch.Tensor:
    """Differentiable render: image = F(params); gradients flow to every tensor
    of `params` that requires grad."""
    names = tuple(n for n in ALL_PARAM_NAMES if params.get(n) is not None)
    return RenderFn.apply(renderer, iteration, face_id, names, *[params[n] for n in names])
