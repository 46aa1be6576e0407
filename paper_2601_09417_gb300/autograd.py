"""torch.autograd.Function around the splatting forward/backward of the C ABI.

The forward calls vbm_raster_fwd; the backward calls vbm_raster_bwd, which
reads the per-pixel compositing state the plan saved (the autograd "context"
lives in the plan, so one plan serves one in-flight forward at a time).
"""

import torch

from . import vbm


class SplatRender(torch.autograd.Function):
    """img[V][3][H][W] = render(params[14][stride]) for the views of `plan`."""

    @staticmethod
    def forward(ctx, params, plan, cams_dev, bg=(0.0, 0.0, 0.0), view_begin=0, view_count=None):
        vc = plan.n_views - view_begin if view_count is None else view_count
        img = torch.zeros((plan.n_views, 3, plan.height, plan.width), dtype=torch.float32, device=params.device)
        plan.forward(params, cams_dev, img, view_begin=view_begin, view_count=vc, bg=bg)
        ctx.plan, ctx.cams, ctx.bg, ctx.vb, ctx.vc = plan, cams_dev, bg, view_begin, vc
        ctx.save_for_backward(params)
        return img

    @staticmethod
    def backward(ctx, dimg):
        (params,) = ctx.saved_tensors
        grad = torch.zeros_like(params)
        ctx.plan.backward(params, ctx.cams, dimg.contiguous(), grad, view_begin=ctx.vb, view_count=ctx.vc,
                          bg=ctx.bg)
        return grad, None, None, None, None, None


def render(params, plan, cams_dev, bg=(0.0, 0.0, 0.0), view_begin=0, view_count=None):
    return SplatRender.apply(params, plan, cams_dev, bg, view_begin, view_count)
