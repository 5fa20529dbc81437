"""Differentiable render for gradient refinement: a torch.autograd.Function over
tsp_render / tsp_render_backward.

``render(means, log_scales, quats, opacity_logits, sh, cams, context)`` returns
the colour images [V, H, W, 3] (views of one size); its backward gives the
gradients with respect to the means, log-scales, (raw) quaternions, opacity
logits and colour coefficients.  The library differentiates the blend with
respect to the mean, linear scales, raw quaternion, opacity and coefficients;
the exp of the log-scales and the sigmoid of the logits are ordinary torch
operations, so autograd composes them.
"""
from __future__ import annotations

import torch

from . import Context


class _Render(torch.autograd.Function):
    @staticmethod
    def forward(ctx, means_opacity, quats, scales, sh, sh_degree, cams, context):
        rgb, _ = context.render(means_opacity, quats, scales, sh, sh_degree, cams)
        img = torch.stack(rgb)
        ctx.save_for_backward(means_opacity, quats, scales, sh, img)
        ctx.sh_degree, ctx.cams, ctx.context = sh_degree, cams, context
        return img

    @staticmethod
    def backward(ctx, grad_img):
        means_opacity, quats, scales, sh, img = ctx.saved_tensors
        grad_img = grad_img.contiguous()
        g = ctx.context.render_backward(means_opacity, quats, scales, sh, ctx.sh_degree, ctx.cams,
                                        list(img), list(grad_img))
        return g["means_opacity"], g["quats"], g["scales"], g["sh"], None, None, None


def render(means, log_scales, quats, opacity_logits, sh, cams, context: Context, sh_degree=None):
    """Colour images [V, H, W, 3] of the Gaussians (means [n,3], log_scales [n,3],
    quats [n,4], opacity_logits [n], sh [n, (d+1)^2, 3]) seen by ``cams``."""
    n = means.shape[0]
    if sh_degree is None:
        sh_degree = int(round(sh.shape[1] ** 0.5)) - 1
    mo = torch.cat([means, torch.sigmoid(opacity_logits)[:, None]], dim=1).contiguous()
    sc = torch.cat([torch.exp(log_scales), torch.zeros((n, 1), device=means.device, dtype=means.dtype)],
                   dim=1).contiguous()
    return _Render.apply(mo, quats.contiguous(), sc, sh.contiguous(), int(sh_degree), cams, context)
