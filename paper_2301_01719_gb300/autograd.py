"""torch.autograd.Function over rt_shade / rt_shade_backward.

Gradients flow to the UVs, the directions and the FP32 texture buffers that
the context borrows (RT_BORROW): the backward kernel recomputes the filter
weights instead of storing them, and sums texel gradients into a buffer of the
borrowed tensor's shape and layout.
"""
from __future__ import annotations

import torch

from . import api


class RadianceShade(torch.autograd.Function):
    @staticmethod
    def forward(actx, rctx, filt, obj_ids, uv, dirs, obj, *textures):
        actx.rctx = rctx
        actx.filt = filt
        actx.obj_ids = obj_ids
        actx.save_for_backward(uv, dirs, obj)
        actx.tex_shapes = [t.shape for t in textures]
        return api.rt_shade(rctx, uv, dirs, obj, filt)

    @staticmethod
    def backward(actx, grad_out):
        uv, dirs, obj = actx.saved_tensors
        grad_out = grad_out.contiguous()
        need_uv, need_dir = actx.needs_input_grad[3], actx.needs_input_grad[4]
        duv = torch.empty_like(uv) if need_uv else None
        ddir = torch.empty_like(dirs) if need_dir else None
        dtex = {}
        tex_grads = []
        for k, (o, shape) in enumerate(zip(actx.obj_ids, actx.tex_shapes)):
            if actx.needs_input_grad[6 + k]:
                g = torch.empty(shape, dtype=torch.float32, device=uv.device)
                dtex[o] = g
                tex_grads.append(g)
            else:
                tex_grads.append(None)
        api.rt_shade_backward(actx.rctx, uv, dirs, obj, actx.filt, grad_out, dtex or None, duv, ddir)
        return (None, None, None, duv, ddir, None, *tex_grads)


def shade(rctx, uv, dirs, obj, filt=api.RT_QUADRILINEAR, textures: dict | None = None):
    """Differentiable synthesis.  textures: {object id: the borrowed FP32 tensor of that object}."""
    textures = textures or {}
    ids = tuple(textures.keys())
    return RadianceShade.apply(rctx, filt, ids, uv, dirs, obj, *[textures[o] for o in ids])
