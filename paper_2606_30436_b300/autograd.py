"""torch.autograd.Function over the C ABI: render in the forward, and in the
backward re-traverse each tile back to front from the saved per-pixel
(T_final, last) instead of storing per-pixel contributor lists.

    img = rasterize(params, cams, cfg)      # params: [K, ld] FP32 tensor, requires_grad
    loss = some_function(img)               # img: frame layout (views packed, planar RGB)
    loss.backward()                         # params.grad: same [K, ld] layout

Saved for the backward: the parameters, the projection records, the pair
list with its tile ranges and block masks, T_final and last -- O(N + P +
pixels), independent of how many Gaussians each pixel blends.  Every step
runs in libgs.so (gs_project, gs_sort, gs_render_fwd, gs_render_bwd).
"""
from __future__ import annotations

import torch

from . import gs


class _Ctx:
    """Device buffers of one rasterisation, kept alive for the backward."""

    def __init__(self, model, cams, cfg, max_pairs):
        self.model = model
        self.buf = gs.Buffers(model, cams, cfg, max_pairs, with_stats=False)


class RasterizeGaussians(torch.autograd.Function):
    @staticmethod
    def forward(ctx, data, n, sh_degree, cams, cfg, max_pairs):
        model = gs.GaussianModel(n, sh_degree, device=data.device, data=data.detach())
        r = _Ctx(model, cams, cfg, max_pairs)
        b = r.buf
        b.status.zero_()
        gs.gs_project(model, b)
        gs.gs_sort(b)
        gs.gs_render_fwd(b)
        if int(b.counts[2].item()) > b.max_pairs:  # grow the pair buffer and redo the binning once
            b.set_max_pairs(int(b.counts[2].item() * 1.25) + 1024)
            b.status.zero_()
            gs.gs_sort(b)
            gs.gs_render_fwd(b)
        ctx.r = r
        return b.img.clone()

    @staticmethod
    def backward(ctx, dL_dimg):
        r = ctx.r
        grads = r.model.like()
        g = dL_dimg.contiguous().float()
        gs.gs_render_bwd(r.model, grads, r.buf, target=None, with_stats=False, dL_dimg=g)
        ctx.r = None
        return grads.data, None, None, None, None, None


def rasterize(params: torch.Tensor, n: int, sh_degree: int, cams, cfg: gs.Config = None, max_pairs: int = None):
    """Differentiable render of all views; returns the frame-layout image."""
    cfg = cfg or gs.Config()
    if max_pairs is None:
        max_pairs = max(1 << 16, 8 * n * len(cams))
    return RasterizeGaussians.apply(params, n, sh_degree, list(cams), cfg, max_pairs)
