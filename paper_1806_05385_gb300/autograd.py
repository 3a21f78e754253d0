"""torch.autograd.Function over the library: forward = stages (a)-(d)
(rasterize + shade), backward = stage (e) (pr_backward).  The visible ids of
the forward pass are saved; barycentrics are recomputed from them in the
backward kernel, so nothing per pixel but the id buffer is kept.
"""
from __future__ import annotations

import torch

from . import binding as B


class Renderer:
    """A device scene handle plus one view; ``render(col, pos, vel)`` is
    differentiable with respect to all three [V,3] float32 CUDA tensors."""

    def __init__(self, tri: torch.Tensor, V: int, view, params=None):
        self.view = B.make_view(view)
        self.W, self.H = int(view.W), int(view.H)
        self.params = params if params is not None else B.make_params()
        z = torch.zeros(V, 3, dtype=torch.float32, device="cuda")
        self.tri = tri.to(device="cuda", dtype=torch.int32).contiguous()
        self.V = V
        self.handle = B.pr_scene_upload(z, z, z, self.tri)

    def close(self):
        if self.handle:
            B.pr_scene_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def render(self, col, pos, vel):
        return RasterShade.apply(col, pos, vel, self)


class RasterShade(torch.autograd.Function):
    @staticmethod
    def forward(ctx, col, pos, vel, r: Renderer):
        col, pos, vel = (x.detach().contiguous().float() for x in (col, pos, vel))
        B.pr_scene_update(r.handle, pos, vel, col)
        n = r.W * r.H
        ids = torch.empty(n, dtype=torch.int32, device="cuda")
        rgb = torch.empty(3 * n, dtype=torch.float32, device="cuda")
        B.pr_rasterize(r.handle, r.view, r.params, ids, None)
        B.pr_shade(r.handle, r.view, ids, rgb)
        ctx.save_for_backward(ids)
        ctx.r = r
        return rgb.view(3, r.H, r.W)

    @staticmethod
    def backward(ctx, grad_rgb):
        (ids,) = ctx.saved_tensors
        r = ctx.r
        g = grad_rgb.contiguous().float().view(-1)
        dcol = torch.zeros(r.V, 3, dtype=torch.float32, device="cuda")
        dpos = torch.zeros_like(dcol)
        dvel = torch.zeros_like(dcol)
        B.pr_backward(r.handle, r.view, ids, g, dcol, dpos, dvel)
        return dcol, dpos, dvel, None
