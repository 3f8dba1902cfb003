"""torch.autograd.Function around the C-ABI renderer (argument marshalling only).

`render(renderer, params, pose_delta, cams)` returns stacked RGB [3 P] and
depth [P] (layout of dcg_render_fwd); its backward calls dcg_render_bwd and
returns the gradient of the planar parameter tensor [F, n] and of
`pose_delta` [V, 6], the left-perturbation twist at zero of each camera pose
(pass zeros; the forward renders the given poses).  When the render state no
longer holds this forward (another forward ran in between) or
`recompute=True`, the backward first re-runs the forward into the state
instead of keeping per-forward sorted lists alive.
"""
from __future__ import annotations

import torch

from . import dcg


class Renderer:
    """One context plus a render state used by the autograd function."""

    def __init__(self, deg: int, max_gaussians: int, max_views: int = 8, max_pixels: int = 8 * 1241 * 376,
                 max_instances: int = 1 << 26, recompute: bool = False, ctx=None):
        self.deg = deg
        self.own = ctx is None
        self.ctx = ctx if ctx is not None else dcg.dcg_create(dcg.config(
            sh_degree=deg, max_active=max_gaussians, max_views=max_views, max_pixels=max_pixels,
            max_instances=max_instances, device_budget=max_gaussians, host_capacity=max_gaussians))
        self.state = dcg.dcg_state_create(self.ctx)
        self.recompute = recompute

    def close(self):
        if self.state is not None:
            dcg.dcg_state_destroy(self.state)
            self.state = None
        if self.own and self.ctx is not None:
            dcg.dcg_destroy(self.ctx)
            self.ctx = None


class _RenderFn(torch.autograd.Function):
    @staticmethod
    def forward(fctx, params, pose_delta, renderer: Renderer, cams):
        n = params.shape[1]
        npix = sum(c.W * c.H for c in cams)
        rgb = torch.empty(3 * npix, device=params.device, dtype=torch.float32)
        depth = torch.empty(npix, device=params.device, dtype=torch.float32)
        p = params.detach()
        g = dcg.gaussians(p, renderer.deg)
        dcg.dcg_render_fwd(renderer.ctx, g, n, cams, rgb, depth, renderer.state)
        fctx.renderer = renderer
        fctx.cams = cams
        fctx.gen = dcg.dcg_state_generation(renderer.state)
        fctx.save_for_backward(p)
        return rgb, depth

    @staticmethod
    def backward(fctx, grad_rgb, grad_depth):
        (p,) = fctx.saved_tensors
        r: Renderer = fctx.renderer
        n = p.shape[1]
        V = len(fctx.cams)
        if r.recompute or dcg.dcg_state_generation(r.state) != fctx.gen:
            npix = grad_depth.numel()
            scratch_rgb = torch.empty(3 * npix, device=p.device)
            scratch_d = torch.empty(npix, device=p.device)
            dcg.dcg_render_fwd(r.ctx, dcg.gaussians(p, r.deg), n, fctx.cams, scratch_rgb, scratch_d, r.state)
        grads = torch.zeros_like(p)
        dpose = torch.zeros(V, 6, device=p.device)
        gr = torch.zeros(3 * grad_depth.numel(), device=p.device) if grad_rgb is None else grad_rgb.contiguous()
        gd = torch.zeros_like(gr[: gr.numel() // 3]) if grad_depth is None else grad_depth.contiguous()
        dcg.dcg_render_bwd(r.ctx, gr, gd, dcg.gaussians(grads, r.deg), dpose, r.state)
        return grads, dpose, None, None


def render(renderer: Renderer, params: torch.Tensor, pose_delta: torch.Tensor, cams):
    """Differentiable RGB + depth of `cams` for planar float32 CUDA params [F, n]."""
    if params.dim() != 2 or params.dtype != torch.float32 or not params.is_cuda:
        raise ValueError("params must be a planar float32 CUDA tensor [F, n]")
    return _RenderFn.apply(params, pose_delta, renderer, cams)
