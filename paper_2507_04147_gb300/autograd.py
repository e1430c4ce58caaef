"""The rasterizer as a differentiable PyTorch operation.

``render(rasterizer, fovea=None)`` renders with the CUDA library (full resolution, or
foveated when a fovea is given) and, on backward, calls ``a3fr_backward`` for the
gradients of the means, log-scales, quaternions, opacity logits and SH coefficients
(3DGS training, Sec. 4.1).  Every step runs in the library; this module only wires it
into autograd.
"""
from __future__ import annotations

import torch

from . import Scene


class GaussianRasterizer:
    """A scene over trainable parameter tensors (CUDA fp32, contiguous, updated in place by
    the optimiser; the library reads them at each render)."""

    def __init__(self, means, log_scales, quats, opacity_logits, sh, sh_degree=None,
                 instance_capacity: int = 0):
        self.params = [means, log_scales, quats, opacity_logits, sh]
        self.scene = Scene(*[p.detach() for p in self.params], sh_degree=sh_degree,
                           instance_capacity=instance_capacity)
        self.scene.keep_aux(True)
        self.renders = 0

    def set_camera(self, eye: int, cam):
        self.scene.set_camera(eye, cam)

    def set_gaze(self, gaze_px, side_stream=None):
        self.scene.set_gaze(gaze_px, side_stream)

    def close(self):
        self.scene.close()


class _Render(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rast: GaussianRasterizer, fovea, *params):
        rast.renders += 1
        ctx.rast, ctx.render_id = rast, rast.renders
        if fovea is None:
            return rast.scene.render_full()
        return rast.scene.render_foveated(fovea)

    @staticmethod
    def backward(ctx, grad_rgb):
        rast = ctx.rast
        if rast.renders != ctx.render_id:
            raise RuntimeError("a3fr backward: the scene has rendered again since this output; "
                               "call backward before the next render")
        g = rast.scene.backward(grad_rgb.contiguous())
        return (None, None, g["means"], g["log_scales"], g["quats"], g["opacity_logits"], g["sh"])


def render(rast: GaussianRasterizer, fovea=None) -> torch.Tensor:
    """Image [eyes, H, W, 3] of the current parameters, differentiable in them."""
    return _Render.apply(rast, fovea, *rast.params)
