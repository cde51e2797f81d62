"""torch.autograd.Function wrappers of libalb's differentiable float32 kernels.

AffineWarpFn(x, angle, scale, tx, ty): bilinear warp with zero border of an NCHW
float32 batch by per-image rotation (degrees, counter-clockwise on screen)
about the centre, scale and shift (fractions of W, H).
PhotometricFn(x, alpha, beta, gamma): y = clamp(alpha x + beta, 0, 1)^gamma.

Forward and backward both run in libalb.so (hand-written CUDA); backward
recomputes the sampling coordinates from the parameters.
"""
from __future__ import annotations

import torch

from . import alb


class AffineWarpFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, angle, scale, tx, ty):
        x = x.contiguous()
        prm = torch.stack([angle, scale, tx, ty], dim=1).to(torch.float32).contiguous()
        y = alb.alb_warp_affine_f32_fwd(x, prm)
        ctx.save_for_backward(x, prm)
        return y

    @staticmethod
    def backward(ctx, gy):
        x, prm = ctx.saved_tensors
        gx, gp = alb.alb_warp_affine_f32_bwd(x, prm, gy.contiguous())
        return gx, gp[:, 0], gp[:, 1], gp[:, 2], gp[:, 3]


class PhotometricFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, alpha, beta, gamma):
        x = x.contiguous()
        prm = torch.stack([alpha, beta, gamma], dim=1).to(torch.float32).contiguous()
        y = alb.alb_photometric_f32_fwd(x, prm)
        ctx.save_for_backward(x, prm)
        return y

    @staticmethod
    def backward(ctx, gy):
        x, prm = ctx.saved_tensors
        gx, gp = alb.alb_photometric_f32_bwd(x, prm, gy.contiguous())
        return gx, gp[:, 0], gp[:, 1], gp[:, 2]


def augment(x, angle, scale, tx, ty, alpha, beta, gamma):
    """Warp then photometric map, both differentiable."""
    return PhotometricFn.apply(AffineWarpFn.apply(x, angle, scale, tx, ty), alpha, beta, gamma)
