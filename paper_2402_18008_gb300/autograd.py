"""Differentiable ACA for networks that regress 4-point offsets (Sec. 5.3,
TensorACA): torch.autograd.Function wrappers whose forward and backward are
the library's CUDA kernels (aca_rect_solve / aca_rect_backward for a
rectangle source, aca_solve / aca_backward for a general source quad).

The output is the unnormalised H of the paper (Eq. 42, resp. Eq. 24-29), a
polynomial in the target coordinates, so its gradient is exact up to FP32
rounding; losses built on reprojections are invariant to the scale of H.
"""
from __future__ import annotations

import torch

from . import _lib


class ACARectFunction(torch.autograd.Function):
    """tgt (8, ld) float32 planes (M2, N2, P2, Q2 x/y) -> H (9, ld)."""

    @staticmethod
    def forward(ctx, tgt: torch.Tensor, rect):
        tgt = tgt.contiguous()
        H = torch.empty((9, tgt.shape[1]), dtype=torch.float32, device=tgt.device)
        _lib.aca_rect_solve(tgt, rect, H)
        ctx.save_for_backward(tgt)
        ctx.rect = tuple(float(v) for v in rect)
        return H

    @staticmethod
    def backward(ctx, grad_H: torch.Tensor):
        (tgt,) = ctx.saved_tensors
        g = torch.empty_like(tgt)
        _lib.aca_rect_backward(tgt, ctx.rect, grad_H.contiguous(), g)
        return g, None


class ACAFunction(torch.autograd.Function):
    """src (8, n), tgt (8, n) float32 planes -> H (9, n); gradient w.r.t. tgt
    only (the source quadrilateral is treated as fixed)."""

    @staticmethod
    def forward(ctx, src: torch.Tensor, tgt: torch.Tensor):
        pts = torch.cat([src, tgt], dim=0).contiguous()
        H = torch.empty((9, pts.shape[1]), dtype=torch.float32, device=pts.device)
        _lib.aca_solve(pts, H)
        ctx.save_for_backward(pts)
        return H

    @staticmethod
    def backward(ctx, grad_H: torch.Tensor):
        (pts,) = ctx.saved_tensors
        g = torch.empty((8, pts.shape[1]), dtype=torch.float32, device=pts.device)
        _lib.aca_backward(pts, grad_H.contiguous(), g)
        return None, g


def aca_rect(tgt: torch.Tensor, rect) -> torch.Tensor:
    return ACARectFunction.apply(tgt, rect)


def aca(src: torch.Tensor, tgt: torch.Tensor) -> torch.Tensor:
    return ACAFunction.apply(src, tgt)
