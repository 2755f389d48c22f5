"""torch.autograd bindings of the DISK filter (argument marshalling only: the
forward and backward passes are the library's CUDA kernels)."""
from __future__ import annotations

import torch

from . import disk


class SVFilterFunction(torch.autograd.Function):
    """Spatially varying filter (Eq. 9 + Eq. 3) with the hand-written
    image-gradient backward (transpose of the cascade)."""

    @staticmethod
    def forward(ctx, img, maps, basis):
        ctx.basis = basis
        ctx.save_for_backward(maps)
        ctx.img_dtype = img.dtype
        return disk.sv_filter(basis, img.contiguous(), maps.contiguous())

    @staticmethod
    def backward(ctx, grad_out):
        (maps,) = ctx.saved_tensors
        g = disk.sv_filter_backward_image(ctx.basis, grad_out.contiguous().to(ctx.img_dtype), maps)
        return g.to(ctx.img_dtype), None, None


def sv_filter(img, maps, basis):
    """Differentiable in ``img``."""
    return SVFilterFunction.apply(img, maps, basis)
