"""torch.autograd bindings of the DISK filter (argument marshalling only: the
forward and backward passes are the library's CUDA kernels)."""
from __future__ import annotations

import torch

from . import disk


class SVFilterFunction(torch.autograd.Function):
    """Spatially varying filter (Eq. 9 + Eq. 3) of an image with a fixed basis;
    the hand-written backward gives the image gradient (transpose of the
    cascade)."""

    @staticmethod
    def forward(ctx, img, maps, basis):
        ctx.basis = basis
        ctx.save_for_backward(maps)
        ctx.img_dtype = img.dtype
        return disk.sv_filter(basis, img.contiguous(), maps.contiguous())

    @staticmethod
    def backward(ctx, grad_out):
        # The library takes the incoming gradient in its own precision (FP32
        # or FP16) and returns the image gradient in FP32; autograd then
        # stores it in the image's dtype (one rounding for an FP16 image, as
        # for any FP16 leaf).  disk.sv_filter_backward_image gives the FP32
        # gradient directly.
        (maps,) = ctx.saved_tensors
        g = disk.sv_filter_backward_image(ctx.basis, grad_out.contiguous(), maps)
        return g.to(ctx.img_dtype), None, None


class SVCascadeFunction(torch.autograd.Function):
    """The filter as a trainable layer: differentiable in the image and in the
    basis theta [B, L, T, 3] (tap offsets and weights of every node; a single
    node is a shift-invariant complex).  Only the inputs are kept; the
    backward recomputes the layer activations from the image.  The forward
    reads theta on the host (the layer halos depend on its values)."""

    @staticmethod
    def forward(ctx, img, maps, theta, node_vals):
        basis = disk.Basis.from_arrays(node_vals, theta.detach().float().cpu().numpy())
        ctx.basis = basis
        img = img.contiguous()
        maps = maps.contiguous()
        ctx.save_for_backward(img, maps)
        return disk.sv_filter(basis, img, maps)

    @staticmethod
    def backward(ctx, grad_out):
        img, maps = ctx.saved_tensors
        gi, gt = disk.sv_filter_backward(ctx.basis, img, grad_out.contiguous().to(img.dtype), maps,
                                         grad_img=ctx.needs_input_grad[0],
                                         grad_theta=ctx.needs_input_grad[2])
        if gi is not None:
            gi = gi.to(img.dtype)
        return gi, None, gt, None


def sv_filter(img, maps, basis):
    """Differentiable in ``img``."""
    return SVFilterFunction.apply(img, maps, basis)


def sv_cascade(img, maps, theta, node_vals):
    """Differentiable in ``img`` and ``theta`` (node_vals: one increasing
    sequence per kernel-space axis)."""
    return SVCascadeFunction.apply(img, maps, theta, node_vals)
