"""torch.autograd.Function around the library's hand-written adjoint.

MtLogPost.apply(heights, ctx) returns the per-chain log-posterior (double,
[C]) of heights [C][L][R][Q] (float32, on the context's device); its backward
multiplies the upstream gradient into the gradient mt_grad computed in the
same call.  Both value and gradient come from the library's kernels.
"""
from __future__ import annotations

import torch


class MtLogPost(torch.autograd.Function):
    @staticmethod
    def forward(fctx, heights, mtctx):
        h = heights.detach().contiguous()
        grad = torch.empty(h.shape, dtype=torch.float64, device=h.device)
        lp = torch.empty(h.shape[0], dtype=torch.float64, device=h.device)
        mtctx.grad(h, grad, lp)
        fctx.save_for_backward(grad)
        fctx.h_dtype = heights.dtype
        return lp

    @staticmethod
    def backward(fctx, g_out):
        (grad,) = fctx.saved_tensors
        g = g_out.to(torch.float64).view(-1, *([1] * (grad.dim() - 1))) * grad
        return g.to(fctx.h_dtype), None


def logpost(heights, mtctx):
    return MtLogPost.apply(heights, mtctx)
