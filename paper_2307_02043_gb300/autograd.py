"""torch.autograd.Function around the mini-batch data term.

forward  : scale * sum_{l in illum} f_l(x)   (LS or Born forward solves)
backward : grad_output * scale * sum_l grad f_l(x), from the library's adjoint
           solve (Section 6: one LS solve for H_l, two for the gradient).
The library computes the loss and the gradient in one call; the gradient is
kept for backward.
"""
from __future__ import annotations

from typing import Sequence

import torch


class LSGradient(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x: torch.Tensor, handle, illum: Sequence[int], scale: float):
        flat = x.detach().contiguous().view(-1)
        grad, loss, _ = handle.grad_batch(flat, list(illum), float(scale))
        ctx.save_for_backward(grad.view_as(x))
        return torch.tensor(loss, dtype=torch.float64, device=x.device)

    @staticmethod
    def backward(ctx, grad_output):
        (grad,) = ctx.saved_tensors
        return grad * grad_output.to(grad.dtype), None, None, None
