"""torch.autograd.Function around the mini-batch data term.

forward  : scale * sum_{l in illum} f_l(x): the forward (LS or Born) solves
           and detector residuals only (Section 6, Eq. 4.1).
backward : grad_output * scale * sum_l grad f_l(x): the adjoint solves and the
           gradient assembly.  When the mini-batch fits the handle's workspace
           (nb <= max_batch), the forward fields of the forward call are reused;
           otherwise, or when the workspace was used in between, the library
           recomputes them chunk by chunk instead of storing every field.
x is saved for backward, so autograd itself rejects an in-place change of x
between the two calls.
"""
from __future__ import annotations

from typing import Sequence

import torch


class LSGradient(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x: torch.Tensor, handle, illum: Sequence[int], scale: float):
        flat = x.detach().contiguous().view(-1)
        loss, _ = handle.loss_batch(flat, list(illum), float(scale))
        ctx.handle = handle
        ctx.illum = list(illum)
        ctx.scale = float(scale)
        ctx.shape = x.shape
        ctx.save_for_backward(flat)
        return torch.tensor(loss, dtype=torch.float64, device=x.device)

    @staticmethod
    def backward(ctx, grad_output):
        (flat,) = ctx.saved_tensors
        grad, reused = ctx.handle.grad_fields(flat, ctx.illum, ctx.scale, reuse=True)
        ctx.handle.last_backward_reused = reused
        return (grad * grad_output.to(grad.dtype)).view(ctx.shape), None, None, None
