"""torch.autograd wrapper of the differentiable form (dm_loss_grad in the C ABI).

TopMaxLoss(desc1, desc2) = sum over the existing top-level patches of
max_q C_L(p, q), for FP32 descriptor fields [H][W][9] on a CUDA device.
Forward: dm_correlate_pyramid + the loss; backward: the adjoint kernels of
the library (argument marshalling only here).
"""
from __future__ import annotations

import torch

from . import dm


class _PyramidHandle:
    """Owns a pyramid handle of dm_correlate_pyramid (host-side views into the
    caller's workspace) and frees it exactly once: at release() after the
    backward, or when the autograd graph holding it is dropped without one."""
    live = 0                     # handles not yet freed (for tests)

    def __init__(self, handle: int):
        self.handle = handle
        _PyramidHandle.live += 1

    def release(self) -> None:
        if self.handle:
            dm.dm_pyramid_free(self.handle)
            self.handle = 0
            _PyramidHandle.live -= 1

    def __del__(self):
        try:
            self.release()
        except Exception:        # interpreter shutdown: the library may be gone
            pass


class _TopMaxLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, desc1, desc2, context):
        d1 = desc1.detach().contiguous()
        d2 = desc2.detach().contiguous()
        H1, W1, _ = d1.shape
        H2, W2, _ = d2.shape
        nbytes = dm.dm_workspace_bytes(context.ctx, W1, H1, W2, H2)["pyramid"]
        ws_pyr = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=d1.device)
        pyr = dm.dm_correlate_pyramid(context.ctx, d1, d2, ws_pyr)
        ws_grad = torch.empty(max(dm.dm_grad_workspace_bytes(context.ctx, W1, H1, W2, H2), 256), dtype=torch.uint8,
                              device=d1.device)
        loss = torch.zeros(1, dtype=torch.float32, device=d1.device)
        dm.dm_loss_grad(context.ctx, pyr, d1, d2, ws_grad, loss)
        ctx.save_for_backward(d1, d2)
        ctx.state = (context, _PyramidHandle(pyr), ws_pyr, ws_grad)
        return loss[0]

    @staticmethod
    def backward(ctx, grad):
        d1, d2 = ctx.saved_tensors
        context, pyr, ws_pyr, ws_grad = ctx.state
        g1 = torch.empty_like(d1)
        g2 = torch.empty_like(d2)
        loss = torch.zeros(1, dtype=torch.float32, device=d1.device)
        dm.dm_loss_grad(context.ctx, pyr.handle, d1, d2, ws_grad, loss, None, g1, g2)
        pyr.release()
        ctx.state = None
        return grad * g1, grad * g2, None


def top_max_loss(desc1: torch.Tensor, desc2: torch.Tensor, context: "dm.Context") -> torch.Tensor:
    """Differentiable sum of the top-level maxima (FP32 path of `context`)."""
    return _TopMaxLoss.apply(desc1, desc2, context)
