"""torch.autograd.Function around ttm_backward (argument marshalling only).

TTMProductLoss.apply(handle, kind, nA, nB, *coresA, *coresB, *coresWC) returns the scalar
<W, A o B> (kind "inner") or ||A o B - C||^2 (kind "sqdist"). The forward pass asks
ttm_backward for the value only (one environment sweep); the gradients w.r.t. the cores
of A and B are computed by the library's environment and adjoint kernels when backward
runs, and scaled by the incoming gradient. W and C receive no gradient.
"""

import torch

from .binding import ttm_backward


class TTMProductLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, handle, kind, nA, nB, *cores):
        A = [c.detach().contiguous() for c in cores[:nA]]
        B = [c.detach().contiguous() for c in cores[nA:nA + nB]]
        WC = [c.detach().contiguous() for c in cores[nA + nB:]]
        val, _, _ = ttm_backward(handle, kind, A, B, WC, want_a=False, want_b=False)
        ctx.handle, ctx.kind = handle, kind
        ctx.nA, ctx.nB, ctx.nWC = nA, nB, len(WC)
        ctx.need = (any(c.requires_grad for c in cores[:nA]), any(c.requires_grad for c in cores[nA:nA + nB]))
        ctx.save_for_backward(*A, *B, *WC)
        return torch.tensor(val, dtype=torch.float64, device=A[0].device)

    @staticmethod
    def backward(ctx, gout):
        saved = ctx.saved_tensors
        A, B, WC = saved[:ctx.nA], saved[ctx.nA:ctx.nA + ctx.nB], saved[ctx.nA + ctx.nB:]
        need_a, need_b = ctx.need
        _, gA, gB = ttm_backward(ctx.handle, ctx.kind, list(A), list(B), list(WC), want_a=need_a, want_b=need_b)
        ga = [gout * g for g in gA] if gA is not None else [None] * ctx.nA
        gb = [gout * g for g in gB] if gB is not None else [None] * ctx.nB
        return (None, None, None, None, *ga, *gb, *([None] * ctx.nWC))


def product_loss(handle, kind, A, B, WC):
    """Convenience wrapper: scalar loss tensor with autograd through the C ABI."""
    return TTMProductLoss.apply(handle, kind, len(A), len(B), *A, *B, *WC)
