"""torch.autograd.Function around ttm_backward (argument marshalling only).

TTMProductLoss.apply(handle, kind, nA, nB, *coresA, *coresB, *coresWC) returns the scalar
<W, A o B> (kind "inner") or ||A o B - C||^2 (kind "sqdist"). The forward pass calls
ttm_backward once, which returns the value and the gradients w.r.t. every core of A and
B from the library's environment and adjoint kernels; backward scales them by the
incoming gradient. W and C receive no gradient.
"""

import torch

from .binding import ttm_backward


class TTMProductLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, handle, kind, nA, nB, *cores):
        A = [c.detach().contiguous() for c in cores[:nA]]
        B = [c.detach().contiguous() for c in cores[nA:nA + nB]]
        WC = [c.detach().contiguous() for c in cores[nA + nB:]]
        need_a = any(c.requires_grad for c in cores[:nA])
        need_b = any(c.requires_grad for c in cores[nA:nA + nB])
        val, gA, gB = ttm_backward(handle, kind, A, B, WC, want_a=need_a, want_b=need_b)
        ctx.nA, ctx.nB, ctx.nWC = nA, nB, len(WC)
        ctx.gA, ctx.gB = gA, gB
        return torch.tensor(val, dtype=torch.float64, device=A[0].device)

    @staticmethod
    def backward(ctx, gout):
        ga = [gout * g for g in ctx.gA] if ctx.gA is not None else [None] * ctx.nA
        gb = [gout * g for g in ctx.gB] if ctx.gB is not None else [None] * ctx.nB
        return (None, None, None, None, *ga, *gb, *([None] * ctx.nWC))


def product_loss(handle, kind, A, B, WC):
    """Convenience wrapper: scalar loss tensor with autograd through the C ABI."""
    return TTMProductLoss.apply(handle, kind, len(A), len(B), *A, *B, *WC)
