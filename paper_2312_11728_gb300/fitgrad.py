"""The fit's total chi2 as a differentiable function of the per-layer alignment, the per-layer
material thickness scales and the tracks' starting parameters (torch.autograd.Function over
mkgb_fit_grad; device tensors on the context's device)."""
from __future__ import annotations

import torch

from . import mkgb


class FitChi2(torch.autograd.Function):
    """total = FitChi2.apply(align [L,6], xscale [L], p0 [n,6], ctx, layers, hits, c0).

    The forward call runs mkgb_fit_grad, which returns the derivatives with the value (its
    reverse sweep over checkpointed steps); backward scales them by the incoming gradient.
    Tracks whose fit fails (status != 0) add nothing."""

    @staticmethod
    def forward(fctx, align, xscale, p0, ctx: mkgb.Context, layers, hits, c0):
        n = layers.shape[0]
        dev = p0.device
        chi2 = torch.zeros(n, dtype=torch.float32, device=dev)
        d_p0 = torch.zeros((n, 6), dtype=torch.float32, device=dev)
        d_al = torch.zeros_like(align, dtype=torch.float32)
        d_xs = torch.zeros_like(xscale, dtype=torch.float32)
        status = torch.zeros(n, dtype=torch.int32, device=dev)
        ctx.fit_grad(layers, hits, p0.detach().contiguous(), c0, align.detach().contiguous(),
                     xscale.detach().contiguous(), chi2, d_p0, d_al, d_xs, status)
        fctx.save_for_backward(d_al, d_xs, d_p0)
        fctx.mark_non_differentiable(status)
        return chi2.sum(), status

    @staticmethod
    def backward(fctx, g, _g_status):
        d_al, d_xs, d_p0 = fctx.saved_tensors
        return g * d_al, g * d_xs, g * d_p0, None, None, None, None
