"""torch.autograd wrapper: x = A^{-1} b with A given in band storage.

Forward: sap_factor + sap_solve.  Backward: lambda = A^{-T} (dl/dx) by
sap_solve_adjoint (the stored block factors reused transposed), then
dl/db = lambda and dl/dband = -lambda x^T restricted to the band
(sap_grad_band).  All arithmetic runs in libsap's kernels."""
from __future__ import annotations

import torch


class SapSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, band, b, N, K, opts_kw):
        from . import sap_factor, sap_solve
        band = band.contiguous()
        b = b.contiguous()
        h = sap_factor(band, N, K, **opts_kw)
        x, info, _ = sap_solve(h, b)
        ctx.h = h
        ctx.save_for_backward(x)
        ctx.info = info
        return x

    @staticmethod
    def backward(ctx, gx):
        from . import sap_grad_band, sap_solve_adjoint
        (x,) = ctx.saved_tensors
        lam, _, _ = sap_solve_adjoint(ctx.h, gx.contiguous())
        gband = sap_grad_band(ctx.h, lam, x) if ctx.needs_input_grad[0] else None
        gb = lam if ctx.needs_input_grad[1] else None
        return gband, gb, None, None, None


def sap_solve_autograd(band: torch.Tensor, b: torch.Tensor, N: int, K: int, **opts_kw) -> torch.Tensor:
    """Differentiable x = A^{-1} b (options as keyword arguments of sap_options_t)."""
    return SapSolve.apply(band, b, N, K, opts_kw)
