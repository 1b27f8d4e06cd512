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


class SapSolveBatched(torch.autograd.Function):
    """x_i = A_i^{-1} b_i for a batch; backward by the batched adjoint solve."""

    @staticmethod
    def forward(ctx, meta, *args):
        from . import sap_factor_batched, sap_solve_batched
        Ns, Ks, opts_kw = meta
        n = len(Ns)
        bands = [a.contiguous() for a in args[:n]]
        bs = [a.contiguous() for a in args[n:]]
        bh = sap_factor_batched(bands, Ns, Ks, **opts_kw)
        xs, infos, _, _ = sap_solve_batched(bh, bs)
        ctx.bh = bh
        ctx.infos = infos
        ctx.save_for_backward(*xs)
        return tuple(xs)

    @staticmethod
    def backward(ctx, *gxs):
        from . import sap_grad_band_batched, sap_solve_adjoint_batched
        xs = list(ctx.saved_tensors)
        n = len(xs)
        gxs = [torch.zeros_like(x) if g is None else g.contiguous() for g, x in zip(gxs, xs)]
        lams, _, _, _ = sap_solve_adjoint_batched(ctx.bh, gxs)
        need_band = any(ctx.needs_input_grad[1:1 + n])
        gbands = sap_grad_band_batched(ctx.bh, lams, xs) if need_band else [None] * n
        gbs = [lam if ctx.needs_input_grad[1 + n + i] else None for i, lam in enumerate(lams)]
        gbands = [g if ctx.needs_input_grad[1 + i] else None for i, g in enumerate(gbands)]
        return (None, *gbands, *gbs)


def sap_solve_batched_autograd(bands, bs, Ns, Ks, **opts_kw):
    """Differentiable x_i = A_i^{-1} b_i for a batch (one shared option set)."""
    return list(SapSolveBatched.apply((list(Ns), list(Ks), opts_kw), *bands, *bs))
