"""torch.autograd.Function for the sampled correntropy loss (Welsch form of Eq. corr at
sampled entries of a tensor-ring model, Def. 1), with the library's hand-written adjoint.

    loss = sum_m sigma^2 (1 - exp(-(x_m - Tr(prod_k Z_k(i_mk)))^2 / (2 sigma^2)))

Forward and backward both run in libtrd's CUDA kernels; the merged subchains are recomputed
in the backward pass rather than stored.  Core tensors use the library layout
(I_k, r_{k+1}, r_k) (row i is row i of the mode-2 unfolding, column alpha + beta r_k).
"""
from __future__ import annotations

from typing import Sequence

import torch

from .binding import TRD


class TRCorrentropy(torch.autograd.Function):
    """loss = TRCorrentropy.apply(handle, idx, x, sigma, *cores)"""

    @staticmethod
    def forward(ctx, handle: TRD, idx: torch.Tensor, x: torch.Tensor, sigma: float, *cores: torch.Tensor):
        cores_c = [c.detach().contiguous() for c in cores]
        loss = handle.sampled_fwd(cores_c, idx, x.detach().contiguous(), float(sigma))
        ctx.handle, ctx.sigma = handle, float(sigma)
        ctx.save_for_backward(idx, x, *cores_c)
        return torch.tensor(loss, dtype=cores[0].dtype, device=cores[0].device)

    @staticmethod
    def backward(ctx, gout: torch.Tensor):
        idx, x, *cores = ctx.saved_tensors
        grads = ctx.handle.sampled_bwd(cores, idx, x.contiguous(), ctx.sigma, float(gout.item()))
        return (None, None, None, None, *grads)


def sampled_correntropy(handle: TRD, cores: Sequence[torch.Tensor], idx: torch.Tensor, x: torch.Tensor,
                        sigma: float) -> torch.Tensor:
    """Differentiable sampled correntropy loss of the TR model `cores` at `idx`."""
    return TRCorrentropy.apply(handle, idx, x, sigma, *cores)
