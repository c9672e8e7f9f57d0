"""torch.autograd wrappers of the differentiable tree aggregation.

    ctx = hdp_create(HDPParams(..., mode="full", levels=1)); hdp_build_trees(ctx, L, R)
    C = HDPAggregate.apply(E, gamma, ctx)          # E: (H, W, X) float32 CUDA, gamma: 0-dim tensor
    d, loss = SoftArgminL1.apply(C, gt, valid, ctx)

Forward and backward both run in libhdp.so (argument marshalling only here).
The backward recomputes the aggregation instead of storing it.  The edge-weight
gradient of the last backward is kept in ctx.edge_grad (per grid edge id).
"""
from __future__ import annotations

import torch

from . import hdp_aggregate_bwd, hdp_aggregate_fwd, hdp_set_gamma, hdp_soft_argmin_l1


class HDPAggregate(torch.autograd.Function):
    @staticmethod
    def forward(fctx, E, gamma, ctx):
        E = E.contiguous()
        hdp_set_gamma(ctx, float(gamma))
        C = torch.empty_like(E)
        hdp_aggregate_fwd(ctx, E, C)
        fctx.save_for_backward(E, gamma)
        fctx.hctx = ctx
        return C

    @staticmethod
    def backward(fctx, gC):
        E, gamma = fctx.saved_tensors
        ctx = fctx.hctx
        hdp_set_gamma(ctx, float(gamma))
        gE = torch.empty_like(E)
        gw = torch.empty(2 * E.shape[0] * E.shape[1], dtype=torch.float32, device=E.device)
        gg = torch.empty(1, dtype=torch.float32, device=E.device)
        hdp_aggregate_bwd(ctx, E, gC.contiguous(), gE, gw, gg)
        ctx.edge_grad = gw
        return gE, gg.reshape(gamma.shape).to(gamma.dtype), None


class SoftArgminL1(torch.autograd.Function):
    """(disparity map, mean |d - gt| over valid pixels) from an aggregated volume."""

    @staticmethod
    def forward(fctx, C, gt, valid, ctx, T=1.0):
        C = C.contiguous()
        H, W, X = C.shape
        d = torch.empty((H, W), dtype=torch.float32, device=C.device)
        loss = torch.zeros(1, dtype=torch.float32, device=C.device)
        gC = torch.empty_like(C)
        hdp_soft_argmin_l1(ctx, C, gt.contiguous(), None if valid is None else valid.contiguous(), T, d, loss, gC)
        fctx.save_for_backward(gC)
        fctx.mark_non_differentiable(d)
        return d, loss.reshape(())

    @staticmethod
    def backward(fctx, gd, gloss):
        (gC,) = fctx.saved_tensors
        return gC * gloss, None, None, None, None
