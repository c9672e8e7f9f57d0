"""torch.autograd wrappers of the differentiable tree aggregation.

    ctx = hdp_create(HDPParams(..., mode="full", levels=1)); hdp_build_trees(ctx, L, R)
    theta = torch.tensor([alpha, tau_c, tau_g], device="cuda", requires_grad=True)
    E = CostVolume.apply(theta, ctx)                # (H, W, X) float32: the matching cost of the loaded layer
    w = image_edge_weights(ctx).requires_grad_()    # optional: real-valued edge weights per grid edge id
    C = HDPAggregate.apply(E, gamma, ctx, w)        # gamma: 0-dim tensor; w may be None
    d, loss = SoftArgminL1.apply(C, gt, valid, ctx)

Forward and backward all run in libhdp.so (argument marshalling only here):
the cost parameters, gamma and the edge weights receive gradients.  The tree
itself stays the one built from the images (it is piecewise constant in the
weights).  The backward recomputes the aggregation instead of storing it.
The edge-weight gradient of the last backward is also kept in ctx.edge_grad
(per grid edge id), whether or not w was given.
"""
from __future__ import annotations

import numpy as np
import torch

from . import (hdp_aggregate_bwd, hdp_aggregate_fwd, hdp_cost_volume, hdp_cost_volume_bwd, hdp_get_stage,
               hdp_set_edge_weights, hdp_set_gamma, hdp_soft_argmin_l1, hdp_tree_level)


def _layer_shape(ctx, level=None):
    l = hdp_tree_level(ctx) if level is None else level
    if l < 0:
        raise RuntimeError("no tree loaded (call hdp_build_trees)")
    W, H, d = ctx.dims[l]
    return l, H, W, d + 1


def image_edge_weights(ctx, level=None, device="cuda"):
    """The image's own weights of the loaded layer (after hdp_build_trees: the top layer) as float32 per grid
    edge id, in intensity units (the pyramid scale 4^l divided out); 0 for the ids that are no edge."""
    l, H, W, _ = _layer_shape(ctx, level)
    w = hdp_get_stage(ctx, l, "weights").astype(np.float64)
    w = np.where(w >= 0, w / float(4 ** l), 0.0).astype(np.float32)
    return torch.from_numpy(w).to(device)


def _scalars(t):
    return [float(v) for v in t.detach().reshape(-1).float().cpu()]


def _use_weights(ctx, w):
    """Load w (or the image's weights when None) for the next aggregation; gamma must be set before."""
    if w is not None or getattr(ctx, "_wf", False):
        hdp_set_edge_weights(ctx, None if w is None else w.detach().float().contiguous())
    ctx._wf = w is not None


class CostVolume(torch.autograd.Function):
    """E = (1 - alpha) min(dc, tau_c) + alpha min(dg, tau_g) over every pixel and label of the loaded layer, for
    theta = (alpha, tau_c, tau_g); the backward gives dL/dtheta."""

    @staticmethod
    def forward(fctx, theta, ctx, level=None):
        alpha, tau_c, tau_g = _scalars(theta)
        _, H, W, X = _layer_shape(ctx, level)
        dev = theta.device if theta.is_cuda else torch.device("cuda")
        E = torch.empty((H, W, X), dtype=torch.float32, device=dev)
        hdp_cost_volume(ctx, alpha, tau_c, tau_g, E)
        fctx.params = (alpha, tau_c, tau_g)
        fctx.hctx = ctx
        fctx.theta_meta = (theta.dtype, theta.device, theta.shape)
        return E

    @staticmethod
    def backward(fctx, gE):
        g = torch.empty(3, dtype=torch.float32, device=gE.device)
        hdp_cost_volume_bwd(fctx.hctx, *fctx.params, gE.contiguous(), g)
        dtype, device, shape = fctx.theta_meta
        return g.to(device=device, dtype=dtype).reshape(shape), None, None


class HDPAggregate(torch.autograd.Function):
    @staticmethod
    def forward(fctx, E, gamma, ctx, w=None):
        E = E.contiguous()
        hdp_set_gamma(ctx, float(gamma))
        _use_weights(ctx, w)
        C = torch.empty_like(E)
        hdp_aggregate_fwd(ctx, E, C)
        if w is None:
            fctx.save_for_backward(E, gamma)
        else:
            fctx.save_for_backward(E, gamma, w)
        fctx.hctx = ctx
        return C

    @staticmethod
    def backward(fctx, gC):
        saved = fctx.saved_tensors
        E, gamma = saved[0], saved[1]
        w = saved[2] if len(saved) > 2 else None
        ctx = fctx.hctx
        hdp_set_gamma(ctx, float(gamma))
        _use_weights(ctx, w)
        gE = torch.empty_like(E)
        gw = torch.empty(2 * E.shape[0] * E.shape[1], dtype=torch.float32, device=E.device)
        gg = torch.empty(1, dtype=torch.float32, device=E.device)
        hdp_aggregate_bwd(ctx, E, gC.contiguous(), gE, gw, gg)
        ctx.edge_grad = gw
        gw_out = None if w is None else gw.to(w.dtype).reshape(w.shape)
        return gE, gg.reshape(gamma.shape).to(gamma.dtype), None, gw_out


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
