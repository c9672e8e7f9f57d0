"""Shared helpers of the GPU parity tests: run one layer on the oracle and on
the CUDA path from the same inputs and compare stage by stage."""
from __future__ import annotations

import numpy as np

import oracle
from oracle.pipeline import OracleParams, pyramid

REL_TOL = 1e-5          # FP32 aggregated cost vs FP64 (relative, R23 form)
GAP_TOL = 1e-6          # WTA may differ only where the oracle's top-two gap is below this (relative)


def oracle_params(hp) -> OracleParams:
    large = hp.width > 640
    beta = hp.beta if hp.beta is not None else ((95, 100) if large else (3, 5))
    delta0 = hp.delta0 if hp.delta0 is not None else (0.004 if large else 0.064)
    return OracleParams(max_disp=hp.max_disp, levels=hp.levels, tree=hp.tree, mode=hp.mode, gamma=hp.gamma,
                        alpha=hp.alpha, tau_c=hp.tau_c, tau_g=hp.tau_g, st_k=hp.st_k, beta=beta, delta0=delta0,
                        gmm=hp.gmm, prior=hp.prior, rt_seed=hp.rt_seed, prefilter=hp.prefilter)


def oracle_layer(op: OracleParams, L, R, l, top, d_l, d_up, D_up, want_costs=True):
    """All stages of layer l on the oracle, given the upper layer's disparities."""
    H, W, _ = L.shape
    gL, gR = oracle.gradient(L), oracle.gradient(R)
    rec = {}
    hdp = op.mode == "hdp" and l < top
    if not hdp:
        pix = np.tile(oracle.full_set(d_l), (W * H, 1))
    else:
        a20, tc3, tg6 = op.cost_ints
        pw = oracle.prior(L, gL, R, gR, l, d_l, a20, tc3, tg6) if op.prior == "sampled" else np.ones(d_l + 1, np.int64)
        masks = oracle.range_table(pw, d_l, d_up, op.gmm_for(l), op.delta0 * 2 ** l)
        pix = oracle.pixel_intervals(W, H, D_up, masks)
        rec.update(prior=pw, table=masks, pix_set=D_up[np.arange(H)[:, None] // 2, np.arange(W)[None, :] // 2].ravel())
    w = op.tree_weights(L)
    order = op.edge_order(w, W, H, l)
    in_tree, dt_root, tint = oracle.build_forest(W, H, order, w, pix, op.beta, op.tree, op.st_k, l)
    bo, parent, depth = oracle.bfs(W, H, in_tree)
    agg = oracle.aggregate(L, gL, R, gR, l, d_l, bo, parent, w, tint, op.gamma, op.alpha, op.tau_c, op.tau_g,
                           want_costs=want_costs)
    # edges that pass DT-Rule 1, in (w, id) order
    if hdp:
        p = order >> 1
        q = np.where(order & 1, p + W, p + 1)
        keep = (pix[p] & pix[q]).any(axis=1)
        edges = order[keep]
    else:
        edges = order
    rec.update(L=L, R=R, gL=gL, gR=gR, pix=pix, weights=w, edges=edges, in_tree=in_tree, dt_root=dt_root,
               tree_intv=tint, bfs=bo, parent=parent, depth=depth, agg=agg)
    return rec


def rel_err(g, o):
    o = np.asarray(o, np.float64)
    g = np.asarray(g, np.float64)
    floor = 1e-6 * max(np.abs(o).mean(), 1e-30)
    return np.abs(g - o) / np.maximum(np.abs(o), floor)


def wta_mismatch(gpu_d, agg):
    """(number of WTA differences, how many of them the near-tie rule allows)."""
    o = agg["wta"]
    diff = np.flatnonzero(gpu_d != o)
    if diff.size == 0:
        return 0, 0
    best, second = agg["best"][diff], agg["second"][diff]
    gap = (second - best) / np.maximum(np.abs(best), 1e-30)
    return int(diff.size), int((gap < GAP_TOL).sum())


def pyramids(left, right, layers):
    return pyramid(left, layers), pyramid(right, layers)


def layer_gaps(agg, idx):
    """The oracle's relative top-two gap at pixels idx."""
    best, second = agg["best"][idx], agg["second"][idx]
    return (second - best) / np.maximum(np.abs(best), 1e-30)


def end_to_end_check(gpu_disp, recs, top):
    """Compare a whole GPU run with the oracle's whole run layer by layer, top down.

    gpu_disp[l] is the GPU's D_l, recs[l] the oracle's record of layer l.  While
    every upper layer agrees, layer l sees identical inputs on both sides, so its
    maps must agree except at counted near ties (oracle gap < GAP_TOL).  Once a
    layer differs (at allowed near ties only), the layers below see different
    predicted ranges and are no longer comparable; they are reported, not
    asserted.  Returns (per-layer list of (layer, mismatches, near ties,
    compared), first layer with an unexplained difference or None)."""
    out, bad = [], None
    comparable = True
    for l in range(top, -1, -1):
        o = recs[l]["agg"]
        diff = np.flatnonzero(np.asarray(gpu_disp[l]).ravel() != o["wta"])
        near = int((layer_gaps(o, diff) < GAP_TOL).sum()) if diff.size else 0
        out.append((l, int(diff.size), near, comparable))
        if comparable and diff.size != near and bad is None:
            bad = l
        if diff.size:
            comparable = False
    return out, bad
