"""The whole HDP stereo method on the CPU oracle, in the paper's order.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 3: the layers are processed top-down, l = L .. 0.  At each layer:
  1. pixel-wise interval prediction (Sec. 3.1): layer L takes [0, d_L]; below
     it the prior P(D_l) is sampled, the posterior table built (Eq. dpm) and
     PixelIntv read from it by the upper layer's disparity (Eq. crtr);
  2. HDP forest construction (Sec. 3.2): edge weights (Eq. weight), DT-Rule 1,
     Kruskal with Rule 2 and DT-Rule 2 (Eq. DTrules), TreeIntv unions;
  3. aggregation over the forest (Sec. 3.3, Eqs. E, W, S, C) and WTA.
No refinement is applied (Sec. 3.3, last paragraph).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import (aggregate, bfs, build_forest, edge_weights, full_set, gradient, pixel_intervals, prior,
               median3, pyr_down, range_table, sort_edges, sort_edges_rt, to_level0)


@dataclass
class OracleParams:
    max_disp: int
    levels: int = 2                 # number of layers, L + 1
    tree: str = "mst"               # "mst" | "st" | "rt" (random spanning tree, Sec. 4.1)
    mode: str = "hdp"               # "hdp" | "full" (single layer, full range)
    gamma: float = 25.5             # Eq. S, 0.1 * 255
    alpha: float = 0.9              # cost weights ([Cost2])
    tau_c: float = 7.0
    tau_g: float = 2.0
    st_k: int = 1200                # ST merge constant (not given in the paper)
    beta: tuple = (3, 5)            # DT-Rule 2 threshold as a rational
    delta0: float = 0.064           # delta_l = delta0 * 2^l
    gmm: list = field(default_factory=list)   # per predicted layer: [[pi, mu, sd], ...]
    prior: str = "sampled"          # "sampled" | "uniform"
    rt_seed: int = 0                # seed of the random tree's edge order
    prefilter: str = "none"         # "none" | "median3" (the M+* variants, Sec. 4.1)

    def tree_weights(self, L):
        """Eq. (weight) on the layer's image, median-filtered first for the M+* variants."""
        return edge_weights(median3(L) if self.prefilter == "median3" else L)

    def edge_order(self, w, W, H, level):
        """Rule 1: (w, id) order for MST and ST; the seeded random order for RT."""
        if self.tree == "rt":
            return sort_edges_rt(w, W, H, self.rt_seed, level)
        return sort_edges(w, W, H)

    def gmm_for(self, l):
        if l < len(self.gmm) and self.gmm[l] is not None:
            return np.asarray(self.gmm[l], np.float64).reshape(-1, 3)
        return np.array([[1.0, 0.0, 1.0]])

    @property
    def cost_ints(self):
        return int(round(20 * self.alpha)), int(round(3 * self.tau_c)), int(round(6 * self.tau_g))


def pyramid(img_u8: np.ndarray, layers: int):
    out = [to_level0(img_u8)]
    for _ in range(1, layers):
        out.append(pyr_down(out[-1]))
    return out


def match(left: np.ndarray, right: np.ndarray, p: OracleParams, keep: bool = False,
          want_costs: bool = False, inject_up=None):
    """Run the method; returns (D_0, per-layer records if keep).

    inject_up: optional {l: D_{l+1} map} used instead of the oracle's own
    upper-layer result (stage tests feed the CUDA path's inputs this way)."""
    layers = 1 if p.mode == "full" else p.levels
    Ls = pyramid(left, layers)
    Rs = pyramid(right, layers)
    d = [p.max_disp]
    for _ in range(1, layers):
        d.append(d[-1] // 2)
    a20, tc3, tg6 = p.cost_ints
    recs = {}
    D_up = None
    for l in reversed(range(layers)):
        L, R = Ls[l], Rs[l]
        H, W, _ = L.shape
        gL, gR = gradient(L), gradient(R)
        rec = {}
        if l == layers - 1:
            pix = np.tile(full_set(d[l]), (W * H, 1))
        else:
            if inject_up is not None and l in inject_up:
                D_up = inject_up[l]
            pw = prior(L, gL, R, gR, l, d[l], a20, tc3, tg6) if p.prior == "sampled" else np.ones(d[l] + 1, np.int64)
            masks = range_table(pw, d[l], d[l + 1], p.gmm_for(l), p.delta0 * (2 ** l))
            pix = pixel_intervals(W, H, D_up, masks)
            rec.update(prior=pw, masks=masks)
        w = p.tree_weights(L)
        order = p.edge_order(w, W, H, l)
        in_tree, dt_root, tint = build_forest(W, H, order, w, pix, p.beta, p.tree, p.st_k, l)
        bfs_order, parent, depth = bfs(W, H, in_tree)
        agg = aggregate(L, gL, R, gR, l, d[l], bfs_order, parent, w, tint, p.gamma, p.alpha, p.tau_c, p.tau_g,
                        want_costs=want_costs)
        D = agg["wta"].reshape(H, W)
        if keep:
            rec.update(L=L, R=R, gL=gL, gR=gR, W=W, H=H, d=d[l], pix=pix, w=w, order=order, in_tree=in_tree,
                       dt_root=dt_root, tree_intv=tint, bfs=bfs_order, parent=parent, depth=depth, agg=agg, D=D,
                       D_up=D_up)
            recs[l] = rec
        D_up = D
    return D_up, recs


def refine(left: np.ndarray, right: np.ndarray, p: OracleParams, want_costs: bool = False):
    """Tree-based refinement at layer 0 (Sec. 3.3, last paragraph; readings in hdp_oracle.c).

    The right view's map is the method run with the views exchanged, which is
    the left-reference method on both images mirrored left-right.  Returns
    (refined D_0, record with D_L, D_R, refD and the refinement aggregation)."""
    from . import lr_check, refine_aggregate
    D_L, recs = match(left, right, p, keep=True)
    D_Rm, _ = match(np.ascontiguousarray(right[:, ::-1]), np.ascontiguousarray(left[:, ::-1]), p)
    D_R = np.ascontiguousarray(D_Rm[:, ::-1])
    refD = lr_check(D_L, D_R)
    r0 = recs[0]
    agg = refine_aggregate(r0["W"], r0["H"], 0, r0["d"], r0["bfs"], r0["parent"], r0["w"], r0["tree_intv"], refD,
                           p.gamma, want_costs=want_costs)
    D = agg["wta"].reshape(r0["H"], r0["W"])
    return D, dict(D_L=D_L, D_R=D_R, refD=refD, agg=agg, rec0=r0)
