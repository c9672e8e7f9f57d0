"""CPU check of the decomposition the region engine relies on for risky layers.

On a layer where DT-Rule 2 may join different pixel sets (a "risky" layer),
the GPU resolves every connected component of the edges that survive DT-Rule 1
on its own CTA, each component's edges in the strict order.  That is exact
because no surviving edge joins two components, so no merge, Int, size or
TreeIntv of one component ever depends on another.  This test replays the
decomposition with the oracle itself: the sequential forest (Sec. 3.2: Rule 2,
DT-Rules 1 and 2, and for the segment tree its criterion and linking pass)
over the whole list must equal the union of the same algorithm run on each
component's sublist, on random grids with overlapping and disjoint sets.
"""
import numpy as np
import pytest

import oracle

scipy_sparse = pytest.importorskip("scipy.sparse")
from scipy.sparse.csgraph import connected_components  # noqa: E402


def _scene(rng, W, H):
    img = rng.integers(0, 256, (H, W, 3)).astype(np.int32)
    img = (img // 32) * 32 + rng.integers(0, 8, (H, W, 3))   # few weight classes, many ties
    # pixel sets: intervals around a blockwise centre, widths 0..2: neighbours
    # share sets, overlap partly or are disjoint
    centre = np.kron(rng.integers(2, 14, ((H + 3) // 4, (W + 3) // 4)), np.ones((4, 4), np.int64))[:H, :W]
    centre = centre + rng.integers(-1, 2, (H, W))
    half = rng.integers(0, 3, (H, W))
    pix = np.stack([oracle.set_from_labels(range(max(0, c - r), min(15, c + r) + 1))
                    for c, r in zip(centre.ravel(), half.ravel())])
    return img, pix


def _components(order, pix, W, N):
    rows, cols = [], []
    for e in order:
        p = e >> 1
        q = p + W if e & 1 else p + 1
        if (pix[p] & pix[q]).any():   # survives DT-Rule 1
            rows.append(p)
            cols.append(q)
    g = scipy_sparse.coo_matrix((np.ones(len(rows)), (rows, cols)), shape=(N, N))
    return connected_components(g, directed=False)


def _risky(order, pix, W, beta):
    for e in order:
        p = e >> 1
        q = p + W if e & 1 else p + 1
        a, b = pix[p], pix[q]
        inter = sum(bin(int(x)).count("1") for x in (a & b))
        uni = sum(bin(int(x)).count("1") for x in (a | b))
        if inter and not np.array_equal(a, b) and inter * beta[1] >= beta[0] * uni:
            return True
    return False


@pytest.mark.parametrize("tree,beta", [("mst", (1, 5)), ("st", (1, 5)), ("st", (3, 5)), ("mst", (3, 5))])
def test_components_of_the_dt_rule1_graph_resolve_independently(tree, beta):
    rng = np.random.default_rng(11)
    W, H = 15, 12
    N = W * H
    tested = 0
    for _ in range(8):
        img, pix = _scene(rng, W, H)
        w = oracle.edge_weights(img)
        order = oracle.sort_edges(w, W, H)
        full = oracle.build_forest(W, H, order, w, pix, beta, tree, st_k=300)
        ncomp, label = _components(order, pix, W, N)
        merged = np.zeros_like(full[0])
        root = np.arange(N, dtype=np.int32)
        tint = pix.copy()
        sizes = np.bincount(label, minlength=ncomp)
        for c in range(ncomp):
            if sizes[c] < 2:
                continue
            sub = np.array([e for e in order if label[e >> 1] == c], np.int32)
            part = oracle.build_forest(W, H, sub, w, pix, beta, tree, st_k=300)
            merged |= part[0]
            mine = label == c
            root[mine] = part[1][mine]
            tint[mine] = part[2][mine]
        assert np.array_equal(merged, full[0])
        assert np.array_equal(root, full[1])
        assert np.array_equal(tint, full[2])
        if ncomp > 1 and (sizes > 1).sum() > 1 and _risky(order, pix, W, beta):
            tested += 1
    assert tested >= 3, "too few scenes with several components on a risky layer"
