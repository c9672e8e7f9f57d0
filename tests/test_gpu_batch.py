"""Batched matching: pairs of different sizes and ranges run concurrently on
their own streams (and as one captured CUDA graph) give exactly the
disparity maps of matching them one at a time."""
import numpy as np
import pytest

import paper_1509_08197_gb300 as hdp
from paper_1509_08197_gb300.scenes import workload_pair

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("depths", ["mixed", "equal", "groups"])
def test_batch_equals_one_at_a_time(depths):
    # mixed depths: every pair runs its own chain; equal depths: level by level,
    # one aggregation launch per pass and tile class over the tiles of every
    # pair of a group of one geometry (here every pair is its own group);
    # groups: two pairs of each of two geometries (different scenes and
    # ranges), so each group's launches take the tiles of two pairs
    dev = torch.device("cuda:0")
    if depths == "groups":
        specs = [("tiny", dict()), ("tiny", dict(width=77, height=41, max_disp=31)),
                 ("tiny", dict(max_disp=23)), ("tiny", dict(width=77, height=41, max_disp=19))]
    else:
        specs = [("tiny", dict()), ("tiny", dict(width=77, height=41, max_disp=31)),
                 ("tiny", dict(width=120, height=90, max_disp=47)), ("third", dict())]
    pairs, params = [], []
    for i, (name, over) in enumerate(specs):
        p = workload_pair(name, index=i, **over)
        pairs.append(p)
        H, W, _ = p.left.shape
        levels = (3 if W < 200 else 4) if depths == "mixed" else 3
        # groups: the 96x72 pairs FP32 with MST, the 77x41 pairs FP16 with ST (one geometry per group)
        storage = "fp16" if (i == 3 if depths != "groups" else i % 2 == 1) else "fp32"
        params.append(hdp.HDPParams(width=W, height=H, max_disp=p.max_disp, levels=levels,
                                    tree="mst" if i % 2 == 0 else "st", storage=storage))
    # two contexts on caller streams, two that own theirs
    ctxs = [hdp.hdp_create(hp, torch.cuda.Stream(device=dev)) if i < 2 else hdp.hdp_create_own_stream(hp)
            for i, hp in enumerate(params)]
    assert hdp.hdp_get_stream(ctxs[3]) is not None
    try:
        L = [torch.from_numpy(p.left).to(dev).contiguous() for p in pairs]
        R = [torch.from_numpy(p.right).to(dev).contiguous() for p in pairs]
        ref = []
        for c, l, r, hp in zip(ctxs, L, R, params):
            out = torch.empty((hp.height, hp.width), dtype=torch.int32, device=dev)
            hdp.hdp_build_trees(c, l, r)
            hdp.hdp_match(c, out)
            hdp.hdp_sync(c)
            ref.append(out.cpu().numpy())
        outs = [torch.full((hp.height, hp.width), -1, dtype=torch.int32, device=dev) for hp in params]
        hdp.hdp_match_batch(ctxs, L, R, outs)
        for c in ctxs:
            hdp.hdp_sync(c)
        for o, r in zip(outs, ref):
            assert np.array_equal(o.cpu().numpy(), r)
        for o in outs:
            o.fill_(-1)
        nk = hdp.hdp_batch_graph_capture(ctxs, L, R, outs)
        assert nk > 100
        hdp.hdp_batch_graph_launch(ctxs[0])
        hdp.hdp_batch_graph_launch(ctxs[0])
        for c in ctxs:
            hdp.hdp_sync(c)
        for o, r in zip(outs, ref):
            assert np.array_equal(o.cpu().numpy(), r)
    finally:
        for c in ctxs:
            hdp.hdp_destroy(c)
