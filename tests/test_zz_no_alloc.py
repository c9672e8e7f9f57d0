"""hdp_match_noalloc: the entry point for callers that cannot allocate device
memory.  It must give the same disparity map as the context-based path
(hdp_create + hdp_build_trees + hdp_match) on the same inputs, on two calls in
a row (the fixed workspace keeps the previous call's contents), and refuse
problems larger than its fixed workspace.  This file is collected last."""
import ctypes

import numpy as np
import pytest

import paper_1509_08197_gb300 as hdp
from paper_1509_08197_gb300.scenes import workload_pair

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _reference(params, pair, dev):
    ctx = hdp.hdp_create(params)
    try:
        out = torch.empty((params.height, params.width), dtype=torch.int32, device=dev)
        hdp.hdp_build_trees(ctx, torch.from_numpy(pair.left).to(dev), torch.from_numpy(pair.right).to(dev))
        hdp.hdp_match(ctx, out)
        hdp.hdp_sync(ctx)
        return out.cpu().numpy()
    finally:
        hdp.hdp_destroy(ctx)


def _noalloc(params, pair, dev):
    out = torch.full((params.height, params.width), -7, dtype=torch.int32, device=dev)
    left = torch.from_numpy(pair.left).to(dev).contiguous()
    right = torch.from_numpy(pair.right).to(dev).contiguous()
    hdp.hdp_match_noalloc(params, left, right, out)
    torch.cuda.synchronize(dev)
    return out.cpu().numpy()


def test_noalloc_matches_context_path_twice():
    dev = torch.device("cuda:0")
    cases = [
        (hdp.HDPParams(width=96, height=72, max_disp=15, levels=2, tree="mst"), workload_pair("tiny")),
        (hdp.HDPParams(width=77, height=41, max_disp=31, levels=3, tree="st", st_k=300),
         workload_pair("tiny", index=1, width=77, height=41, max_disp=31)),
    ]
    for params, pair in cases:
        ref = _reference(params, pair, dev)
        first = _noalloc(params, pair, dev)
        second = _noalloc(params, pair, dev)
        # disparities are integers: the same kernels on the same inputs give the same map
        assert np.array_equal(first, ref)
        assert np.array_equal(second, ref)


def test_noalloc_rejects_problems_above_its_workspace():
    big = hdp.HDPParams(width=1390, height=1110, max_disp=255, levels=5)
    dev = torch.device("cuda:0")
    left = torch.zeros((1110, 1390, 3), dtype=torch.uint8, device=dev)
    out = torch.zeros((1110, 1390), dtype=torch.int32, device=dev)
    with pytest.raises(hdp.HDPError):
        hdp.hdp_match_noalloc(big, left, left, out)
