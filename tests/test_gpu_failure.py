"""Failure path of the bounded device waits, without faulting the GPU.

Every spin in the library (grid barriers of cooperative kernels, decoupled
look-backs of the scans and of the aggregation tiles) gives up after a bounded
number of polls, records a timeout in the context's device status and lets
its kernel return.  hdp_wait_probe drives two of those waits into their limit
on something that never arrives; the test checks that the timeout is reported
by hdp_sync as HDP_ERR_TIMEOUT, that the report clears the status, and that
the context then matches a pair exactly as a fresh context does."""
import numpy as np
import pytest

import paper_1509_08197_gb300 as hdp
from paper_1509_08197_gb300.scenes import workload_pair

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _match(ctx, pair, dev):
    out = torch.empty((ctx.params.height, ctx.params.width), dtype=torch.int32, device=dev)
    hdp.hdp_build_trees(ctx, torch.from_numpy(pair.left).to(dev), torch.from_numpy(pair.right).to(dev))
    hdp.hdp_match(ctx, out)
    hdp.hdp_sync(ctx)
    return out.cpu().numpy()


@pytest.mark.parametrize("kind", [0, 1])
def test_a_wait_that_runs_out_reports_timeout_and_the_context_recovers(kind):
    dev = torch.device("cuda:0")
    pair = workload_pair("tiny")
    hp = hdp.HDPParams(width=96, height=72, max_disp=15, levels=2, tree="st", st_k=300)
    ctx = hdp.hdp_create(hp)
    try:
        before = _match(ctx, pair, dev)
        hdp.hdp_wait_probe(ctx, kind, 1000)
        with pytest.raises(hdp.HDPError) as e:
            hdp.hdp_sync(ctx)
        assert f"({hdp.HDP_ERR_TIMEOUT})" in str(e.value)
        hdp.hdp_sync(ctx)                  # reported once, then cleared
        after = _match(ctx, pair, dev)     # grid barriers and scans work again
    finally:
        hdp.hdp_destroy(ctx)
    assert np.array_equal(before, after)


def test_wait_probe_rejects_bad_arguments():
    hp = hdp.HDPParams(width=96, height=72, max_disp=15, levels=2)
    ctx = hdp.hdp_create(hp)
    try:
        for kind, limit in ((2, 10), (0, 0), (1, 1 << 25)):
            with pytest.raises(hdp.HDPError):
                hdp.hdp_wait_probe(ctx, kind, limit)
    finally:
        hdp.hdp_destroy(ctx)
