"""Launch-shape knobs change only the speed: every setting, and the
autotuner's pick, gives bit-identical forests, costs and disparity maps."""
import numpy as np
import pytest

import paper_1509_08197_gb300 as hdp
from paper_1509_08197_gb300.scenes import workload_pair

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _match(ctx, L, R, H, W):
    out = torch.empty((H, W), dtype=torch.int32, device=L.device)
    hdp.hdp_build_trees(ctx, L, R)
    hdp.hdp_match(ctx, out)
    hdp.hdp_sync(ctx)
    return out.cpu().numpy(), hdp.hdp_get_stage(ctx, 0, "in_tree"), hdp.hdp_get_stage(ctx, 0, "costs")


@pytest.mark.parametrize("tree", ["mst", "st"])
def test_knobs_do_not_change_results(tree):
    pair = workload_pair("third")
    H, W, _ = pair.left.shape
    dev = torch.device("cuda:0")
    L = torch.from_numpy(pair.left).to(dev).contiguous()
    R = torch.from_numpy(pair.right).to(dev).contiguous()
    ctx = hdp.hdp_create(hdp.HDPParams(width=W, height=H, max_disp=79, levels=3, tree=tree))
    try:
        t0 = hdp.hdp_get_tuning(ctx)
        assert t0.as_dict() == dict(agg_ctas_per_sm=8, region_ctas_per_sm=1, big_class_edges=2048,
                                    one_cta_nodes=131072, boruvka_edges_per_cta=4096, region_max_nodes=1 << 24,
                                    tile_small_nodes=1 << 17, tile_small_nodes_hdp=1 << 19, col_min_labels=64)
        ref = _match(ctx, L, R, H, W)
        for kw in (dict(agg_ctas_per_sm=1, region_ctas_per_sm=1, big_class_edges=64, one_cta_nodes=1024,
                        boruvka_edges_per_cta=512, region_max_nodes=0),
                   dict(agg_ctas_per_sm=2, region_ctas_per_sm=3, big_class_edges=4096, one_cta_nodes=1 << 24,
                        boruvka_edges_per_cta=1 << 20, region_max_nodes=1 << 30),
                   dict(agg_ctas_per_sm=3, region_ctas_per_sm=2, big_class_edges=256, one_cta_nodes=1 << 24,
                        boruvka_edges_per_cta=2048, region_max_nodes=0)):
            hdp.hdp_set_tuning(ctx, _tuning(t0, **kw))
            got = _match(ctx, L, R, H, W)
            for a, b in zip(ref, got):
                assert np.array_equal(a, b)
        hdp.hdp_set_tuning(ctx, t0)
        with pytest.raises(hdp.HDPError):
            hdp.hdp_set_tuning(ctx, _tuning(t0, agg_ctas_per_sm=0))
        with pytest.raises(hdp.HDPError):
            hdp.hdp_set_tuning(ctx, _tuning(t0, col_min_labels=32))   # the column kernel needs 64 label slots
    finally:
        hdp.hdp_destroy(ctx)


def _tuning(base, **kw):
    t = hdp.Tuning(**base.as_dict())
    for k, v in kw.items():
        setattr(t, k, v)
    return t


@pytest.mark.parametrize("mode", ["hdp", "full"])
def test_layout_knobs_keep_the_integer_stages(mode):
    # tile sizes and the column/warp kernel choice: forests and orders bit for
    # bit, costs within FP32 rounding, maps identical except near ties; the
    # autotuner's pick likewise
    from parity_util import REL_TOL, rel_err
    pair = workload_pair("third")
    H, W, _ = pair.left.shape
    dev = torch.device("cuda:0")
    L = torch.from_numpy(pair.left).to(dev).contiguous()
    R = torch.from_numpy(pair.right).to(dev).contiguous()
    hp = hdp.HDPParams(width=W, height=H, max_disp=79, levels=3, tree="st") if mode == "hdp" else \
        hdp.HDPParams(width=W, height=H, max_disp=79, levels=1, mode="full", tree="st")
    ctx = hdp.hdp_create(hp)
    try:
        t0 = hdp.hdp_get_tuning(ctx)
        ref = _match(ctx, L, R, H, W)
        picks = [dict(col_min_labels=257), dict(tile_small_nodes=1 << 30, tile_small_nodes_hdp=1 << 30),
                 dict(tile_small_nodes=0, tile_small_nodes_hdp=0, col_min_labels=128)]
        for kw in picks:
            try:
                hdp.hdp_set_tuning(ctx, _tuning(t0, **kw))
            except hdp.HDPError:
                continue   # more tiles than the look-back scratch holds: refused, nothing run
            d, tree, costs = _match(ctx, L, R, H, W)
            assert np.array_equal(tree, ref[1])
            assert costs.shape == ref[2].shape and rel_err(costs, ref[2]).max() <= REL_TOL
            assert (d != ref[0]).mean() < 1e-3
        hdp.hdp_set_tuning(ctx, t0)
        best = hdp.hdp_autotune(ctx, L, R, reps=1)
        assert best.as_dict() == hdp.hdp_get_tuning(ctx).as_dict()
        d, tree, costs = _match(ctx, L, R, H, W)
        assert np.array_equal(tree, ref[1]) and rel_err(costs, ref[2]).max() <= REL_TOL
        assert (d != ref[0]).mean() < 1e-3
    finally:
        hdp.hdp_destroy(ctx)
