"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Each layer is run on the GPU with the oracle's upper-layer disparities
injected, so every stage is compared on identical inputs: pyramid, edge
weights and order, forest edges, tree roots and TreeIntv, BFS order, parents
and depths, prior, interval table and pixel sets bit-exactly; aggregated
costs within 1e-5 relative; WTA identical except near ties (counted).
"""
import numpy as np
import pytest

import oracle
import paper_1509_08197_gb300 as hdp
from paper_1509_08197_gb300.scenes import workload_pair

from parity_util import (GAP_TOL, REL_TOL, end_to_end_check, oracle_layer, oracle_params, pyramids, rel_err,
                         wta_mismatch)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _run_layers(hp, pair, check_costs=True, layers=None, tuning=None):
    """Run every layer on both sides; return per-layer comparison records."""
    dev = torch.device("cuda:0")
    ctx = hdp.hdp_create(hp)
    try:
        if tuning:
            t = hdp.hdp_get_tuning(ctx)
            for k, v in tuning.items():
                setattr(t, k, v)
            hdp.hdp_set_tuning(ctx, t)
        left = torch.from_numpy(pair.left).to(dev).contiguous()
        right = torch.from_numpy(pair.right).to(dev).contiguous()
        hdp.hdp_build_trees(ctx, left, right)
        op = oracle_params(hp)
        Ls, Rs = pyramids(pair.left, pair.right, len(ctx.dims))
        out = {}
        D_up = None
        for l in range(ctx.top, -1, -1):
            W, H, d = ctx.dims[l]
            d_up = ctx.dims[l + 1][2] if l < ctx.top else 0
            if l < ctx.top:
                hdp.hdp_set_stage(ctx, l + 1, "disp", D_up.astype(np.int32).ravel())
            hdp.hdp_run_level(ctx, l)
            o = oracle_layer(op, Ls[l], Rs[l], l, ctx.top, d, d_up, D_up, want_costs=check_costs)
            g = {k: hdp.hdp_get_stage(ctx, l, k) for k in
                 ("pyr_left", "pyr_right", "weights", "edges", "in_tree", "dt_root", "tree_intv", "bfs", "parent",
                  "depth", "disp", "info")}
            if check_costs:
                g["costs"] = hdp.hdp_get_stage(ctx, l, "costs")
            if l < ctx.top and hp.mode == "hdp":
                g["prior"] = hdp.hdp_get_stage(ctx, l, "prior")
                g["table"] = hdp.hdp_get_stage(ctx, l, "table")
                g["pix_set"] = hdp.hdp_get_stage(ctx, l, "pix_set")
            out[l] = (g, o)
            D_up = o["agg"]["wta"].reshape(H, W)
        return out
    finally:
        hdp.hdp_destroy(ctx)


def _assert_layer(l, g, o, hp, d, wta=True):
    W = o["L"].shape[1]
    assert np.array_equal(g["pyr_left"][..., :3], o["L"]), f"layer {l}: left pyramid"
    assert np.array_equal(g["pyr_right"][..., :3], o["R"]), f"layer {l}: right pyramid"
    assert np.array_equal(g["pyr_left"][..., 3], o["gL"]), f"layer {l}: gradient"
    assert np.array_equal(g["weights"], o["weights"].astype(np.int32)), f"layer {l}: edge weights"
    if "prior" in g:
        assert np.array_equal(g["prior"], o["prior"]), f"layer {l}: prior"
        assert np.array_equal(g["table"], o["table"]), f"layer {l}: interval table"
        assert np.array_equal(g["pix_set"], o["pix_set"]), f"layer {l}: pixel sets"
    assert np.array_equal(g["edges"], o["edges"]), f"layer {l}: sorted edges"
    assert np.array_equal(g["in_tree"], o["in_tree"]), f"layer {l}: forest edges"
    assert np.array_equal(g["dt_root"], o["dt_root"]), f"layer {l}: tree roots"
    assert np.array_equal(g["tree_intv"], o["tree_intv"]), f"layer {l}: TreeIntv"
    assert np.array_equal(g["bfs"], o["bfs"]), f"layer {l}: BFS order"
    assert np.array_equal(g["parent"], o["parent"]), f"layer {l}: parents"
    assert np.array_equal(g["depth"], o["depth"]), f"layer {l}: depths"
    if "costs" in g:
        assert g["costs"].shape == o["agg"]["costs"].shape
        err = rel_err(g["costs"], o["agg"]["costs"])
        assert err.max() <= REL_TOL, f"layer {l}: max relative cost error {err.max():.3g}"
    if not wta:
        return
    n, allowed = wta_mismatch(g["disp"], o["agg"])
    assert n == allowed, f"layer {l}: {n} WTA differences, only {allowed} are near ties (gap < {GAP_TOL})"


def test_tiny_hdp_mst():
    pair = workload_pair("tiny")
    hp = hdp.HDPParams(width=96, height=72, max_disp=15, levels=2, tree="mst")
    res = _run_layers(hp, pair)
    for l, (g, o) in res.items():
        _assert_layer(l, g, o, hp, None)


@pytest.mark.parametrize("case", ["tiny_hdp", "third_hdp", "third_hdp_risky", "third_full"])
def test_random_tree(case):
    # HDP+RT (Sec. 4.1): the seeded random edge order through the same engines;
    # every stage bit-exact, costs within REL_TOL, WTA up to near ties
    if case == "tiny_hdp":
        pair = workload_pair("tiny")
        hp = hdp.HDPParams(width=96, height=72, max_disp=15, levels=2, tree="rt", rt_seed=11)
    elif case == "third_hdp":
        pair = workload_pair("third")
        hp = hdp.HDPParams(width=463, height=370, max_disp=79, levels=4, tree="rt", rt_seed=12)
    elif case == "third_hdp_risky":
        pair = workload_pair("third")
        hp = hdp.HDPParams(width=463, height=370, max_disp=79, levels=3, tree="rt", rt_seed=13, beta=(1, 5))
    else:
        pair = workload_pair("third")
        hp = hdp.HDPParams(width=463, height=370, max_disp=79, levels=1, mode="full", tree="rt", rt_seed=14)
    res = _run_layers(hp, pair)
    if case == "third_hdp_risky":
        assert int(res[0][0]["info"][5]) == 1 and int(res[0][0]["info"][3]) == 7
    for l, (g, o) in res.items():
        _assert_layer(l, g, o, hp, None)


@pytest.mark.parametrize("case", ["tiny_hdp_mst", "third_hdp_st", "third_full_st"])
def test_median_prefilter(case):
    # M+* variants (Sec. 4.1): tree weights from the 3x3 median-filtered layer image
    if case == "tiny_hdp_mst":
        pair = workload_pair("tiny")
        hp = hdp.HDPParams(width=96, height=72, max_disp=15, levels=2, prefilter="median3")
    elif case == "third_hdp_st":
        pair = workload_pair("third")
        hp = hdp.HDPParams(width=463, height=370, max_disp=79, levels=4, tree="st", prefilter="median3")
    else:
        pair = workload_pair("third")
        hp = hdp.HDPParams(width=463, height=370, max_disp=79, levels=1, mode="full", tree="st",
                           prefilter="median3")
    res = _run_layers(hp, pair)
    for l, (g, o) in res.items():
        _assert_layer(l, g, o, hp, None)


def test_injected_prior_rebuilds_the_table():
    # the priors and tables of predicted layers run on the context's side
    # stream after hdp_build_trees; a prior set afterwards must win, and the
    # layer's table must be rebuilt from it
    pair = workload_pair("tiny")
    hp = hdp.HDPParams(width=96, height=72, max_disp=15, levels=2, tree="mst")
    dev = torch.device("cuda:0")
    ctx = hdp.hdp_create(hp)
    try:
        left = torch.from_numpy(pair.left).to(dev).contiguous()
        right = torch.from_numpy(pair.right).to(dev).contiguous()
        hdp.hdp_build_trees(ctx, left, right)
        op = oracle_params(hp)
        d0, d1 = ctx.dims[0][2], ctx.dims[1][2]
        custom = np.random.default_rng(7).integers(1, 60, d0 + 1).astype(np.int64)
        hdp.hdp_set_stage(ctx, 0, "prior", custom)
        hdp.hdp_run_level(ctx, 1)
        hdp.hdp_run_level(ctx, 0)
        assert np.array_equal(hdp.hdp_get_stage(ctx, 0, "prior"), custom)
        want = oracle.range_table(custom, d0, d1, op.gmm_for(0), op.delta0)
        assert np.array_equal(hdp.hdp_get_stage(ctx, 0, "table"), want)
    finally:
        hdp.hdp_destroy(ctx)


def test_tiny_hdp_st_and_full():
    pair = workload_pair("tiny")
    for hp in (hdp.HDPParams(width=96, height=72, max_disp=15, levels=2, tree="st", st_k=300),
               hdp.HDPParams(width=96, height=72, max_disp=15, levels=1, mode="full", tree="mst"),
               hdp.HDPParams(width=96, height=72, max_disp=15, levels=1, mode="full", tree="st")):
        res = _run_layers(hp, pair)
        for l, (g, o) in res.items():
            _assert_layer(l, g, o, hp, None)


@pytest.mark.parametrize("tree", ["mst", "st"])
def test_third_size_hdp(tree):
    # 463x370, range 0-79, 4 layers (small-image delta0/beta: DT-Rule 2 can merge different sets)
    pair = workload_pair("third")
    hp = hdp.HDPParams(width=463, height=370, max_disp=79, levels=4, tree=tree)
    res = _run_layers(hp, pair)
    for l, (g, o) in res.items():
        _assert_layer(l, g, o, hp, None)


@pytest.mark.parametrize("tree,one_cta", [("mst", False), ("st", False), ("mst", True), ("st", True)])
def test_risky_layers_take_the_reservation_engine(tree, one_cta):
    # beta = 1/5: DT-Rule 2 joins many different sets, so the lower layers are
    # "risky" and only reservations are exact there: windows with each local
    # tree's TreeIntv in shared memory, over each component of the edges that
    # survive DT-Rule 1 on its own CTA (engine 7), or over the whole list on
    # one CTA when the region engine is switched off (engine 6)
    pair = workload_pair("third")
    hp = hdp.HDPParams(width=463, height=370, max_disp=79, levels=3, tree=tree, beta=(1, 5))
    res = _run_layers(hp, pair, tuning=dict(region_max_nodes=1) if one_cta else None)
    risky = {l: int(g["info"][5]) for l, (g, o) in res.items()}
    engine = {l: int(g["info"][3]) for l, (g, o) in res.items()}
    assert risky[0] == 1 and risky[1] == 1, risky
    assert all(engine[l] == (6 if one_cta else 7) for l in risky if risky[l]), engine
    for l, (g, o) in res.items():
        _assert_layer(l, g, o, hp, None)


def test_engines_of_the_segment_tree():
    # first pass by regions on the HDP layers, windowed on the (small) top layer
    pair = workload_pair("third")
    # beta = 99/100: no two different PixelIntv sets of this scene qualify
    hp = hdp.HDPParams(width=463, height=370, max_disp=79, levels=3, tree="st", beta=(99, 100))
    res = _run_layers(hp, pair, check_costs=False)
    engine = {l: int(g["info"][3]) for l, (g, o) in res.items()}
    risky = {l: int(g["info"][5]) for l, (g, o) in res.items()}
    assert not any(risky.values()), risky
    assert engine[0] == 5 and engine[1] == 5 and engine[2] == 3, engine
    for l, (g, o) in res.items():
        _assert_layer(l, g, o, hp, None)
    # hybrid first pass on a full-range layer of >= 131072 nodes
    hp = hdp.HDPParams(width=463, height=370, max_disp=79, levels=1, mode="full", tree="st")
    res = _run_layers(hp, pair, check_costs=False)
    assert int(res[0][0]["info"][3]) == 4
    _assert_layer(0, res[0][0], res[0][1], hp, None)


def test_ragged_sizes_and_uniform_prior():
    # odd sizes (partial pyramid squares, ragged tiles), uniform prior, beta 0.95
    pair = workload_pair("tiny", width=77, height=41, max_disp=31)
    hp = hdp.HDPParams(width=77, height=41, max_disp=31, levels=3, tree="mst", prior="uniform", beta=(19, 20),
                       delta0=0.01)
    res = _run_layers(hp, pair)
    for l, (g, o) in res.items():
        _assert_layer(l, g, o, hp, None)


def _end_to_end(hp, pair):
    """Whole runs on both sides (no injection); returns the GPU's maps of every layer and the oracle's records."""
    from oracle.pipeline import match
    _, recs = match(pair.left, pair.right, oracle_params(hp), keep=True)
    ctx = hdp.hdp_create(hp)
    try:
        dev = torch.device("cuda:0")
        out = torch.empty((hp.height, hp.width), dtype=torch.int32, device=dev)
        hdp.hdp_build_trees(ctx, torch.from_numpy(pair.left).to(dev), torch.from_numpy(pair.right).to(dev))
        hdp.hdp_match(ctx, out)
        hdp.hdp_sync(ctx)
        maps = {l: hdp.hdp_get_stage(ctx, l, "disp") for l in range(ctx.top + 1)}
        D = out.cpu().numpy()
        D2 = hdp.hdp_match_host(ctx, pair.left, pair.right)
        top = ctx.top
    finally:
        hdp.hdp_destroy(ctx)
    assert np.array_equal(D.ravel(), maps[0])
    assert np.array_equal(D, D2)
    return maps, recs, top


def test_end_to_end_match_and_host_path():
    # no injection: each side runs the whole method on its own; the maps must be
    # identical except at counted near ties of the oracle (gap < GAP_TOL)
    pair = workload_pair("tiny")
    hp = hdp.HDPParams(width=96, height=72, max_disp=15, levels=2)
    maps, recs, top = _end_to_end(hp, pair)
    per_layer, bad = end_to_end_check(maps, recs, top)
    assert bad is None, f"unexplained WTA differences: {per_layer}"


def test_headline_end_to_end_1390x1110():
    # the configuration the throughput is quoted on: 1390x1110, range 0-255,
    # 5 layers, HDP + segment tree, beta 0.95, delta0 0.004, FP32
    pair = workload_pair("full")
    hp = hdp.HDPParams(width=1390, height=1110, max_disp=255, levels=5, tree="st")
    maps, recs, top = _end_to_end(hp, pair)
    per_layer, bad = end_to_end_check(maps, recs, top)
    assert bad is None, f"unexplained WTA differences: {per_layer}"


def test_headline_stages_1390x1110():
    # every stage of every layer of the headline configuration, the oracle's
    # upper-layer disparities injected: 256-label rows on the top layers and
    # 1.5M-node regions on layer 0
    pair = workload_pair("full")
    hp = hdp.HDPParams(width=1390, height=1110, max_disp=255, levels=5, tree="st")
    res = _run_layers(hp, pair)
    for l, (g, o) in res.items():
        _assert_layer(l, g, o, hp, None)


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_full_range_st_d255_big_layer(storage):
    # a full-range segment-tree layer of 171,310 nodes (hybrid first pass) with
    # 256 labels per row: FP32 costs within REL_TOL, FP16 within its storage bound
    pair = workload_pair("third", max_disp=255)
    hp = hdp.HDPParams(width=463, height=370, max_disp=255, levels=1, mode="full", tree="st", storage=storage)
    res = _run_layers(hp, pair)
    g, o = res[0]
    assert int(g["info"][3]) == 4, "hybrid first pass expected"
    if storage == "fp32":
        _assert_layer(0, g, o, hp, None)
    else:
        _assert_layer(0, {k: v for k, v in g.items() if k not in ("costs", "disp")}, o, hp, None, wta=False)
        _assert_fp16_layer(0, hp, pair, g, o)


def _assert_fp16_layer(l, hp, pair, g16, o):
    """FP16 storage: costs within 2e-3 relative of FP64, WTA flips only within twice that gap."""
    # storage rounds each stored entry to 11 significant bits (relative 2^-11);
    # a value goes through at most two stores plus FP32 recurrences
    err = rel_err(g16["costs"], o["agg"]["costs"])
    assert err.max() < 2e-3, f"layer {l}: fp16 max relative error {err.max():.3g}"
    agg = o["agg"]
    diff = np.flatnonzero(g16["disp"] != agg["wta"])
    gap = (agg["second"][diff] - agg["best"][diff]) / np.maximum(np.abs(agg["best"][diff]), 1e-30)
    assert (gap < 4e-3).all(), f"layer {l}: fp16 flips with gap up to {gap.max():.3g}"


@pytest.mark.parametrize("case", ["hdp_mst_463x370", "full_st_96x72"])
def test_fp16_storage_error(case):
    # HDP layers mix row widths (tiles with and without TMA bulk copies); the
    # full-range case has 16-label rows, so every tile moves by bulk copies
    if case == "hdp_mst_463x370":
        pair = workload_pair("third")
        base = dict(width=463, height=370, max_disp=79, levels=4, tree="mst")
    else:
        pair = workload_pair("tiny")
        base = dict(width=96, height=72, max_disp=15, levels=1, mode="full", tree="st")
    r16 = _run_layers(hdp.HDPParams(storage="fp16", **base), pair)
    for l in r16:
        g16, o = r16[l]
        _assert_fp16_layer(l, None, pair, g16, o)


def test_host_path_replays_its_graph():
    # on a context with its own stream, hdp_match_host captures its device work
    # on the first call and replays it; a tuning change drops the graph
    pair = workload_pair("tiny", index=3)
    hp = hdp.HDPParams(width=96, height=72, max_disp=15, levels=2, tree="st", st_k=300)
    ref_ctx = hdp.hdp_create(hp)
    ctx = hdp.hdp_create_own_stream(hp)
    try:
        ref = hdp.hdp_match_host(ref_ctx, pair.left, pair.right)       # default stream: eager
        maps = [hdp.hdp_match_host(ctx, pair.left, pair.right) for _ in range(3)]
        t = hdp.hdp_get_tuning(ctx)
        t.agg_ctas_per_sm = 3
        hdp.hdp_set_tuning(ctx, t)
        maps.append(hdp.hdp_match_host(ctx, pair.left, pair.right))
        other = workload_pair("tiny", index=4)
        D_other = hdp.hdp_match_host(ctx, other.left, other.right)    # new inputs through the same graph
        D_other_ref = hdp.hdp_match_host(ref_ctx, other.left, other.right)
    finally:
        hdp.hdp_destroy(ctx)
        hdp.hdp_destroy(ref_ctx)
    for m in maps:
        assert np.array_equal(m, ref)
    assert np.array_equal(D_other, D_other_ref)
