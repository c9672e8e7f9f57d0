"""Tree-based refinement (Sec. 3.3, last paragraph) on the GPU against the FP64 oracle.

Both sides compute the left map, the right map (the method on the mirrored,
exchanged views), the left-right check and the aggregation of |x - D_L| over
layer 0's forest.  The maps of both views must equal the oracle's (these pairs
have no near ties upstream), the checked map bit for bit, the refinement's
aggregated costs within REL_TOL and its WTA up to counted near ties."""
import numpy as np
import pytest

import oracle
import paper_1509_08197_gb300 as hdp
from oracle.pipeline import refine
from paper_1509_08197_gb300.scenes import workload_pair

from parity_util import REL_TOL, oracle_params, rel_err, wta_mismatch

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("case", ["tiny_hdp_mst", "tiny_full_st", "ragged_hdp_st"])
def test_refinement_matches_the_oracle(case):
    if case == "tiny_hdp_mst":
        pair = workload_pair("tiny")
        hp = hdp.HDPParams(width=96, height=72, max_disp=15, levels=2, tree="mst")
    elif case == "tiny_full_st":
        pair = workload_pair("tiny")
        hp = hdp.HDPParams(width=96, height=72, max_disp=15, levels=1, mode="full", tree="st", st_k=300)
    else:
        pair = workload_pair("tiny", index=2, width=77, height=41, max_disp=31)
        hp = hdp.HDPParams(width=77, height=41, max_disp=31, levels=3, tree="st", st_k=300)
    D_ref, rec = refine(pair.left, pair.right, oracle_params(hp), want_costs=True)
    dev = torch.device("cuda:0")
    L = torch.from_numpy(pair.left).to(dev)
    R = torch.from_numpy(pair.right).to(dev)
    out = torch.empty((hp.height, hp.width), dtype=torch.int32, device=dev)
    ctx = hdp.hdp_create(hp)
    try:
        hdp.hdp_build_trees(ctx, L, R)
        hdp.hdp_match(ctx, out)
        D_L = hdp.hdp_get_stage(ctx, 0, "disp").reshape(hp.height, hp.width)
        hdp.hdp_refine(ctx, L, R, out)
        hdp.hdp_sync(ctx)
        D = out.cpu().numpy()
        refD = hdp.hdp_get_stage(ctx, 0, "ref_d").reshape(hp.height, hp.width)
        D_R = hdp.hdp_get_stage(ctx, 0, "disp_r").reshape(hp.height, hp.width)
        costs = hdp.hdp_get_stage(ctx, 0, "costs")
        assert np.array_equal(hdp.hdp_get_stage(ctx, 0, "disp").reshape(D.shape), D)
    finally:
        hdp.hdp_destroy(ctx)
    assert np.array_equal(D_L, rec["D_L"]), "left map"
    assert np.array_equal(D_R, rec["D_R"]), "right map"
    assert np.array_equal(refD, oracle.lr_check(D_L, D_R)), "left-right check"
    assert (refD >= 0).mean() > 0.2   # the check is not degenerate
    err = rel_err(costs, rec["agg"]["costs"])
    assert err.max() <= REL_TOL, f"refinement costs: max relative error {err.max():.3g}"
    n, allowed = wta_mismatch(D.ravel(), rec["agg"])
    assert n == allowed, f"{n} refined disparities differ, {allowed} near ties"
    assert np.array_equal(D, D_ref) or n > 0


def test_refine_stages_need_a_refinement():
    hp = hdp.HDPParams(width=96, height=72, max_disp=15, levels=2)
    ctx = hdp.hdp_create(hp)
    try:
        with pytest.raises(hdp.HDPError):
            hdp.hdp_get_stage(ctx, 0, "ref_d")
    finally:
        hdp.hdp_destroy(ctx)
