"""GMM_l by EM (Sec. 2.2) on the GPU against the FP64 oracle.

The ground-truth pyramid and the offset histograms are integer work and must
be bit-exact; the EM fit runs in FP32 and must agree with the oracle's FP64 fit
after the same iterations within EM_TOL (weights and spreads relative, means
absolute in units of the widest spread)."""
import numpy as np
import pytest

import oracle
import paper_1509_08197_gb300 as hdp
from paper_1509_08197_gb300.scenes import integer_gt, training_pairs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

EM_TOL = 2e-4


def _gt_maps(n=2):
    return [integer_gt(p) for p in training_pairs("third", n)]


def test_gt_pyramid_and_offsets_are_exact():
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(41)
    for (H, W) in [(370, 463), (41, 77), (1, 9), (2, 2)]:
        g = rng.integers(-1, 80, size=(H, W)).astype(np.int32)
        g[rng.random((H, W)) < 0.1] = -1
        lo = torch.from_numpy(g).to(dev)
        up = hdp.hdp_gt_down(lo)
        want_up = oracle.gt_down(g)
        assert np.array_equal(up.cpu().numpy(), want_up)
        for rgn in (39, 3):
            h = torch.zeros(2 * rgn + 1, dtype=torch.int64, device=dev)
            hdp.hdp_offset_hist(up, lo, rgn, h)
            hdp.hdp_offset_hist(up, lo, rgn, h)    # accumulates
            want = oracle.offset_hist(want_up, g, rgn)
            assert np.array_equal(h.cpu().numpy(), 2 * want)


def _close(g, o):
    g = np.asarray(g, np.float64)
    o = np.asarray(o, np.float64)
    scale = o[:, 2].max()
    assert np.allclose(g[:, 0], o[:, 0], rtol=EM_TOL, atol=EM_TOL * 1e-2), (g, o)
    assert np.allclose(g[:, 1], o[:, 1], rtol=0, atol=EM_TOL * scale), (g, o)
    assert np.allclose(g[:, 2], o[:, 2], rtol=EM_TOL, atol=0), (g, o)


@pytest.mark.parametrize("K", [1, 2, 3])
def test_em_matches_the_oracle_on_training_offsets(K):
    dev = torch.device("cuda:0")
    maps = _gt_maps()
    d = [79, 39, 19, 9]
    for l in range(3):
        h = np.zeros(2 * d[l + 1] + 1, np.int64)
        for g in maps:
            lo = g
            for _ in range(l):
                lo = oracle.gt_down(lo)
            oracle.offset_hist(oracle.gt_down(lo), lo, d[l + 1], h)
        want = oracle.gmm_em(h, d[l + 1], K, 200)
        got = hdp.hdp_gmm_em(torch.from_numpy(h).to(dev), d[l + 1], K, 200).cpu().numpy()
        _close(got, want)


def test_em_matches_the_oracle_on_a_sampled_mixture():
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(42)
    n = 300000
    core = rng.random(n) < 0.6
    x = np.where(core, rng.normal(-2.0, 1.2, n), rng.normal(5.0, 9.0, n))
    o = np.clip(np.rint(x), -127, 127).astype(int)
    h = np.bincount(o + 127, minlength=255).astype(np.int64)
    for K, iters in ((2, 1), (2, 50), (2, 400), (4, 100)):
        want = oracle.gmm_em(h, 127, K, iters)
        got = hdp.hdp_gmm_em(torch.from_numpy(h).to(dev), 127, K, iters).cpu().numpy()
        _close(got, want)


def test_fit_gmm_end_to_end():
    # the binding's composition (GPU pyramid, histograms, EM per layer) equals the oracle's
    maps = _gt_maps()
    got = hdp.fit_gmm(maps, 79, 4, K=2, iters=150)
    d = [79, 39, 19, 9]
    los = list(maps)
    for l in range(3):
        h = np.zeros(2 * d[l + 1] + 1, np.int64)
        ups = []
        for lo in los:
            up = oracle.gt_down(lo)
            oracle.offset_hist(up, lo, d[l + 1], h)
            ups.append(up)
        los = ups
        _close(got[l], oracle.gmm_em(h, d[l + 1], 2, 150))


def test_em_rejects_bad_arguments():
    lib = hdp.load()
    assert lib.hdp_gmm_em(None, 10, 2, 10, 0.5, None, None) == hdp.HDP_ERR_ARG
    dev = torch.device("cuda:0")
    h = torch.zeros(21, dtype=torch.int64, device=dev)
    out = torch.empty(27, dtype=torch.float32, device=dev)
    import ctypes
    P = ctypes.c_void_p
    assert lib.hdp_gmm_em(P(h.data_ptr()), 10, 9, 10, 0.5, P(out.data_ptr()), None) == hdp.HDP_ERR_ARG
    assert lib.hdp_gmm_em(P(h.data_ptr()), 256, 2, 10, 0.5, P(out.data_ptr()), None) == hdp.HDP_ERR_ARG
    assert lib.hdp_gmm_em(P(h.data_ptr()), 10, 2, 10, 0.0, P(out.data_ptr()), None) == hdp.HDP_ERR_ARG
