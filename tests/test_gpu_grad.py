"""Differentiable tree aggregation on the GPU (through the C ABI) against the
FP64 oracle: forward Eq. C, the adjoint (dL/dE, dL/dw, dL/dgamma), FP64 central
differences (h = 1e-6) on 24x24 crops, and the soft-argmin + L1 readout."""
import numpy as np
import pytest

import oracle
import paper_1509_08197_gb300 as hdp
from paper_1509_08197_gb300.scenes import workload_pair

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

H = W = 24
D = 63
X = D + 1
GAMMA = 25.5


def _case(seed=0):
    pair = workload_pair("grad")
    L = np.ascontiguousarray(pair.left[40:40 + H, 60:60 + W])
    R = np.ascontiguousarray(pair.right[40:40 + H, 60:60 + W])
    gt = pair.gt[40:40 + H, 60:60 + W].astype(np.float32)
    dev = torch.device("cuda:0")
    hp = hdp.HDPParams(width=W, height=H, max_disp=D, levels=1, mode="full", tree="mst", gamma=GAMMA)
    ctx = hdp.hdp_create(hp)
    hdp.hdp_build_trees(ctx, torch.from_numpy(L).to(dev), torch.from_numpy(R).to(dev))
    Li = oracle.to_level0(L)
    w = oracle.edge_weights(Li)
    order = oracle.sort_edges(w, W, H)
    in_tree, _, _ = oracle.build_forest(W, H, order, w, np.tile(oracle.full_set(D), (W * H, 1)))
    bo, parent, _ = oracle.bfs(W, H, in_tree)
    wn = oracle.node_weights(W, H, parent, w)
    rng = np.random.default_rng(seed)
    E = rng.uniform(0, 2.5, size=(W * H, X))
    Ri = oracle.to_level0(R)
    return ctx, dev, dict(w=w, bo=bo, parent=parent, wn=wn, E=E, gt=gt, rng=rng, Li=Li, Ri=Ri,
                          gL=oracle.gradient(Li), gR=oracle.gradient(Ri))


def _s(o, gamma=GAMMA):
    return np.where(o["parent"] >= 0, np.exp(-o["wn"] / gamma), 0.0)


def _edge_id(v, p):
    if p == v - 1:
        return 2 * p
    if p == v + 1:
        return 2 * v
    if p == v - W:
        return 2 * p + 1
    return 2 * v + 1


def test_forward_matches_oracle():
    ctx, dev, o = _case()
    try:
        E = torch.from_numpy(o["E"].astype(np.float32).reshape(H, W, X)).to(dev)
        C = torch.empty_like(E)
        hdp.hdp_aggregate_fwd(ctx, E, C)
        hdp.hdp_sync(ctx)
        ref = oracle.aggregate_given(o["bo"], o["parent"], _s(o), E.cpu().numpy().reshape(-1, X).astype(np.float64))
        err = np.abs(C.cpu().numpy().reshape(-1, X) - ref) / np.abs(ref)
        assert err.max() < 1e-5
    finally:
        hdp.hdp_destroy(ctx)


def test_backward_matches_adjoint_and_central_differences():
    ctx, dev, o = _case(1)
    try:
        E32 = o["E"].astype(np.float32)
        g = o["rng"].normal(size=(W * H, X)).astype(np.float32)
        E = torch.from_numpy(E32.reshape(H, W, X)).to(dev)
        gC = torch.from_numpy(g.reshape(H, W, X)).to(dev)
        gE = torch.empty_like(E)
        gw = torch.empty(2 * H * W, dtype=torch.float32, device=dev)
        gg = torch.empty(1, dtype=torch.float32, device=dev)
        hdp.hdp_aggregate_bwd(ctx, E, gC, gE, gw, gg)
        hdp.hdp_sync(ctx)
        E64, g64 = E32.astype(np.float64), g.astype(np.float64)
        gE_o, gw_o, gg_o = oracle.aggregate_adjoint(o["bo"], o["parent"], o["wn"], GAMMA, E64, g64)
        gE_g = gE.cpu().numpy().reshape(-1, X)
        assert np.abs(gE_g - gE_o).max() <= 1e-4 * np.abs(gE_o).max()
        gw_g = gw.cpu().numpy()
        for v in range(W * H):
            p = o["parent"][v]
            if p >= 0:
                assert gw_g[_edge_id(v, p)] == pytest.approx(gw_o[v], rel=2e-3, abs=1e-3 * np.abs(gw_o).max())
        assert float(gg.cpu()) == pytest.approx(gg_o, rel=2e-3)

        # FP64 central differences of L = sum(g * C) with h = 1e-6
        def L(E_, wn_, gamma_):
            s = np.where(o["parent"] >= 0, np.exp(-wn_ / gamma_), 0.0)
            return float((g64 * oracle.aggregate_given(o["bo"], o["parent"], s, E_)).sum())
        h = 1e-6
        rng = o["rng"]
        for _ in range(4):
            i, x = int(rng.integers(0, W * H)), int(rng.integers(0, X))
            Ep, Em = E64.copy(), E64.copy()
            Ep[i, x] += h
            Em[i, x] -= h
            fd = (L(Ep, o["wn"], GAMMA) - L(Em, o["wn"], GAMMA)) / (2 * h)
            assert gE_g[i, x] == pytest.approx(fd, rel=1e-3, abs=1e-4)
        for v in np.flatnonzero(o["parent"] >= 0)[::97]:
            wp, wm = o["wn"].copy(), o["wn"].copy()
            wp[v] += h
            wm[v] -= h
            fd = (L(E64, wp, GAMMA) - L(E64, wm, GAMMA)) / (2 * h)
            assert gw_g[_edge_id(v, o["parent"][v])] == pytest.approx(fd, rel=5e-3, abs=1e-3 * np.abs(gw_o).max())
        fd = (L(E64, o["wn"], GAMMA + h) - L(E64, o["wn"], GAMMA - h)) / (2 * h)
        assert float(gg.cpu()) == pytest.approx(fd, rel=2e-3)
    finally:
        hdp.hdp_destroy(ctx)


def test_soft_argmin_l1_and_autograd_chain():
    from paper_1509_08197_gb300.autograd import HDPAggregate, SoftArgminL1
    ctx, dev, o = _case(2)
    try:
        rng = o["rng"]
        valid_np = rng.uniform(size=(H, W)) > 0.2
        E = torch.from_numpy(o["E"].astype(np.float32).reshape(H, W, X)).to(dev).requires_grad_(True)
        gamma = torch.tensor(GAMMA, dtype=torch.float32, device=dev, requires_grad=True)
        gt = torch.from_numpy(o["gt"]).to(dev)
        valid = torch.from_numpy(valid_np.astype(np.uint8)).to(dev)
        C = HDPAggregate.apply(E, gamma, ctx)
        d, loss = SoftArgminL1.apply(C, gt, valid, ctx)
        loss.backward()
        torch.cuda.synchronize()
        # FP64 reference of the whole chain
        E64 = o["E"].astype(np.float32).astype(np.float64)

        def Lfull(E_, gamma_):
            s = np.where(o["parent"] >= 0, np.exp(-o["wn"] / gamma_), 0.0)
            Cr = oracle.aggregate_given(o["bo"], o["parent"], s, E_)
            dr = oracle.soft_argmin(Cr)
            return float(np.abs(dr - o["gt"].ravel())[valid_np.ravel()].mean()), dr
        Lr, dr = Lfull(E64, GAMMA)
        assert np.abs(d.detach().cpu().numpy().ravel() - dr).max() < 1e-3
        assert float(loss.detach()) == pytest.approx(Lr, rel=1e-4)
        h = 1e-6
        gEg = E.grad.cpu().numpy().reshape(-1, X)
        for _ in range(4):
            i = int(rng.choice(np.flatnonzero(valid_np.ravel())))
            x = int(rng.integers(0, X))
            Ep, Em = E64.copy(), E64.copy()
            Ep[i, x] += h
            Em[i, x] -= h
            fd = (Lfull(Ep, GAMMA)[0] - Lfull(Em, GAMMA)[0]) / (2 * h)
            assert gEg[i, x] == pytest.approx(fd, rel=5e-3, abs=1e-6)
        fd = (Lfull(E64, GAMMA + h)[0] - Lfull(E64, GAMMA - h)[0]) / (2 * h)
        assert float(gamma.grad) == pytest.approx(fd, rel=5e-3, abs=1e-7)
    finally:
        hdp.hdp_destroy(ctx)


# cost parameters off the integer grids of hdp_params; no dc (a multiple of 1/3) or dg (of 1/6) lies within
# 1e-6 of tau_c or tau_g, so central differences with h = 1e-6 do not cross a truncation point
THETA = (0.83, 7.1, 2.05)


def _theta32(th):
    return [float(np.float32(v)) for v in th]


def test_cost_volume_matches_oracle():
    ctx, dev, o = _case()
    try:
        E = torch.empty((H, W, X), dtype=torch.float32, device=dev)
        hdp.hdp_cost_volume(ctx, *THETA, E)
        hdp.hdp_sync(ctx)
        ref = oracle.cost_volume(o["Li"], o["gL"], o["Ri"], o["gR"], 0, X, *_theta32(THETA))
        assert np.abs(E.cpu().numpy().reshape(-1, X) - ref).max() <= 2e-6 * max(1.0, np.abs(ref).max())
        with pytest.raises(hdp.HDPError):
            hdp.hdp_cost_volume(ctx, 0.5, -1.0, 2.0, E)    # a negative truncation is refused
        assert hdp.hdp_tree_level(ctx) == 0
        with pytest.raises(TypeError):                    # a volume of the wrong size never reaches the kernels
            hdp.hdp_cost_volume(ctx, *THETA, E[:-1].contiguous())
        with pytest.raises(TypeError):
            hdp.hdp_set_edge_weights(ctx, torch.zeros(2 * H * W - 1, device=dev))
    finally:
        hdp.hdp_destroy(ctx)


def _loss_oracle(o, E, wn, gamma, valid_np):
    s = np.where(o["parent"] >= 0, np.exp(-wn / gamma), 0.0)
    dr = oracle.soft_argmin(oracle.aggregate_given(o["bo"], o["parent"], s, E))
    return float(np.abs(dr - o["gt"].ravel())[valid_np.ravel()].mean())


def test_cost_parameter_and_gamma_gradients_match_central_differences():
    from paper_1509_08197_gb300.autograd import CostVolume, HDPAggregate, SoftArgminL1
    ctx, dev, o = _case(3)
    try:
        valid_np = o["rng"].uniform(size=(H, W)) > 0.2
        theta = torch.tensor(THETA, dtype=torch.float32, device=dev, requires_grad=True)
        gamma = torch.tensor(GAMMA, dtype=torch.float32, device=dev, requires_grad=True)
        gt = torch.from_numpy(o["gt"]).to(dev)
        valid = torch.from_numpy(valid_np.astype(np.uint8)).to(dev)
        E = CostVolume.apply(theta, ctx)
        C = HDPAggregate.apply(E, gamma, ctx)
        _, loss = SoftArgminL1.apply(C, gt, valid, ctx)
        loss.backward()
        torch.cuda.synchronize()

        def Lfull(th, gam):
            Eo = oracle.cost_volume(o["Li"], o["gL"], o["Ri"], o["gR"], 0, X, *th)
            return _loss_oracle(o, Eo, o["wn"], gam, valid_np)
        th0 = _theta32(THETA)
        assert float(loss.detach()) == pytest.approx(Lfull(th0, GAMMA), rel=1e-4)
        h = 1e-6
        g = theta.grad.cpu().numpy()
        for k in range(3):
            tp, tm = list(th0), list(th0)
            tp[k] += h
            tm[k] -= h
            fd = (Lfull(tp, GAMMA) - Lfull(tm, GAMMA)) / (2 * h)
            assert g[k] == pytest.approx(fd, rel=5e-3, abs=1e-6), f"parameter {k}"
        fd = (Lfull(th0, GAMMA + h) - Lfull(th0, GAMMA - h)) / (2 * h)
        assert float(gamma.grad) == pytest.approx(fd, rel=5e-3, abs=1e-7)
    finally:
        hdp.hdp_destroy(ctx)


def test_edge_weights_as_an_input():
    from paper_1509_08197_gb300.autograd import HDPAggregate, SoftArgminL1, image_edge_weights
    ctx, dev, o = _case(4)
    try:
        rng = o["rng"]
        valid_np = rng.uniform(size=(H, W)) > 0.2
        w_img = image_edge_weights(ctx, device=dev)
        assert np.array_equal(w_img.cpu().numpy(), np.where(o["w"] >= 0, o["w"], 0).astype(np.float32))
        w_np = np.maximum(w_img.cpu().numpy() + rng.uniform(-0.4, 0.4, size=2 * H * W).astype(np.float32), 0)
        w = torch.from_numpy(w_np).to(dev).requires_grad_(True)
        E = torch.from_numpy(o["E"].astype(np.float32).reshape(H, W, X)).to(dev)
        gamma = torch.tensor(GAMMA, dtype=torch.float32, device=dev)
        gt = torch.from_numpy(o["gt"]).to(dev)
        valid = torch.from_numpy(valid_np.astype(np.uint8)).to(dev)
        C = HDPAggregate.apply(E, gamma, ctx, w)
        _, loss = SoftArgminL1.apply(C, gt, valid, ctx)
        loss.backward()
        torch.cuda.synchronize()
        E64 = o["E"].astype(np.float32).astype(np.float64)
        wn = oracle.node_weights(W, H, o["parent"], w_np.astype(np.float64))
        assert float(loss.detach()) == pytest.approx(_loss_oracle(o, E64, wn, GAMMA, valid_np), rel=1e-4)
        gw = w.grad.cpu().numpy()
        tree = np.zeros(2 * H * W, bool)
        for v in np.flatnonzero(o["parent"] >= 0):
            tree[_edge_id(v, o["parent"][v])] = True
        assert np.all(gw[~tree] == 0)   # the tree is fixed: other edges carry no gradient
        h = 1e-6
        scale = np.abs(gw).max()
        for v in np.flatnonzero(o["parent"] >= 0)[::61]:
            wp, wm = wn.copy(), wn.copy()
            wp[v] += h
            wm[v] -= h
            fd = (_loss_oracle(o, E64, wp, GAMMA, valid_np) - _loss_oracle(o, E64, wm, GAMMA, valid_np)) / (2 * h)
            assert gw[_edge_id(v, o["parent"][v])] == pytest.approx(fd, rel=5e-3, abs=2e-3 * scale)
        # without weights the next call aggregates with the image's own again
        C2 = HDPAggregate.apply(E, gamma, ctx)
        ref = oracle.aggregate_given(o["bo"], o["parent"], _s(o), E64)
        assert (np.abs(C2.cpu().numpy().reshape(-1, X) - ref) / np.abs(ref)).max() < 1e-5
    finally:
        hdp.hdp_destroy(ctx)
