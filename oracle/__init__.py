"""FP64 CPU oracle for HDP stereo matching (arXiv 1509.08197).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the package smoke check and
by the CPU-baseline leg of bench.py, never by the product path.  It shares no
code with the CUDA implementation.

The arithmetic lives in hdp_oracle.c (plain C, FP64, one function per step of
the paper); this module compiles it with gcc on first use and wraps it with
ctypes.  pipeline.py strings the steps together in the paper's order;
brute.py holds brute-force checkers for tiny inputs.

Parity status of each function (what pins it) is listed in tests/test_oracle_pins.py;
every function here has at least one pin that does not re-run its own code.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hdp_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

WORDS = 8  # 256-bit label sets


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, FP64, no FP contraction) next to its source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-strict-aliasing",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _declare(_lib)
    return _lib


P = ctypes.c_void_p
I = ctypes.c_int
I64 = ctypes.c_int64
D = ctypes.c_double


def _declare(L):
    sig = {
        "orc_pyr_down": (I, [P, I, I, P]),
        "orc_gradient": (I, [P, I, I, P]),
        "orc_cost_m": (D, [P, P, P, P, I, I, I, I, I, D, D, D]),
        "orc_cost_mq": (I64, [P, P, P, P, I, I, I, I, I, I, I, I]),
        "orc_cost_volume": (I, [P, P, P, P, I, I, I, I, D, D, D, P]),
        "orc_edge_weights": (I, [P, I, I, P]),
        "orc_median3": (I, [P, I, I, P]),
        "orc_sort_edges": (I, [P, I, I, P]),
        "orc_splitmix64": (ctypes.c_uint64, [ctypes.c_uint64, ctypes.c_uint64]),
        "orc_sort_edges_rt": (I, [P, I, I, ctypes.c_uint64, I, P]),
        "orc_build_forest": (I, [I, I, P, I, P, P, I, I, I, I64, I, P, P, P]),
        "orc_bfs": (I, [I, I, P, P, P, P]),
        "orc_aggregate": (I, [I, I, I, I, P, P, P, P, D, D, D, D, P, P, P, P, P, P, P, P, P]),
        "orc_prior": (I, [P, P, P, P, I, I, I, I, I, I, I, P, P]),
        "orc_gmm_density": (D, [I, P, D]),
        "orc_range_table": (I, [P, I, I, I, P, D, P, P]),
        "orc_pixel_intervals": (I, [I, I, P, I, P, P]),
        "orc_aggregate_given": (I, [I64, I, P, P, P, P, P, P]),
        "orc_gt_down": (I, [P, I, I, P]),
        "orc_lr_check": (I, [P, P, I, I, P]),
        "orc_refine_aggregate": (I, [I, I, I, I, D, P, P, P, P, P, P, P, P, P, P]),
        "orc_offset_hist": (I, [P, I, P, I, I, I, P]),
        "orc_gmm_em": (I, [P, I, I, I, D, P, P]),
        "orc_aggregate_adjoint": (I, [I64, I, P, P, P, D, P, P, P, P, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


def _p(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ---------------------------------------------------------------- wrappers ---
def to_level0(img_u8: np.ndarray) -> np.ndarray:
    """uint8 (H, W, 3) -> int32 (H, W, 3) at scale 4^0."""
    return _c(img_u8, np.int32)


def pyr_down(img: np.ndarray) -> np.ndarray:
    img = _c(img, np.int32)
    H, W, _ = img.shape
    out = np.empty(((H + 1) // 2, (W + 1) // 2, 3), np.int32)
    lib().orc_pyr_down(_p(img), W, H, _p(out))
    return out


def gradient(img: np.ndarray) -> np.ndarray:
    img = _c(img, np.int32)
    H, W, _ = img.shape
    g = np.empty((H, W), np.int32)
    lib().orc_gradient(_p(img), W, H, _p(g))
    return g


def cost_m(L, gL, R, gR, level, px, py, x, alpha=0.9, tau_c=7.0, tau_g=2.0):
    H, W, _ = L.shape
    return lib().orc_cost_m(_p(L), _p(gL), _p(R), _p(gR), W, level, px, py, x, alpha, tau_c, tau_g)


def cost_volume(L, gL, R, gR, level, X, alpha=0.9, tau_c=7.0, tau_g=2.0):
    """Dense FP64 cost volume [H*W][X] of a layer (orc_cost_m at every pixel and label)."""
    L, gL, R, gR = _c(L, np.int32), _c(gL, np.int32), _c(R, np.int32), _c(gR, np.int32)
    H, W, _ = L.shape
    E = np.empty((H * W, X), np.float64)
    lib().orc_cost_volume(_p(L), _p(gL), _p(R), _p(gR), W, H, level, X, alpha, tau_c, tau_g, _p(E))
    return E


def cost_mq(L, gL, R, gR, level, px, py, x, a20=18, tc3=21, tg6=12):
    H, W, _ = L.shape
    return lib().orc_cost_mq(_p(L), _p(gL), _p(R), _p(gR), W, level, px, py, x, a20, tc3, tg6)


def median3(img: np.ndarray) -> np.ndarray:
    """3 x 3 per-channel median with replicated borders (the M+* prefilter, Sec. 4.1)."""
    img = _c(img, np.int32)
    H, W, _ = img.shape
    out = np.empty_like(img)
    lib().orc_median3(_p(img), W, H, _p(out))
    return out


def edge_weights(img: np.ndarray) -> np.ndarray:
    img = _c(img, np.int32)
    H, W, _ = img.shape
    w = np.empty(2 * H * W, np.int64)
    lib().orc_edge_weights(_p(img), W, H, _p(w))
    return w


def sort_edges(w: np.ndarray, W: int, H: int) -> np.ndarray:
    w = _c(w, np.int64)
    order = np.empty(2 * W * H, np.int32)
    n = lib().orc_sort_edges(_p(w), W, H, _p(order))
    return order[:n].copy()


def splitmix64(seed: int, i: int) -> int:
    """The i-th output of SplitMix64 from state `seed` (the random tree's generator)."""
    return int(lib().orc_splitmix64(seed & (2 ** 64 - 1), i & (2 ** 64 - 1)))


def sort_edges_rt(w: np.ndarray, W: int, H: int, seed: int, level: int) -> np.ndarray:
    """Random-tree order (Sec. 4.1): valid edges by (31-bit SplitMix64 key, id)."""
    w = _c(w, np.int64)
    order = np.empty(2 * W * H, np.int32)
    n = lib().orc_sort_edges_rt(_p(w), W, H, seed & (2 ** 64 - 1), int(level), _p(order))
    if n < 0:
        raise MemoryError("orc_sort_edges_rt")
    return order[:n].copy()


def build_forest(W, H, order, w, pix_intv, beta=(0, 1), tree="mst", st_k=0, level=0):
    """Returns (in_tree[2N] uint8, dt_root[N] int32, tree_intv[N, 8] uint32)."""
    order = _c(order, np.int32)
    w = _c(w, np.int64)
    pix_intv = _c(pix_intv, np.uint32).reshape(-1)
    N = W * H
    in_tree = np.zeros(2 * N, np.uint8)
    root = np.empty(N, np.int32)
    tint = np.empty(N * WORDS, np.uint32)
    rc = lib().orc_build_forest(W, H, _p(order), len(order), _p(w), _p(pix_intv), int(beta[0]), int(beta[1]),
                                1 if tree == "st" else 0, int(st_k), int(level), _p(in_tree), _p(root), _p(tint))
    if rc:
        raise MemoryError("orc_build_forest")
    return in_tree, root, tint.reshape(N, WORDS)


def bfs(W, H, in_tree):
    in_tree = _c(in_tree, np.uint8)
    N = W * H
    order = np.empty(N, np.int32)
    parent = np.empty(N, np.int32)
    depth = np.empty(N, np.int32)
    rc = lib().orc_bfs(W, H, _p(in_tree), _p(order), _p(parent), _p(depth))
    if rc:
        raise RuntimeError(f"orc_bfs failed ({rc})")
    return order, parent, depth


def set_sizes(sets: np.ndarray) -> np.ndarray:
    """Number of labels in each 256-bit set (rows of 8 uint32)."""
    s = _c(sets, np.uint32).reshape(-1, WORDS)
    return np.unpackbits(s.view(np.uint8), axis=1).sum(1).astype(np.int64)


def aggregate(L, gL, R, gR, level, d_l, order, parent, w, tree_intv, gamma=25.5,
              alpha=0.9, tau_c=7.0, tau_g=2.0, want_costs=True):
    """Returns dict(costs (ragged, pixel-major, labels ascending) or None, row_off, wta, best, second)."""
    H, W, _ = L.shape
    N = W * H
    tint = _c(tree_intv, np.uint32).reshape(N, WORDS)
    k = set_sizes(tint)
    row_off = np.zeros(N + 1, np.int64)
    np.cumsum(k, out=row_off[1:])
    costs = np.empty(int(row_off[-1]), np.float64) if want_costs else None
    wta = np.empty(N, np.int32)
    best = np.empty(N, np.float64)
    second = np.empty(N, np.float64)
    rc = lib().orc_aggregate(W, H, level, d_l, _p(_c(L, np.int32)), _p(_c(gL, np.int32)), _p(_c(R, np.int32)),
                             _p(_c(gR, np.int32)), alpha, tau_c, tau_g, gamma, _p(_c(order, np.int32)),
                             _p(_c(parent, np.int32)), _p(_c(w, np.int64)), _p(tint), _p(row_off),
                             _p(costs), _p(wta), _p(best), _p(second))
    if rc:
        raise MemoryError("orc_aggregate")
    return dict(costs=costs, row_off=row_off, wta=wta, best=best, second=second)


def prior(L, gL, R, gR, level, d_l, a20=18, tc3=21, tg6=12, want_centres=False):
    """Prior weights (count + 1); with want_centres also (H//5, W//5, 2) int32 of (dL, dR)."""
    H, W, _ = L.shape
    out = np.empty(d_l + 1, np.int64)
    cen = np.empty((H // 5) * (W // 5) * 2, np.int32) if want_centres else None
    lib().orc_prior(_p(_c(L, np.int32)), _p(_c(gL, np.int32)), _p(_c(R, np.int32)), _p(_c(gR, np.int32)),
                    W, H, level, d_l, a20, tc3, tg6, _p(out), _p(cen))
    return (out, cen.reshape(H // 5, W // 5, 2)) if want_centres else out


def gmm_density(gmm, o):
    g = _c(gmm, np.float64).reshape(-1, 3)
    return lib().orc_gmm_density(len(g), _p(g), float(o))


def range_table(prior_w, d_l, d_up, gmm, delta, want_post=False):
    prior_w = _c(prior_w, np.int64)
    g = _c(gmm, np.float64).reshape(-1, 3)
    masks = np.empty((d_up + 1) * WORDS, np.uint32)
    post = np.empty((d_up + 1) * (d_l + 1), np.float64) if want_post else None
    lib().orc_range_table(_p(prior_w), d_l, d_up, len(g), _p(g), float(delta), _p(masks), _p(post))
    masks = masks.reshape(d_up + 1, WORDS)
    return (masks, post.reshape(d_up + 1, d_l + 1)) if want_post else masks


def pixel_intervals(W, H, d_up_map, masks):
    d_up_map = _c(d_up_map, np.int32)
    Hu, Wu = d_up_map.shape
    out = np.empty(W * H * WORDS, np.uint32)
    lib().orc_pixel_intervals(W, H, _p(d_up_map), Wu, _p(_c(masks, np.uint32)), _p(out))
    return out.reshape(W * H, WORDS)


def full_set(d_l: int) -> np.ndarray:
    """The 256-bit set {0, ..., d_l}."""
    m = np.zeros(WORDS, np.uint32)
    for j in range(d_l + 1):
        m[j >> 5] |= np.uint32(1) << np.uint32(j & 31)
    return m


def set_from_labels(labels) -> np.ndarray:
    m = np.zeros(WORDS, np.uint32)
    for j in labels:
        m[j >> 5] |= np.uint32(1) << np.uint32(j & 31)
    return m


def labels_of(mask) -> list:
    m = np.asarray(mask, np.uint32)
    return [j for j in range(256) if (int(m[j >> 5]) >> (j & 31)) & 1]


def aggregate_given(order, parent, s, E, want_up=False):
    """Eq. C for a given volume E (N, X), all labels defined; s = per-node similarity to parent."""
    E = _c(E, np.float64)
    N, X = E.shape
    C = np.empty_like(E)
    U = np.empty_like(E) if want_up else None
    rc = lib().orc_aggregate_given(N, X, _p(_c(order, np.int32)), _p(_c(parent, np.int32)), _p(_c(s, np.float64)),
                                   _p(E), _p(C), _p(U))
    if rc:
        raise MemoryError("orc_aggregate_given")
    return (C, U) if want_up else C


def aggregate_adjoint(order, parent, w_node, gamma, E, g):
    """(dL/dE, dL/dw per node, dL/dgamma) of L with dL/dC = g."""
    E = _c(E, np.float64)
    g = _c(g, np.float64)
    N, X = E.shape
    gE = np.empty_like(E)
    gw = np.empty(N, np.float64)
    gg = np.zeros(1, np.float64)
    rc = lib().orc_aggregate_adjoint(N, X, _p(_c(order, np.int32)), _p(_c(parent, np.int32)),
                                     _p(_c(w_node, np.float64)), float(gamma), _p(E), _p(g), _p(gE), _p(gw), _p(gg))
    if rc:
        raise MemoryError("orc_aggregate_adjoint")
    return gE, gw, float(gg[0])


def node_weights(W, H, parent, w_edges, level=0):
    """Weight (real units) of the edge from each node to its parent; 0 for roots."""
    N = W * H
    out = np.zeros(N, np.float64)
    for v in range(N):
        p = parent[v]
        if p < 0:
            continue
        if p == v - 1:
            e = 2 * p
        elif p == v + 1:
            e = 2 * v
        elif p == v - W:
            e = 2 * p + 1
        else:
            e = 2 * v + 1
        out[v] = w_edges[e] / float(4 ** level)
    return out


def soft_argmin(C, T=1.0):
    """d(p) = sum_x x softmax(-C(p, .)/T)(x) per row of C (N, X), FP64."""
    C = np.asarray(C, np.float64)
    z = -(C - C.min(1, keepdims=True)) / T
    e = np.exp(z)
    pr = e / e.sum(1, keepdims=True)
    return (pr * np.arange(C.shape[1])[None, :]).sum(1)


# ------------------------------------------------------------- GMM by EM ---
def gt_down(gt: np.ndarray) -> np.ndarray:
    """Ground truth of the next layer (Sec. 2.2 training data): int32 labels, -1 invalid."""
    gt = _c(gt, np.int32)
    H, W = gt.shape
    up = np.empty(((H + 1) // 2, (W + 1) // 2), np.int32)
    lib().orc_gt_down(_p(gt), W, H, _p(up))
    return up


def offset_hist(up: np.ndarray, lo: np.ndarray, rng: int, hist: np.ndarray = None) -> np.ndarray:
    """Add the offsets o = up(P) - floor(lo(c)/2) of valid pixels to hist[o + rng] (int64, 2 rng + 1 bins)."""
    up = _c(up, np.int32)
    lo = _c(lo, np.int32)
    if hist is None:
        hist = np.zeros(2 * rng + 1, np.int64)
    H, W = lo.shape
    lib().orc_offset_hist(_p(up), up.shape[1], _p(lo), W, H, int(rng), _p(hist))
    return hist


def gmm_em(hist: np.ndarray, rng: int, K: int, iters: int, sd_min: float = 0.5, want_ll: bool = False):
    """EM fit of a K-component GMM to offset histogram data; returns (K, 3) rows of (pi, mu, sd)."""
    hist = _c(hist, np.int64)
    out = np.empty(3 * K, np.float64)
    ll = np.empty(iters + 1, np.float64) if want_ll else None
    if lib().orc_gmm_em(_p(hist), int(rng), int(K), int(iters), float(sd_min), _p(out), _p(ll)):
        raise ValueError("orc_gmm_em: empty histogram or K < 1")
    return (out.reshape(K, 3), ll) if want_ll else out.reshape(K, 3)


# ------------------------------------------------------------- refinement ---
def lr_check(DL: np.ndarray, DR: np.ndarray) -> np.ndarray:
    """refD = D_L where the left-right check passes (D_R(x - D_L, y) = D_L), else -1."""
    DL = _c(DL, np.int32)
    DR = _c(DR, np.int32)
    H, W = DL.shape
    out = np.empty((H, W), np.int32)
    lib().orc_lr_check(_p(DL), _p(DR), W, H, _p(out))
    return out


def refine_aggregate(W, H, level, d_l, order, parent, w, tree_intv, refD, gamma=25.5, want_costs=True):
    """Eq. C for the refinement cost |x - refD(p)| (0 where refD < 0) over the forest; dict like aggregate()."""
    N = W * H
    tint = _c(tree_intv, np.uint32).reshape(N, WORDS)
    k = set_sizes(tint)
    row_off = np.zeros(N + 1, np.int64)
    np.cumsum(k, out=row_off[1:])
    costs = np.empty(int(row_off[-1]), np.float64) if want_costs else None
    wta = np.empty(N, np.int32)
    best = np.empty(N, np.float64)
    second = np.empty(N, np.float64)
    rc = lib().orc_refine_aggregate(W, H, level, d_l, float(gamma), _p(_c(order, np.int32)), _p(_c(parent, np.int32)),
                                    _p(_c(w, np.int64)), _p(tint), _p(_c(refD, np.int32).reshape(-1)), _p(row_off),
                                    _p(costs), _p(wta), _p(best), _p(second))
    if rc:
        raise MemoryError("orc_refine_aggregate")
    return dict(costs=costs, row_off=row_off, wta=wta, best=best, second=second)
