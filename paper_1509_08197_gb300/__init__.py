"""HDP stereo matching on GB300: Python binding of libhdp.so.

The binding only marshals arguments to the C ABI declared in include/hdp.h
(functions of the same names); every step of the method runs in the CUDA
library.  There is no CPU fallback: if libhdp.so cannot be loaded the calls
raise.  Device buffers are passed as torch CUDA tensors (PyTorch provides
device memory and streams only); host buffers as numpy arrays.

    ctx = hdp_create(params)               # params: HDPParams
    hdp_build_trees(ctx, left, right)      # torch.uint8 (H, W, 3) on cuda
    hdp_match(ctx, out)                    # torch.int32 (H, W) on cuda
    hdp_destroy(ctx)
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libhdp.so")

MAX_LEVELS = 8
MAX_GMM = 8

HDP_OK, HDP_ERR_ARG, HDP_ERR_CUDA, HDP_ERR_OOM, HDP_ERR_TIMEOUT, HDP_ERR_STATE = 0, -1, -2, -3, -4, -5
TREE = {"mst": 0, "st": 1, "rt": 2}
MODE = {"hdp": 0, "full": 1}
PRIOR = {"sampled": 0, "uniform": 1}
STORAGE = {"fp32": 0, "fp16": 1}
PREFILTER = {"none": 0, "median3": 1}
STAGE = dict(pyr_left=0, pyr_right=1, weights=2, edges=3, in_tree=4, dt_root=5, tree_intv=6, bfs=7, parent=8,
             depth=9, prior=10, table=11, pix_set=12, costs=13, disp=14, info=15, ref_d=16, disp_r=17)
_STAGE_DTYPE = dict(pyr_left=np.int32, pyr_right=np.int32, weights=np.int32, edges=np.int32, in_tree=np.uint8,
                    dt_root=np.int32, tree_intv=np.uint32, bfs=np.int32, parent=np.int32, depth=np.int32,
                    prior=np.int64, table=np.uint32, pix_set=np.int32, costs=np.float32, disp=np.int32,
                    info=np.int64, ref_d=np.int32, disp_r=np.int32)


class _Params(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int), ("height", ctypes.c_int), ("max_disp", ctypes.c_int),
                ("levels", ctypes.c_int), ("tree", ctypes.c_int), ("mode", ctypes.c_int),
                ("gamma", ctypes.c_float), ("alpha", ctypes.c_float), ("tau_c", ctypes.c_float),
                ("tau_g", ctypes.c_float), ("st_k", ctypes.c_int), ("beta_num", ctypes.c_int),
                ("beta_den", ctypes.c_int), ("delta0", ctypes.c_double), ("prior", ctypes.c_int),
                ("gmm_k", ctypes.c_int * MAX_LEVELS),
                ("gmm", ((ctypes.c_double * 3) * MAX_GMM) * MAX_LEVELS),
                ("storage", ctypes.c_int), ("rt_seed", ctypes.c_uint64), ("prefilter", ctypes.c_int)]


@dataclass
class HDPParams:
    width: int
    height: int
    max_disp: int
    levels: int = 4
    tree: str = "mst"
    mode: str = "hdp"
    gamma: float = 25.5
    alpha: float = 0.9
    tau_c: float = 7.0
    tau_g: float = 2.0
    st_k: int = 1200
    beta: tuple = None            # (num, den); default by image width (Sec. 4.1)
    delta0: float = None
    prior: str = "sampled"
    gmm: list = field(default_factory=list)   # per predicted layer: [[pi, mu, sd], ...] or None
    storage: str = "fp32"
    rt_seed: int = 0              # tree="rt": seed of the random edge order (Sec. 4.1)
    prefilter: str = "none"       # "median3": the M+* variants (Sec. 4.1), tree weights from a 3x3 median

    def to_c(self) -> _Params:
        large = self.width > 640
        beta = self.beta if self.beta is not None else ((95, 100) if large else (3, 5))
        delta0 = self.delta0 if self.delta0 is not None else (0.004 if large else 0.064)
        p = _Params()
        p.width, p.height, p.max_disp, p.levels = self.width, self.height, self.max_disp, self.levels
        p.tree, p.mode = TREE[self.tree], MODE[self.mode]
        p.gamma, p.alpha, p.tau_c, p.tau_g = self.gamma, self.alpha, self.tau_c, self.tau_g
        p.st_k = self.st_k
        p.beta_num, p.beta_den = int(beta[0]), int(beta[1])
        p.delta0 = float(delta0)
        p.prior = PRIOR[self.prior]
        for l, comp in enumerate(self.gmm[:MAX_LEVELS]):
            if comp is None:
                continue
            comp = np.asarray(comp, np.float64).reshape(-1, 3)
            p.gmm_k[l] = len(comp)
            for k, (pi, mu, sd) in enumerate(comp):
                p.gmm[l][k][0], p.gmm[l][k][1], p.gmm[l][k][2] = pi, mu, sd
        p.storage = STORAGE[self.storage]
        p.rt_seed = int(self.rt_seed) & (2 ** 64 - 1)
        p.prefilter = PREFILTER[self.prefilter]
        return p


_lib = None


def load(path: str = LIB_PATH):
    """Load libhdp.so (build it with paper_1509_08197_gb300.build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing (run paper_1509_08197_gb300.build.build())")
    L = ctypes.CDLL(path)
    P, I, I64, SZ = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t
    sigs = {
        "hdp_default_params": (None, [P, I, I, I]),
        "hdp_create": (I, [P, P, P]),
        "hdp_create_own_stream": (I, [P, P]),
        "hdp_get_stream": (P, [P]),
        "hdp_workspace_bytes": (SZ, [P]),
        "hdp_get_tuning": (I, [P, P]),
        "hdp_set_tuning": (I, [P, P]),
        "hdp_autotune": (I, [P, P, P, I, I, P]),
        "hdp_build_trees": (I, [P, P, P, I]),
        "hdp_match": (I, [P, P]),
        "hdp_match_host": (I, [P, P, P, P]),
        "hdp_refine": (I, [P, P, P, I, P]),
        "hdp_run_level": (I, [P, I]),
        "hdp_sync": (I, [P]),
        "hdp_wait_probe": (I, [P, I, ctypes.c_uint]),
        "hdp_destroy": (I, [P]),
        "hdp_last_error": (ctypes.c_char_p, [P]),
        "hdp_stage_bytes": (I64, [P, I, I]),
        "hdp_get_stage": (I, [P, I, I, P, SZ]),
        "hdp_set_stage": (I, [P, I, I, P, SZ]),
        "hdp_set_timing": (I, [P, I]),
        "hdp_get_timings": (I, [P, P, I]),
        "hdp_graph_capture": (I, [P, P, P, I, P, P]),
        "hdp_graph_launch": (I, [P]),
        "hdp_match_noalloc": (I, [P, P, P, I, P, P]),
        "hdp_gt_down": (I, [P, I, I, P, P]),
        "hdp_offset_hist": (I, [P, P, I, I, I, P, P]),
        "hdp_gmm_em": (I, [P, I, I, I, ctypes.c_float, P, P]),
        "hdp_aggregate_fwd": (I, [P, P, P]),
        "hdp_aggregate_bwd": (I, [P, P, P, P, P, P]),
        "hdp_set_gamma": (I, [P, ctypes.c_float]),
        "hdp_soft_argmin_l1": (I, [P, P, P, P, ctypes.c_float, P, P, P]),
        "hdp_cost_volume": (I, [P, ctypes.c_float, ctypes.c_float, ctypes.c_float, P]),
        "hdp_cost_volume_bwd": (I, [P, ctypes.c_float, ctypes.c_float, ctypes.c_float, P, P]),
        "hdp_set_edge_weights": (I, [P, P]),
        "hdp_tree_level": (I, [P]),
        "hdp_match_batch": (I, [P, I, P, P, P, P]),
        "hdp_batch_graph_capture": (I, [P, I, P, P, P, P, P]),
        "hdp_batch_graph_launch": (I, [P]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


class Tuning(ctypes.Structure):
    """hdp_tuning: launch-shape knobs.  The launch knobs give identical results; the layout knobs (tile sizes,
    column or warp kernel) keep every integer stage identical and move aggregated costs within FP32 rounding."""
    _fields_ = [("agg_ctas_per_sm", ctypes.c_int), ("region_ctas_per_sm", ctypes.c_int),
                ("big_class_edges", ctypes.c_int), ("one_cta_nodes", ctypes.c_int),
                ("boruvka_edges_per_cta", ctypes.c_int), ("region_max_nodes", ctypes.c_int),
                ("tile_small_nodes", ctypes.c_int), ("tile_small_nodes_hdp", ctypes.c_int),
                ("col_min_labels", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class HDPError(RuntimeError):
    pass


class Context:
    """An hdp_ctx handle with the parameters and layer sizes it was created for."""

    def __init__(self, handle, params: HDPParams):
        self.handle = handle
        self.params = params
        self.dims = []
        W, H, d = params.width, params.height, params.max_disp
        n = 1 if params.mode == "full" else params.levels
        for _ in range(n):
            self.dims.append((W, H, d))
            W, H, d = (W + 1) // 2, (H + 1) // 2, d // 2

    @property
    def top(self):
        return len(self.dims) - 1


def _check(ctx, rc, what):
    if rc != HDP_OK:
        msg = load().hdp_last_error(ctx.handle if ctx else None)
        raise HDPError(f"{what} failed ({rc}): {msg.decode() if msg else ''}")


def _ptr(t):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
        raise TypeError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _image(t, params):
    """A device image of this problem: contiguous torch.uint8 (height, width, 3) on a CUDA device."""
    import torch
    want = (params.height, params.width, 3)
    if not isinstance(t, torch.Tensor) or t.dtype != torch.uint8 or tuple(t.shape) != want:
        raise TypeError(f"expected a torch.uint8 tensor of shape {want}")
    return _ptr(t)


def _dmap(t, params):
    """A device disparity map of this problem: contiguous torch.int32 (height, width) on a CUDA device."""
    import torch
    want = (params.height, params.width)
    if not isinstance(t, torch.Tensor) or t.dtype != torch.int32 or tuple(t.shape) != want:
        raise TypeError(f"expected a torch.int32 tensor of shape {want}")
    return _ptr(t)


def _stream(stream):
    """The cudaStream_t of `stream`; None means torch's current stream."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def hdp_create(params: HDPParams, stream=None) -> Context:
    """A context bound to `stream` (torch's current stream when None)."""
    L = load()
    h = ctypes.c_void_p()
    s = _stream(stream)
    cp = params.to_c()
    rc = L.hdp_create(ctypes.byref(cp), s, ctypes.byref(h))
    if rc != HDP_OK:
        raise HDPError(f"hdp_create failed ({rc})")
    return Context(h, params)


def hdp_create_own_stream(params: HDPParams) -> Context:
    """A context with its own non-blocking stream (destroyed with it)."""
    L = load()
    h = ctypes.c_void_p()
    cp = params.to_c()
    rc = L.hdp_create_own_stream(ctypes.byref(cp), ctypes.byref(h))
    if rc != HDP_OK:
        raise HDPError(f"hdp_create_own_stream failed ({rc})")
    return Context(h, params)


def hdp_get_stream(ctx: Context):
    """The context's stream as a torch.cuda.ExternalStream (None: the default stream)."""
    import torch
    ptr = load().hdp_get_stream(ctx.handle)
    return torch.cuda.ExternalStream(ptr) if ptr else None


def hdp_get_tuning(ctx: Context) -> Tuning:
    t = Tuning()
    _check(ctx, load().hdp_get_tuning(ctx.handle, ctypes.byref(t)), "hdp_get_tuning")
    return t


def hdp_set_tuning(ctx: Context, t: Tuning):
    _check(ctx, load().hdp_set_tuning(ctx.handle, ctypes.byref(t)), "hdp_set_tuning")


def hdp_autotune(ctx: Context, left, right, reps: int = 2) -> Tuning:
    """Coordinate descent over the launch-shape knobs on this pair (device images)."""
    t = Tuning()
    W = ctx.params.width
    _check(ctx, load().hdp_autotune(ctx.handle, _image(left, ctx.params), _image(right, ctx.params), 3 * W, int(reps),
                                    ctypes.byref(t)),
           "hdp_autotune")
    return t


def hdp_workspace_bytes(ctx: Context) -> int:
    return load().hdp_workspace_bytes(ctx.handle)


def hdp_build_trees(ctx: Context, left, right):
    """left, right: torch.uint8 (H, W, 3) contiguous CUDA tensors."""
    W = ctx.params.width
    _check(ctx, load().hdp_build_trees(ctx.handle, _image(left, ctx.params), _image(right, ctx.params), 3 * W),
           "hdp_build_trees")


def hdp_match(ctx: Context, out):
    """out: torch.int32 (H, W) contiguous CUDA tensor."""
    _check(ctx, load().hdp_match(ctx.handle, _dmap(out, ctx.params)), "hdp_match")


def hdp_refine(ctx: Context, left, right, out):
    """Tree-based refinement at layer 0 (right view by mirroring, left-right check, re-aggregation): the
    refined map into out (torch.int32 (H, W) CUDA tensor); left/right as for hdp_build_trees."""
    W = ctx.params.width
    _check(ctx, load().hdp_refine(ctx.handle, _image(left, ctx.params), _image(right, ctx.params), 3 * W,
                                  _dmap(out, ctx.params)), "hdp_refine")


def hdp_match_host(ctx: Context, left: np.ndarray, right: np.ndarray, out: np.ndarray = None) -> np.ndarray:
    H, W = ctx.params.height, ctx.params.width
    left = np.ascontiguousarray(left, np.uint8)
    right = np.ascontiguousarray(right, np.uint8)
    if left.shape != (H, W, 3) or right.shape != (H, W, 3):
        raise TypeError(f"expected uint8 images of shape {(H, W, 3)}")
    if out is None:
        out = np.empty((H, W), np.int32)
    if out.shape != (H, W) or out.dtype != np.int32 or not out.flags.c_contiguous:
        raise TypeError(f"expected a contiguous int32 output of shape {(H, W)}")
    _check(ctx, load().hdp_match_host(ctx.handle, left.ctypes.data, right.ctypes.data, out.ctypes.data),
           "hdp_match_host")
    return out


def hdp_run_level(ctx: Context, level: int):
    _check(ctx, load().hdp_run_level(ctx.handle, level), "hdp_run_level")


def hdp_sync(ctx: Context):
    _check(ctx, load().hdp_sync(ctx.handle), "hdp_sync")


def hdp_wait_probe(ctx: Context, kind: int, limit: int):
    """Enqueue a bounded device wait made to run out (0: grid barrier, 1: look-back); hdp_sync then raises."""
    _check(ctx, load().hdp_wait_probe(ctx.handle, int(kind), int(limit)), "hdp_wait_probe")


def hdp_destroy(ctx: Context):
    if ctx.handle:
        rc = load().hdp_destroy(ctx.handle)
        ctx.handle = None
        if rc != HDP_OK:
            raise HDPError(f"hdp_destroy reported {rc}")


def hdp_get_stage(ctx: Context, level: int, what: str) -> np.ndarray:
    L = load()
    n = L.hdp_stage_bytes(ctx.handle, level, STAGE[what])
    if n < 0:
        _check(ctx, int(n), f"hdp_stage_bytes({what})")
    dt = np.dtype(_STAGE_DTYPE[what])
    out = np.empty(int(n) // dt.itemsize, dt)
    _check(ctx, L.hdp_get_stage(ctx.handle, level, STAGE[what], out.ctypes.data, int(n)), f"hdp_get_stage({what})")
    W, H, d = ctx.dims[level]
    if what in ("pyr_left", "pyr_right"):
        out = out.reshape(H, W, 4)
    elif what in ("tree_intv", "table"):
        out = out.reshape(-1, 8)
    return out


def hdp_set_stage(ctx: Context, level: int, what: str, arr: np.ndarray):
    dt = np.dtype(_STAGE_DTYPE[what])
    arr = np.ascontiguousarray(arr, dt)
    _check(ctx, load().hdp_set_stage(ctx.handle, level, STAGE[what], arr.ctypes.data, arr.nbytes),
           f"hdp_set_stage({what})")


def hdp_set_timing(ctx: Context, on: bool = True):
    _check(ctx, load().hdp_set_timing(ctx.handle, 1 if on else 0), "hdp_set_timing")


STAGE_NAMES = ("interval prediction", "edges + sort", "forest", "orders + layout", "aggregation + WTA")


def hdp_get_timings(ctx: Context) -> np.ndarray:
    """(levels, 5) device milliseconds of each stage of the last run (timing on)."""
    out = np.zeros(5 * len(ctx.dims), np.float32)
    _check(ctx, load().hdp_get_timings(ctx.handle, out.ctypes.data, out.size), "hdp_get_timings")
    return out.reshape(len(ctx.dims), 5)


def hdp_graph_capture(ctx: Context, left, right, out) -> int:
    """Capture build + match on these device buffers as a CUDA graph; returns its kernel count."""
    n = ctypes.c_int(0)
    _check(ctx, load().hdp_graph_capture(ctx.handle, _image(left, ctx.params), _image(right, ctx.params),
                                         3 * ctx.params.width, _dmap(out, ctx.params), ctypes.byref(n)),
           "hdp_graph_capture")
    return n.value


def hdp_graph_launch(ctx: Context):
    _check(ctx, load().hdp_graph_launch(ctx.handle), "hdp_graph_launch")


NOALLOC_BYTES = 64 << 20


def hdp_match_noalloc(params: HDPParams, left, right, out, stream=None):
    """Match without allocating device memory, for callers that may not
    allocate: the workspace is a fixed 64 MiB array inside libhdp.so (see
    include/hdp.h).  Runs on `stream` (torch's current stream when None) and
    returns when the map is written; raises HDPError with the C status (for
    example HDP_ERR_TIMEOUT when a bounded device wait gave up).  Calls that
    overlap on the GPU race, and the call cannot be graph-captured."""
    cp = params.to_c()
    rc = load().hdp_match_noalloc(ctypes.byref(cp), _image(left, params), _image(right, params), 3 * params.width,
                                  _dmap(out, params), _stream(stream))
    if rc != HDP_OK:
        raise HDPError(f"hdp_match_noalloc failed ({rc})")


def _raw(rc, what):
    if rc != HDP_OK:
        raise HDPError(f"{what} failed ({rc})")


def hdp_gt_down(gt, stream=None):
    """Ground truth of the next layer: gt int32 (H, W) CUDA tensor (-1 invalid) -> int32 (ceil(H/2), ceil(W/2))."""
    import torch
    if not isinstance(gt, torch.Tensor) or gt.dtype != torch.int32 or gt.dim() != 2:
        raise TypeError("expected an int32 (H, W) CUDA tensor")
    H, W = gt.shape
    up = torch.empty(((H + 1) // 2, (W + 1) // 2), dtype=torch.int32, device=gt.device)
    _raw(load().hdp_gt_down(_ptr(gt), W, H, _ptr(up), _stream(stream)), "hdp_gt_down")
    return up


def hdp_offset_hist(up, lo, rng: int, hist, stream=None):
    """Add the offsets up(P) - floor(lo(c)/2) of lo's valid pixels to hist (int64 (2 rng + 1,) CUDA tensor)."""
    import torch
    H, W = lo.shape
    if lo.dtype != torch.int32 or up.dtype != torch.int32 or tuple(up.shape) != ((H + 1) // 2, (W + 1) // 2):
        raise TypeError("expected int32 maps, up of shape (ceil(H/2), ceil(W/2))")
    if hist.dtype != torch.int64 or hist.numel() != 2 * rng + 1:
        raise TypeError("expected an int64 histogram of 2 * range + 1 bins")
    _raw(load().hdp_offset_hist(_ptr(up), _ptr(lo), W, H, int(rng), _ptr(hist), _stream(stream)), "hdp_offset_hist")


def hdp_gmm_em(hist, rng: int, K: int, iters: int, sd_min: float = 0.5, out=None, stream=None):
    """EM fit of K components to the histogram on the GPU; returns the float32 (K, 3) CUDA tensor (pi, mu, sd)."""
    import torch
    if out is None:
        out = torch.empty((K, 3), dtype=torch.float32, device=hist.device)
    _raw(load().hdp_gmm_em(_ptr(hist), int(rng), int(K), int(iters), float(sd_min), _ptr(out), _stream(stream)),
         "hdp_gmm_em")
    return out


def fit_gmm(gt_maps, max_disp: int, levels: int, K: int = 2, iters: int = 200, sd_min: float = 0.5, device=None):
    """GMM_l of every predicted layer (l = 0 .. levels-2) fitted by EM on ground-truth maps (Sec. 2.2).

    gt_maps: int32 (H, W) numpy label maps (-1 invalid) at layer 0, one per training pair, all of range
    0..max_disp.  Every step runs in the CUDA library; returns the per-layer [[pi, mu, sd], ...] lists
    for HDPParams.gmm."""
    import torch
    dev = device or torch.device("cuda", torch.cuda.current_device())
    d = [max_disp]
    for _ in range(levels - 1):
        d.append(d[-1] // 2)
    hists = [torch.zeros(2 * d[l + 1] + 1, dtype=torch.int64, device=dev) for l in range(levels - 1)]
    for g in gt_maps:
        lo = torch.from_numpy(np.ascontiguousarray(g, np.int32)).to(dev)
        for l in range(levels - 1):
            up = hdp_gt_down(lo)
            hdp_offset_hist(up, lo, d[l + 1], hists[l])
            lo = up
    return [hdp_gmm_em(hists[l], d[l + 1], K, iters, sd_min).cpu().numpy().astype(np.float64).tolist()
            for l in range(levels - 1)]


def _optr(t):
    return None if t is None else _ptr(t)


def hdp_tree_level(ctx: Context) -> int:
    """The layer whose forest and layout are loaded, or -1 before hdp_build_trees."""
    return int(load().hdp_tree_level(ctx.handle))


def _loaded(ctx: Context):
    """(N, X) of the loaded layer: pixels and labels of its volumes."""
    l = hdp_tree_level(ctx)
    if l < 0:
        raise HDPError("no tree loaded (call hdp_build_trees)")
    W, H, d = ctx.dims[l]
    return W * H, d + 1


def _f32n(t, n, what):
    """A float32 CUDA tensor of exactly n elements (the kernels index n of them)."""
    p = _f32(t)
    if t.numel() != n:
        raise TypeError(f"{what}: expected {n} float32 elements, got {t.numel()}")
    return p


def _u8n(t, n, what):
    import torch
    if not isinstance(t, torch.Tensor) or t.dtype != torch.uint8 or t.numel() != n:
        raise TypeError(f"{what}: expected a uint8 CUDA tensor of {n} elements")
    return _ptr(t)


def hdp_aggregate_fwd(ctx: Context, E, C):
    """C = A E over the loaded full-range tree; E, C: float32 (H, W, X) CUDA tensors."""
    N, X = _loaded(ctx)
    _check(ctx, load().hdp_aggregate_fwd(ctx.handle, _f32n(E, N * X, "E"), _f32n(C, N * X, "C")),
           "hdp_aggregate_fwd")


def hdp_aggregate_bwd(ctx: Context, E, gC, gE, gw, ggamma):
    """dL/dE (H, W, X), dL/dw per grid edge id (2*H*W,), dL/dgamma (1,) from dL/dC."""
    N, X = _loaded(ctx)
    _check(ctx, load().hdp_aggregate_bwd(ctx.handle, _f32n(E, N * X, "E"), _f32n(gC, N * X, "gC"),
                                         _f32n(gE, N * X, "gE"), _f32n(gw, 2 * N, "gw"), _f32n(ggamma, 1, "ggamma")),
           "hdp_aggregate_bwd")


def hdp_set_gamma(ctx: Context, gamma: float):
    _check(ctx, load().hdp_set_gamma(ctx.handle, float(gamma)), "hdp_set_gamma")


def hdp_soft_argmin_l1(ctx: Context, C, gt=None, valid=None, T=1.0, disp=None, loss=None, gC=None):
    N, X = _loaded(ctx)
    _check(ctx, load().hdp_soft_argmin_l1(ctx.handle, _f32n(C, N * X, "C"), None if gt is None else _f32n(gt, N, "gt"),
                                          None if valid is None else _u8n(valid, N, "valid"), float(T),
                                          None if disp is None else _f32n(disp, N, "disp"),
                                          None if loss is None else _f32n(loss, 1, "loss"),
                                          None if gC is None else _f32n(gC, N * X, "gC")), "hdp_soft_argmin_l1")


def _f32(t):
    import torch
    if not isinstance(t, torch.Tensor) or t.dtype != torch.float32:
        raise TypeError("expected a float32 CUDA tensor")
    return _ptr(t)


def hdp_cost_volume(ctx: Context, alpha: float, tau_c: float, tau_g: float, E):
    """E (H, W, X) float32 CUDA tensor <- the matching cost with real-valued parameters."""
    N, X = _loaded(ctx)
    _check(ctx, load().hdp_cost_volume(ctx.handle, float(alpha), float(tau_c), float(tau_g), _f32n(E, N * X, "E")),
           "hdp_cost_volume")


def hdp_cost_volume_bwd(ctx: Context, alpha: float, tau_c: float, tau_g: float, gE, gparams):
    """gparams (3,) float32 CUDA tensor <- dL/d(alpha, tau_c, tau_g) from gE = dL/dE."""
    N, X = _loaded(ctx)
    _check(ctx, load().hdp_cost_volume_bwd(ctx.handle, float(alpha), float(tau_c), float(tau_g),
                                           _f32n(gE, N * X, "gE"), _f32n(gparams, 3, "gparams")),
           "hdp_cost_volume_bwd")


def hdp_set_edge_weights(ctx: Context, w=None):
    """Real-valued weights per grid edge id (float32 CUDA tensor of 2*H*W) for the loaded tree, or None for the
    image's own."""
    N, _ = _loaded(ctx)
    _check(ctx, load().hdp_set_edge_weights(ctx.handle, None if w is None else _f32n(w, 2 * N, "w")),
           "hdp_set_edge_weights")


def _batch_arrays(ctxs, lefts, rights, outs):
    n = len(ctxs)
    H = (ctypes.c_void_p * n)(*[c.handle for c in ctxs])
    if not (len(lefts) == len(rights) == len(outs) == n):
        raise TypeError("one left image, right image and output per context")
    L = (ctypes.c_void_p * n)(*[_image(t, c.params).value for t, c in zip(lefts, ctxs)])
    R = (ctypes.c_void_p * n)(*[_image(t, c.params).value for t, c in zip(rights, ctxs)])
    Pt = (ctypes.c_int * n)(*[3 * c.params.width for c in ctxs])
    O = (ctypes.c_void_p * n)(*[_dmap(t, c.params).value for t, c in zip(outs, ctxs)])
    return n, H, L, R, Pt, O


def hdp_match_batch(ctxs, lefts, rights, outs):
    """Match len(ctxs) pairs concurrently (each context on its own stream)."""
    n, H, L, R, Pt, O = _batch_arrays(ctxs, lefts, rights, outs)
    _check(ctxs[0], load().hdp_match_batch(H, n, L, R, Pt, O), "hdp_match_batch")


def hdp_batch_graph_capture(ctxs, lefts, rights, outs) -> int:
    n, H, L, R, Pt, O = _batch_arrays(ctxs, lefts, rights, outs)
    k = ctypes.c_int(0)
    _check(ctxs[0], load().hdp_batch_graph_capture(H, n, L, R, Pt, O, ctypes.byref(k)), "hdp_batch_graph_capture")
    return k.value


def hdp_batch_graph_launch(ctx0):
    _check(ctx0, load().hdp_batch_graph_launch(ctx0.handle), "hdp_batch_graph_launch")


def exported_symbols():
    """Names declared in include/hdp.h (for the load/export check)."""
    return ["hdp_default_params", "hdp_create", "hdp_create_own_stream", "hdp_get_stream", "hdp_get_tuning",
            "hdp_set_tuning", "hdp_autotune", "hdp_workspace_bytes", "hdp_build_trees", "hdp_match",
            "hdp_match_host", "hdp_run_level", "hdp_sync", "hdp_wait_probe", "hdp_destroy", "hdp_last_error", "hdp_stage_bytes",
            "hdp_get_stage", "hdp_set_stage", "hdp_set_timing", "hdp_get_timings", "hdp_graph_capture",
            "hdp_graph_launch", "hdp_match_noalloc", "hdp_aggregate_fwd", "hdp_aggregate_bwd", "hdp_set_gamma",
            "hdp_soft_argmin_l1", "hdp_match_batch", "hdp_batch_graph_capture", "hdp_batch_graph_launch",
            "hdp_gt_down", "hdp_offset_hist", "hdp_gmm_em", "hdp_refine", "hdp_cost_volume", "hdp_cost_volume_bwd",
            "hdp_set_edge_weights", "hdp_tree_level"]
