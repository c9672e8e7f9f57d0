"""Seeded synthetic rectified stereo pairs.

This module only produces inputs; it holds none of the matching method's
arithmetic, so both the CUDA path and the CPU oracle can be fed from it.

A scene is a Voronoi partition of the left image into planar disparity
regions d(x, y) = a + bx*x + by*y.  Each region is painted with a base colour
plus multi-octave value noise (amplitude 0 for "textureless" regions).  The
right image is forward-warped from the left one with a z-buffer (the larger
disparity wins); holes are filled from the background neighbour on the same
row and the losing left pixels are marked occluded.  Gaussian noise is added
to both views, which are then clamped and rounded to uint8.

The workloads the paper evaluates on (Middlebury 2006 third/half/full size,
KITTI 1242x375, a 640x480 web-camera set) are not available; these scenes
mimic only their sizes and disparity ranges.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class StereoPair:
    left: np.ndarray        # (H, W, 3) uint8
    right: np.ndarray       # (H, W, 3) uint8
    gt: np.ndarray          # (H, W) float32 ground-truth disparity of the left view
    occluded: np.ndarray    # (H, W) bool, left pixels hidden in the right view
    max_disp: int


def _value_noise(rng, H, W, octaves, base_cell):
    """Sum of bilinearly interpolated random lattices, one per octave, in [-1, 1]."""
    out = np.zeros((H, W), np.float64)
    amp, total = 1.0, 0.0
    cell = float(base_cell)
    ys = np.arange(H, dtype=np.float64)
    xs = np.arange(W, dtype=np.float64)
    for _ in range(max(octaves, 1)):
        gh = int(np.ceil(H / cell)) + 2
        gw = int(np.ceil(W / cell)) + 2
        lat = rng.uniform(-1.0, 1.0, size=(gh, gw))
        fy = ys / cell
        fx = xs / cell
        y0 = np.floor(fy).astype(np.int64)
        x0 = np.floor(fx).astype(np.int64)
        ty = (fy - y0)[:, None]
        tx = (fx - x0)[None, :]
        a = lat[y0][:, x0]
        b = lat[y0][:, x0 + 1]
        c = lat[y0 + 1][:, x0]
        d = lat[y0 + 1][:, x0 + 1]
        out += amp * ((a * (1 - tx) + b * tx) * (1 - ty) + (c * (1 - tx) + d * tx) * ty)
        total += amp
        amp *= 0.5
        cell = max(cell / 2.0, 1.0)
    return out / total


def _voronoi_labels(rng, H, W, regions):
    sx = rng.uniform(0, W, size=regions)
    sy = rng.uniform(0, H, size=regions)
    labels = np.empty((H, W), np.int32)
    xs = np.arange(W, dtype=np.float64)[None, :, None]
    step = max(1, 4_000_000 // max(1, W * regions))
    for y0 in range(0, H, step):
        ys = np.arange(y0, min(H, y0 + step), dtype=np.float64)[:, None, None]
        d2 = (xs - sx[None, None, :]) ** 2 + (ys - sy[None, None, :]) ** 2
        labels[y0:y0 + ys.shape[0]] = np.argmin(d2, axis=2)
    return labels


def make_pair(seed: int, width: int, height: int, max_disp: int, regions: int = 12,
              octaves: int = 2, textureless_frac: float = 0.0, noise_sigma: float = 2.0,
              similar_colour_frac: float = 0.0, texture_amp: float = 40.0,
              texture_cell: float = 8.0) -> StereoPair:
    """Build one seeded stereo pair.

    similar_colour_frac: fraction of regions that copy the base colour of a
    neighbouring region while keeping their own disparity plane (large
    similar-colour areas with varying depth).
    """
    rng = np.random.default_rng(seed)
    H, W, d = int(height), int(width), int(max_disp)
    labels = _voronoi_labels(rng, H, W, regions)

    a = rng.uniform(0.1 * d, 0.9 * d, size=regions)
    bx = rng.uniform(-0.3 * d / W, 0.3 * d / W, size=regions)
    by = rng.uniform(-0.3 * d / W, 0.3 * d / W, size=regions)
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    cx = xx.mean()
    cy = yy.mean()
    gt = a[labels] + bx[labels] * (xx - cx) + by[labels] * (yy - cy)
    gt = np.clip(gt, 0.0, float(d))

    base = rng.uniform(30.0, 225.0, size=(regions, 3))
    if similar_colour_frac > 0 and regions > 1:
        n_copy = int(round(similar_colour_frac * regions))
        # region adjacency from the label map, so a copied colour sits next to its source
        right_pairs = np.stack([labels[:, :-1].ravel(), labels[:, 1:].ravel()], 1)
        down_pairs = np.stack([labels[:-1, :].ravel(), labels[1:, :].ravel()], 1)
        pairs = np.concatenate([right_pairs, down_pairs])
        pairs = pairs[pairs[:, 0] != pairs[:, 1]]
        pairs = np.unique(pairs, axis=0)
        victims = rng.permutation(regions)[:n_copy]
        for v in victims:
            nb = pairs[pairs[:, 0] == v, 1]
            if nb.size:
                base[v] = base[rng.choice(nb)]
    amp = np.full(regions, texture_amp)
    if textureless_frac > 0:
        n_flat = int(round(textureless_frac * regions))
        amp[rng.permutation(regions)[:n_flat]] = 0.0

    noise = np.stack([_value_noise(rng, H, W, octaves, texture_cell) for _ in range(3)], -1)
    left_f = base[labels] + amp[labels][..., None] * noise
    left_f = np.clip(left_f, 0.0, 255.0)

    # forward warp with a z-buffer: target column x - round(d); larger disparity wins
    di = np.rint(gt).astype(np.int64)
    tx = xx.astype(np.int64) - di
    valid = tx >= 0
    src = np.flatnonzero(valid.ravel())
    tgt = (yy.astype(np.int64) * W + tx).ravel()[src]
    key = di.ravel()[src] * (H * W) + src          # disparity first, then source index
    zbuf = np.full(H * W, -1, np.int64)
    np.maximum.at(zbuf, tgt, key)
    hit = zbuf >= 0
    winner = np.where(hit, zbuf % (H * W), -1)
    right_f = np.zeros((H * W, 3), np.float64)
    right_f[hit] = left_f.reshape(-1, 3)[winner[hit]]
    wdisp = np.full(H * W, np.inf)
    wdisp[hit] = di.ravel()[winner[hit]]

    occluded = np.ones(H * W, bool)
    occluded[winner[hit]] = False
    occluded = occluded.reshape(H, W)

    # hole filling: take the nearer-to-background (smaller disparity) of the nearest
    # valid neighbours on the same row
    right_f = right_f.reshape(H, W, 3)
    hitm = hit.reshape(H, W)
    wdisp = wdisp.reshape(H, W)
    idx = np.where(hitm, np.arange(W)[None, :], -1)
    left_nb = np.maximum.accumulate(idx, axis=1)
    idx_r = np.where(hitm, np.arange(W)[None, :], W)
    right_nb = np.minimum.accumulate(idx_r[:, ::-1], axis=1)[:, ::-1]
    rows = np.arange(H)[:, None].repeat(W, 1)
    ln_ok = left_nb >= 0
    rn_ok = right_nb < W
    ld = np.where(ln_ok, wdisp[rows, np.clip(left_nb, 0, W - 1)], np.inf)
    rd = np.where(rn_ok, wdisp[rows, np.clip(right_nb, 0, W - 1)], np.inf)
    use_left = ld <= rd
    fill_col = np.where(use_left, left_nb, right_nb)
    fill_ok = ~hitm & (ln_ok | rn_ok)
    fc = np.clip(fill_col, 0, W - 1)
    right_f[fill_ok] = right_f[rows[fill_ok], fc[fill_ok]]
    right_f[~hitm & ~(ln_ok | rn_ok)] = left_f[~hitm & ~(ln_ok | rn_ok)]

    left = np.clip(np.rint(left_f + rng.normal(0, noise_sigma, left_f.shape)), 0, 255).astype(np.uint8)
    right = np.clip(np.rint(right_f + rng.normal(0, noise_sigma, right_f.shape)), 0, 255).astype(np.uint8)
    return StereoPair(left=left, right=right, gt=gt.astype(np.float32), occluded=occluded, max_disp=d)


# Workload recipes: sizes, ranges and scene statistics of the evaluated setups.
WORKLOADS = {
    # 96x72, range 0-15, 2 layers, MST
    "tiny": dict(width=96, height=72, max_disp=15, regions=12, octaves=2),
    # Middlebury-2006-third-size-like: 463x370, range 0-79, 4 layers
    "third": dict(width=463, height=370, max_disp=79, regions=40, octaves=4, textureless_frac=0.05),
    # Middlebury-2006-full-size-like: 1390x1110, range 0-255, 5 layers
    "full": dict(width=1390, height=1110, max_disp=255, regions=120, octaves=4,
                 textureless_frac=0.05, similar_colour_frac=0.3),
    # differentiable-aggregation crops: 256x256, range 0-63
    "grad": dict(width=256, height=256, max_disp=63, regions=16, octaves=3),
}


def workload_pair(name: str, index: int = 0, **over) -> StereoPair:
    """Seeded pair for a named workload recipe; seed = recipe index * 1000 + pair index."""
    order = list(WORKLOADS)
    kw = dict(WORKLOADS[name])
    kw.update(over)
    return make_pair(seed=(order.index(name) + 1) * 1000 + index, **kw)


def integer_gt(pair: StereoPair) -> np.ndarray:
    """The pair's ground truth as integer labels: floor(gt + 1/2) clipped to
    0..max_disp, -1 at occluded pixels (int32, (H, W))."""
    d = np.clip(np.floor(pair.gt.astype(np.float64) + 0.5), 0, pair.max_disp).astype(np.int32)
    d[pair.occluded] = -1
    return d


def training_pairs(name: str, count: int, first_index: int = 100):
    """Seeded training scenes of a recipe (pair indices first_index.., disjoint from the evaluated pairs)."""
    return [workload_pair(name, index=first_index + i) for i in range(count)]
