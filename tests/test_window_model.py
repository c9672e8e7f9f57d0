"""CPU model of the segment-tree first pass by windows, against the oracle.

The GPU resolves a window of the strict (w, id) order class by class when it
holds few weight classes: at the start of class w a tree whose criterion
(w - Int) * |C| > k fails is frozen (its state cannot change without a
merge, and every later edge is at least as heavy), and the class is the
minimum spanning forest by index among the other trees (a merge sets Int = w,
which passes for the rest of the class), built by Boruvka rounds.  Windows
with many classes are resolved in sequential order.  This test replays that
decomposition on random grids with few weight classes and checks that the
forest equals the oracle's sequential Kruskal (Sec. 3.2, ST criterion), so
the argument the kernel relies on is pinned independently of the kernel.
"""
import numpy as np
import pytest

import oracle


def _find(par, v):
    while par[v] != v:
        par[v] = par[par[v]]
        v = par[v]
    return v


def _ends(e, W):
    p = e >> 1
    return p, (p + W if e & 1 else p + 1)


def _class_boruvka(edges, w, W, par, size, intw, kq, in_tree):
    """One weight class: freeze the failing trees, then Boruvka by index."""
    frozen = set()
    for e in edges:
        for r in (_find(par, v) for v in _ends(e, W)):
            if (w - intw[r]) * size[r] > kq:
                frozen.add(r)
    live = list(edges)
    while True:
        best = {}
        nxt = []
        for e in live:
            a, b = (_find(par, v) for v in _ends(e, W))
            if a == b or a in frozen or b in frozen:
                continue
            nxt.append((e, a, b))
            best[a] = min(best.get(a, e), e)
            best[b] = min(best.get(b, e), e)
        if not nxt:
            return
        hooked = []
        for e, a, b in nxt:
            ha, hb = best[a] == e, best[b] == e
            if not (ha or hb):
                continue
            in_tree[e] = 1
            if ha and hb:
                r, to = max(a, b), min(a, b)
            elif ha:
                r, to = a, b
            else:
                r, to = b, a
            par[r] = to
            hooked.append(r)
        pre = {r: size[r] for r in hooked}
        for r in hooked:
            R = _find(par, r)
            size[R] += pre[r]
            intw[R] = w
        live = [e for e, _, _ in nxt if not in_tree[e]]


def _sequential(edges, wts, W, par, size, intw, kq, in_tree, crit):
    for e in edges:
        a, b = (_find(par, v) for v in _ends(e, W))
        if a == b:
            continue
        w = wts[e]
        if crit and ((w - intw[a]) * size[a] > kq or (w - intw[b]) * size[b] > kq):
            continue
        if size[a] < size[b]:
            a, b = b, a
        par[b] = a
        size[a] += size[b]
        intw[a] = w
        in_tree[e] = 1


def _dr_window(win, wts, W, par, size, intw, kq, in_tree, switch_below):
    """Reservation rounds as the kernel runs them (the earliest pending edge of
    a tree holds its reservation; an edge holding both is decided on the
    current state; a tree failing the criterion there is frozen), then, once a
    round resolves fewer than switch_below edges, the rest in window order."""
    w0 = min(int(wts[e]) for e in win)
    frozen = set()
    for e in win:
        for r in (_find(par, v) for v in _ends(e, W)):
            if (w0 - intw[r]) * size[r] > kq:
                frozen.add(r)
    pos = {e: i for i, e in enumerate(win)}   # reservations go by window position (the strict order)
    live = list(win)
    rnd = 0
    while live:
        roots, best = {}, {}
        for e in live:
            a, b = (_find(par, v) for v in _ends(e, W))
            if a == b or a in frozen or b in frozen:
                continue
            roots[e] = (a, b)
            best[a] = min(best.get(a, pos[e]), pos[e])
            best[b] = min(best.get(b, pos[e]), pos[e])
        done = set(e for e in live if e not in roots)
        resolved = 0
        for e, (a, b) in roots.items():
            ha, hb = best[a] == pos[e], best[b] == pos[e]
            if not (ha or hb):
                continue
            w = int(wts[e])
            fa = ha and (w - intw[a]) * size[a] > kq
            fb = hb and (w - intw[b]) * size[b] > kq
            if fa or fb:
                if fa:
                    frozen.add(a)
                if fb:
                    frozen.add(b)
                done.add(e)
                resolved += 1
                continue
            if not (ha and hb):
                continue
            if size[a] < size[b]:
                a, b = b, a
            par[b] = a
            size[a] += size[b]
            intw[a] = w
            in_tree[e] = 1
            done.add(e)
            resolved += 1
        live = [e for e in live if e not in done]
        if live and rnd >= 1 and resolved < switch_below:
            _sequential(live, wts, W, par, size, intw, kq, in_tree, crit=True)
            return
        rnd += 1


def _model_forest(W, H, order, wts, kq, window, max_classes, switch_below=0):
    N = W * H
    par = list(range(N))
    size = [1] * N
    intw = [0] * N
    in_tree = np.zeros(2 * N, np.uint8)
    for s in range(0, len(order), window):
        win = [int(e) for e in order[s:s + window]]
        ws = [int(wts[e]) for e in win]
        if len(set(ws)) <= max_classes:
            for w in sorted(set(ws)):
                _class_boruvka([e for e in win if wts[e] == w], w, W, par, size, intw, kq, in_tree)
        elif switch_below:
            _dr_window(win, wts, W, par, size, intw, kq, in_tree, switch_below)
        else:
            _sequential(win, wts, W, par, size, intw, kq, in_tree, crit=True)
    _sequential([int(e) for e in order], wts, W, par, size, intw, kq, in_tree, crit=False)   # linking pass
    return in_tree


@pytest.mark.parametrize("seed", range(6))
def test_class_by_class_windows_equal_sequential_kruskal(seed):
    # 8 weight classes (0, 3, ..., 21), so that a window of 8..32 edges holds
    # one to four of them; without the freeze at each class start this model
    # disagrees with the oracle in about half of these cases
    rng = np.random.default_rng(seed)
    W, H = int(rng.integers(14, 24)), int(rng.integers(10, 18))
    img = (rng.integers(0, 8, size=(H, W, 3)) * 3).astype(np.int32)
    wts = oracle.edge_weights(img)
    order = oracle.sort_edges(wts, W, H)
    pix = np.tile(oracle.full_set(3), (W * H, 1))
    for k in (2, 6, 20, 60):
        want, _, _ = oracle.build_forest(W, H, order, wts, pix, tree="st", st_k=k, level=0)
        for window, max_classes in ((8, 2), (16, 3), (32, 4), (len(order), 64)):
            got = _model_forest(W, H, order, wts, k, window, max_classes)
            assert np.array_equal(got, want), (seed, k, window)


@pytest.mark.parametrize("seed", range(6))
def test_reservation_rounds_with_sequential_finish_equal_sequential_kruskal(seed):
    # windows of many weight classes: reservation rounds, then the rest of the
    # window in order once a round resolves few edges (the sequential finish)
    rng = np.random.default_rng(100 + seed)
    W, H = int(rng.integers(14, 24)), int(rng.integers(10, 18))
    img = rng.integers(0, 64, size=(H, W, 3)).astype(np.int32)
    wts = oracle.edge_weights(img)
    order = oracle.sort_edges(wts, W, H)
    pix = np.tile(oracle.full_set(3), (W * H, 1))
    for k in (3, 30, 300):
        want, _, _ = oracle.build_forest(W, H, order, wts, pix, tree="st", st_k=k, level=0)
        for window, switch_below in ((16, 1), (32, 2), (64, 4), (len(order), 8)):
            got = _model_forest(W, H, order, wts, k, window, max_classes=0, switch_below=switch_below)
            assert np.array_equal(got, want), (seed, k, window, switch_below)
