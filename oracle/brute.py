"""Brute-force checkers for tiny inputs, used to pin the C oracle.

TEST INFRASTRUCTURE ONLY.  Each function restates a definition from the
paper directly (no union-find, no two-pass recurrences), in plain Python or
numpy, so that an error in the oracle's faster formulation shows up as a
mismatch.
"""
from __future__ import annotations

import heapq
import itertools
from collections import deque

import numpy as np


def grid_edges(W, H):
    """All valid edge ids of the 4-connected W x H grid with their end points."""
    out = []
    for y in range(H):
        for x in range(W):
            p = y * W + x
            if x + 1 < W:
                out.append((2 * p, p, p + 1))
            if y + 1 < H:
                out.append((2 * p + 1, p, p + W))
    return out


def prim_total_weight(W, H, w):
    """Prim's algorithm (a different MST algorithm from Kruskal) on the grid; returns the total weight."""
    N = W * H
    adj = [[] for _ in range(N)]
    for e, p, q in grid_edges(W, H):
        adj[p].append((int(w[e]), e, q))
        adj[q].append((int(w[e]), e, p))
    seen = np.zeros(N, bool)
    total = 0
    for s in range(N):
        if seen[s]:
            continue
        seen[s] = True
        heap = list(adj[s])
        heapq.heapify(heap)
        while heap:
            wt, e, v = heapq.heappop(heap)
            if seen[v]:
                continue
            seen[v] = True
            total += wt
            for item in adj[v]:
                if not seen[item[2]]:
                    heapq.heappush(heap, item)
    return total


def brute_spanning_tree(W, H, w):
    """Exhaustive search over edge subsets for the spanning tree minimising the
    total of (w * BIG + e): the unique MST under the strict (w, id) order."""
    edges = grid_edges(W, H)
    N = W * H
    big = 4 * len(edges) * 2 * N
    best, best_set = None, None
    for subset in itertools.combinations(range(len(edges)), N - 1):
        parent = list(range(N))

        def f(v):
            while parent[v] != v:
                v = parent[v]
            return v
        ok = True
        for i in subset:
            _, p, q = edges[i]
            a, b = f(p), f(q)
            if a == b:
                ok = False
                break
            parent[a] = b
        if not ok:
            continue
        cost = sum(int(w[edges[i][0]]) * big + edges[i][0] for i in subset)
        if best is None or cost < best:
            best, best_set = cost, {edges[i][0] for i in subset}
    return best_set


def naive_forest(W, H, order, w, pix_sets, beta, tree="mst", k=0):
    """Replay of the HDP forest rules (Sec. 3.2) with explicit component labels.

    Components are label arrays relabelled on every merge; TreeIntv, |C| and
    Int(C) are recomputed from the member pixels and accepted edges each time
    they are needed, instead of being carried along as in the oracle."""
    N = W * H
    label = np.arange(N)
    sets = [frozenset(s) for s in pix_sets]
    accepted = set()
    acc_w = {}   # edge -> weight for accepted edges

    def members(c):
        return np.flatnonzero(label == c)

    def tree_set(c):
        out = set()
        for v in members(c):
            out |= sets[v]
        return out

    def int_c(c):
        m = set(members(c).tolist())
        ws = [acc_w[e] for e in accepted if (e >> 1) in m]
        return max(ws) if ws else 0

    passes = 2 if tree == "st" else 1
    for ps in range(passes):
        for e in order:
            p = e >> 1
            q = p + W if e & 1 else p + 1
            if not (sets[p] & sets[q]):
                continue
            a, b = label[p], label[q]
            if a == b:
                continue
            Ta, Tb = tree_set(a), tree_set(b)
            if len(Ta & Tb) * beta[1] < beta[0] * len(Ta | Tb):
                continue
            if tree == "st" and ps == 0:
                wa, wb = int(w[e]), int(w[e])
                na, nb = len(members(a)), len(members(b))
                if wa * na > int_c(a) * na + k or wb * nb > int_c(b) * nb + k:
                    continue
            label[label == b] = a
            accepted.add(e)
            acc_w[e] = int(w[e])
    return accepted


def tree_adjacency(W, H, in_tree):
    N = W * H
    adj = [[] for _ in range(N)]
    for e, p, q in grid_edges(W, H):
        if in_tree[e]:
            adj[p].append((q, e))
            adj[q].append((p, e))
    return adj


def brute_aggregate(W, H, in_tree, w_real, E, gamma):
    """Eq. (C) evaluated directly: C(p, x) = sum over q in DT(p) of
    exp(-W(p, q)/gamma) E(q, x), with W the sum of edge weights on the tree path
    (Eq. W), found by a breadth-first walk from every p.  E: (N, X) array with
    NaN where undefined; returns (N, X)."""
    N = W * H
    adj = tree_adjacency(W, H, in_tree)
    C = np.full_like(E, np.nan, dtype=np.float64)
    for p in range(N):
        dist = {p: 0.0}
        dq = deque([p])
        while dq:
            v = dq.popleft()
            for u, e in adj[v]:
                if u not in dist:
                    dist[u] = dist[v] + float(w_real[e])
                    dq.append(u)
        defined = ~np.isnan(E[p])
        acc = np.zeros(E.shape[1])
        for q, d in dist.items():
            acc[defined] += np.exp(-d / gamma) * E[q, defined]
        C[p, defined] = acc[defined]
    return C
