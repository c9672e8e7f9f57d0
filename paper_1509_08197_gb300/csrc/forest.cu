// HDP forest construction (Sec. 3.2): Kruskal semantics over the strict
// (w, edge id) order with Rule 2, DT-Rule 2 (Eq. DTrules) and, for the
// segment tree, the merge criterion w <= Int(C) + k/|C|.
//
// Five engines produce the sequential-Kruskal result exactly:
//  * Boruvka over the sorted list (the list index is the strict order) when
//    no state-dependent rule is active: plain MST, full-range layers, the
//    segment tree's linking pass, and HDP layers with no "risky" edge.
//    Without risky edges every tree keeps the set of its pixels (merges only
//    join equal sets), so DT-Rule 2 reduces to "same PixelIntv" and the result
//    is the minimum spanning forest of the same-set subgraph.
//  * Windows in shared memory (segment-tree first pass of the top layer):
//    windows of consecutive edges whose trees are copied into shared memory.
//    A window of few weight classes goes class by class: inside a class a
//    tree's criterion cannot change before it merges, and a merge sets
//    Int = w, which passes for the rest of the class, so a class is the
//    minimum spanning forest by index among its passing trees (Boruvka in
//    shared memory).  Other windows use deterministic reservations, and one
//    warp finishes them sequentially once the rounds stall.  A tree whose
//    criterion fails at its earliest pending edge is frozen for good.
//  * Regions (segment-tree first pass of predicted layers without risky
//    edges): connected same-set regions are independent, so persistent CTAs
//    take whole regions (small ones packed together) window by window.  On a
//    risky layer the regions are the connected components of the edges that
//    survive DT-Rule 1 (no edge joins two of them), and every pass runs there
//    with the windows of the risky engine below.
//  * Hybrid first pass (big full-range layers): a weight class with many
//    edges is a Boruvka by edge id over the whole grid, for the same reason;
//    runs of small classes form windows resolved as above.
//  * Windows for risky HDP layers (an edge between different sets whose
//    Jaccard ratio reaches beta, so DT-Rule 2 may join different sets and
//    same-set regions are not independent): every pass over the whole list
//    (or over each component, above) in one CTA, window by window, by
//    deterministic reservations in shared memory, with each local tree's
//    TreeIntv there too.  An edge that holds the
//    reservation of both its trees is decided on their current state,
//    exactly as the sequential algorithm decides it.
#include "hdp_impl.cuh"

#define FOREST_THREADS 512

int edge_bits(int N)
{
    int b = 1;
    while ((1LL << b) < 2LL * N) ++b;
    return b;
}

struct ForestArgs {
    const uint32_t* keys;
    const int* d_n;
    int ebits, W, N;
    const int* pixset;   // null: every set is the full range
    const int* canon;
    const uint32_t* table;
    const uint32_t* full_mask;
    int* parent;
    int* size;
    int* intw;
    int* best;
    int* best2;          // second reservation array: Boruvka alternates between the two
    uint8_t* in_tree;
    int *listA, *listB, *raA, *rbA, *raB, *rbB, *hooked;
    int* ctr;
    const int* risky;
    const int* cls_start;
    const int* d_ncls;
    long long kq;
    uint32_t* T;
    int bnum, bden;
    int passes, crit_first;
    int big_class;       // k_fh_hybrid: weight classes with at least this many edges run as a grid Boruvka
    int risky_only;      // region kernels: 1 = serve risky layers only (MST: k_boruvka takes the others)
    int* stats;          // [2]: reservation rounds and windows of the windowed engines (reported per layer)
    int* engine;
    DevStatus* st;
};

__device__ __forceinline__ void decode(uint32_t key, int ebits, int W, int& e, int& w, int& p, int& q)
{
    e = (int)(key & ((1u << ebits) - 1u));
    w = (int)(key >> ebits);
    p = e >> 1;
    q = (e & 1) ? p + W : p + 1;
}

__device__ __forceinline__ bool same_set(const ForestArgs& a, int p, int q)
{
    return !a.pixset || a.canon[a.pixset[p]] == a.canon[a.pixset[q]];
}

// the end points' PixelIntv intersect: the edge survives DT-Rule 1
__device__ __forceinline__ bool sets_meet(const ForestArgs& a, int p, int q)
{
    if (!a.pixset) return true;
    const uint32_t* mp = a.table + (size_t)a.pixset[p] * HDP_WORDS;
    const uint32_t* mq = a.table + (size_t)a.pixset[q] * HDP_WORDS;
    uint32_t m = 0;
#pragma unroll
    for (int w = 0; w < HDP_WORDS; ++w) m |= mp[w] & mq[w];
    return m != 0u;
}

// Regions of the region engine.  A layer without a risky edge: connected
// same-set regions (no accepted edge joins different sets).  A risky layer:
// connected components of the edges that survive DT-Rule 1 (no edge joins two
// components, so each is its own sequential problem).
__device__ __forceinline__ bool region_edge(const ForestArgs& a, int p, int q, bool rk)
{
    return rk ? sets_meet(a, p, q) : same_set(a, p, q);
}

// the region kernels' mode: -1 = nothing to do, else 1 for a risky layer
__device__ __forceinline__ int region_mode(const ForestArgs& a)
{
    const bool rk = a.risky && __ldcg(a.risky);
    return a.risky_only && !rk ? -1 : (int)rk;
}

__device__ __forceinline__ void append(const ForestArgs& a, int which, int idx, int ra, int rb)
{
    const int pos = grid_ticket(a.ctr + which);
    int* L = which ? a.listB : a.listA;
    int* RA = which ? a.raB : a.raA;
    int* RB = which ? a.rbB : a.rbA;
    L[pos] = idx;
    RA[pos] = ra;
    RB[pos] = rb;
}

__device__ __forceinline__ int* best_of(const ForestArgs& a, int par) { return par ? a.best2 : a.best; }

// Boruvka rounds on the candidate list `cur` (best_of(par) holds each root's
// smallest candidate index).  Every root hooks onto the other end of its
// smallest edge; a pair that chose the same edge keeps the smaller root.
// Two reservation arrays alternate, so clearing one overlaps the selection
// into the other: two grid barriers per round.
__device__ bool boruvka_rounds(const ForestArgs& a, int& cur, int& par, bool record_hooks, int wclass = 0)
{
    const unsigned nb = gridDim.x;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    for (int it = 0; it < 64; ++it) {
        const int m = __ldcg(a.ctr + cur);
        if (m == 0) return true;
        const int* L = cur ? a.listB : a.listA;
        const int* RA = cur ? a.raB : a.raA;
        const int* RB = cur ? a.rbB : a.rbA;
        int* best = best_of(a, par);
        int* bnext = best_of(a, par ^ 1);
        int* hk = a.hooked + (par ? (size_t)a.N : 0);   // this round's hooked roots (two lists alternate)
        const int nxt = cur ^ 1;
        for (int j = tid; j < m; j += nth) {
            int idx = L[j], ra = RA[j], rb = RB[j];
            int ba = __ldcg(best + ra), bb = __ldcg(best + rb);
            if (ba == idx || bb == idx) a.in_tree[a.keys[idx] & ((1u << a.ebits) - 1u)] = 1;
            if (ba == idx && !(bb == idx && ra < rb)) {
                __stcg(a.parent + ra, rb);
                if (record_hooks) hk[grid_ticket(a.ctr + 2 + par)] = ra;
            }
            if (bb == idx && !(ba == idx && rb < ra)) {
                __stcg(a.parent + rb, ra);
                if (record_hooks) hk[grid_ticket(a.ctr + 2 + par)] = rb;
            }
        }
        if (tid == 0) {
            a.ctr[nxt] = 0;
            a.ctr[2 + (par ^ 1)] = 0;   // the other hooked list was consumed last round, before a barrier
        }
        if (!grid_sync(a.st, nb)) return false;
        if (record_hooks) {
            // roots hooked in this round fold their (complete) sizes into the
            // roots they now hang from; those are roots after every hook of the
            // round and receive no hook themselves, so the sums are exact
            const int nh = __ldcg(a.ctr + 2 + par);
            for (int j = tid; j < nh; j += nth) {
                const int r = hk[j];
                const int R = uf_find(a.parent, r);
                atomicAdd(a.size + R, __ldcg(a.size + r));
                __stcg(a.intw + R, wclass);
                __stcg(a.parent + r, R);   // shortcut: hook chains would lengthen every later find
            }
        }
        for (int j = tid; j < m; j += nth) {
            __stcg(best + RA[j], INT_MAX);
            __stcg(best + RB[j], INT_MAX);
            int idx = L[j], e, w, p, q;
            decode(a.keys[idx], a.ebits, a.W, e, w, p, q);
            int ra = uf_find(a.parent, p), rb = uf_find(a.parent, q);
            if (ra != rb) {
                min_by_key(bnext, ra, idx);
                min_by_key(bnext, rb, idx);
                append(a, nxt, idx, ra, rb);
            }
        }
        if (!grid_sync(a.st, nb)) return false;
        cur = nxt;
        par ^= 1;
    }
    dev_fail(a.st, DEV_TIMEOUT, 20);
    return false;
}

// Minimum spanning forest of the eligible edges (MST, or the linking pass of
// the segment tree on top of the first pass).  Runs only when no risky edge
// exists.
__global__ void k_boruvka(ForestArgs a)
{
    if (a.risky && __ldcg(a.risky)) return;   // k_fh_risky takes the layer
    const int n = *a.d_n;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    if (tid == 0 && *a.engine == 0) *a.engine = 1;
    for (int idx = tid; idx < n; idx += nth) {
        int e, w, p, q;
        decode(a.keys[idx], a.ebits, a.W, e, w, p, q);
        if (!same_set(a, p, q)) continue;
        int ra = uf_find(a.parent, p), rb = uf_find(a.parent, q);
        if (ra != rb) {
            min_by_key(a.best, ra, idx);
            min_by_key(a.best, rb, idx);
            append(a, 0, idx, ra, rb);
        }
    }
    if (!grid_sync(a.st, gridDim.x)) return;
    int cur = 0, par = 0;
    boruvka_rounds(a, cur, par, false);
}

// ---- segment-tree first pass, windowed, for one CTA (layers up to
// FH_LOCAL_MAX_NODES nodes, pure regime).  The sorted list is cut into windows
// of LW_EDGES consecutive edges.  For a window, the current roots of every
// live edge's end points are gathered from the union-find in global memory and
// given local ids in shared memory, together with their size and Int.  The
// window is then resolved entirely in shared memory by deterministic
// reservations: each round, every unresolved edge reserves both of its local
// roots with its window position (atomicMin of a round-stamped value, so no
// reset pass is needed); an edge that holds both reservations is the earliest
// unresolved edge on both trees, so it is decided on their current state
// exactly as the sequential algorithm decides it.  At the end of the window
// the merged local state is written back.
#define LW_EDGES 2048
#define LW_THREADS 512

template <int NE>
struct LocalWinT {
    uint32_t key[NE];
    uint16_t la[NE], lb[NE];
    uint32_t best[2 * NE];
    int parent[2 * NE];
    int size[2 * NE];
    int intw[2 * NE];
    int glob[2 * NE];
    uint16_t rep[2 * NE];   // representative end point code -> local id
    int nroots;
    int wmin, wmax;         // smallest and largest weight in the window
    int ntrans;             // weight changes along the window
    int wnext;              // next weight class of the window
    int nhook;              // trees hooked in a Boruvka round
};
typedef LocalWinT<LW_EDGES> LocalWin;

__device__ __forceinline__ int lw_find(int* parent, int x)
{
    for (int it = 0; it < 2 * LW_EDGES; ++it) {
        int p = parent[x];
        if (p == x) return x;
        int gp = parent[p];
        if (gp != p) parent[x] = gp;
        x = gp;
        if (gp == p) return p;
    }
    return x;
}

// Union-find root in global memory.  L2 = false: plain loads (no other CTA
// writes the entries this CTA reads while the kernel runs: one CTA, or
// disjoint regions); L2 = true: through L2 (other SMs wrote them before the
// last grid barrier).
template <bool L2>
__device__ __forceinline__ int g_find(int* parent, int v)
{
    if (L2) return uf_find(parent, v);
    for (int it = 0; it < (1 << 26); ++it) {
        int p = parent[v];
        if (p == v) return v;
        int gp = parent[p];
        if (gp == p) return p;
        parent[v] = gp;
        v = gp;
    }
    return v;
}

// Roots of the end points of up to M edges (a[k], b[k] for the edges in
// `live`), walked in lockstep with path halving: one hop of every unfinished
// chain per step, so the chains' load latencies overlap.
template <bool L2, int M>
__device__ __forceinline__ void g_find_many(int* parent, int* a, int* b, unsigned live)
{
    int v[2 * M];
    unsigned pend = 0;
#pragma unroll
    for (int k = 0; k < M; ++k) {
        v[2 * k] = a[k];
        v[2 * k + 1] = b[k];
        if (live >> k & 1u) pend |= 3u << (2 * k);
    }
    for (int it = 0; pend && it < (1 << 26); ++it) {
        int pv[2 * M], gv[2 * M];
#pragma unroll
        for (int j = 0; j < 2 * M; ++j)   // parents of every unfinished chain, loads in flight together
            pv[j] = (pend >> j & 1u) ? (L2 ? __ldcg(parent + v[j]) : parent[v[j]]) : v[j];
        unsigned hop = 0;
#pragma unroll
        for (int j = 0; j < 2 * M; ++j)
            if (pv[j] != v[j]) hop |= 1u << j;
        pend &= hop;
#pragma unroll
        for (int j = 0; j < 2 * M; ++j)   // grandparents
            gv[j] = (hop >> j & 1u) ? (L2 ? __ldcg(parent + pv[j]) : parent[pv[j]]) : 0;
#pragma unroll
        for (int j = 0; j < 2 * M; ++j) {
            if (!(hop >> j & 1u)) continue;
            if (gv[j] == pv[j]) {
                v[j] = pv[j];
                pend &= ~(1u << j);
            } else {
                if (L2) __stcg(parent + v[j], gv[j]);
                else parent[v[j]] = gv[j];
                v[j] = gv[j];
            }
        }
    }
#pragma unroll
    for (int k = 0; k < M; ++k) {
        a[k] = v[2 * k];
        b[k] = v[2 * k + 1];
    }
}

// Pending edges below this count per round hand the rest of a window to one warp.
#define LW_SEQ_BELOW 16
// Windows with fewer weight changes than this go class by class (Boruvka).
#define LW_CLASS_RUNS 32

// Sequential Kruskal over the pending edges of a window (bitmap bm, window
// order), run by one full warp.  The pending edges are first listed densely
// (after the bitmap, in the same scratch), so that every group of 32 is full.
// Each lane takes one edge of a group and caches the state of its two trees
// in registers: root, frozen flag, size, Int, and whether each side's
// criterion passes at this edge's weight.  The group is then decided edge by
// edge from that edge's cache, broadcast by shuffles, and every merge or
// freeze is applied to the caches of all lanes (so no shared-memory round
// trip sits on the serial path).  Lane 0 writes the same changes to shared
// memory for the next group.  A ballot over the caches jumps to the next
// edge that can still merge, so cycles and edges of frozen trees cost no step.
template <int NE>
__device__ __noinline__ void lw_sequential(const ForestArgs& a, LocalWinT<NE>& S, const uint32_t* bm, int cnt)
{
    static_assert(2 * NE <= (1 << 14), "local ids take 14 bits");
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    uint16_t* list = reinterpret_cast<uint16_t*>(const_cast<uint32_t*>(bm) + NE / 32);
    int np = 0;
    for (int g = 0; g < (cnt + 31) / 32; ++g) {
        const uint32_t m = bm[g];
        if (m >> lane & 1u) list[np + __popc(m & ((1u << lane) - 1u))] = (uint16_t)(32 * g + lane);
        np += __popc(m);
    }
    __syncwarp();
    const long long kq = a.kq;
    for (int g0 = 0; g0 < np; g0 += 32) {
        const int nb = min(32, np - g0);
        const uint32_t m = nb == 32 ? FULL : (1u << nb) - 1u;
        int x = 0, y = 0, e = 0, w = 0, sx = 0, sy = 0, ix = 0, iy = 0;
        bool zx = true, zy = true, px = false, py = false;   // frozen; criterion passes
        if (lane < nb) {
            const int i = list[g0 + lane];
            int p, q;
            x = lw_find(S.parent, S.la[i]);
            y = lw_find(S.parent, S.lb[i]);
            decode(S.key[i], a.ebits, a.W, e, w, p, q);
            zx = S.best[x] == 0u;
            zy = S.best[y] == 0u;
            sx = S.size[x]; sy = S.size[y];
            ix = S.intw[x]; iy = S.intw[y];
            px = (long long)(w - ix) * sx <= kq;
            py = (long long)(w - iy) * sy <= kq;
        }
        __syncwarp();   // every lane has read before lane 0 writes
        uint32_t pend = m;
        for (;;) {
            // the next edge of the group whose trees differ and are not frozen;
            // the edges before it are cycles or touch a frozen tree on the
            // current caches, which hold their state in the sequential order
            const unsigned act = __ballot_sync(FULL, (pend >> lane & 1u) && x != y && !zx && !zy);
            if (!act) break;
            const int k = __ffs(act) - 1;
            pend &= ~(uint32_t)((2ull << k) - 1ull);   // decided: every edge up to k
            const unsigned v = __shfl_sync(FULL, (unsigned)x | (unsigned)y << 14 | (unsigned)!px << 28 |
                                                     (unsigned)!py << 29, k);
            const int xk = (int)(v & 0x3fffu), yk = (int)((v >> 14) & 0x3fffu);
            const bool fx = (v >> 28) & 1u, fy = (v >> 29) & 1u;
            if (fx || fy) {   // criterion fails: that tree can never merge again
                if (fx) { zx |= x == xk; zy |= y == xk; }
                if (fy) { zx |= x == yk; zy |= y == yk; }
                if (lane == 0) {
                    if (fx) S.best[xk] = 0u;
                    if (fy) S.best[yk] = 0u;
                }
                continue;
            }
            const int sxk = __shfl_sync(FULL, sx, k), syk = __shfl_sync(FULL, sy, k), wk = __shfl_sync(FULL, w, k);
            int big = xk, small = yk;
            if (sxk < syk) { big = yk; small = xk; }
            const int ns = sxk + syk;
            if (x == small) x = big;
            if (y == small) y = big;
            if (x == big) { sx = ns; ix = wk; px = (long long)(w - ix) * sx <= kq; }
            if (y == big) { sy = ns; iy = wk; py = (long long)(w - iy) * sy <= kq; }
            if (lane == 0) {
                S.parent[small] = big;
                S.size[big] = ns;
                S.intw[big] = wk;
            }
            if (lane == k) a.in_tree[e] = 1;
        }
        __syncwarp();   // lane 0's writes are seen by the next group's reads
    }
}

// One weight class w of a window: its live edges (roots in S.la / S.lb,
// frozen trees marked best == 0) resolve as the minimum spanning forest by
// index among the trees that pass at w, by Boruvka rounds in shared
// memory: every tree takes its smallest edge (which belongs to the forest by
// the cut property, the indices being distinct) and hooks onto the other end;
// a pair that took the same edge keeps the smaller root.  Hooked trees fold
// their sizes into their new roots, whose Int becomes w.  Only 2-cycles can
// form, so each round at least halves the trees that still have live edges.
template <int NT, int NE>
__device__ __noinline__ void lw_boruvka(const ForestArgs& a, LocalWinT<NE>& S, unsigned live, int w)
{
    constexpr int LW_PER = NE / NT;
    constexpr uint32_t MARK = 1u << 14;   // marks MARK | i: above 0 (frozen), below 0xffffffff (free)
    const int t = threadIdx.x;
    uint16_t* hooked = S.rep;             // free after the gather
    // a tree that fails at w (on its state at the class start) can never merge again
#pragma unroll
    for (int k = 0; k < LW_PER; ++k) {
        if (!(live >> k & 1u)) continue;
        const int i = t + k * NT;
        const int x = lw_find(S.parent, S.la[i]), y = lw_find(S.parent, S.lb[i]);
        if (S.best[x] != 0u && (long long)(w - S.intw[x]) * S.size[x] > a.kq) S.best[x] = 0u;
        if (S.best[y] != 0u && (long long)(w - S.intw[y]) * S.size[y] > a.kq) S.best[y] = 0u;
    }
    __syncthreads();
    int round = 0;
    for (; round <= NE; ++round) {
        int xa[LW_PER], xb[LW_PER];
        if (t == 0) S.nhook = 0;
#pragma unroll
        for (int k = 0; k < LW_PER; ++k) {
            xa[k] = xb[k] = 0;
            if (!(live >> k & 1u)) continue;
            const int i = t + k * NT;
            xa[k] = lw_find(S.parent, S.la[i]);
            xb[k] = lw_find(S.parent, S.lb[i]);
            S.la[i] = (uint16_t)xa[k];
            S.lb[i] = (uint16_t)xb[k];
            if (xa[k] == xb[k] || S.best[xa[k]] == 0u || S.best[xb[k]] == 0u) {
                live &= ~(1u << k);   // a cycle, or a frozen tree
            } else {
                atomicMin(&S.best[xa[k]], MARK | (uint32_t)i);
                atomicMin(&S.best[xb[k]], MARK | (uint32_t)i);
            }
        }
        const unsigned marked = live;
        if (!__syncthreads_or(live != 0)) break;
#pragma unroll
        for (int k = 0; k < LW_PER; ++k) {
            if (!(live >> k & 1u)) continue;
            const int i = t + k * NT;
            const uint32_t me = MARK | (uint32_t)i;
            const bool ha = S.best[xa[k]] == me, hb = S.best[xb[k]] == me;
            if (!ha && !hb) continue;
            live &= ~(1u << k);
            int e, we, p, q;
            decode(S.key[i], a.ebits, a.W, e, we, p, q);
            a.in_tree[e] = 1;
            int r = xb[k], to = xa[k];
            if (ha && hb) {
                r = max(xa[k], xb[k]);
                to = min(xa[k], xb[k]);
            } else if (ha) {
                r = xa[k];
                to = xb[k];
            }
            S.parent[r] = to;
            hooked[atomicAdd(&S.nhook, 1)] = (uint16_t)r;
        }
        __syncthreads();
        // hooked roots are roots after every hook of the round and receive no
        // size themselves, so the folded sums are exact
        const int nh = S.nhook;
        for (int j = t; j < nh; j += NT) {
            const int r = hooked[j];
            const int R = lw_find(S.parent, r);
            atomicAdd(&S.size[R], S.size[r]);
            S.intw[R] = w;
        }
#pragma unroll
        for (int k = 0; k < LW_PER; ++k)
            if (marked >> k & 1u) {
                S.best[xa[k]] = 0xffffffffu;
                S.best[xb[k]] = 0xffffffffu;
            }
        __syncthreads();
    }
    if (round > NE) dev_fail(a.st, DEV_TIMEOUT, 42);
    if (t == 0 && a.stats) {
        atomicAdd(a.stats, round + 1);   // Boruvka rounds
        atomicAdd(a.stats + 1, 1);       // windows
    }
}

// One window [base, base + cnt) of the list `keys` (a run of the strict
// order), resolved by the calling CTA of NT threads.  loc[] is INT_MAX on
// entry and on exit.
// RISKY (layers with a risky edge): every edge of the list takes part,
// DT-Rule 2 is decided on the trees' TreeIntv, kept in ST (HDP_WORDS words per
// local tree) and merged with the trees; kq is the criterion's k (a huge
// value for a pass without the criterion).  Windows then use reservations
// only: the class-by-class shortcut and the sequential finish assume trees
// that never join different sets.
template <bool L2, int NT, int NE, bool RISKY = false>
__device__ void lw_window(const ForestArgs& a, const uint32_t* keys, int* loc, LocalWinT<NE>& S, int base, int cnt,
                          uint32_t* ST = nullptr, long long kq_in = -1)
{
    constexpr int LW_PER = NE / NT;
    const long long kq = RISKY ? kq_in : a.kq;
    const int t = threadIdx.x;
    if (t == 0) {
        S.nroots = 0;
        S.wmin = INT_MAX;
        S.wmax = -1;
        S.ntrans = 0;
    }
    __syncthreads();
    // gather: current global roots of both end points; one representative
    // end point per distinct root (smallest code) allocates its local id.
    // The loads of a thread's edges are issued together (keys, then sets,
    // then the finds in lockstep), so their latencies overlap.
    int ra[LW_PER], rb[LW_PER];
    uint32_t kk[LW_PER];
    int wk[LW_PER];
    unsigned live = 0;
    int wl = INT_MAX, wh = -1, ntr = 0;
#pragma unroll
    for (int k = 0; k < LW_PER; ++k) {
        const int i = t + k * NT;
        ra[k] = rb[k] = -1;
        if (i < cnt) {
            kk[k] = keys[base + i];
            live |= 1u << k;
        }
    }
#pragma unroll
    for (int k = 0; k < LW_PER; ++k) {
        if (!(live >> k & 1u)) continue;
        int e, w, p, q;
        decode(kk[k], a.ebits, a.W, e, w, p, q);
        wl = min(wl, w);
        wh = max(wh, w);
        wk[k] = w;
        ra[k] = p;
        rb[k] = q;
        const int i = t + k * NT;
        if (i > 0) {
            int ep, wp, pp, qp;
            decode(keys[base + i - 1], a.ebits, a.W, ep, wp, pp, qp);
            ntr += wp != w;
        }
    }
#pragma unroll
    for (int k = 0; k < LW_PER; ++k)
        if (!RISKY && (live >> k & 1u) && !same_set(a, ra[k], rb[k])) live &= ~(1u << k);
    g_find_many<L2, LW_PER>(a.parent, ra, rb, live);
#pragma unroll
    for (int k = 0; k < LW_PER; ++k) {
        if (!(live >> k & 1u)) continue;
        const int i = t + k * NT;
        if (ra[k] == rb[k]) {
            live &= ~(1u << k);
            continue;
        }
        S.key[i] = kk[k];
        atomicMin(loc + ra[k], 2 * i);
        atomicMin(loc + rb[k], 2 * i + 1);
    }
    if (wl != INT_MAX) {
        atomicMin(&S.wmin, wl);
        atomicMax(&S.wmax, wh);
    }
    if (ntr) atomicAdd(&S.ntrans, ntr);
    __syncthreads();
    // a tree whose criterion already fails at the window's smallest weight
    // can never merge again in this pass (every later edge of its region is
    // at least as heavy and its state cannot change without a merge): it
    // starts frozen, which best == 0 marks (0 is below every reservation
    // stamp).  (A window may hold several whole regions, each in the strict
    // order; the smallest weight over all of them keeps the test exact.)
    const long long w0 = S.wmin;
    int ca[LW_PER], cb[LW_PER];
#pragma unroll
    for (int k = 0; k < LW_PER; ++k) {
        ca[k] = cb[k] = 0;
        if (!(live >> k & 1u)) continue;
        const int i = t + k * NT;
        ca[k] = __ldcg(loc + ra[k]);
        cb[k] = __ldcg(loc + rb[k]);
        for (int side = 0; side < 2; ++side) {
            const int code = side ? cb[k] : ca[k], r = side ? rb[k] : ra[k];
            if (code == 2 * i + side) {
                const int id = atomicAdd(&S.nroots, 1);
                S.rep[code] = (uint16_t)id;
                S.glob[id] = r;
                S.parent[id] = id;
                const int sz = L2 ? __ldcg(a.size + r) : a.size[r];
                const int iw = L2 ? __ldcg(a.intw + r) : a.intw[r];
                S.size[id] = sz;
                S.intw[id] = iw;
                S.best[id] = (w0 - iw) * sz > kq ? 0u : 0xffffffffu;
                if (RISKY)
#pragma unroll
                    for (int h = 0; h < HDP_WORDS; ++h)
                        ST[id * HDP_WORDS + h] = L2 ? __ldcg(a.T + (size_t)r * HDP_WORDS + h) : a.T[(size_t)r * HDP_WORDS + h];
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < LW_PER; ++k) {
        if (!(live >> k & 1u)) continue;
        const int i = t + k * NT;
        S.la[i] = S.rep[ca[k]];
        S.lb[i] = S.rep[cb[k]];
    }
    __syncthreads();
    if (!RISKY && S.ntrans < LW_CLASS_RUNS) {
        // few weight classes (the usual window of a big region): inside a
        // class the trees that pass at its weight keep passing as they merge
        // (Int becomes w) and the others cannot merge, so each class resolves
        // as the minimum spanning forest by index among its passing trees;
        // the classes go in increasing weight (regions sharing the window are
        // independent, so one class step serves all of them)
        int wc = S.wmin;
        for (int c = 0; c <= LW_CLASS_RUNS && wc != INT_MAX; ++c) {
            unsigned lc = 0;
#pragma unroll
            for (int k = 0; k < LW_PER; ++k)
                if ((live >> k & 1u) && wk[k] == wc) lc |= 1u << k;
            lw_boruvka<NT, NE>(a, S, lc, wc);
            if (t == 0) S.wnext = INT_MAX;
            __syncthreads();
            int m = INT_MAX;
#pragma unroll
            for (int k = 0; k < LW_PER; ++k)
                if ((live >> k & 1u) && wk[k] > wc) m = min(m, wk[k]);
            if (m != INT_MAX) atomicMin(&S.wnext, m);
            __syncthreads();
            wc = S.wnext;
            __syncthreads();
        }
        live = 0;
    } else
    // deterministic reservations in shared memory; the earliest unresolved
    // edge always holds both of its reservations, so every round resolves at
    // least one edge and the loop ends within NE rounds
    for (int round = 0; round <= NE; ++round) {
        const uint32_t stamp = (uint32_t)(0xffff - round) << 13;
        const unsigned live0 = live;
        int xa[LW_PER], xb[LW_PER];
#pragma unroll
        for (int k = 0; k < LW_PER; ++k) {
            xa[k] = xb[k] = 0;
            if (!(live >> k & 1u)) continue;
            const int i = t + k * NT;
            xa[k] = lw_find(S.parent, S.la[i]);
            xb[k] = lw_find(S.parent, S.lb[i]);
            // the next round starts from today's roots (a hop or two), not
            // from the end points' original local ids; only this thread reads them
            S.la[i] = (uint16_t)xa[k];
            S.lb[i] = (uint16_t)xb[k];
            if (xa[k] == xb[k] || S.best[xa[k]] == 0u || S.best[xb[k]] == 0u) {
                live &= ~(1u << k);   // a cycle, or a frozen tree: rejected
            } else {
                atomicMin(&S.best[xa[k]], stamp | (uint32_t)i);
                atomicMin(&S.best[xb[k]], stamp | (uint32_t)i);
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < LW_PER; ++k) {
            if (!(live >> k & 1u)) continue;
            const int i = t + k * NT;
            const uint32_t me = stamp | (uint32_t)i;
            const bool ha = S.best[xa[k]] == me, hb = S.best[xb[k]] == me;
            if (!ha && !hb) continue;
            int e, w, p, q;
            decode(S.key[i], a.ebits, a.W, e, w, p, q);
            const long long sa = S.size[xa[k]], sb = S.size[xb[k]];
            const long long ia = S.intw[xa[k]], ib = S.intw[xb[k]];
            // the earliest unresolved edge of a tree sees its final state: if
            // the criterion fails there, the tree is frozen and the edge rejected
            const bool fa = ha && (w - ia) * sa > kq, fb = hb && (w - ib) * sb > kq;
            if (fa || fb) {
                if (fa) S.best[xa[k]] = 0u;
                if (fb) S.best[xb[k]] = 0u;
                live &= ~(1u << k);
                continue;
            }
            if (!ha || !hb) continue;
            live &= ~(1u << k);
            if (RISKY) {   // DT-Rule 2: Jaccard ratio of the two TreeIntv at least beta
                int inter = 0, uni = 0;
#pragma unroll
                for (int h = 0; h < HDP_WORDS; ++h) {
                    const uint32_t ta = ST[xa[k] * HDP_WORDS + h], tb = ST[xb[k] * HDP_WORDS + h];
                    inter += __popc(ta & tb);
                    uni += __popc(ta | tb);
                }
                if ((long long)inter * a.bden < (long long)a.bnum * uni) continue;
            }
            int big = xa[k], small = xb[k];                                  // both pass: merge
            if (sa < sb) { big = xb[k]; small = xa[k]; }
            S.parent[small] = big;
            S.size[big] = (int)(sa + sb);
            S.intw[big] = w;
            if (RISKY)
#pragma unroll
                for (int h = 0; h < HDP_WORDS; ++h) ST[big * HDP_WORDS + h] |= ST[small * HDP_WORDS + h];
            a.in_tree[e] = 1;
        }
        const int lt = __syncthreads_count(live != 0);          // threads still holding edges
        const int rt = __syncthreads_count(live != live0);      // threads that resolved one this round
        if (lt == 0 || (!RISKY && round >= 1 && rt < LW_SEQ_BELOW)) {
            if (lt != 0) {
                // Few edges resolve per round: the rest wait in chains on a few
                // big trees, and every further round would re-examine all of
                // them.  Warp 0 finishes the window as the sequential algorithm
                // does: the pending edges in window order, on the current trees.
                // This is exact: every tree that a pending edge touches holds
                // only merged edges of lower index (an edge merges only while
                // it holds the reservation of both its trees), so the lowest
                // pending edge always sees its sequential state.
                uint32_t* bm = reinterpret_cast<uint32_t*>(S.rep);   // NE bits, then NE 16-bit slots (rep is free after the gather)
                for (int j = t; j < NE / 32; j += NT) bm[j] = 0u;
                __syncthreads();
#pragma unroll
                for (int k = 0; k < LW_PER; ++k)
                    if (live >> k & 1u) {
                        const int i = t + k * NT;
                        atomicOr(bm + (i >> 5), 1u << (i & 31));
                    }
                live = 0;
                __syncthreads();
                if (t < 32) lw_sequential(a, S, bm, cnt);
                __syncthreads();
            }
            if (t == 0 && a.stats) {
                atomicAdd(a.stats, round + 1);   // reservation rounds
                atomicAdd(a.stats + 1, 1);       // windows
            }
            break;
        }
    }
    if (live) dev_fail(a.st, DEV_TIMEOUT, 40);   // unreachable by the argument above
    // write back: merged local roots hang from their new root's global id
    const int nr = S.nroots;
    for (int x = t; x < nr; x += NT) {
        const int r = S.glob[x];
        const int rx = lw_find(S.parent, x);
        if (rx != x) {
            if (L2) __stcg(a.parent + r, S.glob[rx]);
            else a.parent[r] = S.glob[rx];
        } else if (L2) {
            __stcg(a.size + r, S.size[x]);
            __stcg(a.intw + r, S.intw[x]);
            if (RISKY)
#pragma unroll
                for (int h = 0; h < HDP_WORDS; ++h) __stcg(a.T + (size_t)r * HDP_WORDS + h, ST[x * HDP_WORDS + h]);
        } else {
            a.size[r] = S.size[x];
            a.intw[r] = S.intw[x];
            if (RISKY)
#pragma unroll
                for (int h = 0; h < HDP_WORDS; ++h) a.T[(size_t)r * HDP_WORDS + h] = ST[x * HDP_WORDS + h];
        }
        atomicExch(loc + r, INT_MAX);
    }
    __syncthreads();
}

__global__ void __launch_bounds__(LW_THREADS, 1) k_fh_local(ForestArgs a, int* loc)
{
    extern __shared__ __align__(16) unsigned char lw_raw[];
    LocalWin& S = *reinterpret_cast<LocalWin*>(lw_raw);
    if (a.risky && __ldcg(a.risky)) return;
    const int n = *a.d_n;
    if (threadIdx.x == 0) *a.engine = 3;
    for (int base = 0; base < n; base += LW_EDGES)
        lw_window<false, LW_THREADS, LW_EDGES>(a, a.keys, loc, S, base, min(LW_EDGES, n - base));
}

// Layers with a risky edge (DT-Rule 2 may join different sets, so regions are
// not independent): every pass over the whole list in one CTA, window by
// window, with each local tree's TreeIntv in shared memory.
#define RK_EDGES 1024
#define RK_THREADS 512
typedef LocalWinT<RK_EDGES> RiskyWin;
__host__ __device__ constexpr size_t risky_smem() { return sizeof(RiskyWin) + 2 * RK_EDGES * HDP_WORDS * sizeof(uint32_t); }

__global__ void __launch_bounds__(RK_THREADS, 1) k_fh_risky(ForestArgs a, int* loc)
{
    extern __shared__ __align__(16) unsigned char lw_raw[];
    RiskyWin& S = *reinterpret_cast<RiskyWin*>(lw_raw);
    uint32_t* ST = reinterpret_cast<uint32_t*>(lw_raw + sizeof(RiskyWin));
    if (!a.risky || !__ldcg(a.risky)) return;
    const int n = *a.d_n;
    if (threadIdx.x == 0) *a.engine = 6;
    for (int pass = 0; pass < a.passes; ++pass) {
        const long long kq = a.crit_first && pass == 0 ? a.kq : (1LL << 60);
        for (int base = 0; base < n; base += RK_EDGES)
            lw_window<false, RK_THREADS, RK_EDGES, true>(a, a.keys, loc, S, base, min(RK_EDGES, n - base), ST, kq);
    }
}

static void launch_risky(ForestArgs& a, Ctx& c)
{
    static bool configured = false;
    if (!configured) {
        cudaFuncSetAttribute(k_fh_risky, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)risky_smem());
        configured = true;
    }
    k_fh_risky<<<1, RK_THREADS, risky_smem(), c.s>>>(a, c.rootof);
}

// Segment-tree first pass for big layers (cooperative, one CTA per SM):
// weight classes of at least a.big_class (<= LW_EDGES) edges run as a grid
// Boruvka (see the file comment); runs of consecutive smaller classes, up to
// LW_EDGES edges, form one window that block 0 resolves in shared memory while
// the others wait at the next grid barrier.

__global__ void __launch_bounds__(LW_THREADS, 1) k_fh_hybrid(ForestArgs a, int* loc)
{
    extern __shared__ __align__(16) unsigned char lw_raw[];
    LocalWin& S = *reinterpret_cast<LocalWin*>(lw_raw);
    if (a.risky && __ldcg(a.risky)) return;
    const int n = *a.d_n, ncls = *a.d_ncls;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    if (tid == 0) *a.engine = 4;
    int cur = 0, par = 0;
    for (int c = 0; c < ncls;) {
        const int s = a.cls_start[c];
        const int e_end = c + 1 < ncls ? a.cls_start[c + 1] : n;
        if (e_end - s >= a.big_class) {
            const long long w = (long long)(a.keys[s] >> a.ebits);
            for (int idx = s + tid; idx < e_end; idx += nth) {
                int e, ww, p, q;
                decode(a.keys[idx], a.ebits, a.W, e, ww, p, q);
                if (!same_set(a, p, q)) continue;
                int ra = uf_find(a.parent, p), rb = uf_find(a.parent, q);
                if (ra == rb) continue;
                long long sa = __ldcg(a.size + ra), sb = __ldcg(a.size + rb);
                long long ia = __ldcg(a.intw + ra), ib = __ldcg(a.intw + rb);
                if ((w - ia) * sa > a.kq || (w - ib) * sb > a.kq) continue;
                min_by_key(best_of(a, par), ra, idx);
                min_by_key(best_of(a, par), rb, idx);
                append(a, cur, idx, ra, rb);
            }
            if (!grid_sync(a.st, gridDim.x)) return;
            if (__ldcg(a.ctr + cur) != 0 && !boruvka_rounds(a, cur, par, true, (int)w)) return;
            ++c;
        } else {
            int c2 = c + 1;
            while (c2 < ncls) {
                const int e2 = c2 + 1 < ncls ? a.cls_start[c2 + 1] : n;
                if (e2 - a.cls_start[c2] >= a.big_class || e2 - s > LW_EDGES) break;
                ++c2;
            }
            const int wend = c2 < ncls ? a.cls_start[c2] : n;
            if (blockIdx.x == 0) lw_window<true, LW_THREADS, LW_EDGES>(a, a.keys, loc, S, s, wend - s);
            if (!grid_sync(a.st, gridDim.x)) return;
            c = c2;
        }
    }
}

// ---- segment-tree first pass by regions (HDP layers, pure regime).  Without
// a risky edge no accepted edge joins different PixelIntv sets, so the
// connected same-set regions are independent: the sequential result inside a
// region depends only on the region's own edges, in the strict order.  The
// edges are stably sorted by region (keeping the strict order inside each);
// persistent CTAs take whole regions and resolve them window by window.
#define RG_THREADS 1024
#define RG_EDGES 2048
#define RG_SMALL (RG_EDGES / 2)   // regions of at most this many edges share windows
typedef LocalWinT<RG_EDGES> RegionWin;

// Connected same-set regions: lock-free union-find over the same-set edges,
// the larger root hooked under the smaller by atomicMin (so a region's root
// is its smallest pixel); parent pointers only decrease, so shortcuts are
// safe, and a lowered parent that cut a node from its old tree is followed by
// joining that old tree too.
__device__ __forceinline__ int cc_find(int* par, int v)
{
    for (int it = 0; it < (1 << 26); ++it) {
        const int p = __ldcg(par + v);
        if (p == v) return v;
        const int gp = __ldcg(par + p);
        if (gp == p) return p;
        __stcg(par + v, gp);   // v is not a root: only shortcuts ever write it
        v = gp;
    }
    return v;
}

// Runs first: one thread per CC_RUN pixels of a row links every pixel to the
// first pixel of its same-set run inside that stretch (parents only decrease),
// so the hooking below skips those horizontal edges and starts from short
// chains.
#define CC_RUN 32
__global__ void k_cc_runs(ForestArgs a, int* par)
{
    const int mode = region_mode(a);
    if (mode < 0) return;
    const int per_row = (a.W + CC_RUN - 1) / CC_RUN;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= per_row * (a.N / a.W)) return;
    const int y = c / per_row, x0 = (c - y * per_row) * CC_RUN, x1 = min(x0 + CC_RUN, a.W);
    int run = y * a.W + x0;
    for (int x = x0 + 1; x < x1; ++x) {
        const int v = y * a.W + x;
        if (region_edge(a, v - 1, v, mode)) par[v] = run;
        else run = v;
    }
}

__device__ __forceinline__ void cc_hook_edge(const ForestArgs& a, int* par, int e, int mode)
{
    const int p = e >> 1;
    if ((e & 1) ? p + a.W >= a.N : (p % a.W) + 1 >= a.W) return;   // no neighbour there
    if (!(e & 1) && (p % a.W) % CC_RUN != CC_RUN - 1) return;      // linked by k_cc_runs
    const int q = (e & 1) ? p + a.W : p + 1;
    if (!region_edge(a, p, q, mode)) return;
    int u = cc_find(par, p), v = cc_find(par, q);
    for (int it = 0; it < (1 << 20); ++it) {
        if (u == v) return;
        if (u < v) { const int t = u; u = v; v = t; }
        // lower u's parent to v: if u was a root, it now hangs under v; else
        // its old parent (smaller than u) still has to be joined with v
        const int old = atomicMin(par + u, v);
        if (old == u) return;
        u = cc_find(par, old);
        v = cc_find(par, v);
    }
    dev_fail(a.st, DEV_TIMEOUT, 41);
}

// The region kernels below stride over a grid of at most a few CTAs per SM,
// so that where they have nothing to do they end at once.
__global__ void k_cc_hook(ForestArgs a, int* par)
{
    const int mode = region_mode(a);
    if (mode < 0) return;
    // edge ids in image order (the regions do not depend on the order), so
    // that neighbouring threads share parent cache lines
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 2 * a.N; e += gridDim.x * blockDim.x)
        cc_hook_edge(a, par, e, mode);
}

// edges per region (region edges, by their first end point's region root)
__global__ void k_region_count(ForestArgs a, const int* label, int* rcnt)
{
    const int mode = region_mode(a);
    if (mode < 0) return;
    // image order: neighbouring lanes share a region
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 2 * a.N; e += gridDim.x * blockDim.x) {
        const int p = e >> 1;
        if ((e & 1) ? p + a.W >= a.N : (p % a.W) + 1 >= a.W) continue;
        const int q = (e & 1) ? p + a.W : p + 1;
        if (region_edge(a, p, q, mode)) count_by_key(rcnt, label[p]);
    }
}

// sort key of every region edge: its region label, with bit rbits set for
// regions of more than RG_SMALL edges (small regions come first); other
// edges get 2^(rbits+1) - 1 and sort last.  nsmall counts the edges of the
// small regions; sort_n receives the list length for the sort (it stays 0,
// and the sort does nothing, where these kernels have nothing to do).
__global__ void k_region_keys(ForestArgs a, const int* label, const int* rcnt, int rbits, uint32_t* rk, uint32_t* rv,
                              int* nvalid, int* nsmall, int* sort_n)
{
    const int mode = region_mode(a);
    if (mode < 0) return;
    const int n = *a.d_n;
    if (blockIdx.x == 0 && threadIdx.x == 0) *sort_n = n;
    int cv = 0, cs = 0;
    for (int b0 = blockIdx.x * blockDim.x; b0 < n; b0 += gridDim.x * blockDim.x) {   // block-uniform trips
        const int idx = b0 + threadIdx.x;
        bool valid = false, small = false;
        if (idx < n) {
            const uint32_t key = a.keys[idx];
            int e, w, p, q;
            decode(key, a.ebits, a.W, e, w, p, q);
            valid = region_edge(a, p, q, mode);
            uint32_t k = (2u << rbits) - 1u;
            if (valid) {
                const int r = label[p];
                small = rcnt[r] <= RG_SMALL;
                k = (uint32_t)r | (small ? 0u : 1u << rbits);
            }
            rk[idx] = k;
            rv[idx] = key;
        }
        cv += __syncthreads_count(valid);
        cs += __syncthreads_count(small);
    }
    // one atomic per block on each grid-wide count
    if (threadIdx.x == 0) {
        if (cv) atomicAdd(nvalid, cv);
        if (cs) atomicAdd(nsmall, cs);
    }
}

// windows over the small regions: all small regions starting in the same
// RG_SMALL-edge bucket of the sorted list share one window (whole regions,
// under 2 * RG_SMALL edges)
__global__ void k_region_buckets(ForestArgs a, const int* d_nvalid, const int* d_nsmall, int* wb_lo, int* wb_hi,
                                 int* nsmall_regions)
{
    if (region_mode(a) < 0) return;
    const int nreg = *a.d_ncls;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nreg; r += gridDim.x * blockDim.x) {
        const int s = a.cls_start[r];
        if (s >= *d_nsmall) continue;
        const int e = r + 1 < nreg ? a.cls_start[r + 1] : *d_nvalid;
        const int b = s / RG_SMALL;
        atomicMin(wb_lo + b, s);
        atomicMax(wb_hi + b, e);
        grid_ticket(nsmall_regions);   // a count: one atomic per group of lanes
    }
}

// A run [s, e) of the region-sorted list on a risky layer (one component, or
// a bucket of whole small ones): every pass over it in windows of RK_EDGES,
// with each local tree's TreeIntv in shared memory (as k_fh_risky does for
// the whole list).
__device__ void region_risky(const ForestArgs& a, const uint32_t* rkeys, int* loc, unsigned char* raw, int s, int e)
{
    RiskyWin& S = *reinterpret_cast<RiskyWin*>(raw);
    uint32_t* ST = reinterpret_cast<uint32_t*>(raw + sizeof(RiskyWin));
    for (int pass = 0; pass < a.passes; ++pass) {
        const long long kq = a.crit_first && pass == 0 ? a.kq : (1LL << 60);
        for (int base = s; base < e; base += RK_EDGES)
            lw_window<false, RG_THREADS, RK_EDGES, true>(a, rkeys, loc, S, base, min(RK_EDGES, e - base), ST, kq);
    }
}

__host__ __device__ constexpr size_t regions_smem()
{
    return sizeof(RegionWin) > risky_smem() ? sizeof(RegionWin) : risky_smem();
}

// Work items: every big region (its windows in order, on one CTA), then one
// window per bucket of small regions.  The windows read the union-find with
// plain (L1-cached) loads: regions are disjoint, so no other CTA writes an
// entry this CTA reads while the kernel runs (words of other regions that
// share a cache line are never read here), and earlier kernels' writes are
// visible by launch order.  Layers without a risky edge: the
// segment tree's first pass (engine 5).  Risky layers: every pass, region by
// region (engine 7).
__global__ void __launch_bounds__(RG_THREADS, 1) k_fh_regions(ForestArgs a, const uint32_t* rkeys, const int* d_nvalid,
                                                           const int* d_nsmall, const int* d_nsmall_regions,
                                                           const int* wb_lo, const int* wb_hi, int* loc, int* ticket)
{
    extern __shared__ __align__(16) unsigned char rg_raw[];
    RegionWin& S = *reinterpret_cast<RegionWin*>(rg_raw);
    __shared__ int s_r;
    const int mode = region_mode(a);
    if (mode < 0) return;
    const int nreg = *a.d_ncls, nv = *d_nvalid, nsr = *d_nsmall_regions;
    const int nbig = nreg - nsr, nbuckets = cdiv(*d_nsmall, RG_SMALL);
    if (blockIdx.x == 0 && threadIdx.x == 0) *a.engine = mode ? 7 : 5;
    for (;;) {
        if (threadIdx.x == 0) s_r = atomicAdd(ticket, 1);
        __syncthreads();
        const int t = s_r;
        __syncthreads();
        if (t < nbig) {
            const int r = nsr + t;
            const int s = a.cls_start[r], e = r + 1 < nreg ? a.cls_start[r + 1] : nv;
            if (mode) {
                region_risky(a, rkeys, loc, rg_raw, s, e);
            } else {
                for (int base = s; base < e; base += RG_EDGES)
                    lw_window<false, RG_THREADS, RG_EDGES>(a, rkeys, loc, S, base, min(RG_EDGES, e - base));
            }
        } else if (t - nbig < nbuckets) {
            const int lo = wb_lo[t - nbig], hi = wb_hi[t - nbig];
            if (lo < hi) {
                if (mode) region_risky(a, rkeys, loc, rg_raw, lo, hi);
                else lw_window<false, RG_THREADS, RG_EDGES>(a, rkeys, loc, S, lo, hi - lo);
            }
        } else {
            break;
        }
    }
}

// k_forest_init plus the stage's other starting state in one launch: no
// forest edge yet, the counters, the engine and window statistics, and the
// grid barrier's state (the error word is kept)
__global__ void k_forest_start(int* parent, int* size, int* intw, int* best, int* best2, int* minid, int* loc,
                               uint8_t* in_tree, int* ints, DevStatus* st, int N)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v == 0) {
        for (int k = 0; k < 5; ++k) ints[IDX_CTR0 + k] = 0;
        ints[IDX_ENGINE] = 0;
        ints[IDX_DRROUNDS] = 0;
        ints[IDX_DRWINDOWS] = 0;
        st->bar_count = 0u;
        st->bar_gen = 0u;
    }
    if (v >= N) return;
    loc[v] = INT_MAX;
    parent[v] = v;
    size[v] = 1;
    intw[v] = 0;
    best[v] = INT_MAX;
    best2[v] = INT_MAX;
    minid[v] = INT_MAX;
    in_tree[2 * v] = 0;
    in_tree[2 * v + 1] = 0;
}

__global__ void k_fill_int_f(int* p, int n, int v)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

__global__ void k_forest_init(int* parent, int* size, int* intw, int* best, int* best2, int* minid, int* loc, int N)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= N) return;
    loc[v] = INT_MAX;
    parent[v] = v;
    size[v] = 1;
    intw[v] = 0;
    best[v] = INT_MAX;
    best2[v] = INT_MAX;
    minid[v] = INT_MAX;
}

// TreeIntv of every singleton tree = its PixelIntv (used by the reservation engine)
__global__ void k_T_init(uint32_t* T, const int* pixset, const uint32_t* table, int N, const int* risky, int always)
{
    if (!always && !__ldcg(risky)) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N * HDP_WORDS; i += gridDim.x * blockDim.x) {
        const int v = i / HDP_WORDS, k = i % HDP_WORDS;
        T[i] = table[(size_t)pixset[v] * HDP_WORDS + k];
    }
}

__global__ void k_class_flags(const uint32_t* keys, const int* d_n, int ebits, uint32_t* flags)
{
    const int n = *d_n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        flags[i] = i == 0 || (keys[i] >> ebits) != (keys[i - 1] >> ebits);
}

__global__ void k_class_scatter(const uint32_t* flags, const uint32_t* pos, const int* d_n, int* cls_start,
                                const uint32_t* total, int* ncls)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) *ncls = (int)*total;
    const int n = *d_n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if (flags[i] && pos[i] < (uint32_t)n) cls_start[pos[i]] = i;
}

__global__ void k_flatten(int* parent, int* rootof, int* minid, int N)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= N) return;
    int r = uf_find(parent, v);
    rootof[v] = r;
    min_by_key(minid, r, v);
}

// dt_root = smallest pixel id of the tree; TreeIntv at union-find roots for
// the engines that do not maintain it (their trees keep one set).
__global__ void k_finish_roots(const int* rootof, const int* minid, int* dtroot, uint32_t* T, const int* pixset,
                               const uint32_t* table, const uint32_t* full_mask, const int* engine, int N)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= N) return;
    int r = rootof[v];
    dtroot[v] = minid[r];
    if (r == v) {
        // the reservation engines of risky layers keep the unions themselves
        bool maintained = pixset != nullptr && (*engine == 2 || *engine == 6 || *engine == 7);
        if (!maintained) {
            const uint32_t* src = pixset ? table + (size_t)pixset[v] * HDP_WORDS : full_mask;
            for (int k = 0; k < HDP_WORDS; ++k) T[(size_t)v * HDP_WORDS + k] = src[k];
        }
    }
}

// 4-bit adjacency of the forest: bit 0 up, 1 left, 2 right, 3 down
__global__ void k_adj(const uint8_t* in_tree, int W, int H, uint8_t* adj)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= W * H) return;
    int x = v % W, y = v / W;
    uint8_t m = 0;
    if (y > 0 && in_tree[2 * (v - W) + 1]) m |= 1;
    if (x > 0 && in_tree[2 * (v - 1)]) m |= 2;
    if (x + 1 < W && in_tree[2 * v]) m |= 4;
    if (y + 1 < H && in_tree[2 * v + 1]) m |= 8;
    adj[v] = m;
}

// blocks_per_sm = 0: as many as fit; barrier-heavy kernels use 1 (fewer arrivals per barrier)
cudaError_t coop_launch(const void* fn, int threads, void** args, cudaStream_t s, int blocks_per_sm, int* used,
                        size_t smem, int max_blocks)
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, smem);
    if (blocks_per_sm > 0 && per > blocks_per_sm) per = blocks_per_sm;
    int blocks = per * sms;
    if (max_blocks > 0 && blocks > max_blocks) blocks = max_blocks;
    if (blocks < 1) blocks = 1;
    if (used) *used = blocks;
    return cudaLaunchCooperativeKernel(fn, dim3(blocks), dim3(threads), args, smem, s);
}


// The region machinery's size-proportional steps, skipped where the region
// kernels have nothing to do (a layer without a risky edge under risky_only)
__global__ void k_region_flatten(ForestArgs a, int* parent, int* rootof, int* rcnt)
{
    if (region_mode(a) < 0) return;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < a.N; v += gridDim.x * blockDim.x) {
        rcnt[v] = 0;   // per-region edge counts, made by k_region_count next
        rootof[v] = uf_find(parent, v);
    }
}

__global__ void k_region_init(ForestArgs a, int* parent, int* size, int* intw, int* best, int* best2, int* minid,
                              int* loc, uint8_t* in_tree)
{
    if (region_mode(a) < 0) return;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < a.N; v += gridDim.x * blockDim.x) {
        loc[v] = INT_MAX;
        parent[v] = v;
        size[v] = 1;
        intw[v] = 0;
        best[v] = INT_MAX;
        best2[v] = INT_MAX;
        minid[v] = INT_MAX;
        in_tree[2 * v] = 0;
        in_tree[2 * v + 1] = 0;
    }
}

// The region engine on an HDP layer: label the regions (lock-free
// union-find), sort the region edges by region (the strict order kept inside
// each), and resolve them region by region on persistent CTAs (k_fh_regions).
// Every kernel reads the layer's risky flag: without a risky edge the regions
// are the same-set regions and the pass is the segment tree's first; with one
// they are the components of the edges that survive DT-Rule 1 and every pass
// runs there (a.passes, a.crit_first).  With a.risky_only set a layer without
// a risky edge makes every kernel return at once.
static void launch_regions(Ctx& c, ForestArgs& a, const LayerDims& d)
{
    const int N = d.N;
    k_cc_runs<<<cdiv(cdiv(d.W, CC_RUN) * d.H, 256), 256, 0, c.s>>>(a, c.parent);
    const int g2 = min(cdiv(2 * N, 256), 4 * c.num_sms), g1 = min(cdiv(N, 256), 4 * c.num_sms);
    k_cc_hook<<<g2, 256, 0, c.s>>>(a, c.parent);
    int* rcnt = c.minid;   // free until k_region_init below
    k_region_flatten<<<g1, 256, 0, c.s>>>(a, c.parent, c.rootof, rcnt);
    int* nvalid = c.ints + IDX_TMP3;
    int* nsmall = c.ints + IDX_CTR3;
    int* nsmall_regions = c.ints + IDX_CTR4;
    cudaMemsetAsync(nvalid, 0, sizeof(int), c.s);
    cudaMemsetAsync(nsmall, 0, 2 * sizeof(int), c.s);   // and nsmall_regions
    k_region_count<<<g2, 256, 0, c.s>>>(a, c.rootof, rcnt);
    int rbits = 1;   // labels < N < 2^rbits, so no big key equals the all-ones "other" key
    while ((1 << rbits) <= N) ++rbits;
    int* sort_n = c.ints + IDX_RSORTN;
    cudaMemsetAsync(sort_n, 0, sizeof(int), c.s);
    k_region_keys<<<g2, 256, 0, c.s>>>(a, c.rootof, rcnt, rbits, (uint32_t*)c.listA, (uint32_t*)c.listB, nvalid,
                                       nsmall, sort_n);
    const int where = radix_sort((uint32_t*)c.listA, (uint32_t*)c.listB, (uint32_t*)c.raA, (uint32_t*)c.raB,
                                 sort_n, 2 * N, rbits + 1, c.tmp, c.scan, c.s);
    const uint32_t* rk = (const uint32_t*)(where ? c.raA : c.listA);
    const uint32_t* rv = (const uint32_t*)(where ? c.raB : c.listB);
    uint32_t* flags = (uint32_t*)c.rbA;
    uint32_t* pos = (uint32_t*)c.rbB;
    uint32_t* total = (uint32_t*)(c.ints + IDX_TMP0);
    k_class_flags<<<g2, 256, 0, c.s>>>(rk, nvalid, 0, flags);
    scan_u32(flags, pos, nvalid, 2 * N, true, c.scan, total, c.s);
    k_class_scatter<<<g2, 256, 0, c.s>>>(flags, pos, nvalid, c.cls_start, total, c.ints + IDX_NCLS);
    int* wb_lo = c.rbA;     // buckets (at most 2N / RG_SMALL): the flag/scan buffers are free again
    int* wb_hi = c.rbB;
    const int nb = cdiv(2 * N, RG_SMALL);
    k_fill_int_f<<<cdiv(nb, 256), 256, 0, c.s>>>(wb_lo, nb, INT_MAX);
    cudaMemsetAsync(wb_hi, 0, sizeof(int) * (size_t)nb, c.s);
    k_region_buckets<<<g1, 256, 0, c.s>>>(a, nvalid, nsmall, wb_lo, wb_hi, nsmall_regions);
    k_region_init<<<g1, 256, 0, c.s>>>(a, c.parent, c.csize, c.intw, c.best, c.best2, c.minid, c.rootof, c.in_tree);
    int* ticket = c.ints + IDX_TMP2;
    cudaMemsetAsync(ticket, 0, sizeof(int), c.s);
    static int rg_per_sm = 0;
    if (rg_per_sm == 0) {
        cudaFuncSetAttribute(k_fh_regions, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)regions_smem());
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&rg_per_sm, k_fh_regions, RG_THREADS, regions_smem());
        if (rg_per_sm < 1) rg_per_sm = 1;
    }
    const int rg = min(rg_per_sm, c.tune.region_ctas_per_sm);
    k_fh_regions<<<c.num_sms * rg, RG_THREADS, regions_smem(), c.s>>>(a, rv, nvalid, nsmall, nsmall_regions, wb_lo,
                                                                     wb_hi, c.rootof, ticket);
}

void launch_forest(Ctx& c, int l, int hdp)
{
    const LayerDims& d = c.dim[l];
    const int N = d.N;
    ForestArgs a{};
    a.keys = c.sorted;
    a.d_n = c.ints + IDX_NEDGES;
    a.ebits = edge_bits(N);
    a.W = d.W;
    a.N = N;
    a.pixset = hdp ? c.pixset : nullptr;
    a.canon = hdp ? c.canon[l] : nullptr;
    a.table = hdp ? c.table[l] : nullptr;
    a.full_mask = c.full_mask + (size_t)l * HDP_WORDS;
    a.parent = c.parent;
    a.size = c.csize;
    a.intw = c.intw;
    a.best = c.best;
    a.best2 = c.best2;
    a.in_tree = c.in_tree;
    a.listA = c.listA; a.listB = c.listB;
    a.raA = c.raA; a.rbA = c.rbA; a.raB = c.raB; a.rbB = c.rbB;
    a.hooked = c.hooked;
    a.ctr = c.ints + IDX_CTR0;
    a.risky = c.ints + IDX_RISKY;
    a.cls_start = c.cls_start;
    a.d_ncls = c.ints + IDX_NCLS;
    a.kq = (long long)c.p.st_k << (2 * l);
    a.T = c.T;
    a.bnum = c.p.beta_num;
    a.bden = c.p.beta_den;
    a.engine = c.ints + IDX_ENGINE;
    a.st = c.st;
    a.stats = c.ints + IDX_DRROUNDS;

    k_forest_start<<<cdiv(N, 256), 256, 0, c.s>>>(c.parent, c.csize, c.intw, c.best, c.best2, c.minid, c.rootof,
                                                  c.in_tree, c.ints, c.st, N);

    const bool st_tree = c.p.tree == HDP_TREE_ST;
    // layers below tune.one_cta_nodes run the first pass in one CTA (windowed
    // reservations in shared memory) and the risky fallback in a single block
    const bool small = N < c.tune.one_cta_nodes;
    a.big_class = min(c.tune.big_class_edges, LW_EDGES);
    if (hdp) {
        // the reservation engine needs every TreeIntv when it may run
        int always = 0;
        // grid-stride over one wave: it returns at once unless the layer is risky
        k_T_init<<<min(cdiv(N * HDP_WORDS, 256), c.num_sms * 8), 256, 0, c.s>>>(c.T, c.pixset, c.table[l], N,
                                                                               c.ints + IDX_RISKY, always);
    }
    void* args[] = {&a};
    // grids sized by the layer (one block per 4K edges at most, one wave at
    // most): small layers get cheap barriers and batched pairs share the GPU
    const int bor_blocks = cdiv(2 * N, c.tune.boruvka_edges_per_cta);
    if (!st_tree) {
        a.passes = 1;
        a.crit_first = 0;
        if (hdp && N < c.tune.region_max_nodes) {
            // a risky HDP layer: its components region by region; every
            // region kernel returns at once on the other layers, which
            // Boruvka takes
            a.risky_only = 1;
            launch_regions(c, a, d);
            a.risky_only = 0;
            cudaMemsetAsync(c.ints + IDX_CTR0, 0, 5 * sizeof(int), c.s);
            cudaMemsetAsync(c.st, 0, 2 * sizeof(unsigned), c.s);
            coop_launch((const void*)k_boruvka, FOREST_THREADS, args, c.s, 1, nullptr, 0, bor_blocks);
        } else {
            coop_launch((const void*)k_boruvka, FOREST_THREADS, args, c.s, 1, nullptr, 0, bor_blocks);
            if (hdp) launch_risky(a, c);
        }
    } else if (hdp && N < c.tune.region_max_nodes) {
        // HDP layer: regions.  Without a risky edge the first pass region by
        // region, then the linking pass by Boruvka; a risky layer takes both
        // passes region by region and Boruvka returns at once.
        a.passes = 2;
        a.crit_first = 1;
        launch_regions(c, a, d);
        cudaMemsetAsync(c.ints + IDX_CTR0, 0, 5 * sizeof(int), c.s);
        cudaMemsetAsync(c.st, 0, 2 * sizeof(unsigned), c.s);
        coop_launch((const void*)k_boruvka, FOREST_THREADS, args, c.s, 1, nullptr, 0, bor_blocks);
    } else if (!small) {
        // first pass by weight classes and windows, then the linking pass by Boruvka
        uint32_t* flags = c.sorted == c.keys0 ? c.keys1 : c.keys0;
        uint32_t* pos = (uint32_t*)c.listA;
        uint32_t* total = (uint32_t*)(c.ints + IDX_TMP0);
        k_class_flags<<<cdiv(2 * N, 256), 256, 0, c.s>>>(c.sorted, c.ints + IDX_NEDGES, a.ebits, flags);
        scan_u32(flags, pos, c.ints + IDX_NEDGES, 2 * N, true, c.scan, total, c.s);
        k_class_scatter<<<cdiv(2 * N, 256), 256, 0, c.s>>>(flags, pos, c.ints + IDX_NEDGES, c.cls_start, total,
                                                           c.ints + IDX_NCLS);
        static bool configured = false;
        if (!configured) {
            cudaFuncSetAttribute(k_fh_hybrid, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(LocalWin));
            configured = true;
        }
        void* hy_args[] = {&a, &c.rootof};
        coop_launch((const void*)k_fh_hybrid, LW_THREADS, hy_args, c.s, 1, nullptr, sizeof(LocalWin),
                    cdiv(2 * N, 2 * c.tune.boruvka_edges_per_cta));
        cudaMemsetAsync(c.ints + IDX_CTR0, 0, 3 * sizeof(int), c.s);
        cudaMemsetAsync(c.st, 0, 2 * sizeof(unsigned), c.s);
        a.passes = 2;
        a.crit_first = 1;
        coop_launch((const void*)k_boruvka, FOREST_THREADS, args, c.s, 1, nullptr, 0, bor_blocks);
        if (hdp) launch_risky(a, c);
    } else {
        // small layer: the windowed first pass in shared memory, then the
        // linking pass by Boruvka; with risky edges both return at once and
        // k_fh_risky runs both passes
        static bool configured = false;
        if (!configured) {
            cudaFuncSetAttribute(k_fh_local, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(LocalWin));
            configured = true;
        }
        k_fh_local<<<1, LW_THREADS, sizeof(LocalWin), c.s>>>(a, c.rootof);
        cudaMemsetAsync(c.ints + IDX_CTR0, 0, 3 * sizeof(int), c.s);
        cudaMemsetAsync(c.st, 0, 2 * sizeof(unsigned), c.s);
        coop_launch((const void*)k_boruvka, FOREST_THREADS, args, c.s, 1, nullptr, 0, bor_blocks);
        a.passes = 2;
        a.crit_first = 1;
        if (hdp) launch_risky(a, c);   // risky: both passes, windowed, in one CTA
    }
    k_flatten<<<cdiv(N, 256), 256, 0, c.s>>>(c.parent, c.rootof, c.minid, N);
    k_finish_roots<<<cdiv(N, 256), 256, 0, c.s>>>(c.rootof, c.minid, c.dtroot, c.T, hdp ? c.pixset : nullptr,
                                                  hdp ? c.table[l] : nullptr, a.full_mask, c.ints + IDX_ENGINE, N);
    k_adj<<<cdiv(N, 256), 256, 0, c.s>>>(c.in_tree, d.W, d.H, c.adj);
}
