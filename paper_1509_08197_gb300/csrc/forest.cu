// HDP forest construction (Sec. 3.2): Kruskal semantics over the strict
// (w, edge id) order with Rule 2, DT-Rule 2 (Eq. DTrules) and, for the
// segment tree, the merge criterion w <= Int(C) + k/|C|.
//
// Three engines produce the sequential-Kruskal result exactly:
//  * Boruvka over the sorted list (the list index is the strict order) when
//    no state-dependent rule is active: plain MST, full-range layers, and HDP
//    layers with no "risky" edge.  Without risky edges every tree keeps the
//    set of its pixels (merges only join equal sets), so DT-Rule 2 reduces to
//    "same PixelIntv" and the result is the minimum spanning forest of the
//    same-set subgraph.
//  * The segment-tree first pass one weight class at a time: inside a class
//    every edge has the same w, and a tree's criterion cannot change before it
//    merges (and a merge sets Int = w, which passes for the rest of the
//    class), so the class reduces to a Boruvka by edge id among the edges
//    whose two trees pass at the start of the class.
//  * Deterministic reservations (general fallback): each round takes a window
//    of the earliest unresolved edges; an edge that holds the reservation of
//    both its trees is resolved on their current state, exactly as the
//    sequential algorithm would.
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
    int *win, *wtmp, *wra, *wrb, *wst;
    int WIN;
    int passes, crit_first;
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

__device__ __forceinline__ void append(const ForestArgs& a, int which, int idx, int ra, int rb)
{
    int pos = atomicAdd(a.ctr + which, 1);
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
                if (record_hooks) hk[atomicAdd(a.ctr + 2 + par, 1)] = ra;
            }
            if (bb == idx && !(ba == idx && rb < ra)) {
                __stcg(a.parent + rb, ra);
                if (record_hooks) hk[atomicAdd(a.ctr + 2 + par, 1)] = rb;
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
            }
        }
        for (int j = tid; j < m; j += nth) {
            __stcg(best + RA[j], INT_MAX);
            __stcg(best + RB[j], INT_MAX);
            int idx = L[j], e, w, p, q;
            decode(a.keys[idx], a.ebits, a.W, e, w, p, q);
            int ra = uf_find(a.parent, p), rb = uf_find(a.parent, q);
            if (ra != rb) {
                atomicMin(bnext + ra, idx);
                atomicMin(bnext + rb, idx);
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
    if (a.risky && __ldcg(a.risky)) return;
    const int n = *a.d_n;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    if (tid == 0) *a.engine = 1;
    for (int idx = tid; idx < n; idx += nth) {
        int e, w, p, q;
        decode(a.keys[idx], a.ebits, a.W, e, w, p, q);
        if (!same_set(a, p, q)) continue;
        int ra = uf_find(a.parent, p), rb = uf_find(a.parent, q);
        if (ra != rb) {
            atomicMin(a.best + ra, idx);
            atomicMin(a.best + rb, idx);
            append(a, 0, idx, ra, rb);
        }
    }
    if (!grid_sync(a.st, gridDim.x)) return;
    int cur = 0, par = 0;
    boruvka_rounds(a, cur, par, false);
}

// Segment-tree first pass, one weight class at a time (see file comment).
__global__ void k_fh(ForestArgs a)
{
    if (a.risky && __ldcg(a.risky)) return;
    const int n = *a.d_n, ncls = *a.d_ncls;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    int cur = 0, par = 0;
    for (int c = 0; c < ncls; ++c) {
        const int s = a.cls_start[c];
        const int e_end = c + 1 < ncls ? a.cls_start[c + 1] : n;
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
            atomicMin(best_of(a, par) + ra, idx);
            atomicMin(best_of(a, par) + rb, idx);
            append(a, cur, idx, ra, rb);
        }
        if (!grid_sync(a.st, gridDim.x)) return;
        if (__ldcg(a.ctr + cur) == 0) continue;
        // sizes and Int = w of the trees merged in this class are folded inside
        // the rounds; a tree's criterion is only read at the start of a class
        if (!boruvka_rounds(a, cur, par, true, (int)w)) return;
    }
}

__device__ int block_excl_sum(int v, int* smem, int* total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    int incl = v;
    for (int d = 1; d < 32; d <<= 1) {
        int o = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += o;
    }
    if (lane == 31) smem[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int x = lane < nw ? smem[lane] : 0;
        int xi = x;
        for (int d = 1; d < 32; d <<= 1) {
            int o = __shfl_up_sync(0xffffffffu, xi, d);
            if (lane >= d) xi += o;
        }
        if (lane < nw) smem[lane] = xi - x;
        if (lane == nw - 1) smem[32] = xi;
    }
    __syncthreads();
    int r = smem[warp] + incl - v;
    *total = smem[32];
    __syncthreads();
    return r;
}

// single block: plain (L1-cached) accesses; the block's own writes are visible
// to it after __syncthreads.  Grid: through L2, which all SMs share.
template <bool SINGLE> __device__ __forceinline__ int ldv(const int* p) { return SINGLE ? *p : __ldcg(p); }
template <bool SINGLE> __device__ __forceinline__ uint32_t ldv(const uint32_t* p) { return SINGLE ? *p : __ldcg(p); }
template <bool SINGLE> __device__ __forceinline__ void stv(int* p, int v) { if (SINGLE) *p = v; else __stcg(p, v); }
template <bool SINGLE> __device__ __forceinline__ void stv(uint32_t* p, uint32_t v) { if (SINGLE) *p = v; else __stcg(p, v); }

// union-find root for one block (plain loads: the block's own writes are
// visible to it after __syncthreads)
template <bool SINGLE>
__device__ __forceinline__ int uf_find_t(int* parent, int v)
{
    if (!SINGLE) return uf_find(parent, v);
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

// Deterministic reservations over windows of the sorted list.  ctr[3] = window
// size, ctr[4] = next fresh list index.  best[] holds window positions.
template <bool SINGLE>
__global__ void k_dr(ForestArgs a, int only_if_risky)
{
    __shared__ int smem[33];
    if (only_if_risky && !ldv<SINGLE>(a.risky)) return;
    const unsigned nb = gridDim.x;
    const int n = *a.d_n;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    const bool full = a.pixset == nullptr;
    if (tid == 0) *a.engine = 2;
    for (int pass = 0; pass < a.passes; ++pass) {
        const bool crit = a.crit_first && pass == 0;
        if (tid == 0) { a.ctr[3] = 0; a.ctr[4] = 0; }
        if (!grid_sync(a.st, nb)) return;
        for (long long round = 0;; ++round) {
            if (round > (1LL << 30)) { dev_fail(a.st, DEV_TIMEOUT, 30); return; }
            if (blockIdx.x == 0) {
                int k = ldv<SINGLE>(a.ctr + 3), nx = ldv<SINGLE>(a.ctr + 4);
                int add = min(a.WIN - k, n - nx);
                for (int t = threadIdx.x; t < add; t += blockDim.x) a.win[k + t] = nx + t;
                __syncthreads();
                if (threadIdx.x == 0) { a.ctr[3] = k + add; a.ctr[4] = nx + add; }
            }
            if (!grid_sync(a.st, nb)) return;
            const int wc = ldv<SINGLE>(a.ctr + 3);
            if (wc == 0) break;
            for (int i = tid; i < wc; i += nth) {
                int idx = ldv<SINGLE>(a.win + i), e, w, p, q;
                decode(a.keys[idx], a.ebits, a.W, e, w, p, q);
                int ra = uf_find_t<SINGLE>(a.parent, p), rb = uf_find_t<SINGLE>(a.parent, q);
                a.wra[i] = ra;
                a.wrb[i] = rb;
                if (ra != rb) {
                    atomicMin(a.best + ra, i);
                    atomicMin(a.best + rb, i);
                }
            }
            if (!grid_sync(a.st, nb)) return;
            for (int i = tid; i < wc; i += nth) {
                int ra = ldv<SINGLE>(a.wra + i), rb = ldv<SINGLE>(a.wrb + i);
                int done = 1;
                if (ra != rb) {
                    if (ldv<SINGLE>(a.best + ra) == i && ldv<SINGLE>(a.best + rb) == i) {
                        int idx = ldv<SINGLE>(a.win + i), e, w, p, q;
                        decode(a.keys[idx], a.ebits, a.W, e, w, p, q);
                        bool ok = true;
                        if (!full) {
                            int inter = 0, uni = 0;
#pragma unroll
                            for (int k = 0; k < HDP_WORDS; ++k) {
                                uint32_t ta = ldv<SINGLE>(a.T + (size_t)ra * HDP_WORDS + k);
                                uint32_t tb = ldv<SINGLE>(a.T + (size_t)rb * HDP_WORDS + k);
                                inter += __popc(ta & tb);
                                uni += __popc(ta | tb);
                            }
                            ok = (long long)inter * a.bden >= (long long)a.bnum * uni;   // DT-Rule 2
                        }
                        long long sa = ldv<SINGLE>(a.size + ra), sb = ldv<SINGLE>(a.size + rb);
                        if (ok && crit) {
                            long long ia = ldv<SINGLE>(a.intw + ra), ib = ldv<SINGLE>(a.intw + rb);
                            ok = (long long)w * sa <= ia * sa + a.kq && (long long)w * sb <= ib * sb + a.kq;
                        }
                        if (ok) {
                            int big = ra, small = rb;
                            if (sa < sb) { big = rb; small = ra; }
                            stv<SINGLE>(a.parent + small, big);
                            stv<SINGLE>(a.size + big, (int)(sa + sb));
                            stv<SINGLE>(a.intw + big, w);
                            if (!full) {
#pragma unroll
                                for (int k = 0; k < HDP_WORDS; ++k) {
                                    uint32_t u = ldv<SINGLE>(a.T + (size_t)ra * HDP_WORDS + k) |
                                                 ldv<SINGLE>(a.T + (size_t)rb * HDP_WORDS + k);
                                    stv<SINGLE>(a.T + (size_t)big * HDP_WORDS + k, u);
                                }
                            }
                            a.in_tree[e] = 1;
                        }
                    } else {
                        done = 0;
                    }
                }
                a.wst[i] = done;
            }
            if (!grid_sync(a.st, nb)) return;
            for (int i = tid; i < wc; i += nth) {
                int ra = ldv<SINGLE>(a.wra + i), rb = ldv<SINGLE>(a.wrb + i);
                if (ra != rb) {
                    stv<SINGLE>(a.best + ra, INT_MAX);
                    stv<SINGLE>(a.best + rb, INT_MAX);
                }
            }
            if (blockIdx.x == 0) {
                // stable compaction of the unresolved window entries
                const int per = cdiv(wc, (int)blockDim.x);
                const int b0 = threadIdx.x * per, b1 = min(wc, b0 + per);
                int cnt = 0;
                for (int i = b0; i < b1; ++i) cnt += ldv<SINGLE>(a.wst + i) == 0;
                int tot = 0;
                int off = block_excl_sum(cnt, smem, &tot);
                for (int i = b0; i < b1; ++i)
                    if (ldv<SINGLE>(a.wst + i) == 0) a.wtmp[off++] = ldv<SINGLE>(a.win + i);
                __syncthreads();
                for (int i = threadIdx.x; i < tot; i += blockDim.x) a.win[i] = a.wtmp[i];
                __syncthreads();
                if (threadIdx.x == 0) a.ctr[3] = tot;
            }
            if (!grid_sync(a.st, nb)) return;
        }
    }
}

__global__ void k_forest_init(int* parent, int* size, int* intw, int* best, int* best2, int* minid, int N)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= N) return;
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
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N * HDP_WORDS) return;
    int v = i / HDP_WORDS, k = i % HDP_WORDS;
    T[i] = table[(size_t)pixset[v] * HDP_WORDS + k];
}

__global__ void k_class_flags(const uint32_t* keys, const int* d_n, int ebits, uint32_t* flags)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= *d_n) return;
    flags[i] = i == 0 || (keys[i] >> ebits) != (keys[i - 1] >> ebits);
}

__global__ void k_class_scatter(const uint32_t* flags, const uint32_t* pos, const int* d_n, int* cls_start,
                                const uint32_t* total, int* ncls)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *ncls = (int)*total;
    if (i >= *d_n) return;
    if (flags[i] && pos[i] < (uint32_t)*d_n) cls_start[pos[i]] = i;
}

__global__ void k_flatten(int* parent, int* rootof, int* minid, int N)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= N) return;
    int r = uf_find(parent, v);
    rootof[v] = r;
    atomicMin(minid + r, v);
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
        bool maintained = pixset != nullptr && *engine == 2;
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
cudaError_t coop_launch(const void* fn, int threads, void** args, cudaStream_t s, int blocks_per_sm, int* used)
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, 0);
    if (blocks_per_sm > 0 && per > blocks_per_sm) per = blocks_per_sm;
    int blocks = per * sms;
    if (blocks < 1) blocks = 1;
    if (used) *used = blocks;
    return cudaLaunchCooperativeKernel(fn, dim3(blocks), dim3(threads), args, 0, s);
}

// layers below this size run the segment-tree passes with the reservation
// engine in a single block (many weight classes, few edges per class)
#define FH_MIN_NODES 131072
#define DR_SINGLE_BLOCK_NODES 131072

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
    a.win = c.win; a.wtmp = c.wtmp; a.wra = c.wra; a.wrb = c.wrb; a.wst = c.wst;
    a.engine = c.ints + IDX_ENGINE;
    a.st = c.st;

    k_forest_init<<<cdiv(N, 256), 256, 0, c.s>>>(c.parent, c.csize, c.intw, c.best, c.best2, c.minid, N);
    cudaMemsetAsync(c.in_tree, 0, 2 * (size_t)N, c.s);
    cudaMemsetAsync(c.ints + IDX_CTR0, 0, 5 * sizeof(int), c.s);
    cudaMemsetAsync(c.st, 0, 2 * sizeof(unsigned), c.s);   // barrier state (keeps err)
    cudaMemsetAsync(c.ints + IDX_ENGINE, 0, sizeof(int), c.s);

    const bool st_tree = c.p.tree == HDP_TREE_ST;
    const bool small = N < DR_SINGLE_BLOCK_NODES;
    if (hdp) {
        // the reservation engine needs every TreeIntv when it may run
        int always = st_tree && small;
        k_T_init<<<cdiv(N * HDP_WORDS, 256), 256, 0, c.s>>>(c.T, c.pixset, c.table[l], N, c.ints + IDX_RISKY, always);
    }
    void* args[] = {&a};
    int only_if_risky = 1;
    void* dr_args[] = {&a, &only_if_risky};
    const void* dr_grid = (const void*)k_dr<false>;
    if (!st_tree) {
        coop_launch((const void*)k_boruvka, FOREST_THREADS, args, c.s, 1, nullptr);
        a.passes = 1;
        a.crit_first = 0;
        a.WIN = small ? 4096 : 16384;
        if (hdp) {
            cudaMemsetAsync(c.st, 0, 2 * sizeof(unsigned), c.s);
            if (small) k_dr<true><<<1, 1024, 0, c.s>>>(a, 1);
            else coop_launch(dr_grid, FOREST_THREADS, dr_args, c.s, 1, nullptr);
        }
    } else if (!small) {
        // first pass by weight classes, then the linking pass by Boruvka
        uint32_t* flags = c.sorted == c.keys0 ? c.keys1 : c.keys0;
        uint32_t* pos = (uint32_t*)c.listA;
        uint32_t* total = (uint32_t*)(c.ints + IDX_TMP0);
        k_class_flags<<<cdiv(2 * N, 256), 256, 0, c.s>>>(c.sorted, c.ints + IDX_NEDGES, a.ebits, flags);
        scan_u32(flags, pos, c.ints + IDX_NEDGES, 2 * N, true, c.tmp, total, c.s);
        k_class_scatter<<<cdiv(2 * N, 256), 256, 0, c.s>>>(flags, pos, c.ints + IDX_NEDGES, c.cls_start, total,
                                                           c.ints + IDX_NCLS);
        coop_launch((const void*)k_fh, FOREST_THREADS, args, c.s, 1, nullptr);
        cudaMemsetAsync(c.ints + IDX_CTR0, 0, 3 * sizeof(int), c.s);
        cudaMemsetAsync(c.st, 0, 2 * sizeof(unsigned), c.s);
        coop_launch((const void*)k_boruvka, FOREST_THREADS, args, c.s, 1, nullptr);
        a.passes = 2;
        a.crit_first = 1;
        a.WIN = 16384;
        if (hdp) {
            cudaMemsetAsync(c.st, 0, 2 * sizeof(unsigned), c.s);
            coop_launch(dr_grid, FOREST_THREADS, dr_args, c.s, 1, nullptr);
        }
    } else {
        a.passes = 2;
        a.crit_first = 1;
        a.WIN = 4096;
        k_dr<true><<<1, 1024, 0, c.s>>>(a, 0);
    }
    k_flatten<<<cdiv(N, 256), 256, 0, c.s>>>(c.parent, c.rootof, c.minid, N);
    k_finish_roots<<<cdiv(N, 256), 256, 0, c.s>>>(c.rootof, c.minid, c.dtroot, c.T, hdp ? c.pixset : nullptr,
                                                  hdp ? c.table[l] : nullptr, a.full_mask, c.ints + IDX_ENGINE, N);
    k_adj<<<cdiv(N, 256), 256, 0, c.s>>>(c.in_tree, d.W, d.H, c.adj);
}
