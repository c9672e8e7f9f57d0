// Orders of the forest.
//
// Breadth-first order (the reading used for the paper's trees: each tree is
// rooted at its smallest pixel id; roots by increasing id, then depth by
// depth with a node's children by increasing id after those of earlier
// nodes).  It equals the depth-ordered (stable) version of the depth-first
// preorder that visits children by increasing id and trees by root id.
//
// Aggregation layout: heavy paths (each node continues with its child of
// largest subtree) are contiguous in the heavy-first preorder; nodes are
// grouped by light depth (number of light edges above them) and row width,
// so every pass over a light level is a set of independent affine scans
// along contiguous rows.
//
// Both orders come from one Euler tour of every tree: list ranking by pointer
// jumping gives each arc's distance to the tour end; from it parents, subtree
// sizes and tour positions; one prefix sum over the tour of (+child values at
// the entering arc, -child values at the leaving arc) gives depth, both
// preorders and the light depth of every node.
#include "hdp_impl.cuh"


__device__ __forceinline__ int nb_of(int v, int k, int W)
{
    return k == 0 ? v - W : k == 1 ? v - 1 : k == 2 ? v + 1 : v + W;
}
__device__ __forceinline__ int arc_index(const uint32_t* aoff, const uint8_t* adj, int v, int k)
{
    return (int)aoff[v] + __popc((unsigned)adj[v] & ((1u << k) - 1u));
}
__device__ __forceinline__ int first_dir(unsigned m) { return __ffs(m) - 1; }


__global__ void k_arc_count(const uint8_t* adj, int N, uint32_t* cnt)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < N) cnt[v] = __popc((unsigned)adj[v]);
}

// Splitters of the list ranking: every tour head, and the arcs whose hashed
// index (Fibonacci hashing) has its top lg bits zero, one arc in 2^lg on
// average.  A head is never a successor, so "the next arc is a splitter" is
// the hash test alone.
__device__ __forceinline__ bool lr_pick(int a, int lg) { return ((uint32_t)a * 0x9E3779B1u) >> (32 - lg) == 0u; }

// successor of arc (v -> u): leave u by the next existing direction after the
// one pointing back to v (cyclic order up, left, right, down); the arc that
// would re-enter the root's first arc ends the tour.  Splitters take a ticket:
// sid[a] is its number (-1 for other arcs) and spl lists them.
__global__ void k_tour_succ(const uint8_t* adj, const uint32_t* aoff, const int* dtroot, int N, int W, int* succ,
                            int* sid, int lg, int* nspl, int* spl)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= N) return;
    const unsigned mv = adj[v];
    const bool root = dtroot[v] == v;
    unsigned m = mv;
    while (m) {
        int k = __ffs(m) - 1;
        m &= m - 1;
        int a = arc_index(aoff, adj, v, k);
        int u = nb_of(v, k, W);
        unsigned mu = adj[u];
        int back = 3 - k, d = back;
        for (int t = 1; t <= 4; ++t) {
            d = (back + t) & 3;
            if (mu & (1u << d)) break;
        }
        bool end = dtroot[u] == u && d == first_dir(mu);
        succ[a] = end ? HDP_END : arc_index(aoff, adj, u, d);
        int id = -1;
        if ((root && k == first_dir(mv)) || lr_pick(a, lg)) {
            id = grid_ticket(nspl);
            spl[id] = a;
        }
        sid[a] = id;
    }
}

// Each splitter walks its segment (up to the next splitter or the tour end),
// giving every arc its owner and its offset in the segment; the segments form
// the reduced list (rs: next segment, rv: length) that pointer jumping ranks.
__global__ void k_lr_walk(const int* __restrict__ succ, const int* __restrict__ sid, const int* __restrict__ spl,
                          const int* nspl, int lg, int limit, int* owner, int* offs, int* rs, int* rv, DevStatus* st)
{
    const int n = *nspl;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        int cur = spl[j], off = 0, nxt = HDP_END;
        for (int it = 0; it <= limit; ++it) {
            owner[cur] = j;
            offs[cur] = off++;
            nxt = succ[cur];
            if (nxt == HDP_END || lr_pick(nxt, lg)) break;
            if (it == limit) {   // longer than the whole arc list: not a tour
                dev_fail(st, DEV_BAD_INPUT, 50);
                nxt = HDP_END;
                break;
            }
            cur = nxt;
        }
        rs[j] = nxt == HDP_END ? HDP_END : sid[nxt];
        rv[j] = off;
    }
}

// distance of arc x to its tour end, from its segment's rank and its offset
__device__ __forceinline__ int tour_rank(const int* R, const int* owner, const int* offs, int x)
{
    return R[owner[x]] - offs[x];
}

// Wyllie pointer jumping: val = number of arcs from the arc to its tour end.
// ctr[0..2] are per-iteration "still jumping" flags.
__global__ void k_rank(int* succ, int* val, int* succ2, int* val2, const int* d_narcs, int* ctr, DevStatus* st)
{
    const int n = *d_narcs;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    int *s0 = succ, *v0 = val, *s1 = succ2, *v1 = val2;
    for (int it = 0; it < 40; ++it) {
        if (tid == 0) ctr[(it + 1) % 3] = 0;
        int changed = 0;
        for (int a = tid; a < n; a += nth) {
            int s = __ldcg(s0 + a);
            int v = __ldcg(v0 + a);
            if (s != HDP_END) {
                v += __ldcg(v0 + s);
                s = __ldcg(s0 + s);
                changed |= s != HDP_END;
            }
            __stcg(v1 + a, v);
            __stcg(s1 + a, s);
        }
        if (__any_sync(0xffffffffu, changed) && (threadIdx.x & 31) == 0) atomicOr(ctr + it % 3, 1);
        if (!grid_sync(st, gridDim.x)) return;
        int* t = s0; s0 = s1; s1 = t;
        t = v0; v0 = v1; v1 = t;
        if (__ldcg(ctr + it % 3) == 0) break;
    }
    if (v0 != val)
        for (int a = tid; a < n; a += nth) val[a] = __ldcg(v0 + a);
}

// The same pointer jumping in one block, for short lists: the lists live in
// shared memory when they fit (RANK_SMALL entries), else in the caller's
// global scratch (s2, v2), and every round ends with a block barrier instead
// of a grid barrier.
#define RANK_SMALL 8192
__global__ void __launch_bounds__(1024) k_rank_small(int* succ, int* val, int* succ2, int* val2, const int* d_n)
{
    extern __shared__ int rk_sm[];
    const int n = *d_n;
    const bool in_smem = n <= RANK_SMALL;
    int *s0 = succ, *v0 = val, *s1 = succ2, *v1 = val2;
    if (in_smem) {
        s0 = rk_sm;
        v0 = rk_sm + RANK_SMALL;
        s1 = rk_sm + 2 * RANK_SMALL;
        v1 = rk_sm + 3 * RANK_SMALL;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            s0[i] = succ[i];
            v0[i] = val[i];
        }
        __syncthreads();
    }
    for (int it = 0; it < 40; ++it) {
        int changed = 0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            int sc = s0[i], v = v0[i];
            if (sc != HDP_END) {
                v += v0[sc];
                sc = s0[sc];
                changed |= sc != HDP_END;
            }
            s1[i] = sc;
            v1[i] = v;
        }
        const int any = __syncthreads_or(changed);
        int* t = s0; s0 = s1; s1 = t;
        t = v0; v0 = v1; v1 = t;
        if (!any) break;
    }
    if (v0 != val)
        for (int i = threadIdx.x; i < n; i += blockDim.x) val[i] = v0[i];
}

// parent = the neighbour whose arc into v comes first in the tour; subtree size
// and tour positions of the entering (down) and leaving (up) arcs
__global__ void k_orient(const uint8_t* adj, const uint32_t* aoff, const int* dtroot, const int* R, const int* owner, const int* offs, int N,
                         int W,
                         int* par, int* pdir, int* sub, int* tpos_down, int* tpos_up, uint32_t* root_tl,
                         uint32_t* root_sz)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= N) return;
    int r = dtroot[v];
    unsigned mr = adj[r];
    int tl = mr ? tour_rank(R, owner, offs, arc_index(aoff, adj, r, first_dir(mr))) : 0;
    if (r == v) {
        par[v] = -1;
        pdir[v] = -1;
        sub[v] = tl / 2 + 1;
        root_tl[v] = tl;
        root_sz[v] = tl / 2 + 1;
        return;
    }
    root_tl[v] = 0;
    root_sz[v] = 0;
    unsigned m = adj[v];
    while (m) {
        int k = __ffs(m) - 1;
        m &= m - 1;
        int u = nb_of(v, k, W);
        int up = arc_index(aoff, adj, v, k);          // v -> u
        int dn = arc_index(aoff, adj, u, 3 - k);      // u -> v
        const int vd = tour_rank(R, owner, offs, dn), vu = tour_rank(R, owner, offs, up);
        if (vd > vu) {
            par[v] = u;
            pdir[v] = k;
            sub[v] = (vd - vu + 1) / 2;
            tpos_down[v] = tl - vd;
            tpos_up[v] = tl - vu;
        }
    }
}

// children values (1, off2, off3, light) written by the parent: off2 follows
// increasing id, off3 places the heavy child (largest subtree, lowest id on
// ties) first
__global__ void k_children(const uint8_t* adj, const int* pdir, const int* sub, int N, int W, I4* vals4, int* hdir)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= N) return;
    unsigned m = adj[v];
    if (pdir[v] >= 0) m &= ~(1u << pdir[v]);
    int hk = -1, hs = -1;
    for (unsigned t = m; t; t &= t - 1) {
        int k = __ffs(t) - 1;
        int s = sub[nb_of(v, k, W)];
        if (s > hs) { hs = s; hk = k; }
    }
    hdir[v] = hk;
    int acc2 = 0, acc3 = hs > 0 ? hs : 0;
    for (unsigned t = m; t; t &= t - 1) {
        int k = __ffs(t) - 1;
        int c = nb_of(v, k, W);
        int s = sub[c];
        int off2 = 1 + acc2;
        acc2 += s;
        int off3, li;
        if (k == hk) { off3 = 1; li = 0; }
        else { off3 = 1 + acc3; acc3 += s; li = 1; }
        vals4[c] = I4{1, off2, off3, li};
    }
}

__global__ void k_tour_fill(const int* dtroot, const int* tpos_down, const int* tpos_up, const uint32_t* tbase,
                            const I4* vals4, int N, const int* d_narcs, I4* tour, DevStatus* st)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= N) return;
    int r = dtroot[v];
    if (r == v) return;
    I4 x = vals4[v];
    long long a = (long long)tbase[r] + tpos_down[v], b = (long long)tbase[r] + tpos_up[v];
    const int n = *d_narcs;
    if (a < 0 || a >= n || b < 0 || b >= n) { dev_fail(st, DEV_BAD_INPUT, 41); return; }
    tour[a] = x;
    tour[b] = I4{-x.x, -x.y, -x.z, -x.w};
}

__global__ void k_keys(const int* dtroot, const int* tpos_down, const uint32_t* tbase, const uint32_t* nbase,
                       const I4* S, int N, int* depth, int* pre2, int* pre3, int* light, int* ntrees)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= N) return;
    int r = dtroot[v];
    if (r == v) {
        depth[v] = 0;
        pre2[v] = pre3[v] = (int)nbase[v];
        light[v] = 0;
        atomicAdd(ntrees, 1);
        return;
    }
    I4 s = S[tbase[r] + tpos_down[v]];
    depth[v] = s.x;
    pre2[v] = (int)nbase[r] + s.y;
    pre3[v] = (int)nbase[r] + s.z;
    light[v] = s.w;
}

__global__ void k_scatter_bfs(const int* pre2, const int* depth, int N, uint32_t* ka, uint32_t* va, DevStatus* st)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= N) return;
    if (pre2[v] < 0 || pre2[v] >= N || depth[v] < 0 || depth[v] >= N) { dev_fail(st, DEV_BAD_INPUT, 42); return; }
    ka[pre2[v]] = (uint32_t)depth[v];
    va[pre2[v]] = (uint32_t)v;
}

__global__ void k_scatter_layout(const int* pre3, const int* light, const int* rootof, const uint32_t* T, int N,
                                 uint32_t* ka, uint32_t* va, DevStatus* st)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= N) return;
    int k = set_popc(T + (size_t)rootof[v] * HDP_WORDS);
    int q = (k + 3) >> 2;            // float4 columns, 1..64
    int lv = light[v];
    if (lv < 0 || lv >= MAX_LIGHT_LEVELS || q < 1 || q > 64 || pre3[v] < 0 || pre3[v] >= N) {
        dev_fail(st, DEV_BAD_INPUT, 40);
        return;
    }
    ka[pre3[v]] = ((uint32_t)lv << 6) | (uint32_t)(q - 1);
    va[pre3[v]] = (uint32_t)v;
}

__device__ __forceinline__ int edge_to_parent(int v, int k, int W)
{
    return k == 0 ? 2 * (v - W) + 1 : k == 1 ? 2 * (v - 1) : k == 2 ? 2 * v : 2 * v + 1;
}

// row metadata, part 1
__global__ void k_rows(const uint32_t* keys_sorted, const int* lay, const int* rootof, const int* par, const int* pdir,
                       const int* weights, const I4* vals4, int N, int W, float inv_scale, int* rowof, int* kp,
                       int* rdt, float* rs, uint32_t* lccnt, const int* hdir, const uint8_t* adj)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int v = lay[i];
    rowof[v] = i;
    kp[i] = 4 * (int)((keys_sorted[i] & 63u) + 1);
    rdt[i] = rootof[v];
    float s = 0.f;
    if (par[v] >= 0) s = expf(-(float)weights[edge_to_parent(v, pdir[v], W)] * inv_scale);
    bool top = par[v] < 0 || vals4[v].w;   // root or light child: first row of a heavy path
    rs[i] = top ? -s : s;   // the sign bit marks path tops (roots store -0)
    if (par[v] < 0) rs[i] = -0.0f;
    unsigned m = adj[v];
    if (pdir[v] >= 0) m &= ~(1u << pdir[v]);
    lccnt[i] = __popc(m) - (hdir[v] >= 0 ? 1 : 0);
}

// row metadata, part 2: parent rows and light-children rows
__global__ void k_rows2(const int* lay, const int* rowof, const int* par, const int* pdir, const int* hdir,
                        const uint8_t* adj, const uint32_t* lcoff, int N, int W, int* prow, int* lcrow)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int v = lay[i];
    prow[i] = par[v] >= 0 ? rowof[par[v]] : -1;
    unsigned m = adj[v];
    if (pdir[v] >= 0) m &= ~(1u << pdir[v]);
    if (hdir[v] >= 0) m &= ~(1u << hdir[v]);
    uint32_t o = lcoff[i], o1 = lcoff[i] + (uint32_t)__popc(m);
    if (o1 > (uint32_t)N) return;
    for (; m; m &= m - 1) lcrow[o++] = rowof[nb_of(v, __ffs(m) - 1, W)];
}

// rows are sorted by key, so each (level, width) run starts where the key changes
__global__ void k_runstart(const uint32_t* keys_sorted, int N, int* runstart)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N && (i == 0 || keys_sorted[i] != keys_sorted[i - 1])) runstart[keys_sorted[i]] = i;
}

// a tile starts at every (light level, width) run start and every
// tile_rows(width) rows after it; tiles may split heavy paths
__global__ void k_tile_flags(const uint32_t* keys_sorted, const int* runstart, int N, int extra, int tf, uint32_t* flag)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    uint32_t key = keys_sorted[i];
    int kp = 4 * (int)((key & 63u) + 1);
    flag[i] = ((i - runstart[key]) % tile_rows_of(kp, extra, tf)) == 0;
}

__global__ void k_tile_fill(const uint32_t* flag, const uint32_t* tid, const uint32_t* keys_sorted, int N, int* tbeg,
                            int* lvl_first, int* lvl_count, int max_tiles, DevStatus* st)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N || !flag[i]) return;
    int t = (int)tid[i];
    if (t >= max_tiles) { dev_fail(st, DEV_BAD_INPUT, 43); return; }
    tbeg[t] = i;
    int lv = (int)(keys_sorted[i] >> 6);
    if (lv >= MAX_LIGHT_LEVELS) return;
    min_by_key(lvl_first, lv, t);   // tiles come sorted by level: one atomic per level and warp
    count_by_key(lvl_count, lv);
}


// The stage's counters and tables in one launch (none is touched before its
// use below): the scan lengths N and N + 1 (with the slots after them, the
// splitter count among them, zeroed), the tree count, slot N of both
// ping-pong key buffers (the light-child counts' total), the run starts and
// the per-level tile tables.
__global__ void k_order_init(int* ints, int N, uint32_t* ka, uint32_t* kb, int* runstart, int* lvl_first,
                             int* lvl_count)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        ints[IDX_N] = N;
        ints[IDX_N + 1] = 0;
        ints[IDX_TMP1] = N + 1;
        ints[IDX_TMP1 + 1] = 0;
        ints[IDX_NTREES] = 0;
        ka[N] = 0u;
        kb[N] = 0u;
    }
    if (i < 2048) runstart[i] = INT_MAX;
    if (i < MAX_LIGHT_LEVELS) {
        lvl_first[i] = INT_MAX;
        lvl_count[i] = 0;
    }
}

void launch_order(Ctx& c, int l)
{
    const LayerDims& d = c.dim[l];
    const int N = d.N;
    cudaStream_t s = c.s;
    const int g = cdiv(N, 256);
    int* dN = c.ints + IDX_N;
    static_assert(MAX_LIGHT_LEVELS <= 2048, "one launch covers the tables");
    static_assert(IDX_TMP1 + 1 == IDX_TMP2, "the splitter count follows the second scan length");
    k_order_init<<<cdiv(2048, 256), 256, 0, s>>>(c.ints, N, c.ka, c.kb, c.runstart, c.lvl_first, c.lvl_count);

    // arcs and their successors
    uint32_t* cnt = c.ka;
    k_arc_count<<<g, 256, 0, s>>>(c.adj, N, cnt);
    scan_u32(cnt, c.aoff, dN, N, true, c.scan, (uint32_t*)(c.ints + IDX_NARCS), s);
    // list ranking by splitters: about one arc in 2^lg starts a segment
    // (layers of 64K..128K nodes take 1 in 32, so that their segment list is
    // short enough for the one-block ranking)
    const int lg = N >= (1 << 19) ? 5 : N >= (1 << 17) ? 4 : N >= (1 << 16) ? 5 : 3;
    int* nspl = c.ints + IDX_TMP2;   // zeroed by k_order_init
    int* sid = c.val;
    int* spl = c.succ2;
    int *owner = c.listA, *offs = c.listB, *rs = c.raA, *rv = c.rbA, *rs2 = c.raB, *rv2 = c.rbB;
    k_tour_succ<<<g, 256, 0, s>>>(c.adj, c.aoff, c.dtroot, N, d.W, c.succ, sid, lg, nspl, spl);
    const int est = (2 * N >> lg) + 1024;   // expected segments, for the grid sizes only
    k_lr_walk<<<min(cdiv(est, 128), c.num_sms * 16), 128, 0, s>>>(c.succ, sid, spl, nspl, lg, 2 * N, owner, offs,
                                                                 rs, rv, c.st);
    if ((2 * N >> lg) <= 3 * RANK_SMALL / 4) {
        // a short list: one block, shared memory
        static bool configured = false;
        if (!configured) {
            cudaFuncSetAttribute(k_rank_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 4 * RANK_SMALL * (int)sizeof(int));
            configured = true;
        }
        k_rank_small<<<1, 1024, 4 * RANK_SMALL * sizeof(int), s>>>(rs, rv, rs2, rv2, nspl);
    } else {
        cudaMemsetAsync(c.ints + IDX_CTR0, 0, 3 * sizeof(int), s);
        cudaMemsetAsync(c.st, 0, 2 * sizeof(unsigned), s);
        int* a0 = rs; int* a1 = rv; int* a2 = rs2; int* a3 = rv2;
        const int* nar = nspl;
        int* ctr = c.ints + IDX_CTR0;
        DevStatus* st = c.st;
        void* args[] = {&a0, &a1, &a2, &a3, &nar, &ctr, &st};
        // about four segments per thread per round, at most one wave
        coop_launch((const void*)k_rank, 256, args, s, 0, nullptr, 0, cdiv(est, 256 * 4));
    }
    k_orient<<<g, 256, 0, s>>>(c.adj, c.aoff, c.dtroot, rv, owner, offs, N, d.W, c.par, c.pdir, c.sub, c.tpos_down,
                               c.tpos_up, c.ka, c.kb);
    k_children<<<g, 256, 0, s>>>(c.adj, c.pdir, c.sub, N, d.W, c.vals4, c.hdir);
    scan_u32(c.ka, c.tbase, dN, N, true, c.scan, nullptr, s);
    scan_u32(c.kb, c.nbase, dN, N, true, c.scan, nullptr, s);
    k_tour_fill<<<g, 256, 0, s>>>(c.dtroot, c.tpos_down, c.tpos_up, c.tbase, c.vals4, N, c.ints + IDX_NARCS, c.tour,
                                  c.st);
    scan_i4_inclusive(c.tour, c.tour, c.ints + IDX_NARCS, 2 * N, c.scan4, s);
    k_keys<<<g, 256, 0, s>>>(c.dtroot, c.tpos_down, c.tbase, c.nbase, c.tour, N, c.depth, c.pre2, c.pre3, c.light,
                             c.ints + IDX_NTREES);

    // (the breadth-first order itself is only an output: launch_bfs, on request)

    // aggregation layout: heavy-first preorder stably sorted by (light level, width)
    k_scatter_layout<<<g, 256, 0, s>>>(c.pre3, c.light, c.rootof, c.T, N, c.ka, c.va, c.st);
    int where = radix_sort(c.ka, c.va, c.kb, c.vb, dN, N, 11, c.tmp, c.scan, s);
    uint32_t* ksorted = where ? c.kb : c.ka;
    cudaMemcpyAsync(c.lay, where ? c.vb : c.va, sizeof(int) * N, cudaMemcpyDeviceToDevice, s);
    uint32_t* lccnt = where ? c.ka : c.kb;   // the free ping-pong buffer
    float inv_scale = 1.0f / (c.p.gamma * (float)(1 << (2 * l)));
    k_rows<<<g, 256, 0, s>>>(ksorted, c.lay, c.rootof, c.par, c.pdir, c.weights, c.vals4, N, d.W, inv_scale, c.rowof,
                             c.kp, c.rdt, c.rs, lccnt, c.hdir, c.adj);
    // N + 1 entries so that lcoff[N] holds the total
    int* dN1 = c.ints + IDX_TMP1;   // N + 1, and lccnt[N] = 0, from k_order_init
    scan_u32(lccnt, c.lcoff, dN1, N + 1, true, c.scan, (uint32_t*)(c.ints + IDX_NLC), s);
    k_rows2<<<g, 256, 0, s>>>(c.lay, c.rowof, c.par, c.pdir, c.hdir, c.adj, c.lcoff, N, d.W, c.prow, c.lcrow);
    scan_u32((const uint32_t*)c.kp, c.roff, dN, N, true, c.scan, (uint32_t*)(c.ints + IDX_K), s);

    // tiles
    k_runstart<<<g, 256, 0, s>>>(ksorted, N, c.runstart);
    c.layer_tf[l] = layer_tile_floats(c, l);   // the aggregation of this layout uses the same size
    k_tile_flags<<<g, 256, 0, s>>>(ksorted, c.runstart, N, c.p.storage == HDP_STORE_FP16 ? 4 : 0, c.layer_tf[l],
                                   c.ustart_flag);
    scan_u32(c.ustart_flag, c.uid, dN, N, true, c.scan, (uint32_t*)(c.ints + IDX_NUNITS), s);
    k_tile_fill<<<g, 256, 0, s>>>(c.ustart_flag, c.uid, ksorted, N, c.ubeg, c.lvl_first, c.lvl_count, (int)c.max_tiles,
                                  c.st);

}

// The breadth-first order of layer l (R15): the preorder with children by id,
// stably sorted by depth.  The aggregation does not need it (it walks the
// heavy-path layout), so it is built only when asked for, from the depths and
// preorder that stay in place while layer l's tree is the current one.
void launch_bfs(Ctx& c, int l)
{
    const int N = c.dim[l].N;
    cudaStream_t s = c.s;
    k_scatter_bfs<<<cdiv(N, 256), 256, 0, s>>>(c.pre2, c.depth, N, c.ka, c.va, c.st);
    int dbits = 1;
    while ((1 << dbits) < N) ++dbits;
    const int where = radix_sort(c.ka, c.va, c.kb, c.vb, c.ints + IDX_N, N, dbits, c.tmp, c.scan, s);
    cudaMemcpyAsync(c.bfs, where ? c.vb : c.va, sizeof(int) * N, cudaMemcpyDeviceToDevice, s);
}
