// Non-local cost aggregation over the HDP forest and WTA (Sec. 3.3,
// Eqs. E, W, S, C) with the linear-time two-pass method of the cited MST
// work:
//   leaf to root  U(v) = E(v) + sum over children c of s_c U(c)
//   root to leaf  C(v) = s_v C(parent) + (1 - s_v^2) U(v),  C(root) = U(root)
// with s_v = exp(-w(v, parent) / gamma).  E(v, x) = M(v, x) for x in the
// TreeIntv of v's tree and is computed on the fly (never stored).
//
// Rows (one per node) are laid out by light level, width and heavy-first
// preorder, so a heavy path is a run of consecutive rows and the pass over a
// light level is an affine recurrence along rows:
//   up   x_r = a_r + m_r x_{r+1},  a_r = E_r + sum_light s_c U_c,  m_r = s_{r+1}
//   down x_r = b_r + m_r x_{r-1},  b_r = (1 - s_r^2) U_r (+ s_r C(parent) at a top)
// with m = 0 across path boundaries.  A warp owns a unit of whole paths and
// walks it in groups of rows, one row per lane group, combining rows with a
// shuffle scan of affine maps and carrying the last row into the next group.
// Light levels run one launch each (deepest first for the up pass).
#include "hdp_impl.cuh"

#define AGG_THREADS 256

struct AggArgs {
    const int4* imL;
    const int4* imR;
    int W, N, full, dl;
    CostK ck;
    const int* lay;
    const float* rs;
    const int* prow;
    const int* rdt;
    const uint32_t* T;
    const uint32_t* lcoff;
    const int* lcrow;
    const uint32_t* roff;
    const int* kp;
    const int* ubeg;
    const int* d_nunits;
    const int* lvl_first;
    const int* lvl_count;
    float* vol;
    __half* volh;
    float* nup;
    float* nd;
    int* tickets;
    int level;
    int32_t* disp;
    DevStatus* st;
};

__device__ __forceinline__ float4 f4(float a) { return make_float4(a, a, a, a); }
__device__ __forceinline__ float4 fma4(float m, float4 x, float4 a)
{
    return make_float4(fmaf(m, x.x, a.x), fmaf(m, x.y, a.y), fmaf(m, x.z, a.z), fmaf(m, x.w, a.w));
}
__device__ __forceinline__ float4 shfl_down4(float4 v, int d)
{
    return make_float4(__shfl_down_sync(0xffffffffu, v.x, d), __shfl_down_sync(0xffffffffu, v.y, d),
                       __shfl_down_sync(0xffffffffu, v.z, d), __shfl_down_sync(0xffffffffu, v.w, d));
}
__device__ __forceinline__ float4 shfl_up4(float4 v, int d)
{
    return make_float4(__shfl_up_sync(0xffffffffu, v.x, d), __shfl_up_sync(0xffffffffu, v.y, d),
                       __shfl_up_sync(0xffffffffu, v.z, d), __shfl_up_sync(0xffffffffu, v.w, d));
}
__device__ __forceinline__ float4 shfl4(float4 v, int src)
{
    return make_float4(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src),
                       __shfl_sync(0xffffffffu, v.z, src), __shfl_sync(0xffffffffu, v.w, src));
}

// label of the n-th element (0-based) of a 256-bit set, -1 if absent
__device__ __forceinline__ int nth_label(const uint32_t* m, int n)
{
#pragma unroll
    for (int w = 0; w < HDP_WORDS; ++w) {
        int c = __popc(m[w]);
        if (n < c) return 32 * w + (int)__fns(m[w], 0, n + 1);
        n -= c;
    }
    return -1;
}

struct RowInfo {
    int k;            // number of labels of the row's tree
    int lab[8];       // labels of this lane's (up to 2 x 4) slots, -1 = padding
};

__device__ __forceinline__ void row_labels(const AggArgs& a, int r, int col0, int fpl, int q, RowInfo& ri)
{
    if (a.full) {
        ri.k = a.dl + 1;
#pragma unroll
        for (int f = 0; f < 2; ++f)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                int slot = 4 * (col0 + 32 * f) + i;
                ri.lab[4 * f + i] = (f < fpl && col0 + 32 * f < q && slot < ri.k) ? slot : -1;
            }
        return;
    }
    uint32_t m[HDP_WORDS];
    const uint32_t* src = a.T + (size_t)a.rdt[r] * HDP_WORDS;
#pragma unroll
    for (int w = 0; w < HDP_WORDS; ++w) m[w] = src[w];
    int k = 0;
#pragma unroll
    for (int w = 0; w < HDP_WORDS; ++w) k += __popc(m[w]);
    ri.k = k;
#pragma unroll
    for (int f = 0; f < 2; ++f) {
        int col = col0 + 32 * f;
        bool ok = f < fpl && col < q;
        int lab = ok && 4 * col < k ? nth_label(m, 4 * col) : -1;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            ri.lab[4 * f + i] = lab;
            if (lab >= 0 && 4 * col + i + 1 < k) {
                // next set bit after lab
                int w = lab >> 5, b = lab & 31;
                int nxt = -1;
                if (b < 31) {
                    unsigned r2 = __fns(m[w], b + 1, 1);
                    if (r2 != 0xffffffffu) nxt = 32 * w + (int)r2;
                }
                for (int ww = w + 1; nxt < 0 && ww < HDP_WORDS; ++ww)
                    if (m[ww]) nxt = 32 * ww + __ffs(m[ww]) - 1;
                lab = nxt;
            } else {
                lab = -1;
            }
        }
    }
}

__device__ __forceinline__ float cost_m(int4 l, int4 r, const CostK& k)
{
    int sum = abs(l.x - r.x) + abs(l.y - r.y) + abs(l.z - r.z);
    int dg = abs(l.w - r.w);
    return (float)(k.A * min(sum, k.Tc) + k.B * min(dg, k.Tg)) * k.inv;
}

template <bool FP16>
__device__ __forceinline__ float4 load_row4(const AggArgs& a, size_t off)
{
    if (FP16) {
        const __half2* h = (const __half2*)(a.volh + off);
        float2 x = __half22float2(h[0]), y = __half22float2(h[1]);
        return make_float4(x.x, x.y, y.x, y.y);
    } else {
        return *(const float4*)(a.vol + off);
    }
}

template <bool FP16>
__device__ __forceinline__ void store_row4(const AggArgs& a, size_t off, float4 v)
{
    if (FP16) {
        __half2* h = (__half2*)(a.volh + off);
        h[0] = __floats2half2_rn(v.x, v.y);
        h[1] = __floats2half2_rn(v.z, v.w);
    } else {
        *(float4*)(a.vol + off) = v;
    }
}

struct Shape {
    int q, lpr, rpw, fpl, col0, rsub;
};
__device__ __forceinline__ Shape unit_shape(int kp)
{
    Shape s;
    s.q = kp >> 2;
    s.lpr = s.q <= 32 ? (1 << (32 - __clz(s.q - 1))) : 32;
    if (s.q == 1) s.lpr = 1;
    s.rpw = 32 / s.lpr;
    s.fpl = (s.q + 31) >> 5;
    int lane = threadIdx.x & 31;
    s.col0 = lane % s.lpr;
    s.rsub = lane / s.lpr;
    return s;
}

template <bool FP16>
__device__ void up_unit(const AggArgs& a, int u, int nunits)
{
    const int b = a.ubeg[u];
    const int e = u + 1 < nunits ? a.ubeg[u + 1] : a.N;
    const Shape sh = unit_shape(a.kp[b]);
    const size_t base = a.roff[b];
    const int kp = sh.q * 4;
    float4 carry[2] = {f4(0.f), f4(0.f)};
    float ncarry = 0.f;
    for (int gend = e; gend > b; gend -= sh.rpw) {
        const int r = gend - sh.rpw + sh.rsub;
        const bool act = r >= b;
        float4 A[2] = {f4(0.f), f4(0.f)};
        float m = 0.f, An = 0.f;
        RowInfo ri;
        if (act) {
            if (r + 1 < e) {
                float s1 = a.rs[r + 1];
                m = signbit(s1) ? 0.f : s1;
            }
            row_labels(a, r, sh.col0, sh.fpl, sh.q, ri);
            const int v = a.lay[r];
            const int px = v % a.W, py = v / a.W;
            const int4 Lp = a.imL[v];
            const int4* Rrow = a.imR + (size_t)py * a.W;
#pragma unroll
            for (int f = 0; f < 2; ++f) {
                float t[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    int x = ri.lab[4 * f + i];
                    t[i] = x >= 0 ? cost_m(Lp, Rrow[max(px - x, 0)], a.ck) : 0.f;
                }
                A[f] = make_float4(t[0], t[1], t[2], t[3]);
            }
            An = 1.f;
            const uint32_t l0 = a.lcoff[r], l1 = a.lcoff[r + 1];
            for (uint32_t j = l0; j < l1; ++j) {
                const int c = a.lcrow[j];
                const float sc = fabsf(a.rs[c]);
                const size_t co = a.roff[c];
                const float nc = FP16 ? a.nup[c] : 1.f;
#pragma unroll
                for (int f = 0; f < 2; ++f) {
                    int col = sh.col0 + 32 * f;
                    if (f < sh.fpl && col < sh.q) A[f] = fma4(sc * nc, load_row4<FP16>(a, co + 4 * col), A[f]);
                }
                if (FP16) An = fmaf(sc, nc, An);
            }
        }
        // suffix scan of affine maps (A, m) across the rows of the group
        for (int dlt = 1; dlt < sh.rpw; dlt <<= 1) {
            const int src = dlt * sh.lpr;
            float4 o0 = shfl_down4(A[0], src), o1 = shfl_down4(A[1], src);
            float om = __shfl_down_sync(0xffffffffu, m, src);
            float on = __shfl_down_sync(0xffffffffu, An, src);
            if (sh.rsub + dlt < sh.rpw) {
                A[0] = fma4(m, o0, A[0]);
                A[1] = fma4(m, o1, A[1]);
                if (FP16) An = fmaf(m, on, An);
                m *= om;
            }
        }
        float4 x0 = fma4(m, carry[0], A[0]);
        float4 x1 = fma4(m, carry[1], A[1]);
        float nx = FP16 ? fmaf(m, ncarry, An) : 1.f;
        if (act) {
            const size_t ro = base + (size_t)(r - b) * kp;
            const float sc = FP16 ? 1.f / nx : 1.f;
            if (sh.col0 < sh.q) store_row4<FP16>(a, ro + 4 * sh.col0, FP16 ? make_float4(x0.x * sc, x0.y * sc, x0.z * sc, x0.w * sc) : x0);
            if (sh.fpl > 1 && sh.col0 + 32 < sh.q)
                store_row4<FP16>(a, ro + 4 * (sh.col0 + 32), FP16 ? make_float4(x1.x * sc, x1.y * sc, x1.z * sc, x1.w * sc) : x1);
            if (FP16 && sh.col0 == 0) a.nup[r] = nx;
        }
        carry[0] = shfl4(x0, sh.col0);
        carry[1] = shfl4(x1, sh.col0);
        if (FP16) ncarry = __shfl_sync(0xffffffffu, nx, 0);
    }
}

template <bool FP16>
__device__ void down_unit(const AggArgs& a, int u, int nunits)
{
    const int b = a.ubeg[u];
    const int e = u + 1 < nunits ? a.ubeg[u + 1] : a.N;
    const Shape sh = unit_shape(a.kp[b]);
    const size_t base = a.roff[b];
    const int kp = sh.q * 4;
    float4 carry[2] = {f4(0.f), f4(0.f)};
    float ncarry = 0.f;
    for (int gs = b; gs < e; gs += sh.rpw) {
        const int r = gs + sh.rsub;
        const bool act = r < e;
        float4 B[2] = {f4(0.f), f4(0.f)};
        float m = 0.f, Bn = 0.f, nu = 1.f;
        if (act) {
            const float s = a.rs[r];
            const bool top = signbit(s);
            const float sv = fabsf(s);
            m = top ? 0.f : sv;
            const float w = 1.f - sv * sv;
            const size_t ro = base + (size_t)(r - b) * kp;
            const int pr = top ? a.prow[r] : -1;
            const size_t po = pr >= 0 ? a.roff[pr] : 0;
            if (FP16) nu = a.nup[r];
            const float np = FP16 && pr >= 0 ? a.nd[pr] : 1.f;
#pragma unroll
            for (int f = 0; f < 2; ++f) {
                int col = sh.col0 + 32 * f;
                if (f < sh.fpl && col < sh.q) {
                    float4 U = load_row4<FP16>(a, ro + 4 * col);
                    if (FP16) U = make_float4(U.x * nu, U.y * nu, U.z * nu, U.w * nu);
                    float4 bb = make_float4(w * U.x, w * U.y, w * U.z, w * U.w);
                    if (pr >= 0) bb = fma4(sv * np, load_row4<FP16>(a, po + 4 * col), bb);
                    B[f] = bb;
                }
            }
            if (FP16) Bn = fmaf(sv, pr >= 0 ? np : 0.f, w * nu);
        }
        // prefix scan of affine maps across the rows of the group
        for (int dlt = 1; dlt < sh.rpw; dlt <<= 1) {
            const int src = dlt * sh.lpr;
            float4 o0 = shfl_up4(B[0], src), o1 = shfl_up4(B[1], src);
            float om = __shfl_up_sync(0xffffffffu, m, src);
            float on = __shfl_up_sync(0xffffffffu, Bn, src);
            if (sh.rsub >= dlt) {
                B[0] = fma4(m, o0, B[0]);
                B[1] = fma4(m, o1, B[1]);
                if (FP16) Bn = fmaf(m, on, Bn);
                m *= om;
            }
        }
        float4 x0 = fma4(m, carry[0], B[0]);
        float4 x1 = fma4(m, carry[1], B[1]);
        float nx = FP16 ? fmaf(m, ncarry, Bn) : 1.f;
        // WTA over this row's slots (lowest label on ties)
        float bv = INFINITY;
        int bl = INT_MAX;
        if (act) {
            RowInfo ri;
            row_labels(a, r, sh.col0, sh.fpl, sh.q, ri);
            float xs[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                int lab = ri.lab[i];
                if (lab >= 0 && (xs[i] < bv || (xs[i] == bv && lab < bl))) { bv = xs[i]; bl = lab; }
            }
            const size_t ro = base + (size_t)(r - b) * kp;
            const float sc = FP16 ? 1.f / nx : 1.f;
            if (sh.col0 < sh.q) store_row4<FP16>(a, ro + 4 * sh.col0, FP16 ? make_float4(x0.x * sc, x0.y * sc, x0.z * sc, x0.w * sc) : x0);
            if (sh.fpl > 1 && sh.col0 + 32 < sh.q)
                store_row4<FP16>(a, ro + 4 * (sh.col0 + 32), FP16 ? make_float4(x1.x * sc, x1.y * sc, x1.z * sc, x1.w * sc) : x1);
            if (FP16 && sh.col0 == 0) a.nd[r] = nx;
        }
        for (int o = sh.lpr >> 1; o > 0; o >>= 1) {
            float ov = __shfl_xor_sync(0xffffffffu, bv, o);
            int ol = __shfl_xor_sync(0xffffffffu, bl, o);
            if (ov < bv || (ov == bv && ol < bl)) { bv = ov; bl = ol; }
        }
        if (act && sh.col0 == 0) a.disp[a.lay[r]] = bl == INT_MAX ? -1 : bl;
        const int last = (sh.rpw - 1) * sh.lpr + sh.col0;
        carry[0] = shfl4(x0, last);
        carry[1] = shfl4(x1, last);
        if (FP16) ncarry = __shfl_sync(0xffffffffu, nx, (sh.rpw - 1) * sh.lpr);
    }
}

template <bool FP16, bool UP>
__global__ void __launch_bounds__(AGG_THREADS) k_agg(AggArgs a)
{
    const int cnt = a.lvl_count[a.level];
    if (cnt == 0) return;
    const int first = a.lvl_first[a.level];
    const int nunits = *a.d_nunits;
    const int lane = threadIdx.x & 31;
    int* tk = a.tickets + (UP ? 0 : MAX_LIGHT_LEVELS) + a.level;
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(tk, 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= cnt) break;
        const int u = first + t;
        if (UP) up_unit<FP16>(a, u, nunits);
        else down_unit<FP16>(a, u, nunits);
    }
}

CostK cost_consts(const Ctx& c, int l)
{
    CostK k;
    int sc = 1 << (2 * l);
    k.A = 2 * (20 - c.a20);
    k.B = c.a20;
    k.Tc = c.tc3 * sc;
    k.Tg = c.tg6 * sc;
    k.inv = (float)(1.0 / (120.0 * sc));
    return k;
}

void launch_aggregate(Ctx& c, int l)
{
    const LayerDims& d = c.dim[l];
    const bool hdp = c.p.mode == HDP_MODE_HDP && l < c.top;
    AggArgs a{};
    a.imL = c.imL[l];
    a.imR = c.imR[l];
    a.W = d.W;
    a.N = d.N;
    a.full = hdp ? 0 : 1;
    a.dl = d.d;
    a.ck = cost_consts(c, l);
    a.lay = c.lay;
    a.rs = c.rs;
    a.prow = c.prow;
    a.rdt = c.rdt;
    a.T = c.T;
    a.lcoff = c.lcoff;
    a.lcrow = c.lcrow;
    a.roff = c.roff;
    a.kp = c.kp;
    a.ubeg = c.ubeg;
    a.d_nunits = c.ints + IDX_NUNITS;
    a.lvl_first = c.lvl_first;
    a.lvl_count = c.lvl_count;
    a.vol = c.vol;
    a.volh = c.volh;
    a.nup = c.nup;
    a.nd = c.nfull;
    a.tickets = c.tickets;
    a.disp = c.disp[l];
    a.st = c.st;
    int levels = 1;
    while ((1 << levels) <= d.N) ++levels;
    if (levels > MAX_LIGHT_LEVELS) levels = MAX_LIGHT_LEVELS;
    cudaMemsetAsync(c.tickets, 0, sizeof(int) * 2 * MAX_LIGHT_LEVELS, c.s);
    const int blocks = c.num_sms * 8;
    const bool fp16 = c.p.storage == HDP_STORE_FP16;
    for (int lv = levels - 1; lv >= 0; --lv) {
        a.level = lv;
        if (fp16) k_agg<true, true><<<blocks, AGG_THREADS, 0, c.s>>>(a);
        else k_agg<false, true><<<blocks, AGG_THREADS, 0, c.s>>>(a);
    }
    for (int lv = 0; lv < levels; ++lv) {
        a.level = lv;
        if (fp16) k_agg<true, false><<<blocks, AGG_THREADS, 0, c.s>>>(a);
        else k_agg<false, false><<<blocks, AGG_THREADS, 0, c.s>>>(a);
    }
}
