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
// with m = 0 across path boundaries.  The rows of a level are cut into tiles of
// about TILE_FLOATS costs; a warp stages its tile in shared memory (all loads
// of the tile in flight together), scans it (per-lane sequential chunks and a
// shuffle scan of affine maps across chunks), and takes the carry from the
// neighbouring tile of the same path with a decoupled look-back: a tile
// publishes its affine aggregate (A, M), then its inclusive boundary value; the
// carry is evaluated innermost-first, so the rounding does not depend on
// timing.  Each pass is one launch over all tiles of the layer: tiles take
// tickets deepest light level first (up) or shallowest first (down), and a
// tile whose rows read another level's rows (a light child's U, a parent's
// C) waits for that tile's done flag, set once its stores have completed.
#include "hdp_impl.cuh"

#define AGG_WARPS 4
#define AGG_THREADS (32 * AGG_WARPS)
#define AGG_CHUNK 64   // light children staged per chunk

struct AggArgs {
    const uint32_t* tstart;   // 1 at the first row of a tile
    const uint32_t* tid;      // exclusive count of tile starts
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
    const int* tbeg;
    const int* d_ntiles;
    float* vol;          // up-pass values U (and the down pass input)
    float* vout;         // down-pass output C (== vol for in-place aggregation)
    const float* Ein;    // optional dense cost volume [N][X] (all labels) instead of the matching cost
    const int* refD;     // optional refinement cost |x - refD[v]| (0 where refD[v] < 0) instead of the matching cost
    int X;
    __half* volh;
    float* nup;
    float* nd;
    int* tickets;
    int* tflags;
    int* dflags;         // per tile and pass: 1 once the tile's rows are final in global memory
    float* aggA;
    float* inclA;
    float* aggM;
    int32_t* disp;
    DevStatus* st;
};

__device__ __forceinline__ float4 f4(float a) { return make_float4(a, a, a, a); }
__device__ __forceinline__ float4 fma4(float m, float4 x, float4 a)
{
    return make_float4(fmaf(m, x.x, a.x), fmaf(m, x.y, a.y), fmaf(m, x.z, a.z), fmaf(m, x.w, a.w));
}
__device__ __forceinline__ float4 add4(float4 a, float4 b) { return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w); }
__device__ __forceinline__ float4 shfl_up4(float4 v, int d)
{
    return make_float4(__shfl_up_sync(0xffffffffu, v.x, d), __shfl_up_sync(0xffffffffu, v.y, d),
                       __shfl_up_sync(0xffffffffu, v.z, d), __shfl_up_sync(0xffffffffu, v.w, d));
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

// labels of slots 4j .. 4j+3 of a row (-1 for padding slots)
__device__ __forceinline__ void slot_labels(const AggArgs& a, int row, int j, int lab[4], int* kout)
{
    if (a.full) {
        const int k = a.dl + 1;
#pragma unroll
        for (int i = 0; i < 4; ++i) lab[i] = 4 * j + i < k ? 4 * j + i : -1;
        if (kout) *kout = k;
        return;
    }
    uint32_t m[HDP_WORDS];
    const uint32_t* src = a.T + (size_t)a.rdt[row] * HDP_WORDS;
#pragma unroll
    for (int w = 0; w < HDP_WORDS; ++w) m[w] = src[w];
    int k = 0;
#pragma unroll
    for (int w = 0; w < HDP_WORDS; ++w) k += __popc(m[w]);
    if (kout) *kout = k;
    int l = 4 * j < k ? nth_label(m, 4 * j) : -1;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        lab[i] = l;
        if (l >= 0 && 4 * j + i + 1 < k) {
            int w = l >> 5, b = l & 31, nxt = -1;
            if (b < 31) {
                unsigned r = __fns(m[w], b + 1, 1);
                if (r != 0xffffffffu) nxt = 32 * w + (int)r;
            }
            for (int ww = w + 1; nxt < 0 && ww < HDP_WORDS; ++ww)
                if (m[ww]) nxt = 32 * ww + __ffs(m[ww]) - 1;
            l = nxt;
        } else {
            l = -1;
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
        const uint2 raw = *(const uint2*)(a.volh + off);
        float2 x = __half22float2(*(const __half2*)&raw.x), y = __half22float2(*(const __half2*)&raw.y);
        return make_float4(x.x, x.y, y.x, y.y);
    } else {
        return *(const float4*)(a.vol + off);
    }
}

// rows written by other SMs during the same kernel: read through L2 only
template <bool FP16>
__device__ __forceinline__ float4 load_row4_cg(const AggArgs& a, size_t off)
{
    if (FP16) {
        const uint2 raw = __ldcg((const uint2*)(a.volh + off));
        float2 x = __half22float2(*(const __half2*)&raw.x), y = __half22float2(*(const __half2*)&raw.y);
        return make_float4(x.x, x.y, y.x, y.y);
    } else {
        return __ldcg((const float4*)(a.vol + off));
    }
}

template <bool FP16>
__device__ __forceinline__ void store_row4(const AggArgs& a, size_t off, float4 v)
{
    if (FP16) {
        __half2 h0 = __floats2half2_rn(v.x, v.y), h1 = __floats2half2_rn(v.z, v.w);
        uint2 raw;
        raw.x = *(const unsigned*)&h0;
        raw.y = *(const unsigned*)&h1;
        *(uint2*)(a.volh + off) = raw;
    } else {
        *(float4*)(a.vol + off) = v;
    }
}

// ---- TMA bulk copies (untiled cp.async.bulk): 16-byte aligned addresses and sizes
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t phase)
{
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(phase) : "memory");
    return ok != 0;
}
// bounded wait for a bulk load; on timeout the error is recorded and the wait
// continues (bounded again) so that no copy into this warp's buffer is left
// in flight
__device__ __forceinline__ void mbar_wait(const DevStatus* cst, uint64_t* bar, uint32_t phase)
{
    DevStatus* st = const_cast<DevStatus*>(cst);
    for (int round = 0; round < 2; ++round) {
        for (unsigned it = 0; it < HDP_SPIN_LIMIT; ++it)
            if (mbar_test(bar, phase)) return;
        dev_fail(st, DEV_TIMEOUT, 53);
    }
}
__device__ __forceinline__ void bulk_store(void* dst, const void* src, uint32_t bytes)
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// the shared-memory source of earlier bulk stores may be overwritten after this
__device__ __forceinline__ void bulk_store_drain() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// every earlier bulk store has completed (written to global memory)
__device__ __forceinline__ void bulk_store_complete() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ int tile_of_row(const AggArgs& a, int r) { return (int)a.tid[r] + (int)a.tstart[r] - 1; }

// the spin on a neighbouring tile's state is bounded; on timeout the carry is
// taken as zero and the device status reports DEV_TIMEOUT
__device__ __forceinline__ int wait_flag(const AggArgs& a, int* f)
{
    unsigned it = 0;
    const unsigned cap = spin_cap(a.st);
    int v;
    while ((v = *(volatile int*)f) == 0) {
        if (++it > cap || dev_err(a.st)) {
            dev_fail(a.st, DEV_TIMEOUT, 50);
            return -1;
        }
        __nanosleep(64);
    }
    __threadfence();
    return v;
}

__device__ __noinline__ void wait_done(const AggArgs& a, int* f)
{
    unsigned it = 0;
    const unsigned cap = spin_cap(a.st);
    while (*(volatile int*)f != 2) {
        if (++it > cap || dev_err(a.st)) {
            dev_fail(a.st, DEV_TIMEOUT, 52);
            return;
        }
        __nanosleep(64);
    }
}

// a light child's U (up pass) or a parent's C (down pass) lives in another
// tile, with an earlier ticket: wait until that tile has published its rows
// (bounded; on timeout the value read may be stale and the device status
// reports DEV_TIMEOUT)
__device__ __forceinline__ void wait_tile(const AggArgs& a, const int* dflags, int t, int ntiles)
{
    if ((unsigned)t >= (unsigned)ntiles) {   // a corrupt layout: record it, read nothing
        dev_fail(a.st, DEV_BAD_INPUT, 55);
        return;
    }
    if (*(volatile const int*)(dflags + t)) return;
    unsigned it = 0;
    const unsigned cap = spin_cap(a.st);
    while (*(volatile const int*)(dflags + t) == 0) {
        if (++it > cap || dev_err(a.st)) {
            dev_fail(a.st, DEV_TIMEOUT, 54);
            return;
        }
        __nanosleep(32);
    }
}

template <bool FP16, bool UP, int TF>
__device__ void tile_pass(const AggArgs& a, int u, float4* X, float* M, float* P, float* PT, float* Q,
                          float4* CIN, int* CO, float* CS, uint64_t* bar, uint32_t& bar_phase)
{
    const int lane = threadIdx.x & 31;
    const int ntiles = *a.d_ntiles;
    const int b = a.tbeg[u];
    const int kp = a.kp[b];
    const int q = kp >> 2;
    const int qe = q + (FP16 ? 1 : 0);          // FP16: an extra column carries the support mass
    int e = b + tile_rows_of(kp, FP16 ? 4 : 0, TF);
    if (u + 1 < ntiles) e = min(e, a.tbeg[u + 1]);
    e = min(e, a.N);
    const int n = e - b;
    const size_t base = a.roff[b];
    // idx / qe and idx / q by a multiply-high with m = ceil(2^32 / d): exact for
    // idx < 2^14 and 2 <= d < 2^8 (here idx < n * qe <= 768, qe <= 65); d = 1,
    // whose m does not fit in 32 bits, is taken apart
    const uint32_t mqe = qe > 1 ? (uint32_t)((0x100000000ull + qe - 1) / qe) : 0u;
    const uint32_t mq = q > 1 ? (uint32_t)((0x100000000ull + q - 1) / q) : 0u;
    int* flags = a.tflags + (UP ? 0 : (size_t)ntiles);
    int* dflags = a.dflags + (UP ? 0 : (size_t)ntiles);
    int* Pi = (int*)P;
    int* PTi = (int*)PT;
    int* Qi = (int*)Q;

    // FP16 rows of a multiple of 8 labels starting on a 16-byte boundary move
    // with TMA bulk copies too (full range: always); other FP16 tiles use
    // vector loads and stores
    const bool tma16 = FP16 && (kp & 7) == 0 && (base & 7) == 0;
    // half rows staged at the tail of X (widened in place by phase 1b)
    const uint32_t s16 = TF * 4 - (uint32_t)(n * kp * 2);
    const __half* X16 = (const __half*)((const char*)X + s16);

    // the previous tile's bulk store reads X: let it finish before X is rewritten
    if (lane == 0) bulk_store_drain();
    __syncwarp();
    if (!UP && (!FP16 || tma16)) {
        // the tile's U rows are one contiguous run: one TMA bulk copy into X
        if (lane == 0) {
            if (FP16) bulk_load((char*)X + s16, a.volh + base, (uint32_t)(n * kp * 2), bar);
            else bulk_load(X, a.vol + base, (uint32_t)(n * kp * sizeof(float)), bar);
        }
    }

    // ---- phase 1a: per-row inputs, one lane per row (every load of a row in
    // flight at once), kept in shared memory for the element loop
    //   up:   Pi = node, PTi = its first light child, M, and Qi = its column
    //         (bits 0-18) | light children (19-20) | label set is one interval
    //         (21) | padding of the row (22-23) | first label (24-31)
    //   down: Pi = parent row offset (-1: none), PT = parent weight, Q = own weight, M
    int c_base = 0, c_end = 0;
    if (UP) {
        c_base = (int)a.lcoff[b];
        c_end = (int)a.lcoff[e];
        for (int r = lane; r < n; r += 32) {
            const int row = b + r;
            const int v = a.lay[row];
            const int c0 = (int)a.lcoff[row];
            Pi[r] = v;
            PTi[r] = c0;
            uint32_t qi = (uint32_t)(v % a.W) | ((uint32_t)((int)a.lcoff[row + 1] - c0) << 19);
            if (!a.full) {
                // the row's labels are its tree's set; most sets are one interval
                const uint32_t* m = a.T + (size_t)a.rdt[row] * HDP_WORDS;
                int k = 0, lo = -1, hi = -1;
#pragma unroll
                for (int w = 0; w < HDP_WORDS; ++w) {
                    const uint32_t x = m[w];
                    if (x) {
                        if (lo < 0) lo = 32 * w + __ffs(x) - 1;
                        hi = 32 * w + 31 - __clz(x);
                        k += __popc(x);
                    }
                }
                if (k > 0 && hi - lo + 1 == k)
                    qi |= (1u << 21) | ((uint32_t)(kp - k) << 22) | ((uint32_t)lo << 24);
            }
            Qi[r] = (int)qi;
            float m = 0.f;
            if (row + 1 < a.N) {
                const float s1 = a.rs[row + 1];
                m = signbit(s1) ? 0.f : s1;
            }
            M[r] = m;
        }
    } else {
        // parent row of a path top, -1 otherwise; CIN (320 floats >= the
        // rows of any tile) is unused until phase 3 (P, PT, Q, M hold the
        // row inputs: Pi aliases P)
        int* Pr = (int*)CIN;
        for (int r = lane; r < n; r += 32) {
            const int row = b + r;
            const float s = a.rs[row];
            const bool top = signbit(s);
            const float sv = fabsf(s), w = 1.f - sv * sv;
            const int pr = top ? a.prow[row] : -1;
            Pr[r] = pr;
            Pi[r] = pr >= 0 ? (int)a.roff[pr] : -1;
            PT[r] = pr >= 0 ? sv : 0.f;
            Q[r] = FP16 ? w * a.nup[row] : w;
            M[r] = top ? 0.f : s;
        }
        // only now wait for the parents' tiles (their C and, in FP16, their
        // masses), with this tile's own loads already in flight
        for (int r = lane; r < n; r += 32) {
            const int pr = Pr[r];
            if (pr < 0) continue;
            wait_tile(a, dflags, tile_of_row(a, pr), ntiles);
            if (FP16) PT[r] *= __ldcg(a.nd + pr);
        }
    }
    __syncwarp();
    if (!UP && (!FP16 || tma16)) {
        mbar_wait(a.st, bar, bar_phase);
        bar_phase ^= 1u;
    }
    if (!UP && tma16) {
        // widen the staged half rows in place into X's layout (q vectors and a
        // mass slot per row), 32 vectors per step, all reads of a step before
        // its writes.  Element e's float slot lies below its own half slot
        // (a tile fits TF floats), and half slots grow with e, so a
        // step never overwrites halves of a later step.
        for (int e0 = 0; e0 < n * qe; e0 += 32) {
            const int e = e0 + lane;
            const int r = qe > 1 ? (int)__umulhi((uint32_t)e, mqe) : e, j = e - r * qe;
            const bool ok = e < n * qe && j < q;
            uint2 raw = make_uint2(0u, 0u);
            if (ok) raw = *(const uint2*)(X16 + (size_t)r * kp + 4 * j);
            __syncwarp();
            if (ok) {
                const float2 lo = __half22float2(*(const __half2*)&raw.x);
                const float2 hi = __half22float2(*(const __half2*)&raw.y);
                X[e] = make_float4(lo.x, lo.y, hi.x, hi.y);
            }
            __syncwarp();
        }
    }

    // ---- phase 1b: the affine inputs of every (row, column) of the tile.  Up:
    // E first (it needs no other tile, so it runs before any wait), then the
    // light children's U added in child order, the children taken in chunks of
    // AGG_CHUNK whose row offsets and weights are staged (after waiting for
    // their tiles) first.  Down: (1 - s^2) U plus s C(parent) at path tops.
    // No unrolling: the kernel is bound by instruction fetch and latency, not
    // by the loop overhead (1390x1110 full range: 6.9 ms unrolled 4 times,
    // 6.0 ms not unrolled)
    if (UP) {
#pragma unroll 1
        for (int idx = lane; idx < n * qe; idx += 32) {
            const int r = qe > 1 ? (int)__umulhi((uint32_t)idx, mqe) : idx, j = idx - r * qe, row = b + r;
            float4 x;
            if (j < q) {
                const uint32_t qi = (uint32_t)Qi[r];
                const int v = Pi[r];
                float t[4];
                if (a.Ein) {
                    const float* er = a.Ein + (size_t)v * a.X;
#pragma unroll
                    for (int i = 0; i < 4; ++i) t[i] = 4 * j + i < a.X ? er[4 * j + i] : 0.f;
                } else {
                    int lab[4];
                    if (qi & (1u << 21)) {   // one interval: slot s holds label lo + s
                        const int lo = (int)(qi >> 24), k = kp - (int)((qi >> 22) & 3u);
#pragma unroll
                        for (int i = 0; i < 4; ++i) lab[i] = 4 * j + i < k ? lo + 4 * j + i : -1;
                    } else {
                        slot_labels(a, row, j, lab, nullptr);
                    }
                    if (a.refD) {   // refinement: distance to the pixel's checked disparity
                        const int rd = a.refD[v];
#pragma unroll
                        for (int i = 0; i < 4; ++i) t[i] = lab[i] >= 0 && rd >= 0 ? (float)abs(lab[i] - rd) : 0.f;
                    } else {
                        const int px = (int)(qi & 0x7ffffu);
                        const int4 Lp = a.imL[v];
                        const int4* Rrow = a.imR + (size_t)(v - px);
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            t[i] = lab[i] >= 0 ? cost_m(Lp, Rrow[max(px - lab[i], 0)], a.ck) : 0.f;
                    }
                }
                x = make_float4(t[0], t[1], t[2], t[3]);
            } else {
                x = make_float4(1.f, 0.f, 0.f, 0.f);   // FP16: the support mass starts at 1
            }
            X[idx] = x;
        }
        __syncwarp();
        for (int cc = c_base; cc < c_end; cc += AGG_CHUNK) {
            const int cn = min(AGG_CHUNK, c_end - cc);
            for (int k = lane; k < cn; k += 32) {
                const int cr = a.lcrow[cc + k];
                wait_tile(a, dflags, tile_of_row(a, cr), ntiles);
                CO[k] = (int)a.roff[cr];
                CS[k] = fabsf(a.rs[cr]) * (FP16 ? __ldcg(a.nup + cr) : 1.f);
            }
            __syncwarp();
#pragma unroll 1
            for (int idx = lane; idx < n * qe; idx += 32) {
                const int r = qe > 1 ? (int)__umulhi((uint32_t)idx, mqe) : idx, j = idx - r * qe;
                const uint32_t qi = (uint32_t)Qi[r];
                const int cb = PTi[r], ce = cb + (int)((qi >> 19) & 3u);
                const int lo = max(cb, cc) - cc, hi = min(ce, cc + cn) - cc;
                if (lo >= hi) continue;
                float4 x = X[idx];
                if (j < q) {
                    for (int k = lo; k < hi; ++k) x = fma4(CS[k], load_row4_cg<FP16>(a, (size_t)CO[k] + 4 * j), x);
                } else {
                    for (int k = lo; k < hi; ++k) x.x += CS[k];
                }
                X[idx] = x;
            }
            __syncwarp();
        }
    } else {
#pragma unroll 1
        for (int idx = lane; idx < n * qe; idx += 32) {
            const int r = qe > 1 ? (int)__umulhi((uint32_t)idx, mqe) : idx, j = idx - r * qe;
            const int po = Pi[r];
            const float cw = Q[r];
            float4 x;
            if (j < q) {
                const float4 U = (!FP16 || tma16) ? X[idx] : load_row4<FP16>(a, base + (size_t)r * kp + 4 * j);
                x = make_float4(cw * U.x, cw * U.y, cw * U.z, cw * U.w);
                if (po >= 0) {
                    const float4 cp = FP16 ? load_row4_cg<FP16>(a, (size_t)po + 4 * j)
                                           : __ldcg((const float4*)(a.vout + po + 4 * j));
                    x = fma4(PT[r], cp, x);
                }
            } else {
                x = make_float4(cw + PT[r], 0.f, 0.f, 0.f);
            }
            X[idx] = x;
        }
        __syncwarp();
    }

    // ---- phase 2: scan in recurrence order t (row = n-1-t going up, t going down)
    const int G = qe >= 32 ? 32 : (qe <= 1 ? 1 : 1 << (32 - __clz(qe - 1)));
    const int C = 32 / G;
    const int col = lane % G, chunk = lane / G;
    const int len = (n + C - 1) / C;
    const int t0 = min(n, chunk * len), t1 = min(n, t0 + len);
    float4 acc[3] = {f4(0.f), f4(0.f), f4(0.f)};
    float accM = 1.f;
    for (int t = t0; t < t1; ++t) {
        const int r = UP ? n - 1 - t : t;
        const float m = M[r];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int j = col + G * k;
            if (j < qe) {
                acc[k] = fma4(m, acc[k], X[r * qe + j]);
                X[r * qe + j] = acc[k];
            }
        }
        accM *= m;
        if (col == 0) P[r] = accM;
    }
    float4 inc[3] = {acc[0], acc[1], acc[2]};
    float incM = accM;
    for (int d = 1; d < C; d <<= 1) {
        float4 o0 = shfl_up4(inc[0], d * G), o1 = shfl_up4(inc[1], d * G), o2 = shfl_up4(inc[2], d * G);
        const float om = __shfl_up_sync(0xffffffffu, incM, d * G);
        if (chunk >= d) {
            inc[0] = fma4(incM, o0, inc[0]);
            inc[1] = fma4(incM, o1, inc[1]);
            inc[2] = fma4(incM, o2, inc[2]);
            incM *= om;
        }
    }
    float4 carry[3] = {shfl_up4(inc[0], G), shfl_up4(inc[1], G), shfl_up4(inc[2], G)};
    float mprev = __shfl_up_sync(0xffffffffu, incM, G);
    if (chunk == 0) {
        carry[0] = carry[1] = carry[2] = f4(0.f);
        mprev = 1.f;
    }
    __syncwarp();
    for (int t = t0; t < t1; ++t) {
        const int r = UP ? n - 1 - t : t;
        const float p = P[r];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int j = col + G * k;
            if (j < qe) X[r * qe + j] = fma4(p, carry[k], X[r * qe + j]);
        }
        if (col == 0) PT[r] = p * mprev;
    }
    __syncwarp();

    // ---- phase 3: carry from the neighbouring tile of the same path.  Tiles of a
    // path sit at consecutive indices; a tile that links to its neighbour
    // publishes its aggregate (A, M), then walks back 32 tiles at a time over
    // published aggregates to the nearest inclusive value (waiting only on a
    // tile that has published nothing yet).  The carry is then applied tile by
    // tile from that inclusive value outwards, so every tile's value is the
    // same chain of fmas whichever inclusive value was found: the rounding does
    // not depend on timing.
    const int rfirst = UP ? n - 1 : 0;   // first row in recurrence order
    const int rlast = UP ? 0 : n - 1;    // boundary row handed to the next tile
    const bool need = M[rfirst] != 0.f;
    const int nf = 4 * qe;
    float* cin = (float*)CIN;
    if (need) {
        const int dir = UP ? 1 : -1;
        int D = 0;            // distance of the inclusive value (0: wait failed)
        // the neighbour's inclusive value is often out already: then this
        // tile's aggregate is never needed (later tiles wait for its own
        // inclusive value instead) and is not published
        const int j1 = u + dir;
        const int f1 = (j1 >= 0 && j1 < ntiles) ? *(volatile int*)(flags + j1) : 3;
        if (__shfl_sync(0xffffffffu, f1, 0) >= 2) {
            D = 1;
        } else {
            float* dst = a.aggA + (size_t)u * SCR_STRIDE;
            const float* xl = (const float*)(X + rlast * qe);
            for (int f = lane; f < nf; f += 32) dst[f] = xl[f];
            if (lane == 0) a.aggM[u] = PT[rlast];
            __threadfence();
            __syncwarp();
            if (lane == 0) atomicExch(flags + u, 1);
        }
        unsigned it = 0;
        for (int off = 0; D == 0;) {
            const int jt = u + dir * (off + lane + 1);
            // a neighbour outside the tile range would be a chain start with value 0
            const int f = (jt >= 0 && jt < ntiles) ? *(volatile int*)(flags + jt) : 3;
            const unsigned incl = __ballot_sync(0xffffffffu, f >= 2);
            const unsigned none = __ballot_sync(0xffffffffu, f == 0);
            if (incl) {
                const int k = __ffs(incl);          // 1-based
                const unsigned before = k == 1 ? 0u : (0xffffffffu >> (33 - k));
                if (!(none & before)) { D = off + k; break; }
            } else if (!none) {
                off += 32;                          // 32 aggregates: keep walking
                continue;
            }
            if (++it > spin_cap(a.st) || dev_err(a.st)) {
                dev_fail(a.st, DEV_TIMEOUT, 51);
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
        if (D > 0) {
            const int jI = u + dir * D;
            for (int f = lane; f < nf; f += 32)
                cin[f] = (jI >= 0 && jI < ntiles) ? __ldcg(a.inclA + (size_t)jI * SCR_STRIDE + f) : 0.f;
        } else {
            for (int f = lane; f < nf; f += 32) cin[f] = 0.f;
        }
        __syncwarp();
        // distances D-1 .. 1, in chunks of 32 from the far end
        for (int c0 = ((D - 2) >> 5) << 5; D > 1 && c0 >= 0; c0 -= 32) {
            const int nk = min(32, D - 1 - c0);     // tiles of this chunk: distances c0 + 1 .. c0 + nk
            // multiplier of the tile at distance c0 + lane + 1, shared by all columns
            const int dk = c0 + lane + 1;
            const int jm = u + dir * dk;
            const float mk = (lane < nk && jm >= 0 && jm < ntiles) ? __ldcg(a.aggM + jm) : 0.f;
            for (int f0 = 0; f0 < nf; f0 += 32) {      // warp-uniform trip counts (shuffles inside)
                const int f = f0 + lane;
                const bool ok = f < nf;
                float cval = ok ? cin[f] : 0.f;
                for (int k1 = nk - 1; k1 >= 0; k1 -= 8) {   // 8 loads in flight, then the fma chain
                    float av[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int k = k1 - i;
                        av[i] = (ok && k >= 0) ? __ldcg(a.aggA + (size_t)(u + dir * (c0 + k + 1)) * SCR_STRIDE + f) : 0.f;
                    }
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int k = k1 - i;
                        const float m = __shfl_sync(0xffffffffu, mk, k >= 0 ? k : 0);
                        if (k >= 0) cval = fmaf(m, cval, av[i]);
                    }
                }
                if (ok) cin[f] = cval;
            }
            __syncwarp();
        }
    } else {
        for (int f = lane; f < nf; f += 32) cin[f] = 0.f;
    }
    __syncwarp();

    // ---- phase 4: final values, stores, inclusive value for the next tile
    for (int idx = lane; idx < n * qe; idx += 32) {
        const int r = qe > 1 ? (int)__umulhi((uint32_t)idx, mqe) : idx, j = idx - r * qe;
        X[idx] = fma4(PT[r], CIN[j], X[idx]);
    }
    __syncwarp();
    if (FP16 && !tma16) {
        for (int idx = lane; idx < n * q; idx += 32) {
            const int r = q > 1 ? (int)__umulhi((uint32_t)idx, mq) : idx, j = idx - r * q;
            float4 x = X[r * qe + j];
            const float inv = 1.f / X[r * qe + q].x;
            x = make_float4(x.x * inv, x.y * inv, x.z * inv, x.w * inv);
            store_row4<FP16>(a, base + (size_t)r * kp + 4 * j, x);
        }
    } else if (!FP16) {
        // X holds the tile's rows exactly as laid out in HBM: one TMA bulk store
        __syncwarp();
        if (lane == 0) bulk_store((UP ? a.vol : a.vout) + base, X, (uint32_t)(n * kp * sizeof(float)));
    }
    if (FP16)
        for (int r = lane; r < n; r += 32) (UP ? a.nup : a.nd)[b + r] = X[r * qe + q].x;
    // the inclusive value is read only by the neighbour that continues this
    // tile's last path (up: the tile above, if this tile's first row is not a
    // path top; down: the tile below, if its first row is not a top)
    bool linked;
    if (UP) {
        linked = !signbit(a.rs[b]) && u > 0;
    } else {
        linked = u + 1 < ntiles && !signbit(a.rs[a.tbeg[u + 1]]);
    }
    if (linked) {
        float* dst = a.inclA + (size_t)u * SCR_STRIDE;
        const float* xl = (const float*)(X + rlast * qe);
        for (int f = lane; f < nf; f += 32) dst[f] = xl[f];
        __threadfence();
        __syncwarp();
        if (lane == 0) atomicExch(flags + u, 2);
    }

    // ---- phase 5 (down pass): WTA, lowest label on ties
    if (!UP) {
        if (q >= 8) {
            for (int r = 0; r < n; ++r) {
                const int row = b + r;
                int k = 0;
                int dummy[4];
                slot_labels(a, row, 0, dummy, &k);
                float bv = INFINITY;
                int bs = INT_MAX;
                for (int j = lane; j < q; j += 32) {
                    const float4 x = X[r * qe + j];
                    const float xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int slot = 4 * j + i;
                        if (slot < k && xs[i] < bv) { bv = xs[i]; bs = slot; }
                    }
                }
                for (int o = 16; o > 0; o >>= 1) {
                    const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
                    const int os = __shfl_xor_sync(0xffffffffu, bs, o);
                    if (ov < bv || (ov == bv && os < bs)) { bv = ov; bs = os; }
                }
                if (lane == 0) {
                    int lab[4];
                    slot_labels(a, row, bs >> 2, lab, nullptr);
                    a.disp[a.lay[row]] = lab[bs & 3];
                }
            }
        } else {
            for (int r = lane; r < n; r += 32) {
                const int row = b + r;
                int k = 0;
                int dummy[4];
                slot_labels(a, row, 0, dummy, &k);
                float bv = INFINITY;
                int bs = 0;
                for (int j = 0; j < q; ++j) {
                    const float4 x = X[r * qe + j];
                    const float xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int slot = 4 * j + i;
                        if (slot < k && xs[i] < bv) { bv = xs[i]; bs = slot; }
                    }
                }
                int lab[4];
                slot_labels(a, row, bs >> 2, lab, nullptr);
                a.disp[a.lay[row]] = lab[bs & 3];
            }
        }
    }
    __syncwarp();
    if (tma16) {
        // narrow in place to normalised halves, 32 vectors per step in
        // increasing order, all reads of a step (vector and its row's mass)
        // before its writes: a vector's half slot ends before the float slot
        // of any vector or mass of a later step
        __half* H16 = (__half*)X;
        for (int e0 = 0; e0 < n * qe; e0 += 32) {
            const int e = e0 + lane;
            const int r = qe > 1 ? (int)__umulhi((uint32_t)e, mqe) : e, j = e - r * qe;
            const bool ok = e < n * qe && j < q;
            float4 v = f4(0.f);
            float inv = 0.f;
            if (ok) {
                v = X[e];
                inv = 1.f / X[r * qe + q].x;
            }
            __syncwarp();
            if (ok) {
                const __half2 h0 = __floats2half2_rn(v.x * inv, v.y * inv);
                const __half2 h1 = __floats2half2_rn(v.z * inv, v.w * inv);
                uint2 raw;
                raw.x = *(const unsigned*)&h0;
                raw.y = *(const unsigned*)&h1;
                *(uint2*)(H16 + (size_t)r * kp + 4 * j) = raw;
            }
            __syncwarp();
        }
        if (lane == 0) bulk_store(a.volh + base, X, (uint32_t)(n * kp * 2));
    }
    // the tile's rows (and masses) are final once its stores have completed:
    // the bulk stores of lane 0 (async proxy) and every lane's plain stores,
    // each ordered before the flag by a fence
    if (lane == 0 && (tma16 || !FP16)) {
        bulk_store_complete();
        asm volatile("fence.proxy.async.global;" ::: "memory");
    }
    __threadfence();
    __syncwarp();
    if (lane == 0) atomicExch(dflags + u, 1);
}

// per warp: X (TF floats) | M, P, PT, Q (tile_rows_max(TF) each) | CIN (80 float4) | CO, CS (AGG_CHUNK each)
template <int TF>
__host__ __device__ constexpr int agg_warp_f4() { return TF / 4 + tile_rows_max(TF) + 80 + AGG_CHUNK / 2; }

template <bool FP16, bool UP, int TF>
__global__ void __launch_bounds__(AGG_THREADS, TF == TILE_FLOATS ? AGG_MINB_2048 : TF == TILE_FLOATS_HDP ? AGG_MINB_1024
                                                                                                    : AGG_MINB_512)
    k_agg(AggArgs a)
{
    constexpr int RM = tile_rows_max(TF);
    extern __shared__ float4 smem[];
    const int cnt = *a.d_ntiles;
    if (cnt == 0) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float4* X = smem + (size_t)warp * agg_warp_f4<TF>();
    float* M = (float*)(X + TF / 4);
    float* P = M + RM;
    float* PT = P + RM;
    float* Q = PT + RM;
    float4* CIN = (float4*)(Q + RM);
    int* CO = (int*)(CIN + 80);
    float* CS = (float*)(CO + AGG_CHUNK);
    __shared__ __align__(8) uint64_t bars[AGG_WARPS];
    uint64_t* bar = bars + warp;
    uint32_t bar_phase = 0;
    if (lane == 0) mbar_init(bar);
    __syncwarp();
    int* tk = a.tickets + (UP ? 0 : MAX_LIGHT_LEVELS);
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(tk, 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= cnt) break;
        // Tiles are numbered by light level, then position.  Up: the deepest
        // level first and, inside a level, bottom tiles first (carries flow
        // upwards, light children are deeper); down: the reverse.  A tile
        // only waits on tiles with earlier tickets (its path neighbours, the
        // tiles of its light children or of its parents), which were handed
        // to running warps, so every wait ends.
        const int u = UP ? cnt - 1 - t : t;
        tile_pass<FP16, UP, TF>(a, u, X, M, P, PT, Q, CIN, CO, CS, bar, bar_phase);
    }
    if (lane == 0) bulk_store_complete();
}

template <int TF>
static size_t agg_smem() { return (size_t)AGG_WARPS * agg_warp_f4<TF>() * sizeof(float4); }

// ---- column kernel: one-label-set layers with wide rows -----------------------
// On a full-range layer (or a big top layer) every row holds the same kp
// labels.  A CTA takes one tile (the same tickets, flags and look-back scratch
// as k_agg; tiles of TILE_FLOATS_COL floats) and a thread owns two adjacent
// label columns 2x, 2x+1 of all its rows: the cost E(v, x) reads the right
// image at (px - x), so the threads of a row read consecutive pixels; the
// recurrence along the rows is sequential per column (no cross-thread scan);
// children's, parents' and the tile's own rows move as float2 (FP32) or half2
// (FP16) per thread, coalesced.  FP16 storage adds thread kp/2 for the support
// mass (scratch slot kp).  Used when kp >= COL_MIN_KP, so a tile has at most
// TILE_FLOATS_COL / COL_MIN_KP rows.
#define COL_MAX_ROWS (TILE_FLOATS_COL / COL_MIN_KP)
#define COL_THREADS_MAX 160   // 128 column pairs + the mass thread, in warps
#define COL_CHUNK 256         // light children staged per chunk

template <bool FP16>
__device__ __forceinline__ float2 col_ld2(const AggArgs& a, const float* v32, size_t off)
{
    if (FP16) return __half22float2(__ldcg((const __half2*)(a.volh + off)));
    return __ldcg((const float2*)(v32 + off));
}

template <bool FP16, bool UP>
__global__ void __launch_bounds__(COL_THREADS_MAX) k_agg_col(AggArgs a, int kp)
{
    extern __shared__ float2 X2[];                // the tile: n rows of S2 column pairs
    __shared__ int sV[COL_MAX_ROWS];              // up: node; down: parent row offset (-1: none)
    __shared__ int sR[COL_MAX_ROWS];              // up: first light child; down: parent row (-1: none)
    __shared__ int sNC[COL_MAX_ROWS];             // up: light children
    __shared__ float sM[COL_MAX_ROWS];            // multiplier to the previous row in recurrence order
    __shared__ float sP[COL_MAX_ROWS];            // coefficient of the carry
    __shared__ float sW[COL_MAX_ROWS];            // down: 1 - s^2 (x the up-pass mass in FP16)
    __shared__ float sPW[COL_MAX_ROWS];           // down: s (x the parent's mass in FP16)
    __shared__ int sCR[COL_CHUNK];                // staged light children: row in the tile,
    __shared__ int sCO[COL_CHUNK];                // row offset,
    __shared__ float sCS[COL_CHUNK];              // weight (x mass in FP16)
    __shared__ int s_t, s_D;
    const int x = threadIdx.x, lane = x & 31, warp = x >> 5, nwarps = blockDim.x >> 5;
    const int P2 = kp >> 1;                       // column pairs of a row
    const int S2 = P2 + (FP16 ? 1 : 0);           // pairs per row in shared memory (FP16: + the mass)
    const bool col = x < S2;                      // owns a pair (or the mass at x == P2)
    const bool lab2 = x < P2;                     // owns label slots 2x, 2x+1
    const int K = a.dl + 1;                       // labels 0..dl; slots K..kp-1 are padding
    const int ntiles = *a.d_ntiles;
    int* flags = a.tflags + (UP ? 0 : (size_t)ntiles);
    int* dflags = a.dflags + (UP ? 0 : (size_t)ntiles);
    int* tk = a.tickets + (UP ? 0 : MAX_LIGHT_LEVELS);
    float* const vdst = UP ? a.vol : a.vout;
    for (;;) {
        __syncthreads();   // the previous tile is done with the shared arrays
        if (x == 0) s_t = atomicAdd(tk, 1);
        __syncthreads();
        const int t = s_t;
        if (t >= ntiles) break;
        // same order as k_agg: every wait is on an earlier ticket
        const int u = UP ? ntiles - 1 - t : t;
        const int b = a.tbeg[u];
        int e = b + tile_rows_of(kp, FP16 ? 4 : 0, TILE_FLOATS_COL);
        if (u + 1 < ntiles) e = min(e, a.tbeg[u + 1]);
        e = min(e, a.N);
        const int n = min(e - b, COL_MAX_ROWS);
        const size_t base = a.roff[b];
        if (x == 0 && e - b > COL_MAX_ROWS) dev_fail(a.st, DEV_BAD_INPUT, 56);   // a layout this kernel cannot hold

        // ---- per-row inputs, one thread per row (a tile may have more rows than the CTA threads)
        for (int r = x; r < n; r += blockDim.x) {
            const int row = b + r;
            if (UP) {
                const int v = a.lay[row];
                const int c0 = (int)a.lcoff[row];
                sV[r] = v;
                sR[r] = c0;
                sNC[r] = (int)a.lcoff[row + 1] - c0;
                float m = 0.f;
                if (row + 1 < a.N) {
                    const float s1 = a.rs[row + 1];
                    m = signbit(s1) ? 0.f : s1;
                }
                sM[r] = m;
            } else {
                const float s = a.rs[row];
                const bool top = signbit(s);
                const float sv = fabsf(s), w = 1.f - sv * sv;
                const int pr = top ? a.prow[row] : -1;
                sR[r] = pr;
                sV[r] = pr >= 0 ? (int)a.roff[pr] : -1;
                sPW[r] = pr >= 0 ? sv : 0.f;
                sW[r] = FP16 ? w * a.nup[row] : w;
                sM[r] = top ? 0.f : s;
            }
        }
        __syncthreads();
        if (x == 0) {   // carry coefficients: products of the multipliers in recurrence order
            float acc = 1.f;
            for (int k = 0; k < n; ++k) {
                const int r = UP ? n - 1 - k : k;
                acc *= sM[r];
                sP[r] = acc;
            }
        }

        // ---- the affine inputs of every (row, column pair)
        if (UP) {
            // E (no other tile needed), then the light children's U in child order
            if (col) {
                const int c0 = 2 * x, c1 = 2 * x + 1;
                const int l0 = lab2 && c0 < K ? c0 : -1, l1 = lab2 && c1 < K ? c1 : -1;
#pragma unroll 4
                for (int r = 0; r < n; ++r) {
                    float2 val = make_float2(1.f, 0.f);   // the mass pair starts at (1, 0)
                    if (lab2) {
                        const int v = sV[r];
                        if (a.Ein) {
                            val.x = c0 < a.X ? __ldg(a.Ein + (size_t)v * a.X + c0) : 0.f;
                            val.y = c1 < a.X ? __ldg(a.Ein + (size_t)v * a.X + c1) : 0.f;
                        } else if (a.refD) {
                            const int rd = __ldg(a.refD + v);
                            val.x = l0 >= 0 && rd >= 0 ? (float)abs(l0 - rd) : 0.f;
                            val.y = l1 >= 0 && rd >= 0 ? (float)abs(l1 - rd) : 0.f;
                        } else {
                            const int px = v % a.W;
                            const int4 Lp = __ldg(a.imL + v);
                            const int4* Rrow = a.imR + (v - px);
                            val.x = l0 >= 0 ? cost_m(Lp, __ldg(Rrow + max(px - l0, 0)), a.ck) : 0.f;
                            val.y = l1 >= 0 ? cost_m(Lp, __ldg(Rrow + max(px - l1, 0)), a.ck) : 0.f;
                        }
                    }
                    X2[r * S2 + x] = val;
                }
            }
            // the children in chunks: one thread per child waits for its tile and
            // stages (row, offset, weight); then every column pair adds them in
            // child order (children of a row are consecutive), the loads of a
            // chunk in flight together
            const int cb = (int)a.lcoff[b], ce = (int)a.lcoff[b + n];
            for (int cc = cb; cc < ce; cc += COL_CHUNK) {
                const int cn = min(COL_CHUNK, ce - cc);
                __syncthreads();   // the previous chunk's staging is consumed
                for (int k = x; k < cn; k += blockDim.x) {
                    const int cr = a.lcrow[cc + k];
                    wait_tile(a, dflags, tile_of_row(a, cr), ntiles);
                    // the row of this tile whose child range holds child cc + k
                    int lo = 0, hi = n - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (sR[mid] <= cc + k) lo = mid; else hi = mid - 1;
                    }
                    sCR[k] = lo;
                    sCO[k] = (int)a.roff[cr];
                    sCS[k] = fabsf(a.rs[cr]) * (FP16 ? __ldcg(a.nup + cr) : 1.f);
                }
                __syncthreads();
                if (col) {
#pragma unroll 8
                    for (int k = 0; k < cn; ++k) {
                        const int r = sCR[k];
                        const float cs = sCS[k];
                        const float2 cv = lab2 ? col_ld2<FP16>(a, a.vol, (size_t)sCO[k] + 2 * x) : make_float2(1.f, 0.f);
                        float2 v = X2[r * S2 + x];
                        v.x = fmaf(cs, cv.x, v.x);
                        v.y = fmaf(cs, cv.y, v.y);
                        X2[r * S2 + x] = v;
                    }
                }
            }
        } else {
            // (1 - s^2) U first (the tile's own rows), then s C(parent) at path tops
            if (col) {
#pragma unroll 4
                for (int r = 0; r < n; ++r) {
                    const float w = sW[r];
                    if (lab2) {
                        const float2 U = col_ld2<FP16>(a, a.vol, base + (size_t)r * kp + 2 * x);
                        X2[r * S2 + x] = make_float2(w * U.x, w * U.y);
                    } else {
                        X2[r * S2 + x] = make_float2(w, 0.f);
                    }
                }
            }
            for (int r = x; r < n; r += blockDim.x) {
                if (sR[r] < 0) continue;
                wait_tile(a, dflags, tile_of_row(a, sR[r]), ntiles);
                if (FP16) sPW[r] *= __ldcg(a.nd + sR[r]);
            }
            __syncthreads();
            if (col) {
#pragma unroll 4
                for (int r = 0; r < n; ++r) {
                    const int po = sV[r];
                    if (po < 0) continue;
                    const float pw = sPW[r];
                    float2 v = X2[r * S2 + x];
                    if (lab2) {
                        const float2 cp = col_ld2<FP16>(a, a.vout, (size_t)po + 2 * x);
                        v.x = fmaf(pw, cp.x, v.x);
                        v.y = fmaf(pw, cp.y, v.y);
                    } else {
                        v.x += pw;
                    }
                    X2[r * S2 + x] = v;
                }
            }
        }
        // ---- the recurrence along the rows, per column
        if (col) {
            float2 acc = make_float2(0.f, 0.f);
            for (int k = 0; k < n; ++k) {
                const int r = UP ? n - 1 - k : k;
                const float m = sM[r];
                const float2 v = X2[r * S2 + x];
                acc.x = fmaf(m, acc.x, v.x);
                acc.y = fmaf(m, acc.y, v.y);
                X2[r * S2 + x] = acc;
            }
        }
        __syncthreads();
        // ---- carry from the neighbouring tile of the same path (the protocol of
        // k_agg: publish the aggregate unless the neighbour's inclusive value is
        // out, walk back to the nearest inclusive value, apply the carry tile by
        // tile from it outwards, so the rounding does not depend on timing)
        const int rfirst = UP ? n - 1 : 0, rlast = UP ? 0 : n - 1;
        const int dir = UP ? 1 : -1;
        float2 cin = make_float2(0.f, 0.f);
        if (sM[rfirst] != 0.f) {
            if (x == 0) {
                const int j1 = u + dir;
                const int f1 = (j1 >= 0 && j1 < ntiles) ? *(volatile int*)(flags + j1) : 3;
                s_D = f1 >= 2 ? 1 : 0;
            }
            __syncthreads();
            if (s_D == 0) {
                if (col) *(float2*)(a.aggA + (size_t)u * SCR_STRIDE + 2 * x) = X2[rlast * S2 + x];
                if (x == 0) a.aggM[u] = sP[rlast];
                __threadfence();
                __syncthreads();
                if (x == 0) atomicExch(flags + u, 1);
                if (warp == 0) {
                    unsigned it = 0;
                    int D = 0;
                    for (int off = 0; D == 0;) {
                        const int jt = u + dir * (off + lane + 1);
                        const int f = (jt >= 0 && jt < ntiles) ? *(volatile int*)(flags + jt) : 3;
                        const unsigned incl = __ballot_sync(0xffffffffu, f >= 2);
                        const unsigned none = __ballot_sync(0xffffffffu, f == 0);
                        if (incl) {
                            const int k = __ffs(incl);
                            const unsigned before = k == 1 ? 0u : (0xffffffffu >> (33 - k));
                            if (!(none & before)) { D = off + k; break; }
                        } else if (!none) {
                            off += 32;
                            continue;
                        }
                        if (++it > spin_cap(a.st) || dev_err(a.st)) {
                            if (lane == 0) dev_fail(a.st, DEV_TIMEOUT, 57);
                            break;
                        }
                        __nanosleep(64);
                    }
                    if (lane == 0) s_D = D;
                }
                __syncthreads();
            }
            __threadfence();
            const int D = s_D;
            if (col && D > 0) {
                const int jI = u + dir * D;
                if (jI >= 0 && jI < ntiles) cin = __ldcg((const float2*)(a.inclA + (size_t)jI * SCR_STRIDE + 2 * x));
                for (int k1 = D - 1; k1 >= 1; k1 -= 8) {   // 8 loads in flight, then the fma chain
                    float2 av[8];
                    float mv[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int k = k1 - i;
                        const int j = u + dir * k;
                        const bool ok = k >= 1 && j >= 0 && j < ntiles;
                        av[i] = ok ? __ldcg((const float2*)(a.aggA + (size_t)j * SCR_STRIDE + 2 * x)) : make_float2(0.f, 0.f);
                        mv[i] = ok ? __ldcg(a.aggM + j) : 0.f;
                    }
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        if (k1 - i >= 1) {
                            cin.x = fmaf(mv[i], cin.x, av[i].x);
                            cin.y = fmaf(mv[i], cin.y, av[i].y);
                        }
                }
            }
        }
        // ---- final values, stores, the inclusive value for the next tile
        if (col)
            for (int r = 0; r < n; ++r) {
                const float p = sP[r];
                float2 v = X2[r * S2 + x];
                v.x = fmaf(p, cin.x, v.x);
                v.y = fmaf(p, cin.y, v.y);
                X2[r * S2 + x] = v;
            }
        __syncthreads();   // every column's final values (and the masses) are in shared memory
        if (FP16) {
            for (int r = x; r < n; r += blockDim.x) (UP ? a.nup : a.nd)[b + r] = X2[r * S2 + P2].x;
            if (lab2)
                for (int r = 0; r < n; ++r) {
                    const float inv = 1.f / X2[r * S2 + P2].x;
                    const float2 v = X2[r * S2 + x];
                    *(__half2*)(a.volh + base + (size_t)r * kp + 2 * x) = __floats2half2_rn(v.x * inv, v.y * inv);
                }
        } else if (lab2) {
            for (int r = 0; r < n; ++r) *(float2*)(vdst + base + (size_t)r * kp + 2 * x) = X2[r * S2 + x];
        }
        bool linked;
        if (UP) linked = !signbit(a.rs[b]) && u > 0;
        else linked = u + 1 < ntiles && !signbit(a.rs[a.tbeg[u + 1]]);
        if (linked) {
            if (col) *(float2*)(a.inclA + (size_t)u * SCR_STRIDE + 2 * x) = X2[rlast * S2 + x];
            __threadfence();
            __syncthreads();
            if (x == 0) atomicExch(flags + u, 2);
        }
        // ---- WTA (down pass): lowest slot on ties; a warp per row, each lane
        // scanning its column pairs in increasing order
        if (!UP) {
            for (int r = warp; r < n; r += nwarps) {
                float bv = INFINITY;
                int bs = INT_MAX;
                for (int j = lane; j < P2; j += 32) {
                    const float2 v = X2[r * S2 + j];
                    if (2 * j < K && v.x < bv) { bv = v.x; bs = 2 * j; }
                    if (2 * j + 1 < K && v.y < bv) { bv = v.y; bs = 2 * j + 1; }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
                    const int os = __shfl_xor_sync(0xffffffffu, bs, o);
                    if (ov < bv || (ov == bv && os < bs)) { bv = ov; bs = os; }
                }
                if (lane == 0) a.disp[a.lay[b + r]] = bs;   // full range: the slot is the label
            }
        }
        // ---- the tile's rows are final: done
        __threadfence();
        __syncthreads();
        if (x == 0) atomicExch(dflags + u, 1);
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

// one resident wave: SMs x the blocks that fit on one SM
template <bool FP16, bool UP, int TF>
static void launch_level(const AggArgs& a, int num_sms, int max_per_sm, cudaStream_t s)
{
    const size_t sm = agg_smem<TF>();
    static int per_sm = 0;
    if (per_sm == 0) {
        cudaFuncSetAttribute(k_agg<FP16, UP, TF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_agg<FP16, UP, TF>, AGG_THREADS, sm);
        if (per_sm < 1) per_sm = 1;
    }
    k_agg<FP16, UP, TF><<<num_sms * min(per_sm, max_per_sm), AGG_THREADS, sm, s>>>(a);
}

template <bool UP, int TF>
static void launch_level_s(const AggArgs& a, bool fp16, int num_sms, int max_per_sm, cudaStream_t s)
{
    if (fp16) launch_level<true, UP, TF>(a, num_sms, max_per_sm, s);
    else launch_level<false, UP, TF>(a, num_sms, max_per_sm, s);
}

template <bool FP16, bool UP>
static void launch_col_t(const AggArgs& a, int kp, int num_sms, cudaStream_t s)
{
    const int threads = (kp / 2 + (FP16 ? 1 : 0) + 31) / 32 * 32;
    const size_t smem = (TILE_FLOATS_COL + 2 * COL_MAX_ROWS) * sizeof(float);
    static bool configured = false;
    if (!configured) {
        cudaFuncSetAttribute(k_agg_col<FP16, UP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        configured = true;
    }
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_agg_col<FP16, UP>, threads, smem);
    per_sm = max(1, min(per_sm, 8));
    k_agg_col<FP16, UP><<<num_sms * per_sm, threads, smem, s>>>(a, kp);
}

template <bool UP>
static void launch_col(const AggArgs& a, bool fp16, int kp, int num_sms, cudaStream_t s)
{
    if (fp16) launch_col_t<true, UP>(a, kp, num_sms, s);
    else launch_col_t<false, UP>(a, kp, num_sms, s);
}

static AggArgs make_agg_args(Ctx& c, int l, const float* Ein, float* vol_up, float* vol_down)
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
    a.tbeg = c.ubeg;
    a.tstart = c.ustart_flag;
    a.tid = c.uid;
    a.d_ntiles = c.ints + IDX_NUNITS;
    a.vol = vol_up ? vol_up : c.vol;
    a.vout = vol_down ? vol_down : a.vol;
    a.Ein = Ein;
    a.refD = c.agg_refD;
    a.X = d.d + 1;
    a.volh = c.volh;
    a.nup = c.nup;
    a.nd = c.nfull;
    a.tickets = c.tickets;
    a.tflags = c.tflags;
    a.dflags = c.tflags + 2 * c.max_tiles;
    a.aggA = c.aggA;
    a.inclA = c.inclA;
    a.aggM = c.aggM;
    a.disp = c.disp[l];
    a.st = c.st;
    return a;
}

// tickets, look-back flags and done flags of both passes, on the context's stream
void aggregate_clear(Ctx& c)
{
    cudaMemsetAsync(c.tickets, 0, sizeof(int) * 2 * MAX_LIGHT_LEVELS, c.s);
    cudaMemsetAsync(c.tflags, 0, sizeof(int) * 4 * c.max_tiles, c.s);
}

void launch_aggregate_ex(Ctx& c, int l, const float* Ein, float* vol_up, float* vol_down)
{
    const LayerDims& d = c.dim[l];
    const AggArgs a = make_agg_args(c, l, Ein, vol_up, vol_down);
    // one launch per pass over every tile of the layer, in dependency order
    aggregate_clear(c);
    const bool fp16 = c.p.storage == HDP_STORE_FP16;
    const int tf = c.layer_tf[l];   // the size the layout was built with
    const int cap = c.tune.agg_ctas_per_sm;
    const int kp = (d.d + 1 + 3) / 4 * 4;
    if (tf == TILE_FLOATS_COL) {
        // one label set, wide rows: a CTA per tile, a thread per label column
        launch_col<true>(a, fp16, kp, c.num_sms, c.s);
        launch_col<false>(a, fp16, kp, c.num_sms, c.s);
        return;
    }
    if (tf == TILE_FLOATS_SMALL) {
        launch_level_s<true, TILE_FLOATS_SMALL>(a, fp16, c.num_sms, cap, c.s);
        launch_level_s<false, TILE_FLOATS_SMALL>(a, fp16, c.num_sms, cap, c.s);
    } else if (tf == TILE_FLOATS_HDP) {
        launch_level_s<true, TILE_FLOATS_HDP>(a, fp16, c.num_sms, cap, c.s);
        launch_level_s<false, TILE_FLOATS_HDP>(a, fp16, c.num_sms, cap, c.s);
    } else {
        launch_level_s<true, TILE_FLOATS>(a, fp16, c.num_sms, cap, c.s);
        launch_level_s<false, TILE_FLOATS>(a, fp16, c.num_sms, cap, c.s);
    }
}

void launch_aggregate(Ctx& c, int l) { launch_aggregate_ex(c, l, nullptr, nullptr, nullptr); }

// ---- one launch per pass over the tiles of many pairs (batches) -------------
// The pairs' arguments travel as one kernel parameter (at most AGG_MULTI_MAX
// pairs, under the 32 KB parameter limit).  Tickets run over the pairs one
// after another, each pair's tiles in its own dependency order, so a tile only
// waits on an earlier ticket of its own pair and every wait ends.
#define AGG_MULTI_MAX 64

struct AggMulti {
    int n;
    AggArgs a[AGG_MULTI_MAX];
};

template <bool FP16, bool UP, int TF>
__global__ void __launch_bounds__(AGG_THREADS, TF == TILE_FLOATS ? AGG_MINB_2048 : TF == TILE_FLOATS_HDP ? AGG_MINB_1024
                                                                                                    : AGG_MINB_512)
    k_agg_multi(const __grid_constant__ AggMulti m)
{
    constexpr int RM = tile_rows_max(TF);
    extern __shared__ float4 smem[];
    __shared__ int pre[AGG_MULTI_MAX + 1];
    if (threadIdx.x == 0) {
        int s = 0;
        for (int p = 0; p < m.n; ++p) {
            pre[p] = s;
            s += *m.a[p].d_ntiles;
        }
        pre[m.n] = s;
    }
    __syncthreads();
    const int total = pre[m.n];
    if (total == 0) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float4* X = smem + (size_t)warp * agg_warp_f4<TF>();
    float* M = (float*)(X + TF / 4);
    float* P = M + RM;
    float* PT = P + RM;
    float* Q = PT + RM;
    float4* CIN = (float4*)(Q + RM);
    int* CO = (int*)(CIN + 80);
    float* CS = (float*)(CO + AGG_CHUNK);
    __shared__ __align__(8) uint64_t bars[AGG_WARPS];
    uint64_t* bar = bars + warp;
    uint32_t bar_phase = 0;
    if (lane == 0) mbar_init(bar);
    __syncwarp();
    // the batch's own ticket: slot 1 of the first pair's tickets of this pass
    int* tk = m.a[0].tickets + (UP ? 0 : MAX_LIGHT_LEVELS) + 1;
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(tk, 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= total) break;
        int p = 0;
        while (p + 1 < m.n && pre[p + 1] <= t) ++p;
        const int tl = t - pre[p], nt = pre[p + 1] - pre[p];
        const int u = UP ? nt - 1 - tl : tl;
        tile_pass<FP16, UP, TF>(m.a[p], u, X, M, P, PT, Q, CIN, CO, CS, bar, bar_phase);
    }
    if (lane == 0) bulk_store_complete();
}

template <bool FP16, bool UP, int TF>
static void launch_multi_t(const AggMulti& m, int num_sms, int max_per_sm, cudaStream_t s)
{
    const size_t sm = agg_smem<TF>();
    static int per_sm = 0;
    if (per_sm == 0) {
        cudaFuncSetAttribute(k_agg_multi<FP16, UP, TF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_agg_multi<FP16, UP, TF>, AGG_THREADS, sm);
        if (per_sm < 1) per_sm = 1;
    }
    k_agg_multi<FP16, UP, TF><<<num_sms * min(per_sm, max_per_sm), AGG_THREADS, sm, s>>>(m);
}

template <bool UP>
static void launch_multi(const AggMulti& m, int tf, bool fp16, int num_sms, int cap, cudaStream_t s)
{
    if (tf == TILE_FLOATS_SMALL) {
        if (fp16) launch_multi_t<true, UP, TILE_FLOATS_SMALL>(m, num_sms, cap, s);
        else launch_multi_t<false, UP, TILE_FLOATS_SMALL>(m, num_sms, cap, s);
    } else if (tf == TILE_FLOATS_HDP) {
        if (fp16) launch_multi_t<true, UP, TILE_FLOATS_HDP>(m, num_sms, cap, s);
        else launch_multi_t<false, UP, TILE_FLOATS_HDP>(m, num_sms, cap, s);
    } else {
        if (fp16) launch_multi_t<true, UP, TILE_FLOATS>(m, num_sms, cap, s);
        else launch_multi_t<false, UP, TILE_FLOATS>(m, num_sms, cap, s);
    }
}

// Layer l of every context, on stream s, after each context's aggregate_clear
// (and the layer's forest and layout) has completed: the warp-kernel pairs
// grouped by (tile size, storage), one launch per group and pass; pairs of the
// column kernel one by one.  Returns the number of launches.
int launch_aggregate_multi(Ctx* const* cs, int n, int l, cudaStream_t s)
{
    int launches = 0;
    static AggMulti m;   // host staging only: kernel parameters are copied at launch (or into the graph)
    const int tfs[3] = {TILE_FLOATS_SMALL, TILE_FLOATS_HDP, TILE_FLOATS};
    for (int fp = 0; fp < 2; ++fp)
        for (int k = 0; k < 3; ++k) {
            int i = 0;
            while (i < n) {
                m.n = 0;
                int num_sms = 0, cap = 8;
                for (; i < n && m.n < AGG_MULTI_MAX; ++i) {
                    Ctx& c = *cs[i];
                    if ((c.p.storage == HDP_STORE_FP16) != (fp == 1) || c.layer_tf[l] != tfs[k]) continue;
                    m.a[m.n++] = make_agg_args(c, l, nullptr, nullptr, nullptr);
                    num_sms = c.num_sms;
                    cap = min(cap, c.tune.agg_ctas_per_sm);
                }
                if (m.n == 0) continue;
                launch_multi<true>(m, tfs[k], fp == 1, num_sms, cap, s);
                launch_multi<false>(m, tfs[k], fp == 1, num_sms, cap, s);
                launches += 2;
            }
        }
    for (int i = 0; i < n; ++i) {
        Ctx& c = *cs[i];
        if (c.layer_tf[l] != TILE_FLOATS_COL) continue;
        const AggArgs a = make_agg_args(c, l, nullptr, nullptr, nullptr);
        const int kp = (c.dim[l].d + 1 + 3) / 4 * 4;
        launch_col<true>(a, c.p.storage == HDP_STORE_FP16, kp, c.num_sms, s);
        launch_col<false>(a, c.p.storage == HDP_STORE_FP16, kp, c.num_sms, s);
        launches += 2;
    }
    return launches;
}
