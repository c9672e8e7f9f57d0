// Graph pyramid (Sec. 2.1), gradient plane and edge list (Eq. weight, DT-Rule 1).
#include "hdp_impl.cuh"

// layer 0: interleaved RGB uint8 (row pitch in bytes) -> int4 (R, G, B, 0)
__global__ void k_level0(const uint8_t* __restrict__ img, int pitch, int W, int H, int4* out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= W * H) return;
    int x = i % W, y = i / W;
    const uint8_t* p = img + (size_t)y * pitch + 3 * x;
    out[i] = make_int4(p[0], p[1], p[2], 0);
}

// S = 2 step: each node of layer l+1 averages the 2x2 square of layer l below
// it; squares cut by the right/bottom border average the children that exist.
// Values stay integers at scale 4^(l+1): dst = (4 / count) * sum(children).
__global__ void k_pyr(const int4* __restrict__ src, int W, int H, int4* dst, int Wn, int Hn)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Wn * Hn) return;
    int X = i % Wn, Y = i / Wn;
    int sx = 0, sy = 0, sz = 0, cnt = 0;
    for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
            int x = 2 * X + dx, y = 2 * Y + dy;
            if (x < W && y < H) {
                int4 v = src[y * W + x];
                sx += v.x; sy += v.y; sz += v.z;
                ++cnt;
            }
        }
    int f = 4 / cnt;
    dst[i] = make_int4(sx * f, sy * f, sz * f, 0);
}

// horizontal gradient of the grey sum, central difference, replicated border:
// g = Sum(x+1) - Sum(x-1) with Sum = R + G + B (real gradient g / (6 * 4^l)).
// On layer 0 (channels are bytes) pk also receives the pixel packed for the
// prior's byte-wise absolute differences.
__global__ void k_grad(int4* img, int W, int H, uint2* pk)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= W * H) return;
    int x = i % W, y = i / W;
    int4 a = img[y * W + min(x + 1, W - 1)];
    int4 b = img[y * W + max(x - 1, 0)];
    const int g = (a.x + a.y + a.z) - (b.x + b.y + b.z);
    img[i].w = g;
    if (pk) {
        const int4 v = img[i];
        pk[i] = make_uint2((uint32_t)v.x | (uint32_t)v.y << 8 | (uint32_t)v.z << 16, (uint32_t)g);
    }
}

void launch_level0(Ctx& c, int which, const uint8_t* d_img, int pitch)
{
    const LayerDims& d = c.dim[0];
    int4* out = which ? c.imR[0] : c.imL[0];
    k_level0<<<cdiv(d.N, 256), 256, 0, c.s>>>(d_img, pitch, d.W, d.H, out);
    k_grad<<<cdiv(d.N, 256), 256, 0, c.s>>>(out, d.W, d.H, c.pk0[which]);
}

void launch_pyramid(Ctx& c)
{
    for (int l = 1; l < c.nlev; ++l) {
        const LayerDims& a = c.dim[l - 1];
        const LayerDims& b = c.dim[l];
        for (int side = 0; side < 2; ++side) {
            int4* src = side ? c.imR[l - 1] : c.imL[l - 1];
            int4* dst = side ? c.imR[l] : c.imL[l];
            k_pyr<<<cdiv(b.N, 256), 256, 0, c.s>>>(src, a.W, a.H, dst, b.W, b.H);
            k_grad<<<cdiv(b.N, 256), 256, 0, c.s>>>(dst, b.W, b.H, nullptr);
        }
    }
}

// One thread per edge id e = 2*(y*W + x) + o (o = 0: right neighbour, 1: lower).
// w = largest per-channel absolute difference (Eq. weight, integer at scale
// 4^l).  With predicted sets (pixset != null), DT-Rule 1 (Eq. cri1) drops
// edges whose end points' PixelIntv do not intersect; an edge between
// different sets whose Jaccard ratio already reaches beta marks the layer as
// "risky" (DT-Rule 2 may then merge different sets).  Every edge id has its
// own key slot: (w << ebits | e) for a surviving edge, all ones otherwise, so
// that a stable sort on the weight bits alone yields the strict (w, id)
// order with the dropped slots last; count receives the survivors.
__global__ void k_edges(const int4* __restrict__ img, int W, int H, int ebits, const int* __restrict__ pixset,
                        const uint32_t* __restrict__ table, const int* __restrict__ canon, int bnum, int bden,
                        uint32_t* keys, int* count, int* weights, int* risky)
{
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int N = W * H;
    bool keep = false;
    uint32_t key = 0;
    if (e < 2 * N) {
        int p = e >> 1, o = e & 1;
        int x = p % W, y = p / W;
        bool valid = o == 0 ? (x + 1 < W) : (y + 1 < H);
        if (!valid) {
            weights[e] = -1;
        } else {
            int q = o == 0 ? p + 1 : p + W;
            int4 a = img[p], b = img[q];
            int w = max(abs(a.x - b.x), max(abs(a.y - b.y), abs(a.z - b.z)));
            weights[e] = w;
            keep = true;
            if (pixset) {
                int ip = pixset[p], iq = pixset[q];
                const uint32_t* mp = table + HDP_WORDS * ip;
                const uint32_t* mq = table + HDP_WORDS * iq;
                int inter = 0, uni = 0;
#pragma unroll
                for (int k = 0; k < HDP_WORDS; ++k) {
                    inter += __popc(mp[k] & mq[k]);
                    uni += __popc(mp[k] | mq[k]);
                }
                if (inter == 0) keep = false;                                  // DT-Rule 1
                else if (canon[ip] != canon[iq] && (long long)inter * bden >= (long long)bnum * uni)
                    *risky = 1;
            }
            key = ((uint32_t)w << ebits) | (uint32_t)e;
        }
    }
    if (e < 2 * N) keys[e] = keep ? key : 0xffffffffu;
    const int kept = __syncthreads_count(keep);   // one atomic per block on the grid-wide count
    if (threadIdx.x == 0 && kept) atomicAdd(count, kept);
}

// Random spanning tree (Sec. 4.1): the edges are shuffled and taken by the
// same union-find rules.  The shuffle is the order of a counter-based key:
// the top 31 bits of the i-th output of SplitMix64 (Steele, Lea and Flood,
// OOPSLA 2014) from state `seed`, i = l * 2^32 + e + 1, ties by edge id.
__device__ __forceinline__ uint32_t rt_key(unsigned long long seed, int l, int e)
{
    unsigned long long z = seed + (((unsigned long long)l << 32) + (unsigned long long)e + 1ull) *
                                      0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (uint32_t)(z >> 33);
}

// sort key of every slot: the edge's random key if it survived (packed key
// not all ones), else all ones (below no survivor); the value is the edge id
__global__ void k_rt_keys(const uint32_t* __restrict__ packed, int n2, unsigned long long seed, int l, uint32_t* rk,
                          uint32_t* rv)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n2) return;
    rk[e] = packed[e] == 0xffffffffu ? 0xffffffffu : rt_key(seed, l, e);
    rv[e] = (uint32_t)e;
}

// back to packed (w << ebits | e) keys in the random order, which every
// forest engine reads (the list position is the order)
__global__ void k_rt_pack(const uint32_t* __restrict__ rk, const uint32_t* __restrict__ rv,
                          const int* __restrict__ weights, int n2, int ebits, uint32_t* out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n2) return;
    const uint32_t e = rv[i];
    out[i] = rk[i] == 0xffffffffu ? 0xffffffffu : ((uint32_t)weights[e] << ebits) | e;
}

// M+* variants (Sec. 4.1): the tree is built on the layer's image after a
// 3x3 median per colour channel (border pixels replicated); the matching
// cost keeps the unfiltered image.  The median of nine is the middle element
// after an odd-even transposition sort (nine rounds of compare-exchange).
__device__ __forceinline__ int median9(int v[9])
{
#pragma unroll
    for (int round = 0; round < 9; ++round)
#pragma unroll
        for (int i = round & 1; i + 1 < 9; i += 2) {
            const int a = v[i], b = v[i + 1];
            v[i] = min(a, b);
            v[i + 1] = max(a, b);
        }
    return v[4];
}

__global__ void k_median3(const int4* __restrict__ img, int W, int H, int4* __restrict__ out)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= W * H) return;
    const int x = p % W, y = p / W;
    int r[9], g[9], b[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const int xx = min(max(x + k % 3 - 1, 0), W - 1), yy = min(max(y + k / 3 - 1, 0), H - 1);
        const int4 v = img[yy * W + xx];
        r[k] = v.x;
        g[k] = v.y;
        b[k] = v.z;
    }
    out[p] = make_int4(median9(r), median9(g), median9(b), img[p].w);
}

void launch_edges(Ctx& c, int l, int hdp)
{
    const LayerDims& d = c.dim[l];
    int ebits = edge_bits(d.N);
    const int4* wimg = c.imL[l];   // the image the tree's weights come from
    if (c.p.prefilter == HDP_PREFILTER_MEDIAN3) {
        k_median3<<<cdiv(d.N, 256), 256, 0, c.s>>>(c.imL[l], d.W, d.H, c.imF);
        wimg = c.imF;
    }
    cudaMemsetAsync(c.ints + IDX_NEDGES, 0, sizeof(int), c.s);
    cudaMemsetAsync(c.ints + IDX_RISKY, 0, sizeof(int), c.s);
    k_edges<<<cdiv(2 * d.N, 256), 256, 0, c.s>>>(wimg, d.W, d.H, ebits, hdp ? c.pixset : nullptr,
                                                   hdp ? c.table[l] : nullptr, hdp ? c.canon[l] : nullptr,
                                                   c.p.beta_num, c.p.beta_den, c.keys0, c.ints + IDX_NEDGES,
                                                   c.weights, c.ints + IDX_RISKY);
    // stable radix sort of all 2N slots on the weight field [ebits, ebits + 8 + 2l):
    // weights at layer l are below 255 * 4^l < 2^(8 + 2l) - 1, so the dropped
    // slots (all ones) come after every survivor
    int* slots = c.ints + IDX_ESLOTS;
    k_set_int<<<1, 1, 0, c.s>>>(slots, 2 * d.N);
    if (c.p.tree == HDP_TREE_RT) {
        // stable sort of all 2N slots on the full 32-bit random key, ids as
        // values (ties stay in id order); the dropped slots come last
        uint32_t* rk = c.keys1;
        uint32_t* rv = (uint32_t*)c.listA;
        k_rt_keys<<<cdiv(2 * d.N, 256), 256, 0, c.s>>>(c.keys0, 2 * d.N, c.p.rt_seed, l, rk, rv);
        int where = radix_sort(rk, rv, c.keys0, (uint32_t*)c.listB, slots, 2 * d.N, 32, c.tmp, c.scan, c.s, 0);
        const uint32_t* sk = where ? c.keys0 : rk;
        const uint32_t* sv = where ? (const uint32_t*)c.listB : rv;
        uint32_t* out = where ? c.keys1 : c.keys0;
        k_rt_pack<<<cdiv(2 * d.N, 256), 256, 0, c.s>>>(sk, sv, c.weights, 2 * d.N, ebits, out);
        c.sorted = out;
        return;
    }
    int where = radix_sort(c.keys0, nullptr, c.keys1, nullptr, slots, 2 * d.N, 8 + 2 * l, c.tmp, c.scan, c.s, ebits);
    c.sorted = where ? c.keys1 : c.keys0;
}
