// Pixel-wise interval prediction (Sec. 2.2 and Sec. 3.1).
#include "hdp_impl.cuh"

__device__ __forceinline__ int cost_q(int4 a, int4 b, const CostK& k)
{
    int sum = abs(a.x - b.x) + abs(a.y - b.y) + abs(a.z - b.z);
    int dg = abs(a.w - b.w);
    return k.A * min(sum, k.Tc) + k.B * min(dg, k.Tg);
}

__device__ __forceinline__ void warp_argmin(int& v, int& x)
{
    for (int o = 16; o > 0; o >>= 1) {
        int ov = __shfl_xor_sync(0xffffffffu, v, o);
        int ox = __shfl_xor_sync(0xffffffffu, x, o);
        if (ov < v || (ov == v && ox < x)) { v = ov; x = ox; }
    }
}

// Prior P(D_l) by sampling (Sec. 3.1): one warp per centre (5a+2, 5b+2) of a
// full 5x5 square.  The centre's disparity is the argmin (lowest label on
// ties) of the 5x5 box sum of the exact integer cost, for the left view; the
// right view is checked at (cx - dL, cy) with the right-reference cost (box
// columns clamped to the image).  Consistent centres vote for dL.  Pixels are
// int4 (R, G, B, gradient) on every layer, or on layer 0, whose channels are
// bytes, uint2 (packed R, G, B; gradient) so that one byte-wise sum of
// absolute differences gives the colour term.
#define PRIOR_THREADS 256

__device__ __forceinline__ int cost_px(int4 a, int4 b, const CostK& k) { return cost_q(a, b, k); }
__device__ __forceinline__ int cost_px(uint2 a, uint2 b, const CostK& k)
{
    const int sum = (int)__vsadu4(a.x, b.x);
    const int dg = abs((int)a.y - (int)b.y);
    return k.A * min(sum, k.Tc) + k.B * min(dg, k.Tg);
}

// one centre, by one warp (sb: the warp's box in shared memory)
template <typename P>
__device__ __forceinline__ void prior_centre(const P* __restrict__ L, const P* __restrict__ R, int W, int dl,
                                             const CostK& ck, unsigned long long* hist, int na, int wid, P* sb)
{
    const int lane = threadIdx.x & 31;
    const int cx = 5 * (wid % na) + 2, cy = 5 * (wid / na) + 2;
    if (lane < 25) sb[lane] = L[(size_t)(cy + lane / 5 - 2) * W + cx + lane % 5 - 2];
    __syncwarp();
    int best = INT_MAX, bx = INT_MAX;
    for (int x = lane; x <= dl; x += 32) {
        int t = 0;
        for (int dy = -2; dy <= 2; ++dy) {
            const P* rowR = R + (size_t)(cy + dy) * W;
            for (int dx = -2; dx <= 2; ++dx) {
                int px = cx + dx;
                t += cost_px(sb[(dy + 2) * 5 + dx + 2], rowR[max(px - x, 0)], ck);
            }
        }
        if (t < best) { best = t; bx = x; }
    }
    warp_argmin(best, bx);
    const int dL = bx;
    const int u = cx - dL;
    if (u < 0) return;
    __syncwarp();
    if (lane < 25) sb[lane] = R[(size_t)(cy + lane / 5 - 2) * W + min(max(u + lane % 5 - 2, 0), W - 1)];
    __syncwarp();
    best = INT_MAX; bx = INT_MAX;
    for (int x = lane; x <= dl; x += 32) {
        int t = 0;
        for (int dy = -2; dy <= 2; ++dy) {
            const P* rowL = L + (size_t)(cy + dy) * W;
            for (int dx = -2; dx <= 2; ++dx) {
                int uu = min(max(u + dx, 0), W - 1);
                t += cost_px(sb[(dy + 2) * 5 + dx + 2], rowL[min(uu + x, W - 1)], ck);
            }
        }
        if (t < best) { best = t; bx = x; }
    }
    warp_argmin(best, bx);
    if (lane == 0 && bx == dL) atomicAdd(hist + dL, 1ull);
}

// warps stride over the centres, so the grid may be smaller than the centres
template <typename P>
__global__ void __launch_bounds__(PRIOR_THREADS) k_prior(const P* __restrict__ L, const P* __restrict__ R, int W,
                                                         int H, int dl, CostK ck, unsigned long long* hist)
{
    // the 25 pixels of the box in the reference view are the same for every
    // label: one copy per warp in shared memory
    __shared__ P box[PRIOR_THREADS / 32][25];
    const int na = W / 5, nb = H / 5;
    P* sb = box[threadIdx.x >> 5];
    const int nw = gridDim.x * (blockDim.x >> 5);
    for (int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; wid < na * nb; wid += nw) {   // whole warps
        prior_centre(L, R, W, dl, ck, hist, na, wid, sb);
        __syncwarp();
    }
}

__global__ void k_prior_finish(const unsigned long long* hist, int dl, long long* prior, int uniform)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j <= dl) prior[j] = uniform ? 1 : (long long)hist[j] + 1;   // Laplace count
}

void launch_prior(Ctx& c, int l, cudaStream_t s)
{
    const LayerDims& d = c.dim[l];
    unsigned long long* hist = c.hist + (size_t)l * 256;
    cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * 256, s);
    int uniform = c.p.prior == HDP_PRIOR_UNIFORM;
    if (!uniform) {
        int centres = (d.W / 5) * (d.H / 5);
        if (centres > 0) {
            // on the side stream at most three blocks per SM: the priors are
            // needed layers later, and a full grid shares every SM with the
            // latency-bound kernels of the coarser layers running meanwhile
            // (the top layer's one-CTA first pass above all)
            int blocks = cdiv(centres * 32, PRIOR_THREADS);
            if (s == c.s2) blocks = min(blocks, 3 * c.num_sms);
            if (l == 0)
                k_prior<uint2><<<blocks, PRIOR_THREADS, 0, s>>>(c.pk0[0], c.pk0[1], d.W, d.H, d.d,
                                                                  cost_consts(c, l), hist);
            else
                k_prior<int4><<<blocks, PRIOR_THREADS, 0, s>>>(c.imL[l], c.imR[l], d.W, d.H, d.d,
                                                                 cost_consts(c, l), hist);
        }
    }
    k_prior_finish<<<1, 256, 0, s>>>(hist, d.d, c.prior[l], uniform);
}

// GMM_l(o) = sum_k pi_k N(o | mu_k, sd_k), evaluated term by term without
// contracted multiply-adds, in the same operation order as the definition.
__device__ double gmm_density(const double* g, int K, double o)
{
    const double inv_sqrt_2pi = 0.39894228040143267794;
    double acc = 0.0;
    for (int k = 0; k < K; ++k) {
        double pi = g[3 * k], mu = g[3 * k + 1], sd = g[3 * k + 2];
        double z = __ddiv_rn(__dsub_rn(o, mu), sd);
        double e = exp(__dmul_rn(__dmul_rn(-0.5, z), z));
        acc = __dadd_rn(acc, __dmul_rn(__dmul_rn(pi, __ddiv_rn(inv_sqrt_2pi, sd)), e));
    }
    return acc;
}

// One block per upper label i (Eq. dpm + Eq. crtr).  Posterior row i is
// GMM_l(i - floor(j/2)) * prior[j] (row normalisation does not change the
// argmax or the ratio test).  Labels are ranked by decreasing posterior, ties
// to the lower j; starting from the argmax, j is added while
// P_j (1 - delta) >= delta * c, c the sum taken so far.  All-zero rows fall
// back to {2i, 2i+1}.
__global__ void k_table(const long long* __restrict__ prior, int dl, int dup, const double* __restrict__ gmm,
                        const int* gmm_k, int l, double delta, uint32_t* masks)
{
    __shared__ double P[256];
    __shared__ int J[256];
    __shared__ uint32_t m[HDP_WORDS];
    const int i = blockIdx.x, t = threadIdx.x;
    int K = gmm_k[l];
    const double* g = gmm + (size_t)l * HDP_MAX_GMM * 3;
    if (t < HDP_WORDS) m[t] = 0;
    if (t <= dl) {
        double o = (double)(i - t / 2);
        P[t] = __dmul_rn(gmm_density(g, K, o), (double)prior[t]);
    } else {
        P[t] = -1.0;
    }
    J[t] = t;
    __syncthreads();
    // bitonic sort, "before" = larger P, then smaller j
    for (int k = 2; k <= 256; k <<= 1) {
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
            int ix = t ^ jj;
            if (ix > t) {
                bool up = (t & k) == 0;
                double pa = P[t], pb = P[ix];
                int ja = J[t], jb = J[ix];
                bool a_before_b = pa > pb || (pa == pb && ja < jb);
                if (up ? !a_before_b : a_before_b) {
                    P[t] = pb; P[ix] = pa;
                    J[t] = jb; J[ix] = ja;
                }
            }
            __syncthreads();
        }
    }
    if (t == 0) {
        if (!(P[0] > 0.0)) {
            for (int j = 2 * i; j <= 2 * i + 1 && j <= dl; ++j) m[j >> 5] |= 1u << (j & 31);
        } else {
            double c = P[0];
            m[J[0] >> 5] |= 1u << (J[0] & 31);
            const double omd = __dsub_rn(1.0, delta);
            for (int r = 1; r <= dl; ++r) {
                if (__dmul_rn(P[r], omd) >= __dmul_rn(delta, c)) {
                    c = __dadd_rn(c, P[r]);
                    m[J[r] >> 5] |= 1u << (J[r] & 31);
                } else {
                    break;
                }
            }
        }
    }
    __syncthreads();
    if (t < HDP_WORDS) masks[(size_t)i * HDP_WORDS + t] = m[t];
}

// canon[i] = smallest row index with the same set as row i
__global__ void k_canon(const uint32_t* masks, int dup, int* canon)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > dup) return;
    int c = i;
    for (int r = 0; r < i; ++r) {
        bool eq = true;
        for (int k = 0; k < HDP_WORDS; ++k) eq = eq && masks[r * HDP_WORDS + k] == masks[i * HDP_WORDS + k];
        if (eq) { c = r; break; }
    }
    canon[i] = c;
}

void launch_table(Ctx& c, int l, cudaStream_t s)
{
    const LayerDims& d = c.dim[l];
    const LayerDims& u = c.dim[l + 1];
    double delta = c.p.delta0 * (double)(1 << l);
    k_table<<<u.d + 1, 256, 0, s>>>(c.prior[l], d.d, u.d, c.gmm, c.gmm_k, l, delta, c.table[l]);
    k_canon<<<cdiv(u.d + 1, 128), 128, 0, s>>>(c.table[l], u.d, c.canon[l]);
}

// PixelIntv(p) = row D_{l+1}(floor(x/2), floor(y/2)) of the table.
__global__ void k_pixsets(const int* __restrict__ dup_map, int Wu, int W, int H, int dup, int* pixset, DevStatus* st)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= W * H) return;
    int x = i % W, y = i / W;
    int v = dup_map[(y >> 1) * Wu + (x >> 1)];
    if (v < 0 || v > dup) {
        dev_fail(st, DEV_BAD_INPUT, 10);
        v = min(max(v, 0), dup);
    }
    pixset[i] = v;
}

void launch_pixsets(Ctx& c, int l)
{
    const LayerDims& d = c.dim[l];
    const LayerDims& u = c.dim[l + 1];
    k_pixsets<<<cdiv(d.N, 256), 256, 0, c.s>>>(c.disp[l + 1], u.W, d.W, d.H, u.d, c.pixset, c.st);
}
