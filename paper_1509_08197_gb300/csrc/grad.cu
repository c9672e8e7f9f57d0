// Differentiable tree aggregation on a full-range layer: Eq. C applied to a
// given cost volume, its adjoint and a soft-argmin readout with an L1 loss.
//
// C = A E with A(p, q) = exp(-W(p, q)/gamma) (Eqs. W, S, C).  A is symmetric,
// so dL/dE = A g for g = dL/dC: the same two passes applied to g.  For the
// tree edge e = (c, parent pi) the pairs whose path crosses e have one end in
// the subtree of c, which gives, with up-pass values E^, g^ and full
// aggregates C, G,
//   dL/dw_e   = -(s_e/gamma) sum_x [ g^(c)(C(pi) - s_e E^(c)) + E^(c)(G(pi) - s_e g^(c)) ],
//   dL/dgamma = -(1/gamma) sum_e w_e dL/dw_e.
// The backward recomputes the forward passes instead of keeping them.
//
// The cost volume itself is differentiable too: E(p, x) = (1 - alpha)
// min(dc, tau_c) + alpha min(dg, tau_g) (the matching cost of Sec. 3.3 with
// real-valued parameters), so
//   dL/dalpha = sum g_E (min(dg, tau_g) - min(dc, tau_c)),
//   dL/dtau_c = sum g_E (1 - alpha) [dc > tau_c],   dL/dtau_g = sum g_E alpha [dg > tau_g]
// (the truncation's derivative taken as 0 where dc = tau_c).  The edge
// weights may be given as real numbers instead of the image's integers; the
// tree stays the one built from the images, only the similarities
// s_e = exp(-w_e / gamma) follow the given weights.
#include "hdp_impl.cuh"

#define GACC_SLOTS 8   // [0] loss or edge sum, [1] valid pixels, [2..4] cost parameters

static int ensure_grad_buffers(Ctx& c)
{
    if (c.gvol[0]) return 0;
    for (int i = 0; i < 4; ++i)
        if (cudaMalloc((void**)&c.gvol[i], sizeof(float) * (c.vol_elems + 8)) != cudaSuccess) return -1;
    if (cudaMalloc((void**)&c.gacc, sizeof(double) * GACC_SLOTS) != cudaSuccess) return -1;
    if (cudaMalloc((void**)&c.wf, sizeof(float) * 2 * (size_t)c.dim[0].N) != cudaSuccess) return -1;
    return 0;
}

// dense [N][X] (pixel-major) <- layout rows
__global__ void k_gather_dense(const float* vol, const uint32_t* roff, const int* rowof, int N, int X, float* out)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)N * X) return;
    int v = (int)(i / X), x = (int)(i % X);
    out[i] = vol[roff[rowof[v]] + x];
}

__device__ __forceinline__ int edge_of(int v, int k, int W)
{
    return k == 0 ? 2 * (v - W) + 1 : k == 1 ? 2 * (v - 1) : k == 2 ? 2 * v : 2 * v + 1;
}

// one warp per node: dL/dw of the edge to its parent
__global__ void k_edge_grad(const float* Eu, const float* Cf, const float* gu, const float* G, const uint32_t* roff,
                            const int* rowof, const float* rs, const int* par, const int* pdir, const int* weights,
                            const float* wf, int N, int W, int X, float inv_scale, float gamma, float* gw, double* acc)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= N) return;
    const int c = warp, p = par[c];
    if (p < 0) return;
    const int rc = rowof[c], rp = rowof[p];
    const float s = fabsf(rs[rc]);
    const size_t oc = roff[rc], op = roff[rp];
    float t = 0.f;
    for (int x = lane; x < X; x += 32) {
        const float eu = Eu[oc + x], g_u = gu[oc + x];
        t += g_u * (Cf[op + x] - s * eu) + eu * (G[op + x] - s * g_u);
    }
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) {
        const int e = edge_of(c, pdir[c], W);
        const float g = -(s / gamma) * t;
        gw[e] = g;
        const double w = wf ? (double)wf[e] : (double)weights[e] * (double)inv_scale;
        atomicAdd(acc, w * (double)g);
    }
}

__global__ void k_ggamma(const double* acc, float gamma, float* out) { *out = (float)(-acc[0] / gamma); }

// similarities of the current layout for a new gamma or new real-valued
// weights wf (intensity units; null: the image's integer weights at scale
// 4^l); the sign bit keeps the path tops
__global__ void k_set_gamma(const int* lay, const int* par, const int* pdir, const int* weights, const float* wf,
                            int N, int W, float inv_scale, float inv_gamma, float* rs)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int v = lay[i];
    if (par[v] < 0) { rs[i] = -0.0f; return; }
    const int e = edge_of(v, pdir[v], W);
    float s = wf ? expf(-wf[e] * inv_gamma) : expf(-(float)weights[e] * inv_scale);
    rs[i] = signbit(rs[i]) ? -s : s;
}

void launch_set_gamma(Ctx& c, float gamma)
{
    const int l = c.tree_level;
    const LayerDims& d = c.dim[l];
    c.p.gamma = gamma;
    k_set_gamma<<<cdiv(d.N, 256), 256, 0, c.s>>>(c.lay, c.par, c.pdir, c.weights, c.use_wf ? c.wf : nullptr, d.N,
                                                 d.W, 1.0f / (gamma * (float)(1 << (2 * l))), 1.0f / gamma, c.rs);
}

int set_edge_weights(Ctx& c, const float* w)
{
    if (w) {
        if (ensure_grad_buffers(c)) return HDP_ERR_OOM;
        cudaMemcpyAsync(c.wf, w, sizeof(float) * 2 * (size_t)c.dim[c.tree_level].N, cudaMemcpyDeviceToDevice, c.s);
    }
    c.use_wf = w != nullptr;
    launch_set_gamma(c, c.p.gamma);
    return 0;
}

// E(p, x) over every pixel and label 0..X-1 of the loaded layer, pixel-major
__global__ void k_cost_volume(const int4* __restrict__ imL, const int4* __restrict__ imR, int W, int N, int X,
                              float inv_c, float inv_g, float alpha, float tau_c, float tau_g, float* __restrict__ E)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)N * X) return;
    const int p = (int)(i / X), x = (int)(i - (long long)p * X);
    const int px = p % W, xr = max(px - x, 0);
    const int4 a = imL[p], b = imR[p - px + xr];
    const float dc = (float)(abs(a.x - b.x) + abs(a.y - b.y) + abs(a.z - b.z)) * inv_c;
    const float dg = (float)abs(a.w - b.w) * inv_g;
    E[i] = (1.f - alpha) * fminf(dc, tau_c) + alpha * fminf(dg, tau_g);
}

#define CPG_THREADS 256

// dL/d(alpha, tau_c, tau_g) from dL/dE: per-thread sums over a grid-stride
// loop, a block reduction, one double atomic per block and parameter
__global__ void __launch_bounds__(CPG_THREADS) k_cost_param_grad(const int4* __restrict__ imL,
                                                                 const int4* __restrict__ imR, int W, int N, int X,
                                                                 float inv_c, float inv_g, float alpha, float tau_c,
                                                                 float tau_g, const float* __restrict__ gE,
                                                                 double* acc)
{
    __shared__ float red[3][CPG_THREADS / 32];
    float ga = 0.f, gc = 0.f, gg = 0.f;
    const long long n = (long long)N * X;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int p = (int)(i / X), x = (int)(i - (long long)p * X);
        const int px = p % W, xr = max(px - x, 0);
        const int4 a = imL[p], b = imR[p - px + xr];
        const float dc = (float)(abs(a.x - b.x) + abs(a.y - b.y) + abs(a.z - b.z)) * inv_c;
        const float dg = (float)abs(a.w - b.w) * inv_g;
        const float g = gE[i];
        ga += g * (fminf(dg, tau_g) - fminf(dc, tau_c));
        if (dc > tau_c) gc += g;
        if (dg > tau_g) gg += g;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ga += __shfl_xor_sync(0xffffffffu, ga, o);
        gc += __shfl_xor_sync(0xffffffffu, gc, o);
        gg += __shfl_xor_sync(0xffffffffu, gg, o);
    }
    if (lane == 0) {
        red[0][warp] = ga;
        red[1][warp] = gc;
        red[2][warp] = gg;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double t = 0.0;
        for (int w = 0; w < CPG_THREADS / 32; ++w) t += (double)red[threadIdx.x][w];
        const double f = threadIdx.x == 0 ? 1.0 : threadIdx.x == 1 ? (double)(1.f - alpha) : (double)alpha;
        atomicAdd(acc + threadIdx.x, t * f);
    }
}

__global__ void k_params_out(const double* acc, float* out)
{
    if (threadIdx.x < 3) out[threadIdx.x] = (float)acc[threadIdx.x];
}

static void cost_scales(const Ctx& c, float& inv_c, float& inv_g)
{
    const float sc = (float)(1 << (2 * c.tree_level));
    inv_c = 1.0f / (3.0f * sc);
    inv_g = 1.0f / (6.0f * sc);
}

void launch_cost_volume(Ctx& c, float alpha, float tau_c, float tau_g, float* E)
{
    const int l = c.tree_level;
    const LayerDims& d = c.dim[l];
    float inv_c, inv_g;
    cost_scales(c, inv_c, inv_g);
    const long long n = (long long)d.N * (d.d + 1);
    k_cost_volume<<<(unsigned)cdiv(n, 256LL), 256, 0, c.s>>>(c.imL[l], c.imR[l], d.W, d.N, d.d + 1, inv_c, inv_g,
                                                            alpha, tau_c, tau_g, E);
}

int launch_cost_param_grad(Ctx& c, float alpha, float tau_c, float tau_g, const float* gE, float* out)
{
    if (ensure_grad_buffers(c)) return HDP_ERR_OOM;
    const int l = c.tree_level;
    const LayerDims& d = c.dim[l];
    float inv_c, inv_g;
    cost_scales(c, inv_c, inv_g);
    double* acc = c.gacc + 2;
    cudaMemsetAsync(acc, 0, sizeof(double) * 3, c.s);
    const long long n = (long long)d.N * (d.d + 1);
    const long long nb = (n + CPG_THREADS - 1) / CPG_THREADS;
    const int blocks = (int)(nb < 4LL * c.num_sms ? nb : 4LL * c.num_sms);
    k_cost_param_grad<<<blocks, CPG_THREADS, 0, c.s>>>(c.imL[l], c.imR[l], d.W, d.N, d.d + 1, inv_c, inv_g, alpha,
                                                       tau_c, tau_g, gE, acc);
    k_params_out<<<1, 32, 0, c.s>>>(acc, out);
    return 0;
}

int grad_forward(Ctx& c, const float* E, float* C)
{
    if (ensure_grad_buffers(c)) return HDP_ERR_OOM;
    const int l = c.tree_level;
    const LayerDims& d = c.dim[l];
    launch_aggregate_ex(c, l, E, c.gvol[0], c.gvol[1]);
    const long long n = (long long)d.N * (d.d + 1);
    k_gather_dense<<<(unsigned)cdiv(n, 256LL), 256, 0, c.s>>>(c.gvol[1], c.roff, c.rowof, d.N, d.d + 1, C);
    return 0;
}

int grad_backward(Ctx& c, const float* E, const float* gC, float* gE, float* gw, float* ggamma)
{
    if (ensure_grad_buffers(c)) return HDP_ERR_OOM;
    const int l = c.tree_level;
    const LayerDims& d = c.dim[l];
    const int X = d.d + 1;
    launch_aggregate_ex(c, l, E, c.gvol[0], c.gvol[1]);    // recompute E^ and C
    launch_aggregate_ex(c, l, gC, c.gvol[2], c.gvol[3]);   // g^ and G = A g
    const long long n = (long long)d.N * X;
    k_gather_dense<<<(unsigned)cdiv(n, 256LL), 256, 0, c.s>>>(c.gvol[3], c.roff, c.rowof, d.N, X, gE);
    cudaMemsetAsync(gw, 0, sizeof(float) * 2 * (size_t)d.N, c.s);
    cudaMemsetAsync(c.gacc, 0, sizeof(double) * 2, c.s);
    const float inv_scale = 1.0f / (float)(1 << (2 * l));
    k_edge_grad<<<cdiv(d.N * 32, 256), 256, 0, c.s>>>(c.gvol[0], c.gvol[1], c.gvol[2], c.gvol[3], c.roff, c.rowof,
                                                      c.rs, c.par, c.pdir, c.weights, c.use_wf ? c.wf : nullptr,
                                                      d.N, d.W, X, inv_scale, c.p.gamma, gw, c.gacc);
    k_ggamma<<<1, 1, 0, c.s>>>(c.gacc, c.p.gamma, ggamma);
    return 0;
}

// soft-argmin readout d = sum_x x softmax(-C/T) and the mean L1 loss to gt over
// valid pixels, with dL/dC = sign(d - gt)/n_valid * (-1/T) p_x (x - d)
__global__ void k_count_valid(const uint8_t* valid, int N, double* acc)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int v = i < N && (!valid || valid[i]);
    v = __reduce_add_sync(0xffffffffu, v);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(acc + 1, (double)v);
}

__global__ void k_soft_argmin_l1(const float* C, const float* gt, const uint8_t* valid, int N, int X, float T,
                                 const double* acc, float* disp, double* loss, float* gC)
{
    const int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (p >= N) return;
    const float* row = C + (size_t)p * X;
    float m = INFINITY;
    for (int x = lane; x < X; x += 32) m = fminf(m, row[x]);
    for (int o = 16; o > 0; o >>= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
    float z = 0.f, sx = 0.f;
    for (int x = lane; x < X; x += 32) {
        const float e = expf(-(row[x] - m) / T);
        z += e;
        sx += e * (float)x;
    }
    for (int o = 16; o > 0; o >>= 1) {
        z += __shfl_xor_sync(0xffffffffu, z, o);
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
    }
    const float dhat = sx / z;
    if (lane == 0 && disp) disp[p] = dhat;
    const bool ok = !valid || valid[p];
    const double nv = acc[1] > 0 ? acc[1] : 1.0;
    if (lane == 0 && loss && ok && gt) atomicAdd(loss, (double)fabsf(dhat - gt[p]) / nv);
    if (gC) {
        const float sg = (ok && gt) ? (dhat > gt[p] ? 1.f : (dhat < gt[p] ? -1.f : 0.f)) / (float)nv : 0.f;
        for (int x = lane; x < X; x += 32) {
            const float e = expf(-(row[x] - m) / T) / z;
            gC[(size_t)p * X + x] = sg * (-1.f / T) * e * ((float)x - dhat);
        }
    }
}

int launch_soft_argmin_l1(Ctx& c, const float* C, const float* gt, const uint8_t* valid, float T, float* disp,
                          float* loss, float* gC)
{
    if (ensure_grad_buffers(c)) return HDP_ERR_OOM;
    const int l = c.tree_level;
    const LayerDims& d = c.dim[l];
    cudaMemsetAsync(c.gacc, 0, sizeof(double) * 2, c.s);
    k_count_valid<<<cdiv(d.N, 256), 256, 0, c.s>>>(valid, d.N, c.gacc);
    double* dl = (double*)c.gacc;   // slot 0 reused for the loss
    k_soft_argmin_l1<<<cdiv(d.N * 32, 256), 256, 0, c.s>>>(C, gt, valid, d.N, d.d + 1, T, c.gacc, disp,
                                                           loss ? dl : nullptr, gC);
    if (loss) {
        // loss (double) -> float output
        k_ggamma<<<1, 1, 0, c.s>>>(dl, -1.0f, loss);
    }
    return 0;
}
