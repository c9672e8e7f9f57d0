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
#include "hdp_impl.cuh"

static int ensure_grad_buffers(Ctx& c)
{
    if (c.gvol[0]) return 0;
    for (int i = 0; i < 4; ++i)
        if (cudaMalloc((void**)&c.gvol[i], sizeof(float) * (c.vol_elems + 8)) != cudaSuccess) return -1;
    if (cudaMalloc((void**)&c.gacc, sizeof(double) * 2) != cudaSuccess) return -1;
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
                            int N, int W, int X, float inv_scale, float gamma, float* gw, double* acc)
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
        atomicAdd(acc, (double)weights[e] * (double)inv_scale * (double)g);
    }
}

__global__ void k_ggamma(const double* acc, float gamma, float* out) { *out = (float)(-acc[0] / gamma); }

// similarities of the current layout for a new gamma (the sign bit keeps the path tops)
__global__ void k_set_gamma(const int* lay, const int* par, const int* pdir, const int* weights, int N, int W,
                            float inv_scale, float* rs)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int v = lay[i];
    if (par[v] < 0) { rs[i] = -0.0f; return; }
    float s = expf(-(float)weights[edge_of(v, pdir[v], W)] * inv_scale);
    rs[i] = signbit(rs[i]) ? -s : s;
}

void launch_set_gamma(Ctx& c, float gamma)
{
    const int l = c.tree_level;
    const LayerDims& d = c.dim[l];
    c.p.gamma = gamma;
    k_set_gamma<<<cdiv(d.N, 256), 256, 0, c.s>>>(c.lay, c.par, c.pdir, c.weights, d.N, d.W,
                                                 1.0f / (gamma * (float)(1 << (2 * l))), c.rs);
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
                                                      c.rs, c.par, c.pdir, c.weights, d.N, d.W, X, inv_scale,
                                                      c.p.gamma, gw, c.gacc);
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
