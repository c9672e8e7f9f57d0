// GMM_l by EM (Sec. 2.2): the offset o = D_{l+1} - floor(D_l / 2) between a
// superpixel's disparity and the mode given by each of its children is
// collected over ground-truth training pairs and a Gaussian mixture is fitted
// to its distribution by EM.
//
//  * k_gt_down: the ground truth of the next layer.  A superpixel takes the
//    mean of its valid children divided by 2, rounded half up,
//    floor((sum + n) / (2 n)); -1 (invalid) without a valid child.
//  * k_offset_hist: histogram of the offsets of every valid pixel with a
//    valid superpixel, in shared memory per block, then one 64-bit atomic per
//    bin and block.  Integer work: exact.
//  * k_gmm_em: EM on the histogram in one CTA, one thread per bin (at most
//    511 bins: |o| <= 255).  E-step in the log domain; M-step weights and
//    means, then spreads about the new means, each by a fixed-order block
//    reduction, so a run is deterministic.  Spreads are floored at sd_min.
//    FP32 arithmetic.
#include "hdp_impl.cuh"

#define EM_THREADS 512
#define EM_MAX_K HDP_MAX_GMM

__global__ void k_gt_down(const int* __restrict__ gt, int W, int H, int* __restrict__ up)
{
    const int Wu = (W + 1) / 2, Hu = (H + 1) / 2;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Wu * Hu) return;
    const int X = i % Wu, Y = i / Wu;
    long long sum = 0;
    int n = 0;
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        const int x = 2 * X + (d & 1), y = 2 * Y + (d >> 1);
        if (x >= W || y >= H) continue;
        const int v = gt[(size_t)y * W + x];
        if (v < 0) continue;
        sum += v;
        ++n;
    }
    up[i] = n ? (int)((sum + n) / (2 * n)) : -1;
}

__global__ void k_offset_hist(const int* __restrict__ up, const int* __restrict__ lo, int W, int H, int range,
                              unsigned long long* __restrict__ hist)
{
    __shared__ unsigned int bins[2 * HDP_MAX_DISP + 1];
    const int nb = 2 * range + 1, Wu = (W + 1) / 2;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) bins[b] = 0u;
    __syncthreads();
    const int N = W * H;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const int x = i % W, y = i / W;
        const int a = lo[i], b = up[(size_t)(y >> 1) * Wu + (x >> 1)];
        if (a < 0 || b < 0) continue;
        const int o = b - a / 2;
        if (o < -range || o > range) continue;
        atomicAdd(&bins[o + range], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
        if (bins[b]) atomicAdd(&hist[b], (unsigned long long)bins[b]);
}

// sum of v over the block in a fixed order (warp shuffles, then the warp
// partials in index order); every thread receives the result
__device__ __forceinline__ float block_sum(float v, float* red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();   // red may still be read by the previous call
    if (lane == 0) red[warp] = v;
    __syncthreads();
    float t = 0.f;
    for (int w = 0; w < EM_THREADS / 32; ++w) t += red[w];
    return t;
}

__global__ void __launch_bounds__(EM_THREADS) k_gmm_em(const unsigned long long* __restrict__ hist, int range, int K,
                                                      int iters, float sd_min, float* __restrict__ out)
{
    __shared__ float red[EM_THREADS / 32];
    __shared__ float pi[EM_MAX_K], mu[EM_MAX_K], sd[EM_MAX_K];
    const int b = threadIdx.x, nb = 2 * range + 1;
    const float h = b < nb ? (float)hist[b] : 0.f;
    const float o = (float)(b - range);
    // start: every mean at the data mean, spreads s/2 .. growing by 4, equal weights
    const float tot = block_sum(h, red);
    const float m = block_sum(h * o, red) / tot;
    float s = sqrtf(block_sum(h * (o - m) * (o - m), red) / tot);
    s = fmaxf(s, sd_min);
    if (b < K) {
        pi[b] = 1.f / (float)K;
        mu[b] = m;
        sd[b] = fmaxf(s * exp2f(2.f * ((float)b - 0.5f * (float)(K - 1))), sd_min);
    }
    __syncthreads();
    float r[EM_MAX_K];
    for (int it = 0; it < iters; ++it) {
        // E-step: responsibilities of this bin, in the log domain
        float lmax = -INFINITY;
#pragma unroll
        for (int k = 0; k < EM_MAX_K; ++k) {
            r[k] = -INFINITY;
            if (k < K && pi[k] > 0.f) {
                const float z = (o - mu[k]) / sd[k];
                r[k] = logf(pi[k]) - logf(sd[k]) - 0.5f * z * z;
            }
            lmax = fmaxf(lmax, r[k]);
        }
        float den = 0.f;
#pragma unroll
        for (int k = 0; k < EM_MAX_K; ++k) {
            r[k] = k < K ? expf(r[k] - lmax) : 0.f;
            den += r[k];
        }
#pragma unroll
        for (int k = 0; k < EM_MAX_K; ++k) r[k] = r[k] / den;
        // M-step
        for (int k = 0; k < K; ++k) {
            const float w = h * r[k];
            const float nk = block_sum(w, red);
            const float sx = block_sum(w * o, red);
            const float mk = nk > 0.f ? sx / nk : 0.f;
            const float sv = block_sum(w * (o - mk) * (o - mk), red);
            __syncthreads();   // every thread has read this iteration's parameters of component k
            if (b == 0) {
                if (nk > 0.f) {
                    pi[k] = nk / tot;
                    mu[k] = mk;
                    sd[k] = fmaxf(sqrtf(sv / nk), sd_min);
                } else {
                    pi[k] = 0.f;
                }
            }
            __syncthreads();
        }
    }
    if (b < K) {
        out[3 * b] = pi[b];
        out[3 * b + 1] = mu[b];
        out[3 * b + 2] = sd[b];
    }
}

void launch_gt_down(const int* gt, int W, int H, int* up, cudaStream_t s)
{
    const int n = ((W + 1) / 2) * ((H + 1) / 2);
    k_gt_down<<<cdiv(n, 256), 256, 0, s>>>(gt, W, H, up);
}

void launch_offset_hist(const int* up, const int* lo, int W, int H, int range, unsigned long long* hist,
                        int num_sms, cudaStream_t s)
{
    const int blocks = min(cdiv(W * H, 256), 4 * num_sms);
    k_offset_hist<<<blocks, 256, 0, s>>>(up, lo, W, H, range, hist);
}

void launch_gmm_em(const unsigned long long* hist, int range, int K, int iters, float sd_min, float* out,
                   cudaStream_t s)
{
    k_gmm_em<<<1, EM_THREADS, 0, s>>>(hist, range, K, iters, sd_min, out);
}
