// Tree-based refinement at layer 0 (Sec. 3.3, last paragraph: the
// refinement of the cited MST/ST methods, integrated into the framework).
//
//  * The right view's disparity map is the method with the views exchanged.
//    Mirroring both images left-right turns "right pixel x matches left pixel
//    x + d" into the left-reference convention, so the same pipeline runs on
//    the mirrored, exchanged pair (k_mirror) and its map is read mirrored.
//  * k_lr_check: a left pixel (x, y) with disparity D_L is stable iff
//    x - D_L >= 0 and D_R(x - D_L, y) = D_L; refD = D_L there, -1 elsewhere.
//    It also writes D_R in the right view's own frame (for inspection).
//  * The refinement cost |x - refD(p)| (0 at unstable pixels) is aggregated
//    over layer 0's forest by the aggregation kernels (AggArgs::refD) and its
//    WTA is the refined map.
#include "hdp_impl.cuh"

__global__ void k_mirror(const uint8_t* __restrict__ src, int pitch, int W, int H, uint8_t* __restrict__ dst)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= W * H) return;
    const int x = i % W, y = i / W;
    const uint8_t* s = src + (size_t)y * pitch + 3 * (size_t)(W - 1 - x);
    uint8_t* d = dst + 3 * (size_t)i;
    d[0] = s[0];
    d[1] = s[1];
    d[2] = s[2];
}

__global__ void k_lr_check(const int* __restrict__ DL, const int* __restrict__ DRm, int W, int H, int* __restrict__ refD,
                           int* __restrict__ refR)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= W * H) return;
    const int x = i % W, y = i / W;
    const int row = y * W;
    refR[i] = DRm[row + (W - 1 - x)];   // the right map in its own frame
    const int d = DL[i], xr = x - d;
    refD[i] = (xr >= 0 && xr < W && DRm[row + (W - 1 - xr)] == d) ? d : -1;
}

void launch_mirror(const uint8_t* src, int pitch, int W, int H, uint8_t* dst, cudaStream_t s)
{
    k_mirror<<<cdiv(W * H, 256), 256, 0, s>>>(src, pitch, W, H, dst);
}

// c.disp[0] holds D_L, c.dispRm the mirrored run's map, and layer 0's forest
// and layout are loaded: check, then aggregate the refinement cost (its WTA
// overwrites c.disp[0])
void launch_refine(Ctx& c)
{
    const LayerDims& d = c.dim[0];
    k_lr_check<<<cdiv(d.N, 256), 256, 0, c.s>>>(c.disp[0], c.dispRm, d.W, d.H, c.refD, c.refR);
    c.agg_refD = c.refD;
    launch_aggregate(c, 0);
    c.agg_refD = nullptr;
}
