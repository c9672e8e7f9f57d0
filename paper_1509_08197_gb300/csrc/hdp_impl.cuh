// Internal state of an HDP context and the per-stage launchers.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <string>

#include "../../include/hdp.h"
#include "common.cuh"
#include "prims.cuh"

#define MAX_LIGHT_LEVELS 32
// aggregation tiles: consecutive rows of one width holding about tf costs.
// Layers with one label set (full range, the top layer: wide rows, big light
// levels) use TILE_FLOATS; predicted layers (narrow rows, light levels with
// fewer tiles than the GPU has warps) use TILE_FLOATS_HDP, which also fits
// more CTAs per SM.  Measured on the 1390x1110 pair: HDP aggregation 2.95 ms
// with 2048-float tiles, 1.95 ms with 1024; full range 6.0 ms with 2048, 7.9
// ms with 1024.
#define TILE_FLOATS 2048
#define TILE_FLOATS_HDP 1024
// layers of fewer nodes than this are latency-bound (a chain of light levels,
// one tile deep each): they take tiles of TILE_FLOATS_SMALL costs, so a
// warp's share of a tile is short.  TILE_FLOATS_SMALL >= 256 + 4 (the widest
// FP16 row with its mass column).
#define TILE_FLOATS_SMALL 512
// big layers with one label set and rows of at least COL_MIN_KP labels: the
// column kernel (a CTA per tile, a thread per label column), taller tiles
#define TILE_FLOATS_COL 8192
#define COL_MIN_KP 64
// aggregation CTAs (4 warps) per SM: launch bounds of the three tile sizes
// and the default cap (occupancy limits each kernel below the cap)
#define AGG_MINB_2048 4
#define AGG_MINB_1024 7
#define AGG_MINB_512 5
#define AGG_CTAS_DEFAULT 8
// defaults of the layout knobs (hdp_tuning): below these node counts layers
// take 512-float tiles
#define SMALL_TILE_NODES (1 << 17)       // layers with one label set (full range, the top layer)
#define SMALL_TILE_NODES_HDP (1 << 19)   // predicted layers (the 1390x1110 pair: layers 1-3)
#define SCR_STRIDE 264   // floats per tile in the look-back scratch (256 labels + mass, padded)
// rows per tile at most: tf / 8 (the narrowest rows, kp = 4, fill half a tile)
__host__ __device__ __forceinline__ constexpr int tile_rows_max(int tf) { return tf / 8; }
// rows of width kp per tile; FP16 storage adds a support-mass float4 per row
// in shared memory (extra = 4), so that a tile always fits tf floats
__host__ __device__ __forceinline__ int tile_rows_of(int kp, int extra, int tf)
{
    const int r = kp + extra >= tf ? 1 : tf / (kp + extra);
    return r < tile_rows_max(tf) ? r : tile_rows_max(tf);
}

struct LayerDims {
    int W, H, N, d;   // size and largest label of the layer
};

// Per-layer cost arithmetic: Mq = A * min(sum|dI|, Tc) + B * min(|dg|, Tg) and
// M = Mq * inv (the matching cost in 0..255 intensity units), exact integers.
struct CostK {
    int A, B, Tc, Tg;
    float inv;
};

struct Ctx {
    hdp_params p;
    hdp_tuning tune = {AGG_CTAS_DEFAULT, 1, 2048, 131072, 4096, 1 << 24, SMALL_TILE_NODES, SMALL_TILE_NODES_HDP,
                       COL_MIN_KP};
    int layer_tf[HDP_MAX_LEVELS] = {};   // tile size each layer's layout was built with (launch_order)
    cudaStream_t s = nullptr;
    // side stream: the priors and interval tables of the predicted layers need
    // only that layer's images, so they run beside the coarser layers' work
    cudaStream_t s2 = nullptr;
    cudaEvent_t ev_fork = nullptr;
    cudaEvent_t ev_side[HDP_MAX_LEVELS] = {};
    int side_pending[HDP_MAX_LEVELS] = {};
    unsigned long long* hist = nullptr;   // [HDP_MAX_LEVELS][256] prior histograms
    int nlev = 0;     // layers processed
    int top = 0;      // index of the top layer
    LayerDims dim[HDP_MAX_LEVELS];
    int num_sms = 0;
    int a20 = 0, tc3 = 0, tg6 = 0;

    // arena
    char* arena = nullptr;
    size_t arena_bytes = 0, arena_used = 0;

    // images: int4 (R, G, B at scale 4^l, horizontal gradient g)
    int4* imL[HDP_MAX_LEVELS] = {};
    int4* imR[HDP_MAX_LEVELS] = {};
    uint2* pk0[2] = {};   // layer 0 packed for the prior: R | G << 8 | B << 16, gradient
    uint8_t* stage_l = nullptr;   // upload buffers (tightly packed RGB)
    uint8_t* stage_r = nullptr;
    int32_t* disp[HDP_MAX_LEVELS] = {};
    int32_t* disp_host_stage = nullptr;

    // interval prediction (layers below the top)
    long long* prior[HDP_MAX_LEVELS] = {};
    uint32_t* table[HDP_MAX_LEVELS] = {};
    int* canon[HDP_MAX_LEVELS] = {};
    double* gmm = nullptr;   // [HDP_MAX_LEVELS][HDP_MAX_GMM][3]
    int* gmm_k = nullptr;    // [HDP_MAX_LEVELS]
    uint32_t* full_mask = nullptr;   // per layer: the set {0..d_l}  [HDP_MAX_LEVELS][8]

    // work buffers, sized for layer 0 and reused by every layer
    int* pixset = nullptr;           // table row of each pixel (null use: full range)
    int* weights = nullptr;          // [2N] edge weights (-1 invalid)
    uint32_t *keys0 = nullptr, *keys1 = nullptr;   // sorted (w << ebits | e)
    uint32_t* sorted = nullptr;      // points at keys0 or keys1
    int* cls_start = nullptr;        // weight-class starts in the sorted list
    int *parent = nullptr, *csize = nullptr, *intw = nullptr, *best = nullptr, *best2 = nullptr;
    int *rootof = nullptr, *minid = nullptr, *dtroot = nullptr;
    uint32_t* T = nullptr;           // [N][8] TreeIntv at union-find roots
    uint8_t* in_tree = nullptr;      // [2N]
    int *listA = nullptr, *listB = nullptr, *raA = nullptr, *rbA = nullptr, *raB = nullptr, *rbB = nullptr;
    int* hooked = nullptr;
    int *win = nullptr, *wtmp = nullptr, *wra = nullptr, *wrb = nullptr, *wst = nullptr;

    // tree order / layout
    uint8_t* adj = nullptr;          // 4-bit tree adjacency (up, left, right, down)
    uint32_t* aoff = nullptr;        // arc offsets per node (N + 1)
    int *succ = nullptr, *val = nullptr, *succ2 = nullptr, *val2 = nullptr;   // [2N] arcs
    int *par = nullptr, *pdir = nullptr, *sub = nullptr, *hdir = nullptr;
    int* tpos_down = nullptr;        // tour position of the arc parent->v
    int* tpos_up = nullptr;
    I4* vals4 = nullptr;             // per node (1, off2, off3, light)
    I4* tour = nullptr;              // [2N]
    uint32_t* tbase = nullptr;       // per node: exclusive scan of tour lengths of roots
    uint32_t* nbase = nullptr;       // per node: exclusive scan of tree sizes of roots
    int *depth = nullptr, *pre2 = nullptr, *pre3 = nullptr, *light = nullptr;
    uint32_t *ka = nullptr, *va = nullptr, *kb = nullptr, *vb = nullptr;   // sort scratch [N]
    int* bfs = nullptr;              // [N]
    int* lay = nullptr;              // layout row -> pixel
    int* rowof = nullptr;            // pixel -> layout row
    int* kp = nullptr;               // padded width per row
    uint32_t* roff = nullptr;        // row offsets in floats (N + 1)
    float* rs = nullptr;             // similarity to parent, negative zero/sign for path tops
    int* prow = nullptr;             // parent row (-1 root)
    int* rdt = nullptr;              // union-find root of the row's tree (TreeIntv index)
    uint32_t* lcoff = nullptr;       // light-children offsets (N + 1)
    int* lcrow = nullptr;            // light-children rows
    int* runstart = nullptr;         // per (level, width) key: first row
    uint32_t* ustart_flag = nullptr; // tile start flags
    uint32_t* uid = nullptr;         // tile ids
    int* ubeg = nullptr;             // tile first row
    size_t max_tiles = 0;
    int* tflags = nullptr;           // [2][max_tiles] look-back states (0 none, 1 aggregate, 2 inclusive)
    float* aggA = nullptr;           // [max_tiles][SCR_STRIDE]
    float* inclA = nullptr;          // [max_tiles][SCR_STRIDE]
    float* aggM = nullptr;           // [max_tiles]
    int* lvl_first = nullptr;        // [MAX_LIGHT_LEVELS] first tile of the level
    int* lvl_count = nullptr;        // [MAX_LIGHT_LEVELS]
    int* tickets = nullptr;          // [2][MAX_LIGHT_LEVELS]
    int* nunits = nullptr;

    // cost volume and masses
    float* vol = nullptr;
    __half* volh = nullptr;
    float *nup = nullptr, *nfull = nullptr;
    size_t vol_elems = 0;
    float *gvol[4] = {nullptr, nullptr, nullptr, nullptr};   // differentiable path: U_E, C_E, U_g, G (lazy)
    double* gacc = nullptr;
    float* wf = nullptr;       // differentiable path: real-valued edge weights per grid edge id (lazy)
    bool use_wf = false;       // the loaded layout's similarities follow wf

    // scalars on the device
    int* ints = nullptr;   // see IDX_* below
    ScanState scan = {};   // single-pass scan scratch (zero between scans)
    ScanStateI4 scan4 = {};
    uint32_t* tmp = nullptr;   // scan / sort scratch
    size_t tmp_words = 0;
    DevStatus* st = nullptr;
    int4* imF = nullptr;   // median-filtered layer image (M+* variants)
    // refinement (refine.cu): the right view's map as computed on mirrored
    // views, the checked left map (refD) and the right map in its own frame
    int* dispRm = nullptr;
    int* refD = nullptr;
    int* refR = nullptr;
    const int* agg_refD = nullptr;   // set only while the refinement pass is enqueued
    int refined = 0;                 // the refinement stages hold the last hdp_refine
    unsigned long long* zero64 = nullptr;   // a word nothing writes (the wait probes read it)

    int tree_level = -1;       // layer whose forest/layout is in the work buffers
    int built = 0;
    std::string err;
};

// slots of Ctx::ints
enum {
    IDX_NEDGES = 0, IDX_RISKY, IDX_NCLS, IDX_NARCS, IDX_N, IDX_CTR0, IDX_CTR1, IDX_CTR2, IDX_CTR3, IDX_CTR4,
    IDX_K, IDX_NTREES, IDX_NLC, IDX_NUNITS, IDX_ENGINE, IDX_CHANGED, IDX_DRROUNDS, IDX_DRWINDOWS, IDX_NNODES, IDX_ESLOTS, IDX_RSORTN,
    IDX_TMP0 = 24, IDX_TMP1, IDX_TMP2, IDX_TMP3, IDX_COUNT = 32
};

// image.cu
// the aggregation tile size of layer l (see TILE_FLOATS_HDP)
// tile size of layer l's aggregation layout under tuning t
inline int tile_floats_for(const Ctx& c, int l, const hdp_tuning& t)
{
    const bool one_set = c.p.mode == HDP_MODE_FULL || l == c.top;
    if (c.dim[l].N < (one_set ? t.tile_small_nodes : t.tile_small_nodes_hdp)) return TILE_FLOATS_SMALL;
    if (one_set && (c.dim[l].d + 1 + 3) / 4 * 4 >= t.col_min_labels) return TILE_FLOATS_COL;
    return one_set ? TILE_FLOATS : TILE_FLOATS_HDP;
}
// for a new layout (the aggregation then reads c.layer_tf[l])
inline int layer_tile_floats(const Ctx& c, int l) { return tile_floats_for(c, l, c.tune); }

void launch_level0(Ctx& c, int which, const uint8_t* d_img, int pitch);
void launch_pyramid(Ctx& c);
void launch_edges(Ctx& c, int l, int hdp);

// range.cu
void launch_prior(Ctx& c, int l, cudaStream_t s);
void launch_table(Ctx& c, int l, cudaStream_t s);
void launch_pixsets(Ctx& c, int l);

// forest.cu
void launch_forest(Ctx& c, int l, int hdp);
int edge_bits(int N);

// order.cu
void launch_order(Ctx& c, int l);
void launch_bfs(Ctx& c, int l);

// aggregate.cu
void launch_aggregate(Ctx& c, int l);
void launch_aggregate_ex(Ctx& c, int l, const float* Ein, float* vol_up, float* vol_down);
// batches: clear a context's aggregation state, then aggregate layer l of many contexts together
void aggregate_clear(Ctx& c);
int launch_aggregate_multi(Ctx* const* cs, int n, int l, cudaStream_t s);

// grad.cu
// GMM_l by EM (gmm.cu)
void launch_gt_down(const int* gt, int W, int H, int* up, cudaStream_t s);
void launch_offset_hist(const int* up, const int* lo, int W, int H, int range, unsigned long long* hist,
                        int num_sms, cudaStream_t s);
void launch_gmm_em(const unsigned long long* hist, int range, int K, int iters, float sd_min, float* out,
                   cudaStream_t s);

// refinement (refine.cu)
void launch_mirror(const uint8_t* src, int pitch, int W, int H, uint8_t* dst, cudaStream_t s);
void launch_refine(Ctx& c);

int grad_forward(Ctx& c, const float* E, float* C);
int grad_backward(Ctx& c, const float* E, const float* gC, float* gE, float* gw, float* ggamma);
void launch_set_gamma(Ctx& c, float gamma);
int set_edge_weights(Ctx& c, const float* w);
void launch_cost_volume(Ctx& c, float alpha, float tau_c, float tau_g, float* E);
int launch_cost_param_grad(Ctx& c, float alpha, float tau_c, float tau_g, const float* gE, float* out);
int launch_soft_argmin_l1(Ctx& c, const float* C, const float* gt, const uint8_t* valid, float T, float* disp,
                          float* loss, float* gC);

// helpers
CostK cost_consts(const Ctx& c, int l);
cudaError_t coop_launch(const void* fn, int threads, void** args, cudaStream_t s, int blocks_per_sm, int* used_blocks,
                        size_t smem = 0, int max_blocks = 0);
