/*
 * hdp.h - C ABI of the GB300 (sm_103a) implementation of hierarchical
 * disparity prediction (HDP) stereo matching with non-local tree aggregation,
 * Luo et al., "Fast Non-local Stereo Matching based on Hierarchical Disparity
 * Prediction", arXiv 1509.08197.
 *
 * Problem statement (Sec. 1 and Sec. 2.1): rectified left/right RGB images and
 * a disparity bound d in, a disparity map of the left view out.  The method
 * runs top-down over a graph pyramid of L+1 layers (Sec. 3): at each layer it
 * predicts per-pixel disparity sets (Sec. 3.1), builds the HDP forest of
 * disparity trees (Sec. 3.2), aggregates the matching cost over the forest
 * and takes the winner-takes-all label (Sec. 3.3).
 *
 * Conventions for every call:
 *   - Pointers named d_* are CUDA device pointers owned by the caller; h_*
 *     are host pointers owned by the caller.  The context owns its own device
 *     workspace, allocated once by hdp_create and released by hdp_destroy.
 *   - All device work is enqueued on the stream given to hdp_create, in order.
 *     Calls return after enqueueing unless stated otherwise.
 *   - Every call returns an hdp_status and never aborts the process.  Errors
 *     raised asynchronously on the device (including a bounded wait that ran
 *     out, HDP_ERR_TIMEOUT) are reported by the next call that synchronises
 *     (hdp_sync, the *_host calls, hdp_get_stage) or by hdp_destroy;
 *     hdp_sync clears a device-side error once it has reported it.
 *     hdp_last_error returns a text description of the last failure.
 *   - A context is not thread-safe; distinct contexts are independent.
 */
#ifndef HDP_H
#define HDP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hdp_ctx hdp_ctx;

typedef enum {
    HDP_OK = 0,
    HDP_ERR_ARG = -1,      /* invalid argument: the call did nothing */
    HDP_ERR_CUDA = -2,     /* a CUDA runtime call failed */
    HDP_ERR_OOM = -3,      /* device allocation failed */
    HDP_ERR_TIMEOUT = -4,  /* a bounded device-side wait gave up */
    HDP_ERR_STATE = -5     /* calls made in the wrong order */
} hdp_status;

enum { HDP_TREE_MST = 0, HDP_TREE_ST = 1, HDP_TREE_RT = 2 };
enum { HDP_MODE_HDP = 0, HDP_MODE_FULL = 1 };
enum { HDP_PRIOR_SAMPLED = 0, HDP_PRIOR_UNIFORM = 1 };
enum { HDP_STORE_FP32 = 0, HDP_STORE_FP16 = 1 };
enum { HDP_PREFILTER_NONE = 0, HDP_PREFILTER_MEDIAN3 = 1 };

#define HDP_MAX_LEVELS 8
#define HDP_MAX_GMM 8
#define HDP_MAX_DISP 255

/*
 * Parameters.  Sizes: width, height >= 2; 1 <= max_disp <= 255 (labels
 * 0..max_disp); 1 <= levels <= 8.
 *   levels  number of pyramid layers L+1 (Sec. 2.1, S = 2 fixed, as in Sec. 4.1);
 *           mode HDP_MODE_FULL ignores it and aggregates one full-range layer.
 *   tree    HDP_TREE_MST (the MST of [MST]), HDP_TREE_ST (segment tree, [ST]:
 *           Kruskal merging w <= Int(C) + st_k/|C| for both trees, then
 *           linking) or HDP_TREE_RT (random spanning tree, Sec. 4.1: the edges
 *           shuffled, then the same union-find rules; the aggregation still
 *           uses the edge weights).
 *   prefilter HDP_PREFILTER_MEDIAN3 gives the M+* variants of Sec. 4.1: the
 *           edge weights (Eq. weight) of every layer come from that layer's
 *           image after a 3x3 median per colour channel (borders replicated);
 *           the matching cost keeps the unfiltered images.  Default NONE.
 *   rt_seed seed of the random tree's shuffle: edges in increasing order of
 *           the top 31 bits of SplitMix64 output number l * 2^32 + e + 1 from
 *           state rt_seed (edge id e, layer l), ties by edge id.
 *   gamma   Eq. (S): similarity exp(-W/gamma), W in 0..255 intensity units.
 *   alpha, tau_c, tau_g  matching cost of [Cost2] (Sec. 3.3); 20*alpha,
 *           3*tau_c and 6*tau_g must be integers (the cost is evaluated exactly).
 *   beta_num/beta_den  DT-Rule 2 threshold beta (Eq. DTrules) as a rational.
 *   delta0  Eq. (crtr) threshold, delta_l = delta0 * 2^l (Sec. 4.1).
 *   prior   P(D_l) sampled on 5x5 squares with a left-right check (Sec. 3.1)
 *           or uniform.
 *   gmm_k[l], gmm[l][k] = {pi, mu, sd}: GMM_l of Sec. 2.2 for predicted layer l;
 *           gmm_k[l] = 0 selects the default single N(0, 1).
 *   storage cost volume storage: FP32, or FP16 normalised by the per-node
 *           support mass (arithmetic is FP32 either way).
 */
typedef struct {
    int width, height;
    int max_disp;
    int levels;
    int tree;
    int mode;
    float gamma;
    float alpha, tau_c, tau_g;
    int st_k;
    int beta_num, beta_den;
    double delta0;
    int prior;
    int gmm_k[HDP_MAX_LEVELS];
    double gmm[HDP_MAX_LEVELS][HDP_MAX_GMM][3];
    int storage;
    unsigned long long rt_seed;
    int prefilter;
} hdp_params;

/*
 * Launch-shape knobs (no counterpart in the paper).  The first six give the
 * same results bit for bit (the forest engines are exact, and the carries of
 * the aggregation are evaluated in a fixed order); only the speed changes.
 * The three layout knobs below keep forests, orders and every other integer
 * stage bit for bit, but a tile size fixes the order of the FP32 additions,
 * so aggregated costs move within rounding and the WTA only at near ties.
 * Defaults in brackets; hdp_set_tuning rejects values outside the ranges.
 *   agg_ctas_per_sm        aggregation CTAs per SM at most, 1..8 [8] (each
 *                          kernel also stops at its own occupancy: 4 CTAs
 *                          of 2048-float tiles, 7 of 1024, 5 of 512)
 *   region_ctas_per_sm     region-engine CTAs per SM, 1..4 [1] (the CTA with
 *                          the largest region is the critical path: alone on
 *                          its SM it runs faster)
 *   big_class_edges        first pass of big full-range layers: a weight class
 *                          with at least this many edges runs as a grid
 *                          Boruvka, smaller ones in shared-memory windows,
 *                          64..4096 [2048]
 *   one_cta_nodes          layers with fewer nodes run the first pass in one
 *                          CTA and the risky fallback in one block,
 *                          1024..1<<24 [131072]
 *   boruvka_edges_per_cta  cooperative grids get one CTA per this many edges
 *                          (at most one wave), 512..1<<20 [4096]
 *   region_max_nodes       HDP layers with fewer nodes run the forest
 *                          region by region: the segment tree's first pass
 *                          over same-set regions, and every pass of a risky
 *                          layer (MST, ST or RT) over the components of the
 *                          edges that survive DT-Rule 1; bigger layers take
 *                          the first pass by weight class and a risky layer
 *                          on one CTA, 0..1<<30 [1<<24]
 * Aggregation layout: how many costs a tile holds and which kernel walks it.
 *   tile_small_nodes       one-label-set layers (full range, the top layer)
 *                          with fewer nodes use tiles of 512 costs (else the
 *                          column kernel or tiles of 2048), 0..1<<30 [1<<17]
 *   tile_small_nodes_hdp   predicted layers with fewer nodes use tiles of 512
 *                          costs, bigger ones 1024, 0..1<<30 [1<<19]
 *   col_min_labels         one-label-set layers of at least tile_small_nodes
 *                          nodes whose rows hold at least this many label
 *                          slots take the column kernel (a CTA per tile of
 *                          8192 costs, a thread per two labels) instead of
 *                          the warp kernel (a warp per tile, four labels per
 *                          lane step), 64..257 [64] (257: never)
 * A tuning whose layouts need more tiles than the context's look-back scratch
 * holds is refused with HDP_ERR_ARG; hdp_create sizes it for the defaults
 * and for one-set layers on the warp kernel (smaller tiles than the defaults
 * on the biggest layer usually do not fit).
 * A layer keeps the tile size its layout was built with until it is built
 * again.
 */
typedef struct {
    int agg_ctas_per_sm;
    int region_ctas_per_sm;
    int big_class_edges;
    int one_cta_nodes;
    int boruvka_edges_per_cta;
    int region_max_nodes;
    int tile_small_nodes;
    int tile_small_nodes_hdp;
    int col_min_labels;
} hdp_tuning;

/* Fill p with the paper's settings (Sec. 4.1) for a width x height image:
 * S = 2, L = 3 (levels = 4), gamma = 25.5, alpha = 0.9, tau_c = 7, tau_g = 2,
 * delta0/beta = 0.004/0.95 for images wider than 640 pixels, else 0.064/0.6;
 * MST, HDP mode, sampled prior, default GMM, FP32 storage, st_k = 1200. */
void hdp_default_params(hdp_params* p, int width, int height, int max_disp);

/* Validate p, allocate the device workspace for it and bind `stream`
 * (a cudaStream_t, NULL = legacy default stream).  *out receives the context.
 * HDP_ERR_ARG on invalid parameters, HDP_ERR_OOM if the workspace does not fit. */
int hdp_create(const hdp_params* p, void* stream, hdp_ctx** out);

/* As hdp_create, but the context creates its own non-blocking stream and
 * destroys it in hdp_destroy.  For batches (hdp_match_batch) of more pairs
 * than the caller has streams: every context of a batch needs its own.  No
 * counterpart in the paper.  Returns HDP_ERR_CUDA if the stream cannot be
 * created; otherwise as hdp_create. */
int hdp_create_own_stream(const hdp_params* p, hdp_ctx** out);

/* The stream the context enqueues its work on (NULL: the legacy default
 * stream).  Owned by the caller unless the context was made by
 * hdp_create_own_stream. */
void* hdp_get_stream(const hdp_ctx* ctx);

/* Read or replace the context's launch-shape knobs (see hdp_tuning). */
int hdp_get_tuning(const hdp_ctx* ctx, hdp_tuning* out);
int hdp_set_tuning(hdp_ctx* ctx, const hdp_tuning* t);

/* Autotuner: coordinate descent over the hdp_tuning knobs on the caller's
 * pair (device images as for hdp_build_trees).  Each candidate runs
 * hdp_build_trees + hdp_match `reps` times (1..16) on the context's stream,
 * timed with CUDA events (fastest run counts); the best setting of each knob
 * is kept before the next knob is tried.  The result is stored in the context
 * and copied to *out (optional).  Synchronises; do not call during stream
 * capture.  Leaves the context as after hdp_match on that pair. */
int hdp_autotune(hdp_ctx* ctx, const uint8_t* d_left, const uint8_t* d_right, int pitch, int reps, hdp_tuning* out);

/* Bytes of device workspace held by the context. */
size_t hdp_workspace_bytes(const hdp_ctx* ctx);

/* Upload stage: read the caller's device images (interleaved RGB uint8, row
 * pitch `pitch` bytes >= 3*width; they are copied, not retained), build both
 * graph pyramids (Sec. 2.1) and the tree of the top layer (Sec. 3.2 with
 * every PixelIntv = [0, d_L]; the only tree that does not depend on a
 * predicted disparity). */
int hdp_build_trees(hdp_ctx* ctx, const uint8_t* d_left, const uint8_t* d_right, int pitch);

/* Run every layer top-down (Sec. 3) and write the layer-0 disparity map,
 * int32 [height][width], to d_disp_out.  Requires hdp_build_trees first. */
int hdp_match(hdp_ctx* ctx, int32_t* d_disp_out);

/* Tree-based refinement (Sec. 3.3, last paragraph: the refinement of the
 * cited MST and ST methods integrated at layer 0).  On the caller's device
 * images (as for hdp_build_trees):
 *   1. the right view's map D_R: the whole method on the pair mirrored
 *      left-right with the views exchanged (which is the right-reference
 *      method), read back mirrored;
 *   2. the left view's map D_L (hdp_build_trees + hdp_match);
 *   3. the left-right check: (x, y) is stable iff x - D_L >= 0 and
 *      D_R(x - D_L, y) = D_L;
 *   4. the cost |x - D_L(p)| at stable pixels and 0 elsewhere, for x in
 *      TreeIntv(DT(p)), aggregated over layer 0's forest (Eq. C), and its
 *      WTA (ties to the lowest label), written to d_disp_out (int32
 *      [height][width]).
 * Afterwards HDP_STAGE_DISP of layer 0 and HDP_STAGE_COSTS hold the refined
 * map and the refinement's aggregated costs, HDP_STAGE_REF_D and
 * HDP_STAGE_DISP_R the checked map and D_R.  Enqueued on the context's stream. */
int hdp_refine(hdp_ctx* ctx, const uint8_t* d_left, const uint8_t* d_right, int pitch, int32_t* d_disp_out);

/* hdp_build_trees + hdp_match on host buffers: copies h_left/h_right (tightly
 * packed RGB uint8) to the device, runs, copies the disparity map back into
 * h_disp_out (int32 [height][width]) and synchronises the stream. */
int hdp_match_host(hdp_ctx* ctx, const uint8_t* h_left, const uint8_t* h_right, int32_t* h_disp_out);

/* Process one layer only (tests and tools): layer `level` must have its input
 * ready, i.e. hdp_build_trees was called and, for level < L, the disparity map
 * of level+1 exists (from hdp_run_level(level+1) or hdp_set_stage). */
int hdp_run_level(hdp_ctx* ctx, int level);

/* Wait for the context's stream (and its internal side stream, which runs
 * the priors and interval tables of the predicted layers after
 * hdp_build_trees; each hdp_run_level joins its layer's share before using
 * it); report device-side errors. */
int hdp_sync(hdp_ctx* ctx);

int hdp_destroy(hdp_ctx* ctx);
const char* hdp_last_error(const hdp_ctx* ctx);

/* Failure-path check (tests and tools; no counterpart in the paper): enqueue
 * on the context's stream one of the library's bounded device waits, made to
 * run out after `limit` polls (1..2^24) on something that never arrives -
 * kind 0 a grid barrier that counts one block more than its grid has, kind 1
 * a decoupled look-back on a predecessor tile that never publishes.  The
 * wait gives up, records the timeout and its kernel returns; nothing but the
 * status block is written.  The next hdp_sync returns HDP_ERR_TIMEOUT and
 * clears the status, after which the context is usable again.  HDP_ERR_ARG
 * for another kind or limit. */
int hdp_wait_probe(hdp_ctx* ctx, int kind, unsigned limit);

/* Device time of each stage, recorded with CUDA events on the context's
 * stream while timing is on.  hdp_get_timings synchronises and writes
 * ms[level * 5 + k] for k = 0 interval prediction, 1 edges + sort, 2 forest,
 * 3 orders + layout, 4 aggregation + WTA (zero for stages that did not run);
 * n_floats must be at least 5 * levels. */
int hdp_set_timing(hdp_ctx* ctx, int on);
int hdp_get_timings(hdp_ctx* ctx, float* ms, int n_floats);

/* Capture hdp_build_trees + hdp_match on the given device buffers as one CUDA
 * graph (the context's stream must not be the legacy default stream) and keep
 * it in the context; *n_kernels receives the number of kernel launches in it.
 * hdp_graph_launch replays it (same buffers, new contents allowed).  With
 * timing on at capture time the graph records the stage events, so
 * hdp_get_timings reports the stages of the last replay. */
int hdp_graph_capture(hdp_ctx* ctx, const uint8_t* d_left, const uint8_t* d_right, int pitch, int32_t* d_disp_out,
                      int* n_kernels);
int hdp_graph_launch(hdp_ctx* ctx);

/* Many independent pairs at once.  ctxs[i] (each created with its own
 * stream; sizes, ranges and parameters may differ) matches d_left[i] /
 * d_right[i] (row pitch pitch[i] bytes) into d_disp_out[i].  The work forks
 * from the stream of ctxs[0], runs the pairs concurrently on their own
 * streams and joins back, so the call can be captured in a CUDA graph.
 * hdp_batch_graph_capture captures the whole batch once (the graph is kept in
 * ctxs[0], *n_kernels receives its kernel count); hdp_batch_graph_launch
 * replays it on the stream of ctxs[0].  The CUDA runtime maps streams onto
 * CUDA_DEVICE_MAX_CONNECTIONS hardware queues (default 8, a process
 * environment variable read when CUDA starts); with many pairs set it to 32
 * (64 mixed pairs: 123 ms with 8, 75 ms with 32). */
int hdp_match_batch(hdp_ctx** ctxs, int n, const uint8_t* const* d_left, const uint8_t* const* d_right, const int* pitch,
                    int32_t* const* d_disp_out);
int hdp_batch_graph_capture(hdp_ctx** ctxs, int n, const uint8_t* const* d_left, const uint8_t* const* d_right,
                            const int* pitch, int32_t* const* d_disp_out, int* n_kernels);
int hdp_batch_graph_launch(hdp_ctx* ctx0);

/* Differentiable aggregation (Eq. C as a function of the cost volume, the
 * edge weights and gamma) over the forest of the layer whose tree is loaded
 * (after hdp_build_trees: the top layer; with HDP_MODE_FULL the whole-image
 * MST or segment tree).  That layer must be full range and the storage FP32.
 * Volumes are dense FP32 [height][width][X] device arrays, X = d_l + 1
 * labels, pixel-major.  The tree itself is held fixed (it is piecewise
 * constant in the weights).
 *   hdp_aggregate_fwd: C = A E, A(p,q) = exp(-W(p,q)/gamma).
 *   hdp_aggregate_bwd: with g = dL/dC: dL/dE = A g (A is symmetric),
 *     dL/dw[e] for every grid edge id e (0 outside the forest; weights in
 *     0..255 intensity units) and dL/dgamma, by the closed forms of the
 *     adjoint; the forward passes are recomputed, not stored.
 *   hdp_set_gamma: change gamma for the loaded tree.
 *   hdp_soft_argmin_l1: d(p) = sum_x x softmax(-C(p,.)/T), the mean |d - gt|
 *     over pixels with valid[p] != 0 (valid may be NULL), and dL/dC; d_disp,
 *     d_loss (one float) and d_gC may each be NULL.
 * The first call allocates four volume-sized buffers and the edge-weight
 * buffer in the context. */
int hdp_aggregate_fwd(hdp_ctx* ctx, const float* d_E, float* d_C);
/* The layer whose forest and layout are loaded (the one the calls above and
 * below work on; volumes there hold width_l * height_l * (d_l + 1) floats),
 * or -1 before hdp_build_trees.  No counterpart in the paper. */
int hdp_tree_level(const hdp_ctx* ctx);
int hdp_aggregate_bwd(hdp_ctx* ctx, const float* d_E, const float* d_gC, float* d_gE, float* d_gw, float* d_ggamma);
int hdp_set_gamma(hdp_ctx* ctx, float gamma);
int hdp_soft_argmin_l1(hdp_ctx* ctx, const float* d_C, const float* d_gt, const uint8_t* d_valid, float T,
                       float* d_disp, float* d_loss, float* d_gC);

/* The inputs of Eq. C made differentiable as well, on the same loaded layer
 * (same requirements as above).
 *   hdp_cost_volume: the matching cost of Sec. 3.3 with real-valued
 *     parameters, E(p, x) = (1 - alpha) min(dc, tau_c) + alpha min(dg, tau_g)
 *     for every pixel p and label x in 0..d_l, dc the mean absolute RGB
 *     difference and dg the absolute horizontal-gradient difference / 6 of
 *     left pixel (px, py) and right pixel (max(px - x, 0), py), in 0..255
 *     intensity units (the pyramid's scale 4^l divided out).  d_E as above.
 *   hdp_cost_volume_bwd: from d_gE = dL/dE, d_gparams (3 floats) receives
 *     dL/dalpha = sum gE (min(dg, tau_g) - min(dc, tau_c)),
 *     dL/dtau_c = sum gE (1 - alpha) [dc > tau_c] and
 *     dL/dtau_g = sum gE alpha [dg > tau_g] (0 taken at dc = tau_c).
 *   alpha, tau_c, tau_g must be finite and tau_c, tau_g >= 0 (HDP_ERR_ARG);
 *   unlike hdp_params they need not sit on the 1/20, 1/3, 1/6 grids.
 *   hdp_set_edge_weights: real-valued weights for the loaded tree's edges,
 *     d_w[e] per grid edge id e of the loaded layer (2 * width_l * height_l
 *     floats, intensity units, copied), so the similarities become
 *     exp(-d_w[e] / gamma); NULL returns to the image's integer weights.  The
 *     tree is not rebuilt.  Every later aggregation on this tree uses them
 *     (hdp_aggregate_fwd/bwd, whose dL/dgamma then sums d_w[e] dL/dw[e],
 *     hdp_set_gamma, hdp_match on the same layer) until a tree is built again
 *     (hdp_build_trees, or a run of another layer).
 * These calls, like hdp_aggregate_fwd, enqueue on the context's stream and
 * return without waiting. */
int hdp_cost_volume(hdp_ctx* ctx, float alpha, float tau_c, float tau_g, float* d_E);
int hdp_cost_volume_bwd(hdp_ctx* ctx, float alpha, float tau_c, float tau_g, const float* d_gE, float* d_gparams);
int hdp_set_edge_weights(hdp_ctx* ctx, const float* d_w);

/* hdp_build_trees + hdp_match without any allocation, for callers that cannot
 * allocate device memory: code running where cudaMalloc is not allowed or
 * would break an allocator they do not control (inside a memory pool or
 * graph-building framework, a real-time loop, a plug-in that owns no
 * allocator).  The paper has no counterpart; this is an interface of this
 * library only.
 *   - The workspace is a fixed 64 MiB device array inside the library.  With
 *     lazy module loading (the CUDA default) a device reserves it when the
 *     library's module is first loaded there, which is this call's first
 *     call on that device; that first call can therefore fail with
 *     HDP_ERR_OOM or HDP_ERR_CUDA.  Make it once at set-up time, not where
 *     allocation is forbidden.  The array stays reserved on that device
 *     until the process exits.
 *   - Problems whose workspace exceeds it (roughly above 256x256 pixels with
 *     max_disp 63, FP32) are rejected with HDP_ERR_ARG and a message.
 *   - d_left/d_right (interleaved RGB uint8, row pitch `pitch` bytes) and
 *     d_disp_out (int32 [height][width]) are the caller's device buffers;
 *     `stream` is a cudaStream_t (NULL = legacy default stream).
 *   - The first call on a device, with that device current, looks up the
 *     array's device address (cudaGetSymbolAddress).
 *   - The call is synchronous: it waits once after uploading a few hundred
 *     bytes of constants and again after the pipeline, then reads the
 *     device status, so a bounded device wait that gave up returns
 *     HDP_ERR_TIMEOUT and an invalid device input HDP_ERR_ARG.  It cannot be
 *     captured in a CUDA graph: on a stream under capture it returns
 *     HDP_ERR_STATE and does nothing.
 *   - Every call uses the same array: calls that overlap on the GPU (two
 *     streams, two host threads) race and corrupt each other's results.
 *   - It calls no cudaMalloc, cudaFree or other allocating routine. */
int hdp_match_noalloc(const hdp_params* p, const uint8_t* d_left, const uint8_t* d_right, int pitch,
                      int32_t* d_disp_out, void* stream);

/* GMM_l by EM (Sec. 2.2; the trained GMM the paper uses is not published, so
 * it is fitted here on ground truth the caller supplies).  The paper models
 * the offset o = D_{l+1} - floor(D_l / 2) of a superpixel's disparity from
 * the mode each of its children gives, collects o over training pairs with
 * ground truth and fits a Gaussian mixture by EM; the result goes into
 * hdp_params.gmm_k / gmm.  Context-free calls, enqueued on `stream` (a
 * cudaStream_t, NULL = legacy default stream); all pointers are device
 * pointers owned by the caller.
 *   hdp_gt_down: ground truth of the next layer.  d_gt int32 [height][width]
 *     labels (-1 = invalid, e.g. occluded) -> d_gt_up int32
 *     [ceil(height/2)][ceil(width/2)]: the mean of the valid children divided
 *     by 2, rounded half up, floor((sum + n) / (2 n)); -1 without a valid
 *     child.  width * height <= 2^23.
 *   hdp_offset_hist: adds, for every pixel (x, y) of the lower map d_lo
 *     (int32 [height][width]) with d_lo >= 0 and a superpixel
 *     u = d_up[y/2][x/2] >= 0 (d_up as written by hdp_gt_down), one count to
 *     d_hist[o + range] with o = u - floor(d_lo / 2), |o| <= range <= 255
 *     (2 range + 1 uint64 bins, zeroed by the caller; counts accumulate over
 *     calls, so several pairs can be summed).  Exact.
 *   hdp_gmm_em: K (1..8) components fitted to the histogram by `iters`
 *     iterations of EM, FP32: start with every mean at the data mean m,
 *     spreads max(s, sd_min) * 4^(k - (K-1)/2) (s the data's spread) and
 *     equal weights; E-step responsibilities in the log domain; M-step
 *     weights and means, then spreads about the new means, floored at
 *     sd_min > 0 (the offsets are integers: no component may collapse onto
 *     one value).  d_out: float [K][3] = (pi, mu, sd) per component.
 * HDP_ERR_ARG on a bad size or pointer; HDP_ERR_CUDA if a launch fails. */
int hdp_gt_down(const int32_t* d_gt, int width, int height, int32_t* d_gt_up, void* stream);
int hdp_offset_hist(const int32_t* d_up, const int32_t* d_lo, int width, int height, int range,
                    unsigned long long* d_hist, void* stream);
int hdp_gmm_em(const unsigned long long* d_hist, int range, int K, int iters, float sd_min, float* d_out,
               void* stream);

/* Per-stage inspection and injection for tests.  `what` selects one of the
 * HDP_STAGE_* buffers of layer `level`; `bytes` must equal its size exactly
 * (query it with hdp_stage_bytes).  hdp_get_stage synchronises the stream.
 * Only HDP_STAGE_DISP and HDP_STAGE_PRIOR can be set. */
enum {
    HDP_STAGE_PYR_LEFT = 0,   /* int32 [H][W][4]: R,G,B at scale 4^l, horizontal gradient g */
    HDP_STAGE_PYR_RIGHT = 1,
    HDP_STAGE_WEIGHTS = 2,    /* int32 [2N]: w of edge id e = 2*(y*W+x)+o, -1 if invalid */
    HDP_STAGE_EDGES = 3,      /* int32 [count]: edges passing DT-Rule 1, in (w, id) order */
    HDP_STAGE_IN_TREE = 4,    /* uint8 [2N]: 1 if edge id is in the forest */
    HDP_STAGE_DT_ROOT = 5,    /* int32 [N]: smallest pixel id of the pixel's tree */
    HDP_STAGE_TREE_INTV = 6,  /* uint32 [N][8]: TreeIntv of the pixel's tree */
    HDP_STAGE_BFS = 7,        /* int32 [N]: breadth-first order of the forest */
    HDP_STAGE_PARENT = 8,     /* int32 [N]: parent pixel, -1 for roots */
    HDP_STAGE_DEPTH = 9,      /* int32 [N] */
    HDP_STAGE_PRIOR = 10,     /* int64 [d_l+1]: prior weights (count + 1) */
    HDP_STAGE_TABLE = 11,     /* uint32 [d_{l+1}+1][8]: PixelIntv per upper label */
    HDP_STAGE_PIX_SET = 12,   /* int32 [N]: row of the table used by each pixel */
    HDP_STAGE_COSTS = 13,     /* float [K]: aggregated cost, pixel-major, labels ascending */
    HDP_STAGE_DISP = 14,      /* int32 [N]: D_l */
    HDP_STAGE_INFO = 15,      /* int64 [16]: K_l, edge count, tree count, engine, ... (below) */
    HDP_STAGE_REF_D = 16,     /* int32 [N], layer 0 after hdp_refine: D_L where the left-right check passes, else -1 */
    HDP_STAGE_DISP_R = 17     /* int32 [N], layer 0 after hdp_refine: the right view's map, in its own frame */
};
/* HDP_STAGE_INFO of the layer whose tree is current: [0] K_l aggregated
 * entries, [1] edges kept by DT-Rule 1, [2] trees, [3] forest engine (1
 * Boruvka over the sorted list, 3 windows of the top layer, 4 hybrid
 * first pass, 5 first pass by regions, 6 windows of a risky layer), [4]
 * aggregation tiles, [5] 1 if the layer has a risky edge, [6] tour arcs,
 * [7] weight classes (hybrid) or regions (region engine), [8] light-child
 * links, [9] and [10] reservation or Boruvka rounds and windows of the
 * windowed engines; the rest is zero. */
int64_t hdp_stage_bytes(hdp_ctx* ctx, int level, int what);
int hdp_get_stage(hdp_ctx* ctx, int level, int what, void* h_dst, size_t bytes);
int hdp_set_stage(hdp_ctx* ctx, int level, int what, const void* h_src, size_t bytes);

#ifdef __cplusplus
}
#endif
#endif /* HDP_H */
