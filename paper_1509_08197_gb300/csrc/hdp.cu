// C ABI of the HDP library: context, workspace and the per-layer pipeline
// (Sec. 3: top-down over the layers; per layer interval prediction, forest
// construction, aggregation and WTA).
#include <stdio.h>
#include <string.h>

#include <cmath>
#include <vector>

#include "hdp_impl.cuh"

struct hdp_ctx {
    Ctx c;
    cudaEvent_t fork = nullptr, join = nullptr;   // batch fork/join events (lazily created)
    int prior_injected[HDP_MAX_LEVELS] = {};
    int timing = 0;
    cudaEvent_t ev[HDP_MAX_LEVELS][6] = {};
    int ev_used[HDP_MAX_LEVELS][6] = {};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    // hdp_match_host: the pyramid on the staging buffers, captured on first use
    cudaGraph_t host_graph = nullptr;
    cudaGraphExec_t host_exec = nullptr;
    bool own_stream = false;   // created by hdp_create_own_stream, destroyed with the context
    int use_side = 1;          // 0 inside a batch: the other pairs already fill the GPU
};

static void drop_host_graph(hdp_ctx* ctx);

static void mark(hdp_ctx* ctx, int l, int k)
{
    if (!ctx->timing) return;
    if (!ctx->ev[l][k]) cudaEventCreate(&ctx->ev[l][k]);
    // inside stream capture only an "external" record becomes a graph node
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(ctx->c.s, &cs);
    cudaEventRecordWithFlags(ctx->ev[l][k], ctx->c.s,
                             cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : cudaEventRecordDefault);
    ctx->ev_used[l][k] = 1;
}

#define TRY_CUDA(call)                                                               \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess) {                                                     \
            ctx->c.err = std::string(#call) + ": " + cudaGetErrorString(e_);         \
            return e_ == cudaErrorMemoryAllocation ? HDP_ERR_OOM : HDP_ERR_CUDA;     \
        }                                                                            \
    } while (0)

static int fail(hdp_ctx* ctx, int code, const std::string& msg)
{
    if (ctx) ctx->c.err = msg;
    return code;
}

extern "C" void hdp_default_params(hdp_params* p, int width, int height, int max_disp)
{
    memset(p, 0, sizeof(*p));
    p->width = width;
    p->height = height;
    p->max_disp = max_disp;
    p->levels = 4;
    p->tree = HDP_TREE_MST;
    p->mode = HDP_MODE_HDP;
    p->gamma = 25.5f;
    p->alpha = 0.9f;
    p->tau_c = 7.0f;
    p->tau_g = 2.0f;
    p->st_k = 1200;
    bool large = width > 640;
    p->beta_num = large ? 95 : 3;
    p->beta_den = large ? 100 : 5;
    p->delta0 = large ? 0.004 : 0.064;
    p->prior = HDP_PRIOR_SAMPLED;
    p->storage = HDP_STORE_FP32;
}

static bool near_int(double v, int* out)
{
    double r = std::round(v);
    if (std::fabs(v - r) > 1e-4) return false;
    *out = (int)r;
    return true;
}

static size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

template <typename T>
static T* carve(Ctx& c, size_t count)
{
    size_t bytes = align_up(sizeof(T) * (count ? count : 1));
    T* p = (T*)(c.arena + c.arena_used);
    c.arena_used += bytes;
    return p;
}

// lay out every buffer; with c.arena == nullptr this only measures
// look-back scratch entries (tiles) the layouts of every layer need under
// tuning t: every tile but the last of a run is full; with one label set per
// layer (full range, top layer) it holds tile_rows_of(kp, extra, tf) rows,
// otherwise at least 4 * tile_rows_max(tf) costs (the narrowest rows); plus
// one partial tile per (light level, width) run
static size_t tiles_needed(const Ctx& c, const hdp_tuning& t)
{
    size_t tiles = 0;
    for (int l = 0; l < c.nlev; ++l) {
        const size_t kp = (size_t)((c.dim[l].d + 1 + 3) / 4 * 4);
        const bool one_set = c.p.mode == HDP_MODE_FULL || l == c.nlev - 1;
        const int extra = c.p.storage == HDP_STORE_FP16 ? 4 : 0;
        const int tf = tile_floats_for(c, l, t);
        const size_t n = one_set ? (size_t)c.dim[l].N / tile_rows_of((int)kp, extra, tf)
                                 : (size_t)c.dim[l].N * kp / (4 * tile_rows_max(tf));
        tiles = std::max(tiles, n);
    }
    return tiles + 2 * 2048 + 16;
}

static void layout_buffers(Ctx& c)
{
    c.arena_used = 0;
    const int N0 = c.dim[0].N;
    const size_t E2 = 2 * (size_t)N0;
    for (int l = 0; l < c.nlev; ++l) {
        c.imL[l] = carve<int4>(c, c.dim[l].N);
        c.imR[l] = carve<int4>(c, c.dim[l].N);
        c.disp[l] = carve<int32_t>(c, c.dim[l].N);
        c.prior[l] = carve<long long>(c, 256);
        c.table[l] = carve<uint32_t>(c, 256 * HDP_WORDS);
        c.canon[l] = carve<int>(c, 256);
    }
    c.imF = carve<int4>(c, c.p.prefilter == HDP_PREFILTER_MEDIAN3 ? N0 : 1);
    c.pk0[0] = carve<uint2>(c, N0);
    c.pk0[1] = carve<uint2>(c, N0);
    c.stage_l = carve<uint8_t>(c, 3 * (size_t)N0);
    c.stage_r = carve<uint8_t>(c, 3 * (size_t)N0);
    c.disp_host_stage = carve<int32_t>(c, N0);
    c.dispRm = carve<int>(c, N0);
    c.refD = carve<int>(c, N0);
    c.refR = carve<int>(c, N0);
    c.gmm = carve<double>(c, HDP_MAX_LEVELS * HDP_MAX_GMM * 3);
    c.gmm_k = carve<int>(c, HDP_MAX_LEVELS);
    c.full_mask = carve<uint32_t>(c, HDP_MAX_LEVELS * HDP_WORDS);
    c.pixset = carve<int>(c, N0);
    c.weights = carve<int>(c, E2);
    c.keys0 = carve<uint32_t>(c, E2);
    c.keys1 = carve<uint32_t>(c, E2);
    c.cls_start = carve<int>(c, E2);
    c.parent = carve<int>(c, N0);
    c.csize = carve<int>(c, N0);
    c.intw = carve<int>(c, N0);
    c.best = carve<int>(c, N0);
    c.best2 = carve<int>(c, N0);
    c.rootof = carve<int>(c, N0);
    c.minid = carve<int>(c, N0);
    c.dtroot = carve<int>(c, N0);
    c.T = carve<uint32_t>(c, (size_t)N0 * HDP_WORDS);
    c.in_tree = carve<uint8_t>(c, E2);
    c.listA = carve<int>(c, E2);
    c.listB = carve<int>(c, E2);
    c.raA = carve<int>(c, E2);
    c.rbA = carve<int>(c, E2);
    c.raB = carve<int>(c, E2);
    c.rbB = carve<int>(c, E2);
    c.hooked = carve<int>(c, 2 * (size_t)N0);
    c.win = carve<int>(c, 16384);
    c.wtmp = carve<int>(c, 16384);
    c.wra = carve<int>(c, 16384);
    c.wrb = carve<int>(c, 16384);
    c.wst = carve<int>(c, 16384);
    c.adj = carve<uint8_t>(c, N0);
    c.aoff = carve<uint32_t>(c, N0 + 1);
    c.succ = carve<int>(c, E2);
    c.val = carve<int>(c, E2);
    c.succ2 = carve<int>(c, E2);
    c.val2 = carve<int>(c, E2);
    c.par = carve<int>(c, N0);
    c.pdir = carve<int>(c, N0);
    c.sub = carve<int>(c, N0);
    c.hdir = carve<int>(c, N0);
    c.tpos_down = carve<int>(c, N0);
    c.tpos_up = carve<int>(c, N0);
    c.vals4 = carve<I4>(c, N0);
    c.tour = carve<I4>(c, E2);
    c.tbase = carve<uint32_t>(c, N0);
    c.nbase = carve<uint32_t>(c, N0);
    c.depth = carve<int>(c, N0);
    c.pre2 = carve<int>(c, N0);
    c.pre3 = carve<int>(c, N0);
    c.light = carve<int>(c, N0);
    c.ka = carve<uint32_t>(c, N0 + 1);
    c.va = carve<uint32_t>(c, N0 + 1);
    c.kb = carve<uint32_t>(c, N0 + 1);
    c.vb = carve<uint32_t>(c, N0 + 1);
    c.bfs = carve<int>(c, N0);
    c.lay = carve<int>(c, N0);
    c.rowof = carve<int>(c, N0);
    c.kp = carve<int>(c, N0);
    c.roff = carve<uint32_t>(c, N0 + 1);
    c.rs = carve<float>(c, N0);
    c.prow = carve<int>(c, N0);
    c.rdt = carve<int>(c, N0);
    c.lcoff = carve<uint32_t>(c, N0 + 1);
    c.lcrow = carve<int>(c, N0);
    c.runstart = carve<int>(c, 2048);
    c.ustart_flag = carve<uint32_t>(c, N0);
    c.uid = carve<uint32_t>(c, N0);
    c.ubeg = carve<int>(c, N0);
    c.lvl_first = carve<int>(c, MAX_LIGHT_LEVELS);
    c.lvl_count = carve<int>(c, MAX_LIGHT_LEVELS);
    c.tickets = carve<int>(c, 2 * MAX_LIGHT_LEVELS);
    c.nup = carve<float>(c, N0);
    c.nfull = carve<float>(c, N0);
    c.ints = carve<int>(c, IDX_COUNT);
    c.st = carve<DevStatus>(c, 1);
    c.zero64 = carve<unsigned long long>(c, 4);
    c.tmp_words = radix_tmp_words((int)E2) + 4096;
    c.tmp = carve<uint32_t>(c, c.tmp_words);
    c.hist = carve<unsigned long long>(c, HDP_MAX_LEVELS * 256);
    // single-pass scans: the longest is over the 2N edge slots (radix
    // histograms are shorter)
    c.scan.max_tiles = scan_state_tiles((int)E2);
    c.scan.state = carve<unsigned long long>(c, c.scan.max_tiles);
    c.scan.ctr = carve<unsigned int>(c, 2);
    c.scan4.max_tiles = c.scan.max_tiles;
    c.scan4.flags = carve<unsigned int>(c, c.scan4.max_tiles);
    c.scan4.aggv = carve<I4>(c, c.scan4.max_tiles);
    c.scan4.inclv = carve<I4>(c, c.scan4.max_tiles);
    c.scan4.ctr = carve<unsigned int>(c, 2);
    size_t K = 0;
    for (int l = 0; l < c.nlev; ++l) K = std::max(K, (size_t)c.dim[l].N * (size_t)((c.dim[l].d + 1 + 3) / 4 * 4));
    c.vol_elems = K;
    // the defaults, and one-set layers on the warp kernel instead of the column kernel
    hdp_tuning warp = c.tune;
    warp.col_min_labels = 257;
    c.max_tiles = std::max(tiles_needed(c, c.tune), tiles_needed(c, warp));
    c.tflags = carve<int>(c, 4 * c.max_tiles);   // look-back flags, then done flags, of both passes
    c.aggA = carve<float>(c, c.max_tiles * SCR_STRIDE);
    c.inclA = carve<float>(c, c.max_tiles * SCR_STRIDE);
    c.aggM = carve<float>(c, c.max_tiles);
    if (c.p.storage == HDP_STORE_FP16) c.volh = carve<__half>(c, K + 8);
    else c.vol = carve<float>(c, K + 8);
}

// Checks p and fills the layer sizes of c; returns a message on failure.
static const char* setup_params(Ctx& c, const hdp_params* p)
{
    c.p = *p;
    if (p->width < 2 || p->height < 2) return "width and height must be >= 2";
    if (p->width >= (1 << 19)) return "width must be below 2^19";   // packed with row data in the aggregation
    if (p->max_disp < 1 || p->max_disp > HDP_MAX_DISP) return "max_disp must be in 1..255";
    if (p->levels < 1 || p->levels > HDP_MAX_LEVELS) return "levels must be in 1..8";
    if (p->tree != HDP_TREE_MST && p->tree != HDP_TREE_ST && p->tree != HDP_TREE_RT) return "unknown tree";
    if (p->mode != HDP_MODE_HDP && p->mode != HDP_MODE_FULL) return "unknown mode";
    if (!(p->gamma > 0)) return "gamma must be > 0";
    if (!near_int(20.0 * p->alpha, &c.a20) || c.a20 < 0 || c.a20 > 20) return "20*alpha must be an integer in 0..20";
    if (!near_int(3.0 * p->tau_c, &c.tc3) || c.tc3 < 0) return "3*tau_c must be a non-negative integer";
    if (!near_int(6.0 * p->tau_g, &c.tg6) || c.tg6 < 0) return "6*tau_g must be a non-negative integer";
    if (p->st_k < 0) return "st_k must be >= 0";
    if (p->beta_den <= 0 || p->beta_num < 0 || p->beta_num > p->beta_den) return "beta must be in [0, 1]";
    if (!(p->delta0 >= 0.0) || p->delta0 >= 1.0) return "delta0 must be in [0, 1)";
    if (p->prior != HDP_PRIOR_SAMPLED && p->prior != HDP_PRIOR_UNIFORM) return "unknown prior";
    if (p->storage != HDP_STORE_FP32 && p->storage != HDP_STORE_FP16) return "unknown storage";
    if (p->prefilter != HDP_PREFILTER_NONE && p->prefilter != HDP_PREFILTER_MEDIAN3) return "unknown prefilter";
    for (int l = 0; l < HDP_MAX_LEVELS; ++l) {
        if (p->gmm_k[l] < 0 || p->gmm_k[l] > HDP_MAX_GMM) return "gmm_k out of range";
        for (int k = 0; k < p->gmm_k[l]; ++k)
            if (!(p->gmm[l][k][2] > 0)) return "gmm standard deviations must be > 0";
    }
    if ((long long)p->width * p->height > (1 << 23)) return "images above 2^23 pixels are not supported";
    c.nlev = p->mode == HDP_MODE_FULL ? 1 : p->levels;
    c.top = c.nlev - 1;
    int W = p->width, H = p->height, d = p->max_disp;
    for (int l = 0; l < c.nlev; ++l) {
        c.dim[l] = LayerDims{W, H, W * H, d};
        if (8 + 2 * l + edge_bits(W * H) > 32) return "edge keys do not fit 32 bits";
        W = (W + 1) / 2;
        H = (H + 1) / 2;
        d = d / 2;
    }
    return nullptr;
}

// Host-side constants of a context: GMM parameters per predicted layer and
// the full label set of every layer.
struct HostConsts {
    double g[HDP_MAX_LEVELS * HDP_MAX_GMM * 3];
    int gk[HDP_MAX_LEVELS];
    uint32_t fm[HDP_MAX_LEVELS * HDP_WORDS];
};

static void host_constants(const Ctx& c, HostConsts& h)
{
    const hdp_params* p = &c.p;
    double* g = h.g;
    int* gk = h.gk;
    uint32_t* fm = h.fm;
    for (int i = 0; i < HDP_MAX_LEVELS * HDP_MAX_GMM * 3; ++i) g[i] = 0.0;
    for (int i = 0; i < HDP_MAX_LEVELS; ++i) gk[i] = 1;
    for (int l = 0; l < HDP_MAX_LEVELS; ++l) {
        if (p->gmm_k[l] == 0) {
            g[(size_t)l * HDP_MAX_GMM * 3 + 0] = 1.0;
            g[(size_t)l * HDP_MAX_GMM * 3 + 1] = 0.0;
            g[(size_t)l * HDP_MAX_GMM * 3 + 2] = 1.0;
        } else {
            gk[l] = p->gmm_k[l];
            for (int k = 0; k < p->gmm_k[l]; ++k)
                for (int t = 0; t < 3; ++t) g[((size_t)l * HDP_MAX_GMM + k) * 3 + t] = p->gmm[l][k][t];
        }
    }
    for (int i = 0; i < HDP_MAX_LEVELS * HDP_WORDS; ++i) fm[i] = 0u;
    for (int l = 0; l < c.nlev; ++l)
        for (int j = 0; j <= c.dim[l].d; ++j) fm[l * HDP_WORDS + (j >> 5)] |= 1u << (j & 31);
}

extern "C" int hdp_create(const hdp_params* p, void* stream, hdp_ctx** out)
{
    if (!p || !out) return HDP_ERR_ARG;
    *out = nullptr;
    hdp_ctx* ctx = new hdp_ctx();
    Ctx& c = ctx->c;
    c.s = (cudaStream_t)stream;
    if (const char* why = setup_params(c, p)) {
        fprintf(stderr, "hdp_create: %s\n", why);
        delete ctx;
        return HDP_ERR_ARG;
    }
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) {
        fprintf(stderr, "hdp_create: %s\n", cudaGetErrorString(ce));
        delete ctx;
        return HDP_ERR_CUDA;
    }
    cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, dev);
    c.arena = nullptr;
    layout_buffers(c);
    c.arena_bytes = c.arena_used;
    ce = cudaMalloc((void**)&c.arena, c.arena_bytes);
    if (ce != cudaSuccess) {
        fprintf(stderr, "hdp_create: cudaMalloc(%zu): %s\n", c.arena_bytes, cudaGetErrorString(ce));
        cudaGetLastError();
        delete ctx;
        return ce == cudaErrorMemoryAllocation ? HDP_ERR_OOM : HDP_ERR_CUDA;
    }
    layout_buffers(c);
    HostConsts hc;
    host_constants(c, hc);
    TRY_CUDA(cudaMemcpy(c.gmm, hc.g, sizeof(hc.g), cudaMemcpyHostToDevice));
    TRY_CUDA(cudaMemcpy(c.gmm_k, hc.gk, sizeof(hc.gk), cudaMemcpyHostToDevice));
    TRY_CUDA(cudaMemcpy(c.full_mask, hc.fm, sizeof(hc.fm), cudaMemcpyHostToDevice));
    TRY_CUDA(cudaMemset(c.st, 0, sizeof(DevStatus)));
    TRY_CUDA(cudaMemset(c.ints, 0, sizeof(int) * IDX_COUNT));
    TRY_CUDA(cudaMemset(c.zero64, 0, 4 * sizeof(unsigned long long)));
    c.scan.st = c.st;
    c.scan4.st = c.st;
    TRY_CUDA(cudaMemset(c.scan.state, 0, sizeof(unsigned long long) * c.scan.max_tiles));
    TRY_CUDA(cudaMemset(c.scan.ctr, 0, 2 * sizeof(unsigned int)));
    TRY_CUDA(cudaMemset(c.scan4.flags, 0, sizeof(unsigned int) * c.scan4.max_tiles));
    TRY_CUDA(cudaMemset(c.scan4.ctr, 0, 2 * sizeof(unsigned int)));
    TRY_CUDA(cudaStreamCreateWithFlags(&c.s2, cudaStreamNonBlocking));
    TRY_CUDA(cudaEventCreateWithFlags(&c.ev_fork, cudaEventDisableTiming));
    for (int l = 0; l < HDP_MAX_LEVELS; ++l) TRY_CUDA(cudaEventCreateWithFlags(&c.ev_side[l], cudaEventDisableTiming));
    *out = ctx;
    return HDP_OK;
}

extern "C" size_t hdp_workspace_bytes(const hdp_ctx* ctx) { return ctx ? ctx->c.arena_bytes : 0; }

static int check_launch(hdp_ctx* ctx, const char* where)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ctx, HDP_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
    return HDP_OK;
}

static void build_layer_tree(hdp_ctx* ctx, int l)
{
    Ctx& c = ctx->c;
    const bool hdp = c.p.mode == HDP_MODE_HDP && l < c.top;
    launch_edges(c, l, hdp);
    mark(ctx, l, 2);
    launch_forest(c, l, hdp);
    mark(ctx, l, 3);
    launch_order(c, l);
    mark(ctx, l, 4);
    c.tree_level = l;
    c.use_wf = false;   // the new layout's similarities come from the image's weights
}

extern "C" int hdp_build_trees(hdp_ctx* ctx, const uint8_t* d_left, const uint8_t* d_right, int pitch)
{
    if (!ctx) return HDP_ERR_ARG;
    Ctx& c = ctx->c;
    if (!d_left || !d_right || pitch < 3 * c.p.width) return fail(ctx, HDP_ERR_ARG, "bad image pointers or pitch");
    // side work of an earlier call that no level joined still reads the images
    for (int l = 0; l < HDP_MAX_LEVELS; ++l)
        if (c.side_pending[l]) {
            TRY_CUDA(cudaStreamWaitEvent(c.s, c.ev_side[l], 0));
            c.side_pending[l] = 0;
        }
    launch_level0(c, 0, d_left, pitch);
    launch_level0(c, 1, d_right, pitch);
    launch_pyramid(c);
    if (c.s2 && ctx->use_side && c.p.mode == HDP_MODE_HDP && c.top > 0) {
        // priors and tables of every predicted layer, beside layers top..1
        TRY_CUDA(cudaEventRecord(c.ev_fork, c.s));
        TRY_CUDA(cudaStreamWaitEvent(c.s2, c.ev_fork, 0));
        for (int l = c.top - 1; l >= 0; --l) {
            launch_prior(c, l, c.s2);
            launch_table(c, l, c.s2);
            TRY_CUDA(cudaEventRecord(c.ev_side[l], c.s2));
            c.side_pending[l] = 1;
        }
    }
    mark(ctx, c.top, 0);
    mark(ctx, c.top, 1);
    build_layer_tree(ctx, c.top);
    c.built = 1;
    for (int l = 0; l < HDP_MAX_LEVELS; ++l) ctx->prior_injected[l] = 0;
    return check_launch(ctx, "hdp_build_trees");
}

// hdp_run_level without the aggregation: interval prediction, edges, forest, orders
static int run_level_pre(hdp_ctx* ctx, int level)
{
    if (!ctx) return HDP_ERR_ARG;
    Ctx& c = ctx->c;
    if (!c.built) return fail(ctx, HDP_ERR_STATE, "hdp_build_trees has not been called");
    if (level < 0 || level > c.top) return fail(ctx, HDP_ERR_ARG, "level out of range");
    const bool hdp = c.p.mode == HDP_MODE_HDP && level < c.top;
    if (hdp || c.tree_level != level) mark(ctx, level, 0);
    if (hdp) {
        if (c.side_pending[level]) {
            TRY_CUDA(cudaStreamWaitEvent(c.s, c.ev_side[level], 0));
            c.side_pending[level] = 0;
            if (ctx->prior_injected[level]) launch_table(c, level, c.s);
        } else {
            if (!ctx->prior_injected[level]) launch_prior(c, level, c.s);
            launch_table(c, level, c.s);
        }
        ctx->prior_injected[level] = 0;
        launch_pixsets(c, level);
    }
    if (c.tree_level != level || hdp) {
        mark(ctx, level, 1);
        build_layer_tree(ctx, level);
    }
    return HDP_OK;
}

extern "C" int hdp_run_level(hdp_ctx* ctx, int level)
{
    int rc = run_level_pre(ctx, level);
    if (rc) return rc;
    Ctx& c = ctx->c;
    if (!ctx->ev_used[level][4]) mark(ctx, level, 4);
    launch_aggregate(c, level);
    mark(ctx, level, 5);
    return check_launch(ctx, "hdp_run_level");
}

extern "C" int hdp_match(hdp_ctx* ctx, int32_t* d_disp_out)
{
    if (!ctx || !d_disp_out) return HDP_ERR_ARG;
    Ctx& c = ctx->c;
    if (!c.built) return fail(ctx, HDP_ERR_STATE, "hdp_build_trees has not been called");
    c.refined = 0;
    for (int l = c.top; l >= 0; --l) {
        int rc = hdp_run_level(ctx, l);
        if (rc) return rc;
    }
    TRY_CUDA(cudaMemcpyAsync(d_disp_out, c.disp[0], sizeof(int32_t) * c.dim[0].N, cudaMemcpyDeviceToDevice, c.s));
    return HDP_OK;
}

extern "C" int hdp_sync(hdp_ctx* ctx)
{
    if (!ctx) return HDP_ERR_ARG;
    Ctx& c = ctx->c;
    TRY_CUDA(cudaStreamSynchronize(c.s));
    if (c.s2) TRY_CUDA(cudaStreamSynchronize(c.s2));
    DevStatus st;
    TRY_CUDA(cudaMemcpy(&st, c.st, sizeof(st), cudaMemcpyDeviceToHost));
    if (st.err == DEV_OK) return HDP_OK;
    // report once, then clear the status block (error, barrier counter and
    // generation) so that the next call on this context starts clean
    TRY_CUDA(cudaMemsetAsync(c.st, 0, sizeof(DevStatus), c.s));
    TRY_CUDA(cudaStreamSynchronize(c.s));
    if (st.err == DEV_TIMEOUT) return fail(ctx, HDP_ERR_TIMEOUT, "a bounded device wait gave up (site " + std::to_string(st.where) + ")");
    return fail(ctx, HDP_ERR_ARG, "invalid device input (site " + std::to_string(st.where) + ")");
}

extern "C" int hdp_wait_probe(hdp_ctx* ctx, int kind, unsigned limit)
{
    if (!ctx) return HDP_ERR_ARG;
    if (kind < 0 || kind > 1 || limit < 1 || limit > HDP_SPIN_LIMIT)
        return fail(ctx, HDP_ERR_ARG, "hdp_wait_probe: kind must be 0 or 1 and limit in 1..2^24");
    Ctx& c = ctx->c;
    launch_wait_probe(kind, limit, c.zero64, c.st, c.s);
    return check_launch(ctx, "hdp_wait_probe");
}

// ------------------------------------------------------------ tuning ---
static const char* tuning_error(const hdp_tuning& t)
{
    if (t.agg_ctas_per_sm < 1 || t.agg_ctas_per_sm > 8) return "agg_ctas_per_sm out of 1..8";
    if (t.region_ctas_per_sm < 1 || t.region_ctas_per_sm > 4) return "region_ctas_per_sm out of 1..4";
    if (t.big_class_edges < 64 || t.big_class_edges > 4096) return "big_class_edges out of 64..4096";
    if (t.one_cta_nodes < 1024 || t.one_cta_nodes > (1 << 24)) return "one_cta_nodes out of 1024..1<<24";
    if (t.boruvka_edges_per_cta < 512 || t.boruvka_edges_per_cta > (1 << 20)) return "boruvka_edges_per_cta out of 512..1<<20";
    if (t.region_max_nodes < 0 || t.region_max_nodes > (1 << 30)) return "region_max_nodes out of 0..1<<30";
    if (t.tile_small_nodes < 0 || t.tile_small_nodes > (1 << 30)) return "tile_small_nodes out of 0..1<<30";
    if (t.tile_small_nodes_hdp < 0 || t.tile_small_nodes_hdp > (1 << 30)) return "tile_small_nodes_hdp out of 0..1<<30";
    if (t.col_min_labels < COL_MIN_KP || t.col_min_labels > 257) return "col_min_labels out of 64..257";
    return nullptr;
}

// a tuning this context can run: valid knobs, and layouts that fit its look-back scratch
static const char* tuning_error(const Ctx& c, const hdp_tuning& t)
{
    if (const char* why = tuning_error(t)) return why;
    if (tiles_needed(c, t) > c.max_tiles) return "these tile sizes need more look-back scratch than the context holds";
    return nullptr;
}

extern "C" int hdp_get_tuning(const hdp_ctx* ctx, hdp_tuning* out)
{
    if (!ctx || !out) return HDP_ERR_ARG;
    *out = ctx->c.tune;
    return HDP_OK;
}

extern "C" int hdp_set_tuning(hdp_ctx* ctx, const hdp_tuning* t)
{
    if (!ctx || !t) return HDP_ERR_ARG;
    if (const char* why = tuning_error(ctx->c, *t)) return fail(ctx, HDP_ERR_ARG, why);
    ctx->c.tune = *t;
    drop_host_graph(ctx);   // captured with the old launch shapes
    return HDP_OK;
}

// fastest of `reps` timed runs of hdp_build_trees + hdp_match with the current knobs
static int tune_time(hdp_ctx* ctx, const uint8_t* L, const uint8_t* R, int pitch, int reps, float* ms)
{
    Ctx& c = ctx->c;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    TRY_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(ctx, HDP_ERR_CUDA, "cudaEventCreate");
    }
    float best = 1e30f;
    int rc = HDP_OK;
    for (int r = 0; r < reps && rc == HDP_OK; ++r) {
        cudaEventRecord(e0, c.s);
        rc = hdp_build_trees(ctx, L, R, pitch);
        if (rc == HDP_OK) rc = hdp_match(ctx, c.disp_host_stage);
        cudaEventRecord(e1, c.s);
        if (rc == HDP_OK) rc = hdp_sync(ctx);
        float t = 0.f;
        if (rc == HDP_OK && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess && t < best) best = t;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms = best;
    return rc;
}

extern "C" int hdp_autotune(hdp_ctx* ctx, const uint8_t* d_left, const uint8_t* d_right, int pitch, int reps,
                            hdp_tuning* out)
{
    if (!ctx) return HDP_ERR_ARG;
    if (reps < 1 || reps > 16) return fail(ctx, HDP_ERR_ARG, "reps out of 1..16");
    Ctx& c = ctx->c;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (c.s && cudaStreamIsCapturing(c.s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
        return fail(ctx, HDP_ERR_STATE, "hdp_autotune during stream capture");
    const int timing = ctx->timing;
    ctx->timing = 0;
    float best = 0.f;
    int rc = tune_time(ctx, d_left, d_right, pitch, reps, &best);   // also warms up
    if (rc == HDP_OK) rc = tune_time(ctx, d_left, d_right, pitch, reps, &best);
    // per knob a few candidates (0 ends a list); the layout knobs choose the
    // tile sizes (how long a carry chain a tile covers) and, for one-set
    // layers, the kernel (a thread per two labels or a warp per tile)
    static const int cand[9][5] = {{2048, 4096, 8192, 16384, 0},
                                   {512, 1024, 2048, 4096, 0},
                                   {32768, 131072, 524288, 0, 0},
                                   {262144, 1 << 20, 1 << 24, 0, 0},
                                   {1, 2, 4, 0, 0},
                                   {4, 5, 6, 8, 0},
                                   {1 << 15, 1 << 17, 1 << 19, 0, 0},
                                   {1 << 17, 1 << 19, 1 << 21, 0, 0},
                                   {64, 128, 257, 0, 0}};
    for (int k = 0; k < 9 && rc == HDP_OK; ++k) {
        hdp_tuning keep = c.tune;
        for (int j = 0; j < 5 && cand[k][j] && rc == HDP_OK; ++j) {
            hdp_tuning t = keep;
            int* f = k == 0 ? &t.boruvka_edges_per_cta : k == 1 ? &t.big_class_edges : k == 2 ? &t.one_cta_nodes
                   : k == 3 ? &t.region_max_nodes : k == 4 ? &t.region_ctas_per_sm : k == 5 ? &t.agg_ctas_per_sm
                   : k == 6 ? &t.tile_small_nodes : k == 7 ? &t.tile_small_nodes_hdp : &t.col_min_labels;
            if (*f == cand[k][j]) continue;
            *f = cand[k][j];
            if (tuning_error(c, t)) continue;   // e.g. more tiles than the look-back scratch holds
            c.tune = t;
            float ms = 0.f;
            rc = tune_time(ctx, d_left, d_right, pitch, reps, &ms);
            if (rc == HDP_OK && ms < best) {
                best = ms;
                keep = t;
            }
        }
        c.tune = keep;
    }
    ctx->timing = timing;
    drop_host_graph(ctx);   // captured with other launch shapes
    if (rc != HDP_OK) return rc;
    if (out) *out = c.tune;
    return HDP_OK;
}

extern "C" int hdp_refine(hdp_ctx* ctx, const uint8_t* d_left, const uint8_t* d_right, int pitch, int32_t* d_disp_out)
{
    if (!ctx || !d_left || !d_right || !d_disp_out) return HDP_ERR_ARG;
    Ctx& c = ctx->c;
    if (pitch < 3 * c.p.width) return fail(ctx, HDP_ERR_ARG, "bad pitch");
    const int W = c.p.width, H = c.p.height;
    // the right view's map: the method on the mirrored, exchanged pair (the
    // staging buffers are free: hdp_build_trees waits for earlier side work)
    for (int l = 0; l < HDP_MAX_LEVELS; ++l)
        if (c.side_pending[l]) {
            TRY_CUDA(cudaStreamWaitEvent(c.s, c.ev_side[l], 0));
            c.side_pending[l] = 0;
        }
    launch_mirror(d_right, pitch, W, H, c.stage_l, c.s);
    launch_mirror(d_left, pitch, W, H, c.stage_r, c.s);
    int rc = hdp_build_trees(ctx, c.stage_l, c.stage_r, 3 * W);
    if (!rc) rc = hdp_match(ctx, c.dispRm);
    // the left view's map, which leaves layer 0's forest loaded
    if (!rc) rc = hdp_build_trees(ctx, d_left, d_right, pitch);
    if (!rc) rc = hdp_match(ctx, d_disp_out);
    if (rc) return rc;
    launch_refine(c);
    TRY_CUDA(cudaMemcpyAsync(d_disp_out, c.disp[0], sizeof(int32_t) * c.dim[0].N, cudaMemcpyDeviceToDevice, c.s));
    c.refined = 1;
    return check_launch(ctx, "hdp_refine");
}

static void drop_host_graph(hdp_ctx* ctx)
{
    if (ctx->host_exec) { cudaGraphExecDestroy(ctx->host_exec); ctx->host_exec = nullptr; }
    if (ctx->host_graph) { cudaGraphDestroy(ctx->host_graph); ctx->host_graph = nullptr; }
}

extern "C" int hdp_match_host(hdp_ctx* ctx, const uint8_t* h_left, const uint8_t* h_right, int32_t* h_disp_out)
{
    if (!ctx || !h_left || !h_right || !h_disp_out) return HDP_ERR_ARG;
    Ctx& c = ctx->c;
    const size_t bytes = 3 * (size_t)c.dim[0].N;
    TRY_CUDA(cudaMemcpyAsync(c.stage_l, h_left, bytes, cudaMemcpyHostToDevice, c.s));
    TRY_CUDA(cudaMemcpyAsync(c.stage_r, h_right, bytes, cudaMemcpyHostToDevice, c.s));
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const bool graphable = c.s && !ctx->timing && cudaStreamIsCapturing(c.s, &cs) == cudaSuccess &&
                           cs == cudaStreamCaptureStatusNone;
    int rc = HDP_OK;
    if (graphable) {
        // the device side of every call is the same work on the same staging
        // buffers: capture it once (first call) and replay it
        if (!ctx->host_exec) {
            if (c.s2) TRY_CUDA(cudaStreamSynchronize(c.s2));   // a capture cannot wait on earlier side work
            for (int l = 0; l < HDP_MAX_LEVELS; ++l) c.side_pending[l] = 0;
            TRY_CUDA(cudaStreamBeginCapture(c.s, cudaStreamCaptureModeThreadLocal));
            rc = hdp_build_trees(ctx, c.stage_l, c.stage_r, 3 * c.p.width);
            if (!rc) rc = hdp_match(ctx, c.disp_host_stage);
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamEndCapture(c.s, &g);
            if (rc) { if (g) cudaGraphDestroy(g); return rc; }
            if (e != cudaSuccess) return fail(ctx, HDP_ERR_CUDA, std::string("host-path capture: ") + cudaGetErrorString(e));
            ctx->host_graph = g;
            TRY_CUDA(cudaGraphInstantiate(&ctx->host_exec, g, 0));
        }
        TRY_CUDA(cudaGraphLaunch(ctx->host_exec, c.s));
    } else {
        rc = hdp_build_trees(ctx, c.stage_l, c.stage_r, 3 * c.p.width);
        if (!rc) rc = hdp_match(ctx, c.disp_host_stage);
        if (rc) return rc;
    }
    TRY_CUDA(cudaMemcpyAsync(h_disp_out, c.disp_host_stage, sizeof(int32_t) * c.dim[0].N, cudaMemcpyDeviceToHost, c.s));
    return hdp_sync(ctx);
}

extern "C" int hdp_destroy(hdp_ctx* ctx)
{
    if (!ctx) return HDP_ERR_ARG;
    int rc = HDP_OK;
    if (ctx->c.arena) {
        cudaError_t e = cudaStreamSynchronize(ctx->c.s);
        if (e != cudaSuccess) rc = HDP_ERR_CUDA;
        else {
            DevStatus st;
            if (cudaMemcpy(&st, ctx->c.st, sizeof(st), cudaMemcpyDeviceToHost) == cudaSuccess && st.err)
                rc = st.err == DEV_TIMEOUT ? HDP_ERR_TIMEOUT : HDP_ERR_ARG;
        }
        cudaFree(ctx->c.arena);
    }
    for (int l = 0; l < HDP_MAX_LEVELS; ++l)
        for (int k = 0; k < 6; ++k)
            if (ctx->ev[l][k]) cudaEventDestroy(ctx->ev[l][k]);
    for (int i = 0; i < 4; ++i)
        if (ctx->c.gvol[i]) cudaFree(ctx->c.gvol[i]);
    if (ctx->c.gacc) cudaFree(ctx->c.gacc);
    if (ctx->c.wf) cudaFree(ctx->c.wf);
    if (ctx->fork) cudaEventDestroy(ctx->fork);
    if (ctx->join) cudaEventDestroy(ctx->join);
    if (ctx->c.s2) {
        cudaStreamSynchronize(ctx->c.s2);
        cudaStreamDestroy(ctx->c.s2);
    }
    if (ctx->c.ev_fork) cudaEventDestroy(ctx->c.ev_fork);
    for (int l = 0; l < HDP_MAX_LEVELS; ++l)
        if (ctx->c.ev_side[l]) cudaEventDestroy(ctx->c.ev_side[l]);
    if (ctx->exec) cudaGraphExecDestroy(ctx->exec);
    if (ctx->graph) cudaGraphDestroy(ctx->graph);
    drop_host_graph(ctx);
    if (ctx->own_stream && ctx->c.s) cudaStreamDestroy(ctx->c.s);
    delete ctx;
    return rc;
}

extern "C" int hdp_create_own_stream(const hdp_params* p, hdp_ctx** out)
{
    if (!p || !out) return HDP_ERR_ARG;
    *out = nullptr;
    cudaStream_t s = nullptr;
    cudaError_t ce = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (ce != cudaSuccess) {
        fprintf(stderr, "hdp_create_own_stream: %s\n", cudaGetErrorString(ce));
        return HDP_ERR_CUDA;
    }
    int rc = hdp_create(p, s, out);
    if (rc != HDP_OK) {
        cudaStreamDestroy(s);
        return rc;
    }
    (*out)->own_stream = true;
    return HDP_OK;
}

extern "C" void* hdp_get_stream(const hdp_ctx* ctx) { return ctx ? (void*)ctx->c.s : nullptr; }

extern "C" const char* hdp_last_error(const hdp_ctx* ctx) { return ctx ? ctx->c.err.c_str() : "null context"; }

// ------------------------------------------------------------ stages ---
static int read_int(hdp_ctx* ctx, int idx, int* out)
{
    Ctx& c = ctx->c;
    TRY_CUDA(cudaStreamSynchronize(c.s));
    TRY_CUDA(cudaMemcpy(out, c.ints + idx, sizeof(int), cudaMemcpyDeviceToHost));
    return HDP_OK;
}

static bool tree_stage(int what)
{
    return what == HDP_STAGE_WEIGHTS || what == HDP_STAGE_EDGES || what == HDP_STAGE_IN_TREE ||
           what == HDP_STAGE_DT_ROOT || what == HDP_STAGE_TREE_INTV || what == HDP_STAGE_BFS ||
           what == HDP_STAGE_PARENT || what == HDP_STAGE_DEPTH || what == HDP_STAGE_COSTS ||
           what == HDP_STAGE_PIX_SET || what == HDP_STAGE_INFO;
}

extern "C" int64_t hdp_stage_bytes(hdp_ctx* ctx, int level, int what)
{
    if (!ctx) return HDP_ERR_ARG;
    Ctx& c = ctx->c;
    if (level < 0 || level > c.top) return HDP_ERR_ARG;
    const int64_t N = c.dim[level].N;
    switch (what) {
    case HDP_STAGE_PYR_LEFT:
    case HDP_STAGE_PYR_RIGHT: return 16 * N;
    case HDP_STAGE_WEIGHTS: return 8 * N;
    case HDP_STAGE_EDGES: {
        int n = 0;
        int rc = read_int(ctx, IDX_NEDGES, &n);
        return rc ? rc : 4 * (int64_t)n;
    }
    case HDP_STAGE_IN_TREE: return 2 * N;
    case HDP_STAGE_DT_ROOT:
    case HDP_STAGE_BFS:
    case HDP_STAGE_PARENT:
    case HDP_STAGE_DEPTH:
    case HDP_STAGE_PIX_SET:
    case HDP_STAGE_DISP: return 4 * N;
    case HDP_STAGE_TREE_INTV: return 32 * N;
    case HDP_STAGE_PRIOR: return 8 * (int64_t)(c.dim[level].d + 1);
    case HDP_STAGE_TABLE: return level < c.top ? 32 * (int64_t)(c.dim[level + 1].d + 1) : HDP_ERR_ARG;
    case HDP_STAGE_COSTS: {
        if (c.tree_level != level) return HDP_ERR_STATE;
        TRY_CUDA(cudaStreamSynchronize(c.s));
        std::vector<int> rdt(N);
        TRY_CUDA(cudaMemcpy(rdt.data(), c.rdt, 4 * N, cudaMemcpyDeviceToHost));
        std::vector<uint32_t> T((size_t)N * HDP_WORDS);
        TRY_CUDA(cudaMemcpy(T.data(), c.T, 32 * N, cudaMemcpyDeviceToHost));
        int64_t K = 0;
        for (int64_t i = 0; i < N; ++i)
            for (int k = 0; k < HDP_WORDS; ++k) K += __builtin_popcount(T[(size_t)rdt[i] * HDP_WORDS + k]);
        return 4 * K;
    }
    case HDP_STAGE_INFO: return 8 * 16;
    case HDP_STAGE_REF_D:
    case HDP_STAGE_DISP_R: return level == 0 && c.refined ? 4 * N : HDP_ERR_STATE;
    default: return HDP_ERR_ARG;
    }
}

extern "C" int hdp_get_stage(hdp_ctx* ctx, int level, int what, void* h_dst, size_t bytes)
{
    if (!ctx || !h_dst) return HDP_ERR_ARG;
    Ctx& c = ctx->c;
    int64_t need = hdp_stage_bytes(ctx, level, what);
    if (need < 0) return (int)need;
    if ((int64_t)bytes != need) return fail(ctx, HDP_ERR_ARG, "stage size mismatch");
    if (tree_stage(what) && c.tree_level != level && what != HDP_STAGE_PIX_SET)
        return fail(ctx, HDP_ERR_STATE, "the work buffers hold another layer");
    int rc = hdp_sync(ctx);
    if (rc) return rc;
    const int N = c.dim[level].N;
    switch (what) {
    case HDP_STAGE_PYR_LEFT: TRY_CUDA(cudaMemcpy(h_dst, c.imL[level], bytes, cudaMemcpyDeviceToHost)); break;
    case HDP_STAGE_PYR_RIGHT: TRY_CUDA(cudaMemcpy(h_dst, c.imR[level], bytes, cudaMemcpyDeviceToHost)); break;
    case HDP_STAGE_WEIGHTS: TRY_CUDA(cudaMemcpy(h_dst, c.weights, bytes, cudaMemcpyDeviceToHost)); break;
    case HDP_STAGE_EDGES: {
        std::vector<uint32_t> k(bytes / 4);
        TRY_CUDA(cudaMemcpy(k.data(), c.sorted, bytes, cudaMemcpyDeviceToHost));
        uint32_t mask = (1u << edge_bits(N)) - 1u;
        int32_t* o = (int32_t*)h_dst;
        for (size_t i = 0; i < k.size(); ++i) o[i] = (int32_t)(k[i] & mask);
        break;
    }
    case HDP_STAGE_IN_TREE: TRY_CUDA(cudaMemcpy(h_dst, c.in_tree, bytes, cudaMemcpyDeviceToHost)); break;
    case HDP_STAGE_DT_ROOT: TRY_CUDA(cudaMemcpy(h_dst, c.dtroot, bytes, cudaMemcpyDeviceToHost)); break;
    case HDP_STAGE_TREE_INTV: {
        std::vector<int> r(N);
        std::vector<uint32_t> T((size_t)N * HDP_WORDS);
        TRY_CUDA(cudaMemcpy(r.data(), c.rootof, 4 * (size_t)N, cudaMemcpyDeviceToHost));
        TRY_CUDA(cudaMemcpy(T.data(), c.T, 32 * (size_t)N, cudaMemcpyDeviceToHost));
        uint32_t* o = (uint32_t*)h_dst;
        for (int v = 0; v < N; ++v)
            for (int k = 0; k < HDP_WORDS; ++k) o[(size_t)v * HDP_WORDS + k] = T[(size_t)r[v] * HDP_WORDS + k];
        break;
    }
    case HDP_STAGE_BFS:
        launch_bfs(c, level);
        TRY_CUDA(cudaStreamSynchronize(c.s));
        TRY_CUDA(cudaMemcpy(h_dst, c.bfs, bytes, cudaMemcpyDeviceToHost));
        break;
    case HDP_STAGE_PARENT: TRY_CUDA(cudaMemcpy(h_dst, c.par, bytes, cudaMemcpyDeviceToHost)); break;
    case HDP_STAGE_DEPTH: TRY_CUDA(cudaMemcpy(h_dst, c.depth, bytes, cudaMemcpyDeviceToHost)); break;
    case HDP_STAGE_PRIOR: TRY_CUDA(cudaMemcpy(h_dst, c.prior[level], bytes, cudaMemcpyDeviceToHost)); break;
    case HDP_STAGE_TABLE: TRY_CUDA(cudaMemcpy(h_dst, c.table[level], bytes, cudaMemcpyDeviceToHost)); break;
    case HDP_STAGE_PIX_SET: TRY_CUDA(cudaMemcpy(h_dst, c.pixset, bytes, cudaMemcpyDeviceToHost)); break;
    case HDP_STAGE_DISP: TRY_CUDA(cudaMemcpy(h_dst, c.disp[level], bytes, cudaMemcpyDeviceToHost)); break;
    case HDP_STAGE_REF_D: TRY_CUDA(cudaMemcpy(h_dst, c.refD, bytes, cudaMemcpyDeviceToHost)); break;
    case HDP_STAGE_DISP_R: TRY_CUDA(cudaMemcpy(h_dst, c.refR, bytes, cudaMemcpyDeviceToHost)); break;
    case HDP_STAGE_COSTS: {
        std::vector<int> rowof(N), rdt(N);
        std::vector<uint32_t> roff(N + 1), T((size_t)N * HDP_WORDS);
        TRY_CUDA(cudaMemcpy(rowof.data(), c.rowof, 4 * (size_t)N, cudaMemcpyDeviceToHost));
        TRY_CUDA(cudaMemcpy(rdt.data(), c.rdt, 4 * (size_t)N, cudaMemcpyDeviceToHost));
        TRY_CUDA(cudaMemcpy(roff.data(), c.roff, 4 * (size_t)N, cudaMemcpyDeviceToHost));
        TRY_CUDA(cudaMemcpy(T.data(), c.T, 32 * (size_t)N, cudaMemcpyDeviceToHost));
        int Kp = 0;
        TRY_CUDA(cudaMemcpy(&Kp, c.ints + IDX_K, sizeof(int), cudaMemcpyDeviceToHost));
        std::vector<float> vol((size_t)(uint32_t)Kp);
        std::vector<float> nd;
        if (c.p.storage == HDP_STORE_FP16) {
            std::vector<__half> h(vol.size());
            TRY_CUDA(cudaMemcpy(h.data(), c.volh, 2 * h.size(), cudaMemcpyDeviceToHost));
            for (size_t i = 0; i < h.size(); ++i) vol[i] = __half2float(h[i]);
            nd.resize(N);
            TRY_CUDA(cudaMemcpy(nd.data(), c.nfull, 4 * (size_t)N, cudaMemcpyDeviceToHost));
        } else {
            TRY_CUDA(cudaMemcpy(vol.data(), c.vol, 4 * vol.size(), cudaMemcpyDeviceToHost));
        }
        float* o = (float*)h_dst;
        size_t w = 0;
        for (int v = 0; v < N; ++v) {
            int r = rowof[v];
            int k = 0;
            for (int t = 0; t < HDP_WORDS; ++t) k += __builtin_popcount(T[(size_t)rdt[r] * HDP_WORDS + t]);
            float sc = nd.empty() ? 1.f : nd[r];
            for (int j = 0; j < k; ++j) o[w++] = vol[roff[r] + j] * sc;
        }
        break;
    }
    case HDP_STAGE_INFO: {
        int v[IDX_COUNT];
        TRY_CUDA(cudaMemcpy(v, c.ints, sizeof(v), cudaMemcpyDeviceToHost));
        int64_t* o = (int64_t*)h_dst;
        memset(o, 0, 16 * 8);
        o[0] = (uint32_t)v[IDX_K];
        o[1] = v[IDX_NEDGES];
        o[2] = v[IDX_NTREES];
        o[3] = v[IDX_ENGINE];
        o[4] = v[IDX_NUNITS];
        o[5] = v[IDX_RISKY];
        o[6] = v[IDX_NARCS];
        o[7] = v[IDX_NCLS];
        o[8] = v[IDX_NLC];
        o[9] = v[IDX_DRROUNDS];      // windowed forest engines: reservation rounds
        o[10] = v[IDX_DRWINDOWS];    // and windows
        break;
    }
    default: return HDP_ERR_ARG;
    }
    return HDP_OK;
}

extern "C" int hdp_set_stage(hdp_ctx* ctx, int level, int what, const void* h_src, size_t bytes)
{
    if (!ctx || !h_src) return HDP_ERR_ARG;
    Ctx& c = ctx->c;
    if (level < 0 || level > c.top) return fail(ctx, HDP_ERR_ARG, "level out of range");
    int64_t need = hdp_stage_bytes(ctx, level, what);
    if (need < 0) return (int)need;
    if ((int64_t)bytes != need) return fail(ctx, HDP_ERR_ARG, "stage size mismatch");
    if (what == HDP_STAGE_DISP) {
        const int32_t* d = (const int32_t*)h_src;
        for (int i = 0; i < c.dim[level].N; ++i)
            if (d[i] < 0 || d[i] > c.dim[level].d) return fail(ctx, HDP_ERR_ARG, "disparity out of range");
        TRY_CUDA(cudaMemcpyAsync(c.disp[level], h_src, bytes, cudaMemcpyHostToDevice, c.s));
        TRY_CUDA(cudaStreamSynchronize(c.s));
        return HDP_OK;
    }
    if (what == HDP_STAGE_PRIOR) {
        if (c.s2) TRY_CUDA(cudaStreamSynchronize(c.s2));   // the side stream may still write this prior
        TRY_CUDA(cudaMemcpyAsync(c.prior[level], h_src, bytes, cudaMemcpyHostToDevice, c.s));
        TRY_CUDA(cudaStreamSynchronize(c.s));
        ctx->prior_injected[level] = 1;
        return HDP_OK;
    }
    return fail(ctx, HDP_ERR_ARG, "stage cannot be set");
}

extern "C" int hdp_set_timing(hdp_ctx* ctx, int on)
{
    if (!ctx) return HDP_ERR_ARG;
    ctx->timing = on ? 1 : 0;
    for (int l = 0; l < HDP_MAX_LEVELS; ++l)
        for (int k = 0; k < 6; ++k) ctx->ev_used[l][k] = 0;
    return HDP_OK;
}

extern "C" int hdp_get_timings(hdp_ctx* ctx, float* ms, int n)
{
    if (!ctx || !ms || n < 5 * ctx->c.nlev) return HDP_ERR_ARG;
    int rc = hdp_sync(ctx);
    if (rc) return rc;
    for (int l = 0; l < ctx->c.nlev; ++l)
        for (int k = 0; k < 5; ++k) {
            float t = 0.f;
            if (ctx->ev_used[l][k] && ctx->ev_used[l][k + 1]) {
                cudaError_t e = cudaEventElapsedTime(&t, ctx->ev[l][k], ctx->ev[l][k + 1]);
                if (e != cudaSuccess) {
                    cudaGetLastError();
                    return fail(ctx, HDP_ERR_CUDA, std::string("timing events: ") + cudaGetErrorString(e));
                }
            }
            ms[l * 5 + k] = t;
        }
    return HDP_OK;
}

extern "C" int hdp_graph_capture(hdp_ctx* ctx, const uint8_t* d_left, const uint8_t* d_right, int pitch,
                                 int32_t* d_out, int* n_kernels)
{
    if (!ctx || !d_out) return HDP_ERR_ARG;
    Ctx& c = ctx->c;
    if (!c.s) return fail(ctx, HDP_ERR_ARG, "graph capture needs a non-default stream");
    if (ctx->exec) { cudaGraphExecDestroy(ctx->exec); ctx->exec = nullptr; }
    if (ctx->graph) { cudaGraphDestroy(ctx->graph); ctx->graph = nullptr; }
    for (int l = 0; l < HDP_MAX_LEVELS; ++l)
        for (int k = 0; k < 6; ++k) ctx->ev_used[l][k] = 0;
    // a capture cannot wait on work recorded before it
    if (c.s2) TRY_CUDA(cudaStreamSynchronize(c.s2));
    for (int l = 0; l < HDP_MAX_LEVELS; ++l) c.side_pending[l] = 0;
    TRY_CUDA(cudaStreamBeginCapture(c.s, cudaStreamCaptureModeThreadLocal));
    int rc = hdp_build_trees(ctx, d_left, d_right, pitch);
    if (!rc) rc = hdp_match(ctx, d_out);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(c.s, &g);
    if (rc) { if (g) cudaGraphDestroy(g); return rc; }
    if (e != cudaSuccess) return fail(ctx, HDP_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
    ctx->graph = g;
    size_t nn = 0;
    TRY_CUDA(cudaGraphGetNodes(g, nullptr, &nn));
    std::vector<cudaGraphNode_t> nodes(nn);
    TRY_CUDA(cudaGraphGetNodes(g, nodes.data(), &nn));
    int k = 0;
    for (auto nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
    }
    if (n_kernels) *n_kernels = k;
    TRY_CUDA(cudaGraphInstantiate(&ctx->exec, g, 0));
    return HDP_OK;
}

extern "C" int hdp_graph_launch(hdp_ctx* ctx)
{
    if (!ctx) return HDP_ERR_ARG;
    if (!ctx->exec) return fail(ctx, HDP_ERR_STATE, "no captured graph");
    TRY_CUDA(cudaGraphLaunch(ctx->exec, ctx->c.s));
    return HDP_OK;
}

// ------------------------------------------------------ no-allocation path ---
// Workspace of hdp_match_noalloc: a fixed device array that lives as long as
// the library is loaded, on every GPU that loads it.
#define HDP_NOALLOC_BYTES (64u << 20)
static __device__ __align__(256) char g_noalloc_scratch[HDP_NOALLOC_BYTES];

#define HDP_NOALLOC_MAX_DEVICES 64
static char* g_noalloc_ptr[HDP_NOALLOC_MAX_DEVICES];

extern "C" int hdp_match_noalloc(const hdp_params* p, const uint8_t* d_left, const uint8_t* d_right, int pitch,
                                 int32_t* d_disp_out, void* stream)
{
    if (!p || !d_left || !d_right || !d_disp_out) return HDP_ERR_ARG;
    {
        // the call synchronises its stream twice, which a stream under capture forbids
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing((cudaStream_t)stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
            cudaGetLastError();
            fprintf(stderr, "hdp_match_noalloc: the stream is being captured; this call cannot be captured\n");
            return HDP_ERR_STATE;
        }
    }
    hdp_ctx local;   // on the stack: no device allocation
    hdp_ctx* ctx = &local;
    Ctx& c = ctx->c;
    c.s = (cudaStream_t)stream;
    if (const char* why = setup_params(c, p)) {
        fprintf(stderr, "hdp_match_noalloc: %s\n", why);
        return HDP_ERR_ARG;
    }
    if (pitch < 3 * p->width) return HDP_ERR_ARG;
    c.arena = nullptr;
    layout_buffers(c);
    if (c.arena_used > HDP_NOALLOC_BYTES) {
        fprintf(stderr, "hdp_match_noalloc: this problem needs %zu bytes of workspace, above the fixed %u\n",
                c.arena_used, (unsigned)HDP_NOALLOC_BYTES);
        return HDP_ERR_ARG;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= HDP_NOALLOC_MAX_DEVICES) return HDP_ERR_CUDA;
    if (!g_noalloc_ptr[dev]) {
        // one-time set-up on this device (it must be current): the device
        // address of the fixed array; host code cannot use the symbol itself
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) {
            fprintf(stderr, "hdp_match_noalloc: cudaGetSymbolAddress: %s\n", cudaGetErrorString(e));
            return HDP_ERR_CUDA;
        }
        g_noalloc_ptr[dev] = (char*)ptr;
    }
    c.arena = g_noalloc_ptr[dev];
    c.arena_bytes = HDP_NOALLOC_BYTES;
    cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, dev);
    layout_buffers(c);
    // the array keeps the previous call's contents: reset what must start at zero
    HostConsts hc;   // on the stack
    host_constants(c, hc);
    TRY_CUDA(cudaMemcpyAsync(c.gmm, hc.g, sizeof(hc.g), cudaMemcpyHostToDevice, c.s));
    TRY_CUDA(cudaMemcpyAsync(c.gmm_k, hc.gk, sizeof(hc.gk), cudaMemcpyHostToDevice, c.s));
    TRY_CUDA(cudaMemcpyAsync(c.full_mask, hc.fm, sizeof(hc.fm), cudaMemcpyHostToDevice, c.s));
    TRY_CUDA(cudaMemsetAsync(c.st, 0, sizeof(DevStatus), c.s));
    TRY_CUDA(cudaMemsetAsync(c.ints, 0, sizeof(int) * IDX_COUNT, c.s));
    c.scan.st = c.st;
    c.scan4.st = c.st;
    TRY_CUDA(cudaMemsetAsync(c.scan.state, 0, sizeof(unsigned long long) * c.scan.max_tiles, c.s));
    TRY_CUDA(cudaMemsetAsync(c.scan.ctr, 0, 2 * sizeof(unsigned int), c.s));
    TRY_CUDA(cudaMemsetAsync(c.scan4.flags, 0, sizeof(unsigned int) * c.scan4.max_tiles, c.s));
    TRY_CUDA(cudaMemsetAsync(c.scan4.ctr, 0, 2 * sizeof(unsigned int), c.s));
    // the host constants above must outlive the copies: wait for them
    TRY_CUDA(cudaStreamSynchronize(c.s));
    int rc = hdp_build_trees(ctx, d_left, d_right, pitch);
    if (!rc) rc = hdp_match(ctx, d_disp_out);
    // wait for the work and read its device status (a bounded wait that gave
    // up, an invalid device input): the status block lives in the shared
    // array, so this call is the only one that can report it
    if (!rc) rc = hdp_sync(ctx);
    if (rc) {
        fprintf(stderr, "hdp_match_noalloc: %s\n", c.err.c_str());
        return rc;
    }
    return HDP_OK;
}

// ---------------------------------------------------------- GMM by EM ---
static int stream_error(const char* where)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        fprintf(stderr, "%s: %s\n", where, cudaGetErrorString(e));
        return HDP_ERR_CUDA;
    }
    return HDP_OK;
}

extern "C" int hdp_gt_down(const int32_t* d_gt, int width, int height, int32_t* d_gt_up, void* stream)
{
    if (!d_gt || !d_gt_up || width < 1 || height < 1 || (long long)width * height > (1 << 23)) return HDP_ERR_ARG;
    launch_gt_down(d_gt, width, height, d_gt_up, (cudaStream_t)stream);
    return stream_error("hdp_gt_down");
}

extern "C" int hdp_offset_hist(const int32_t* d_up, const int32_t* d_lo, int width, int height, int range,
                               unsigned long long* d_hist, void* stream)
{
    if (!d_up || !d_lo || !d_hist || width < 1 || height < 1 || (long long)width * height > (1 << 23) ||
        range < 0 || range > HDP_MAX_DISP)
        return HDP_ERR_ARG;
    int dev = 0, sms = 1;
    if (cudaGetDevice(&dev) != cudaSuccess) return HDP_ERR_CUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    launch_offset_hist(d_up, d_lo, width, height, range, d_hist, sms, (cudaStream_t)stream);
    return stream_error("hdp_offset_hist");
}

extern "C" int hdp_gmm_em(const unsigned long long* d_hist, int range, int K, int iters, float sd_min, float* d_out,
                          void* stream)
{
    if (!d_hist || !d_out || range < 0 || range > HDP_MAX_DISP || K < 1 || K > HDP_MAX_GMM || iters < 0 ||
        iters > 100000 || !(sd_min > 0.f))
        return HDP_ERR_ARG;
    launch_gmm_em(d_hist, range, K, iters, sd_min, d_out, (cudaStream_t)stream);
    return stream_error("hdp_gmm_em");
}

// ------------------------------------------------------ differentiable path ---
extern "C" int hdp_tree_level(const hdp_ctx* ctx)
{
    if (!ctx) return HDP_ERR_ARG;
    return ctx->c.built ? ctx->c.tree_level : -1;
}

static int grad_ready(hdp_ctx* ctx)
{
    Ctx& c = ctx->c;
    if (!c.built || c.tree_level < 0) return fail(ctx, HDP_ERR_STATE, "no tree loaded (call hdp_build_trees)");
    const bool full = c.p.mode == HDP_MODE_FULL || c.tree_level == c.top;
    if (!full) return fail(ctx, HDP_ERR_STATE, "the loaded layer is not full range");
    if (c.p.storage != HDP_STORE_FP32) return fail(ctx, HDP_ERR_ARG, "the differentiable path needs FP32 storage");
    return HDP_OK;
}

extern "C" int hdp_aggregate_fwd(hdp_ctx* ctx, const float* d_E, float* d_C)
{
    if (!ctx || !d_E || !d_C) return HDP_ERR_ARG;
    int rc = grad_ready(ctx);
    if (rc) return rc;
    rc = grad_forward(ctx->c, d_E, d_C);
    if (rc) return fail(ctx, rc, "workspace for the differentiable path");
    return check_launch(ctx, "hdp_aggregate_fwd");
}

extern "C" int hdp_aggregate_bwd(hdp_ctx* ctx, const float* d_E, const float* d_gC, float* d_gE, float* d_gw,
                                 float* d_ggamma)
{
    if (!ctx || !d_E || !d_gC || !d_gE || !d_gw || !d_ggamma) return HDP_ERR_ARG;
    int rc = grad_ready(ctx);
    if (rc) return rc;
    rc = grad_backward(ctx->c, d_E, d_gC, d_gE, d_gw, d_ggamma);
    if (rc) return fail(ctx, rc, "workspace for the differentiable path");
    return check_launch(ctx, "hdp_aggregate_bwd");
}

extern "C" int hdp_set_gamma(hdp_ctx* ctx, float gamma)
{
    if (!ctx || !(gamma > 0)) return HDP_ERR_ARG;
    int rc = grad_ready(ctx);
    if (rc) return rc;
    launch_set_gamma(ctx->c, gamma);
    return check_launch(ctx, "hdp_set_gamma");
}

extern "C" int hdp_soft_argmin_l1(hdp_ctx* ctx, const float* d_C, const float* d_gt, const uint8_t* d_valid, float T,
                                  float* d_disp, float* d_loss, float* d_gC)
{
    if (!ctx || !d_C || !(T > 0)) return HDP_ERR_ARG;
    if ((d_loss || d_gC) && !d_gt) return HDP_ERR_ARG;
    int rc = grad_ready(ctx);
    if (rc) return rc;
    rc = launch_soft_argmin_l1(ctx->c, d_C, d_gt, d_valid, T, d_disp, d_loss, d_gC);
    if (rc) return fail(ctx, rc, "workspace for the differentiable path");
    return check_launch(ctx, "hdp_soft_argmin_l1");
}

extern "C" int hdp_set_edge_weights(hdp_ctx* ctx, const float* d_w)
{
    if (!ctx) return HDP_ERR_ARG;
    int rc = grad_ready(ctx);
    if (rc) return rc;
    rc = set_edge_weights(ctx->c, d_w);
    if (rc) return fail(ctx, rc, "workspace for the differentiable path");
    return check_launch(ctx, "hdp_set_edge_weights");
}

static bool cost_params_ok(float alpha, float tau_c, float tau_g)
{
    return std::isfinite(alpha) && std::isfinite(tau_c) && std::isfinite(tau_g) && tau_c >= 0.f && tau_g >= 0.f;
}

extern "C" int hdp_cost_volume(hdp_ctx* ctx, float alpha, float tau_c, float tau_g, float* d_E)
{
    if (!ctx || !d_E || !cost_params_ok(alpha, tau_c, tau_g)) return HDP_ERR_ARG;
    int rc = grad_ready(ctx);
    if (rc) return rc;
    launch_cost_volume(ctx->c, alpha, tau_c, tau_g, d_E);
    return check_launch(ctx, "hdp_cost_volume");
}

extern "C" int hdp_cost_volume_bwd(hdp_ctx* ctx, float alpha, float tau_c, float tau_g, const float* d_gE,
                                   float* d_gparams)
{
    if (!ctx || !d_gE || !d_gparams || !cost_params_ok(alpha, tau_c, tau_g)) return HDP_ERR_ARG;
    int rc = grad_ready(ctx);
    if (rc) return rc;
    rc = launch_cost_param_grad(ctx->c, alpha, tau_c, tau_g, d_gE, d_gparams);
    if (rc) return fail(ctx, rc, "workspace for the differentiable path");
    return check_launch(ctx, "hdp_cost_volume_bwd");
}

// ------------------------------------------------------------------ batch ---
#define HDP_BATCH_MAX 1024

// pairs whose layers have the same sizes, mode and storage (their tiles fall
// in the same classes at every level but the top one)
static bool same_geometry(const Ctx& a, const Ctx& b)
{
    if (a.nlev != b.nlev || a.p.storage != b.p.storage || a.p.mode != b.p.mode) return false;
    for (int l = 0; l < a.nlev; ++l)
        if (a.dim[l].W != b.dim[l].W || a.dim[l].H != b.dim[l].H) return false;
    return true;
}

extern "C" int hdp_match_batch(hdp_ctx** ctxs, int n, const uint8_t* const* d_left, const uint8_t* const* d_right,
                               const int* pitch, int32_t* const* d_out)
{
    if (!ctxs || n <= 0 || !d_left || !d_right || !pitch || !d_out) return HDP_ERR_ARG;
    for (int i = 0; i < n; ++i)
        if (!ctxs[i]) return HDP_ERR_ARG;
    hdp_ctx* ctx = ctxs[0];
    for (int i = 1; i < n; ++i)
        if (ctxs[i]->c.s == ctx->c.s) return fail(ctx, HDP_ERR_ARG, "every context of a batch needs its own stream");
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i]->fork) TRY_CUDA(cudaEventCreateWithFlags(&ctxs[i]->fork, cudaEventDisableTiming));
        if (!ctxs[i]->join) TRY_CUDA(cudaEventCreateWithFlags(&ctxs[i]->join, cudaEventDisableTiming));
    }
    TRY_CUDA(cudaEventRecord(ctx->fork, ctx->c.s));
    for (int i = 1; i < n; ++i) TRY_CUDA(cudaStreamWaitEvent(ctxs[i]->c.s, ctx->fork, 0));
    // no side streams inside a batch: the pairs already fill the GPU, and twice
    // the concurrent branches made the batch graph 1.6x slower
    bool same_layers = true;
    for (int i = 1; i < n; ++i) same_layers = same_layers && ctxs[i]->c.nlev == ctx->c.nlev;
    if (!same_layers || n > HDP_BATCH_MAX) {
        // pairs of different depths: every pair runs its own chain
        for (int i = 0; i < n; ++i) {
            ctxs[i]->use_side = 0;
            int rc = hdp_build_trees(ctxs[i], d_left[i], d_right[i], pitch[i]);
            if (!rc) rc = hdp_match(ctxs[i], d_out[i]);
            ctxs[i]->use_side = 1;
            if (rc) return rc;
        }
    } else {
        // level by level in groups of pairs of one geometry (the same layer sizes,
        // so the same tile classes): each pair prepares the level on its own
        // stream (interval prediction, edges, forest, orders), then one
        // aggregation launch per pass and tile class takes the tiles of every
        // pair of the group (a6-a7 in one launch per level), then the group's
        // pairs go on.  Groups wait only for their own pairs, so one group's
        // aggregation overlaps another's forests.
        Ctx* cs[HDP_BATCH_MAX];
        int order[HDP_BATCH_MAX], gstart[HDP_BATCH_MAX + 1];
        int ng = 0, m = 0;
        for (int i = 0; i < n; ++i) {
            ctxs[i]->use_side = 0;
            int rc = hdp_build_trees(ctxs[i], d_left[i], d_right[i], pitch[i]);
            ctxs[i]->use_side = 1;
            if (rc) return rc;
            ctxs[i]->c.refined = 0;
        }
        // groups in order of first appearance, pairs in batch order inside each
        for (int i = 0; i < n; ++i) {
            bool seen = false;
            for (int j = 0; j < i && !seen; ++j) seen = same_geometry(ctxs[i]->c, ctxs[j]->c);
            if (seen) continue;
            gstart[ng++] = m;
            for (int j = i; j < n; ++j)
                if (same_geometry(ctxs[i]->c, ctxs[j]->c)) order[m++] = j;
        }
        gstart[ng] = m;
        for (int k = 0; k < n; ++k) cs[k] = &ctxs[order[k]]->c;
        for (int l = ctx->c.top; l >= 0; --l) {
            for (int g = 0; g < ng; ++g) {
                hdp_ctx* lead = ctxs[order[gstart[g]]];
                for (int k = gstart[g]; k < gstart[g + 1]; ++k) {
                    hdp_ctx* x = ctxs[order[k]];
                    int rc = run_level_pre(x, l);
                    if (rc) return rc;
                    aggregate_clear(x->c);
                    if (x != lead) {
                        TRY_CUDA(cudaEventRecord(x->join, x->c.s));
                        TRY_CUDA(cudaStreamWaitEvent(lead->c.s, x->join, 0));
                    }
                }
                launch_aggregate_multi(cs + gstart[g], gstart[g + 1] - gstart[g], l, lead->c.s);
                int rc = check_launch(lead, "hdp_match_batch");
                if (rc) return rc;
                TRY_CUDA(cudaEventRecord(lead->fork, lead->c.s));
                for (int k = gstart[g] + 1; k < gstart[g + 1]; ++k)
                    TRY_CUDA(cudaStreamWaitEvent(ctxs[order[k]]->c.s, lead->fork, 0));
            }
        }
        for (int i = 0; i < n; ++i)
            TRY_CUDA(cudaMemcpyAsync(d_out[i], ctxs[i]->c.disp[0], sizeof(int32_t) * ctxs[i]->c.dim[0].N,
                                     cudaMemcpyDeviceToDevice, ctxs[i]->c.s));
    }
    for (int i = 1; i < n; ++i) {
        TRY_CUDA(cudaEventRecord(ctxs[i]->join, ctxs[i]->c.s));
        TRY_CUDA(cudaStreamWaitEvent(ctx->c.s, ctxs[i]->join, 0));
    }
    return HDP_OK;
}

extern "C" int hdp_batch_graph_capture(hdp_ctx** ctxs, int n, const uint8_t* const* d_left,
                                       const uint8_t* const* d_right, const int* pitch, int32_t* const* d_out,
                                       int* n_kernels)
{
    if (!ctxs || n <= 0 || !ctxs[0]) return HDP_ERR_ARG;
    hdp_ctx* ctx = ctxs[0];
    Ctx& c = ctx->c;
    if (!c.s) return fail(ctx, HDP_ERR_ARG, "graph capture needs a non-default stream");
    if (ctx->exec) { cudaGraphExecDestroy(ctx->exec); ctx->exec = nullptr; }
    if (ctx->graph) { cudaGraphDestroy(ctx->graph); ctx->graph = nullptr; }
    // events are created before capture (creation is not a stream operation)
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i]) return HDP_ERR_ARG;
        if (!ctxs[i]->fork) TRY_CUDA(cudaEventCreateWithFlags(&ctxs[i]->fork, cudaEventDisableTiming));
        if (!ctxs[i]->join) TRY_CUDA(cudaEventCreateWithFlags(&ctxs[i]->join, cudaEventDisableTiming));
    }
    for (int i = 0; i < n; ++i) {
        if (ctxs[i]->c.s2) TRY_CUDA(cudaStreamSynchronize(ctxs[i]->c.s2));
        for (int l = 0; l < HDP_MAX_LEVELS; ++l) ctxs[i]->c.side_pending[l] = 0;
    }
    TRY_CUDA(cudaStreamBeginCapture(c.s, cudaStreamCaptureModeGlobal));
    int rc = hdp_match_batch(ctxs, n, d_left, d_right, pitch, d_out);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(c.s, &g);
    if (rc) { if (g) cudaGraphDestroy(g); return rc; }
    if (e != cudaSuccess) return fail(ctx, HDP_ERR_CUDA, std::string("batch capture: ") + cudaGetErrorString(e));
    ctx->graph = g;
    size_t nn = 0;
    TRY_CUDA(cudaGraphGetNodes(g, nullptr, &nn));
    std::vector<cudaGraphNode_t> nodes(nn);
    TRY_CUDA(cudaGraphGetNodes(g, nodes.data(), &nn));
    int k = 0;
    for (auto nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
    }
    if (n_kernels) *n_kernels = k;
    TRY_CUDA(cudaGraphInstantiate(&ctx->exec, g, 0));
    return HDP_OK;
}

extern "C" int hdp_batch_graph_launch(hdp_ctx* ctx) { return hdp_graph_launch(ctx); }
