/*
 * Plain, slow, single-threaded FP64 CPU oracle for hierarchical disparity
 * prediction (HDP) stereo matching, arXiv 1509.08197.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or calls
 * this file; only the tests, the package smoke check and the CPU-baseline leg
 * of the benchmark do.  It shares no code, header or table with the CUDA
 * implementation.
 *
 * Each function follows one step of the paper and says which.  Where the paper
 * is silent the reading used is stated in the comment.  Images are
 * interleaved RGB int32 "at scale 4^l": layer-l intensities multiplied by 4^l,
 * which keeps the S=2 pyramid averages exact integers.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -shared -fPIC -o liboracle.so hdp_oracle.c -lm
 * (-ffp-contract=off keeps FP64 rounding identical on x86-64 and aarch64).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_WORDS 8 /* 256-bit disparity sets: labels 0..255 */

static int64_t scale4(int level) { return (int64_t)1 << (2 * level); }
static int imin(int a, int b) { return a < b ? a : b; }
static int imax(int a, int b) { return a > b ? a : b; }
static int64_t lmin(int64_t a, int64_t b) { return a < b ? a : b; }
static int64_t labs64(int64_t a) { return a < 0 ? -a : a; }

/* ------------------------------------------------------------------------ */
/* Sec. 2.1, graph pyramid: G_{l+1} averages each S x S square of G_l
 * (S = 2).  W_{l+1} = ceil(W_l / 2), H_{l+1} = ceil(H_l / 2).  Reading for
 * the partial squares at the right/bottom border: average over the children
 * that exist (1, 2 or 4).  With src at scale 4^l and dst at scale 4^(l+1),
 * dst = (4 / count) * sum(children), exact in integers.                      */
int orc_pyr_down(const int32_t* src, int W, int H, int32_t* dst)
{
    int Wn = (W + 1) / 2, Hn = (H + 1) / 2;
    for (int Y = 0; Y < Hn; ++Y)
        for (int X = 0; X < Wn; ++X) {
            int64_t sum[3] = {0, 0, 0};
            int count = 0;
            for (int dy = 0; dy < 2; ++dy)
                for (int dx = 0; dx < 2; ++dx) {
                    int x = 2 * X + dx, y = 2 * Y + dy;
                    if (x >= W || y >= H) continue;
                    ++count;
                    for (int c = 0; c < 3; ++c) sum[c] += src[3 * ((int64_t)y * W + x) + c];
                }
            for (int c = 0; c < 3; ++c)
                dst[3 * ((int64_t)Y * Wn + X) + c] = (int32_t)(sum[c] * (4 / count));
        }
    return 0;
}

/* Horizontal intensity gradient used by the matching cost ([Cost2], Sec. 3.3):
 * grey G = (R+G+B)/3, central difference (G(x+1) - G(x-1)) / 2 with the border
 * replicated.  Stored as g = Sum(x+1) - Sum(x-1), Sum = R+G+B at scale 4^l,
 * so the real gradient is g / (6 * 4^l).                                     */
int orc_gradient(const int32_t* img, int W, int H, int32_t* g)
{
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int xm = imax(x - 1, 0), xp = imin(x + 1, W - 1);
            const int32_t* a = img + 3 * ((int64_t)y * W + xp);
            const int32_t* b = img + 3 * ((int64_t)y * W + xm);
            g[(int64_t)y * W + x] = (a[0] + a[1] + a[2]) - (b[0] + b[1] + b[2]);
        }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.3, pixel matching cost M(p, x) of [Cost2]: truncated mean absolute
 * RGB difference and truncated absolute horizontal-gradient difference,
 *   M = (1 - alpha) * min(dc, tau_c) + alpha * min(dg, tau_g),
 * in 0..255 intensity units.  Left pixel (px, py) is matched with right pixel
 * (px - x, py); reading: a column left of the image is clamped to column 0.
 * This is the definition, evaluated in FP64.                                 */
double orc_cost_m(const int32_t* L, const int32_t* gL, const int32_t* R, const int32_t* gR,
                  int W, int level, int px, int py, int x,
                  double alpha, double tau_c, double tau_g)
{
    int xr = px - x;
    if (xr < 0) xr = 0;
    const int32_t* a = L + 3 * ((int64_t)py * W + px);
    const int32_t* b = R + 3 * ((int64_t)py * W + xr);
    double sc = (double)scale4(level);
    double dc = (fabs((double)a[0] - b[0]) + fabs((double)a[1] - b[1]) + fabs((double)a[2] - b[2])) / (3.0 * sc);
    double dg = fabs((double)gL[(int64_t)py * W + px] - (double)gR[(int64_t)py * W + xr]) / (6.0 * sc);
    return (1.0 - alpha) * fmin(dc, tau_c) + alpha * fmin(dg, tau_g);
}

/* The dense cost volume E[p][x] = M(p, x) of one layer, every pixel p
 * (row-major) and label x in 0..X-1: orc_cost_m at each entry.  The
 * differentiable path evaluates it for real-valued alpha, tau_c, tau_g.     */
int orc_cost_volume(const int32_t* L, const int32_t* gL, const int32_t* R, const int32_t* gR,
                    int W, int H, int level, int X, double alpha, double tau_c, double tau_g, double* E)
{
    for (int py = 0; py < H; ++py)
        for (int px = 0; px < W; ++px)
            for (int x = 0; x < X; ++x)
                E[((int64_t)py * W + px) * X + x] = orc_cost_m(L, gL, R, gR, W, level, px, py, x, alpha, tau_c, tau_g);
    return 0;
}

/* The same cost written as an exact integer: with a20 = 20*alpha,
 * tc3 = 3*tau_c and tg6 = 6*tau_g integers,
 *   120 * 4^l * M = 2*(20 - a20) * min(sum_c |dI_c|, tc3*4^l) + a20 * min(|dg|, tg6*4^l).
 * Used wherever the cost decides an integer (argmin for the prior), so both
 * implementations take that decision exactly.                               */
int64_t orc_cost_mq(const int32_t* L, const int32_t* gL, const int32_t* R, const int32_t* gR,
                    int W, int level, int px, int py, int x, int a20, int tc3, int tg6)
{
    int xr = px - x;
    if (xr < 0) xr = 0;
    const int32_t* a = L + 3 * ((int64_t)py * W + px);
    const int32_t* b = R + 3 * ((int64_t)py * W + xr);
    int64_t sc = scale4(level);
    int64_t sum = labs64((int64_t)a[0] - b[0]) + labs64((int64_t)a[1] - b[1]) + labs64((int64_t)a[2] - b[2]);
    int64_t dg = labs64((int64_t)gL[(int64_t)py * W + px] - gR[(int64_t)py * W + xr]);
    return 2 * (int64_t)(20 - a20) * lmin(sum, tc3 * sc) + (int64_t)a20 * lmin(dg, tg6 * sc);
}

/* Right-view cost used by the left-right consistency check: right pixel
 * (u, v) matched with left pixel (u + x, v), clamped to the last column.      */
static int64_t cost_mq_right(const int32_t* L, const int32_t* gL, const int32_t* R, const int32_t* gR,
                             int W, int level, int u, int v, int x, int a20, int tc3, int tg6)
{
    int xl = u + x;
    if (xl > W - 1) xl = W - 1;
    const int32_t* a = R + 3 * ((int64_t)v * W + u);
    const int32_t* b = L + 3 * ((int64_t)v * W + xl);
    int64_t sc = scale4(level);
    int64_t sum = labs64((int64_t)a[0] - b[0]) + labs64((int64_t)a[1] - b[1]) + labs64((int64_t)a[2] - b[2]);
    int64_t dg = labs64((int64_t)gR[(int64_t)v * W + u] - gL[(int64_t)v * W + xl]);
    return 2 * (int64_t)(20 - a20) * lmin(sum, tc3 * sc) + (int64_t)a20 * lmin(dg, tg6 * sc);
}

/* ------------------------------------------------------------------------ */
/* M+* variants (Sec. 4.1): the cited MST and ST methods median-filter the
 * image before building their trees; the paper removes that filter and
 * names the versions that keep it M+*.  Reading: a 3 x 3 median per colour
 * channel (border pixels replicated) of the layer's image, used for the edge
 * weights (Eq. weight) only; the matching cost keeps the unfiltered images.
 * The median of the nine values is the fifth smallest.                     */
static int cmp_i32(const void* A, const void* B)
{
    int32_t a = *(const int32_t*)A, b = *(const int32_t*)B;
    return (a > b) - (a < b);
}

int orc_median3(const int32_t* img, int W, int H, int32_t* out)
{
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x)
            for (int c = 0; c < 3; ++c) {
                int32_t v[9];
                int n = 0;
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        int yy = imin(imax(y + dy, 0), H - 1), xx = imin(imax(x + dx, 0), W - 1);
                        v[n++] = img[3 * ((size_t)yy * W + xx) + c];
                    }
                qsort(v, 9, sizeof(int32_t), cmp_i32);
                out[3 * ((size_t)y * W + x) + c] = v[4];
            }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Eq. (weight): w(p, q) = |I(p) - I(q)| on the 4-connected grid.  Reading for
 * colour images: the largest per-channel absolute difference, as in the
 * cited MST method.  Edge id e = 2*(y*W + x) + o: o = 0 joins (x, y) and
 * (x+1, y); o = 1 joins (x, y) and (x, y+1).  w[e] = -1 for ids that leave the
 * image.  Weights stay at scale 4^l (integers).                              */
int orc_edge_weights(const int32_t* img, int W, int H, int64_t* w)
{
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int64_t p = (int64_t)y * W + x;
            for (int o = 0; o < 2; ++o) {
                int qx = x + (o == 0), qy = y + (o == 1);
                if (qx >= W || qy >= H) { w[2 * p + o] = -1; continue; }
                int64_t q = (int64_t)qy * W + qx;
                int64_t m = 0;
                for (int c = 0; c < 3; ++c) {
                    int64_t dlt = labs64((int64_t)img[3 * p + c] - img[3 * q + c]);
                    if (dlt > m) m = dlt;
                }
                w[2 * p + o] = m;
            }
        }
    return 0;
}

static const int64_t* g_sort_w;
static int cmp_edge(const void* A, const void* B)
{
    int32_t a = *(const int32_t*)A, b = *(const int32_t*)B;
    if (g_sort_w[a] != g_sort_w[b]) return g_sort_w[a] < g_sort_w[b] ? -1 : 1;
    return (a > b) - (a < b);
}

/* Rule 1 of the spanning-tree algorithm (Sec. 3.2): edges are taken in order
 * of increasing weight; ties are broken by increasing edge id, which makes
 * the order strict and the minimum spanning tree unique.  Returns the number
 * of valid edges written to `order`.                                         */
int orc_sort_edges(const int64_t* w, int W, int H, int32_t* order)
{
    int n = 0;
    for (int64_t e = 0; e < 2 * (int64_t)W * H; ++e)
        if (w[e] >= 0) order[n++] = (int32_t)e;
    g_sort_w = w;
    qsort(order, (size_t)n, sizeof(int32_t), cmp_edge);
    return n;
}

/* Random spanning tree, RT (Sec. 4.1): the edges are shuffled at random and
 * the same union-find construction takes them in that order.  Reading: the
 * shuffle is the order of a counter-based random key per edge, ties (equal
 * keys) broken by edge id.  The key of edge e at layer l is the top 31 bits
 * of the i-th output of SplitMix64 started from state `seed`, with
 * i = l * 2^32 + e + 1; SplitMix64 is the generator of Steele, Lea and Flood,
 * "Fast splittable pseudorandom number generators" (OOPSLA 2014): the state
 * advances by the odd constant 0x9E3779B97F4A7C15 and each output is the
 * state passed through two xor-shift-multiply rounds and a final xor-shift.  */
uint64_t orc_splitmix64(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + i * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static uint32_t rt_key(uint64_t seed, int level, int64_t e)
{
    return (uint32_t)(orc_splitmix64(seed, ((uint64_t)level << 32) + (uint64_t)e + 1u) >> 33);
}

static const uint32_t* g_rt_key;
static int cmp_rt(const void* A, const void* B)
{
    int32_t a = *(const int32_t*)A, b = *(const int32_t*)B;
    if (g_rt_key[a] != g_rt_key[b]) return g_rt_key[a] < g_rt_key[b] ? -1 : 1;
    return (a > b) - (a < b);
}

/* Rule 1 of the random tree: every valid edge in increasing (key, id) order;
 * returns the number written to `order` (key: scratch of 2*W*H words). */
int orc_sort_edges_rt(const int64_t* w, int W, int H, uint64_t seed, int level, int32_t* order)
{
    const int64_t n2 = 2 * (int64_t)W * H;
    uint32_t* key = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n2 > 0 ? n2 : 1));
    if (!key) return -1;
    int n = 0;
    for (int64_t e = 0; e < n2; ++e) {
        key[e] = rt_key(seed, level, e);
        if (w[e] >= 0) order[n++] = (int32_t)e;
    }
    g_rt_key = key;
    qsort(order, (size_t)n, sizeof(int32_t), cmp_rt);
    free(key);
    return n;
}

/* ------------------------------------------------------------------------ */
/* Sets of disparity labels (PixelIntv / TreeIntv, Sec. 3.1-3.2) as 256-bit
 * masks; |.| is the number of labels in the set.                            */
static int set_count(const uint32_t* a)
{
    int n = 0;
    for (int i = 0; i < ORC_WORDS; ++i) n += __builtin_popcount(a[i]);
    return n;
}
static int set_count_and(const uint32_t* a, const uint32_t* b)
{
    int n = 0;
    for (int i = 0; i < ORC_WORDS; ++i) n += __builtin_popcount(a[i] & b[i]);
    return n;
}
static int set_count_or(const uint32_t* a, const uint32_t* b)
{
    int n = 0;
    for (int i = 0; i < ORC_WORDS; ++i) n += __builtin_popcount(a[i] | b[i]);
    return n;
}

static int32_t uf_find(int32_t* parent, int32_t v)
{
    int32_t r = v;
    while (parent[r] != r) r = parent[r];
    while (parent[v] != r) { int32_t n = parent[v]; parent[v] = r; v = n; }
    return r;
}

/* Sec. 3.2, HDP forest construction, plus the plain MST and the segment tree
 * (ST) it is combined with.  Sequential Kruskal over the strict (w, e) order:
 *   - DT-Rule 1 (Eq. cri1): an edge whose end points have disjoint PixelIntv
 *     is discarded;
 *   - Rule 2: the two ends must lie in different trees;
 *   - DT-Rule 2 (Eq. DTrules): |T_p & T_q| / |T_p | T_q| >= beta, evaluated
 *     exactly as |T_p & T_q| * beta_den >= beta_num * |T_p | T_q|;
 *   - on a merge, TreeIntv becomes the union of the two sets.
 * tree_type 0: MST.  tree_type 1: ST, read from the cited segment-tree method
 * (the paper only cites it): a first Kruskal pass merges two trees only if
 * additionally w <= Int(C) + k/|C| for both (Int = largest merged weight,
 * |C| = pixel count; evaluated as w*|C| <= Int*|C| + k*4^l), then a second
 * pass over the same order links what is left under the other rules.
 * With every set equal to the full range, DT-Rules 1 and 2 always hold and
 * this is the ordinary MST / ST.
 * Outputs: in_tree[e] = 1 for accepted edges; dt_root[p] = smallest pixel id
 * of p's tree; tree_intv[p] = TreeIntv of p's tree (8 words per pixel).      */
int orc_build_forest(int W, int H, const int32_t* order, int n_order, const int64_t* w,
                     const uint32_t* pix_intv, int beta_num, int beta_den,
                     int tree_type, int64_t st_k, int level,
                     uint8_t* in_tree, int32_t* dt_root, uint32_t* tree_intv)
{
    int64_t N = (int64_t)W * H;
    int32_t* parent = (int32_t*)malloc(sizeof(int32_t) * N);
    int32_t* rnk = (int32_t*)calloc((size_t)N, sizeof(int32_t));
    int64_t* size = (int64_t*)malloc(sizeof(int64_t) * N);
    int64_t* intw = (int64_t*)calloc((size_t)N, sizeof(int64_t));
    uint32_t* T = (uint32_t*)malloc(sizeof(uint32_t) * ORC_WORDS * N);
    if (!parent || !rnk || !size || !intw || !T) return -1;
    for (int64_t p = 0; p < N; ++p) { parent[p] = (int32_t)p; size[p] = 1; }
    memcpy(T, pix_intv, sizeof(uint32_t) * ORC_WORDS * N);
    memset(in_tree, 0, (size_t)(2 * N));
    int64_t kq = st_k * scale4(level);

    int passes = tree_type == 1 ? 2 : 1;
    for (int pass = 0; pass < passes; ++pass) {
        int criterion = (tree_type == 1 && pass == 0);
        for (int i = 0; i < n_order; ++i) {
            int32_t e = order[i];
            int32_t p = e >> 1;
            int32_t q = (e & 1) ? p + W : p + 1;
            /* DT-Rule 1 on the pixel-wise sets */
            if (set_count_and(pix_intv + ORC_WORDS * (int64_t)p, pix_intv + ORC_WORDS * (int64_t)q) == 0) continue;
            int32_t a = uf_find(parent, p), b = uf_find(parent, q);
            if (a == b) continue;                       /* Rule 2 */
            const uint32_t* Ta = T + ORC_WORDS * (int64_t)a;
            const uint32_t* Tb = T + ORC_WORDS * (int64_t)b;
            int64_t inter = set_count_and(Ta, Tb), uni = set_count_or(Ta, Tb);
            if (inter * beta_den < (int64_t)beta_num * uni) continue;   /* DT-Rule 2 */
            if (criterion) {
                int64_t wq = w[e];
                if (wq * size[a] > intw[a] * size[a] + kq) continue;
                if (wq * size[b] > intw[b] * size[b] + kq) continue;
            }
            /* merge: union by rank, TreeIntv union, ST bookkeeping */
            if (rnk[a] < rnk[b]) { int32_t t = a; a = b; b = t; }
            parent[b] = a;
            if (rnk[a] == rnk[b]) rnk[a]++;
            for (int k = 0; k < ORC_WORDS; ++k) T[ORC_WORDS * (int64_t)a + k] |= T[ORC_WORDS * (int64_t)b + k];
            size[a] += size[b];
            intw[a] = w[e];   /* edges arrive in increasing weight */
            in_tree[e] = 1;
        }
    }
    /* root of each tree: its smallest pixel id */
    int32_t* minid = (int32_t*)malloc(sizeof(int32_t) * N);
    for (int64_t p = 0; p < N; ++p) minid[p] = INT32_MAX;
    for (int64_t p = 0; p < N; ++p) {
        int32_t r = uf_find(parent, (int32_t)p);
        if ((int32_t)p < minid[r]) minid[r] = (int32_t)p;
    }
    for (int64_t p = 0; p < N; ++p) {
        int32_t r = uf_find(parent, (int32_t)p);
        dt_root[p] = minid[r];
        memcpy(tree_intv + ORC_WORDS * p, T + ORC_WORDS * (int64_t)r, sizeof(uint32_t) * ORC_WORDS);
    }
    free(minid); free(parent); free(rnk); free(size); free(intw); free(T);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Root and breadth-first order of the forest.  The aggregated cost (Eq. C)
 * does not depend on the root, so the choice only fixes an order.  Reading:
 * each tree is rooted at its smallest pixel id; the order lists all roots by
 * increasing id, then depth by depth, a node's children by increasing id
 * after the children of the nodes before it.  parent[root] = -1.            */
int orc_bfs(int W, int H, const uint8_t* in_tree, int32_t* order, int32_t* parent, int32_t* depth)
{
    int64_t N = (int64_t)W * H;
    uint8_t* seen = (uint8_t*)calloc((size_t)N, 1);
    int32_t* stack = (int32_t*)malloc(sizeof(int32_t) * N);
    if (!seen || !stack) return -1;
    int64_t head = 0, tail = 0;
    /* roots: the first pixel met (in increasing id) of each tree */
    for (int64_t s = 0; s < N; ++s) {
        if (seen[s]) continue;
        order[tail++] = (int32_t)s;
        parent[s] = -1;
        depth[s] = 0;
        int64_t sp = 0;
        stack[sp++] = (int32_t)s;
        seen[s] = 1;
        while (sp) {   /* mark the whole tree */
            int32_t v = stack[--sp];
            int x = v % W, y = v / W;
            int32_t nb[4]; int ok[4];
            nb[0] = v - W; ok[0] = y > 0 && in_tree[2 * (int64_t)(v - W) + 1];
            nb[1] = v - 1; ok[1] = x > 0 && in_tree[2 * (int64_t)(v - 1)];
            nb[2] = v + 1; ok[2] = x + 1 < W && in_tree[2 * (int64_t)v];
            nb[3] = v + W; ok[3] = y + 1 < H && in_tree[2 * (int64_t)v + 1];
            for (int k = 0; k < 4; ++k)
                if (ok[k] && !seen[nb[k]]) { seen[nb[k]] = 1; stack[sp++] = nb[k]; }
        }
    }
    memset(seen, 0, (size_t)N);
    for (int64_t i = 0; i < tail; ++i) seen[order[i]] = 1;
    while (head < tail) {
        int32_t v = order[head++];
        int x = v % W, y = v / W;
        /* neighbours in increasing id: up, left, right, down */
        int32_t nb[4]; int ok[4];
        nb[0] = v - W; ok[0] = y > 0 && in_tree[2 * (int64_t)(v - W) + 1];
        nb[1] = v - 1; ok[1] = x > 0 && in_tree[2 * (int64_t)(v - 1)];
        nb[2] = v + 1; ok[2] = x + 1 < W && in_tree[2 * (int64_t)v];
        nb[3] = v + W; ok[3] = y + 1 < H && in_tree[2 * (int64_t)v + 1];
        for (int k = 0; k < 4; ++k)
            if (ok[k] && !seen[nb[k]]) {
                seen[nb[k]] = 1;
                parent[nb[k]] = v;
                depth[nb[k]] = depth[v] + 1;
                order[tail++] = nb[k];
            }
    }
    free(seen); free(stack);
    return tail == N ? 0 : -2;
}

/* ------------------------------------------------------------------------ */
static int set_has(const uint32_t* a, int x) { return (a[x >> 5] >> (x & 31)) & 1u; }

/* Sec. 3.3, aggregation over the forest (Eqs. E, W, S, C) and WTA.
 *   E(p, x) = M(p, x) for x in TreeIntv(DT(p)), undefined otherwise;
 *   S(p, q) = exp(-W(p, q) / gamma), W = sum of edge weights on the tree path;
 *   C(p, x) = sum over q in DT(p) of S(p, q) E(q, x).
 * Computed with the linear-time two-pass method of the cited MST paper:
 * leaf-to-root  U(v) = E(v) + sum_children s_c U(c),
 * root-to-leaf  C(v) = s_v C(parent) + (1 - s_v^2) U(v),  C(root) = U(root),
 * with s_v = exp(-w(v, parent) / gamma), one disparity at a time.
 * Weights are real units (w / 4^l).  Outputs (any may be NULL):
 *   C_out[row_off[p] + slot] for pixel p and its slot-th label in ascending order;
 *   wta[p] = argmin over its labels, ties to the lowest label;
 *   best[p], second[p] = smallest and second-smallest aggregated cost.      */
int orc_aggregate(int W, int H, int level, int d_l,
                  const int32_t* L, const int32_t* gL, const int32_t* R, const int32_t* gR,
                  double alpha, double tau_c, double tau_g, double gamma,
                  const int32_t* order, const int32_t* parent, const int64_t* w,
                  const uint32_t* tree_intv, const int64_t* row_off,
                  double* C_out, int32_t* wta, double* best, double* second)
{
    int64_t N = (int64_t)W * H;
    double* s = (double*)malloc(sizeof(double) * N);
    double* U = (double*)malloc(sizeof(double) * N);
    double* C = (double*)malloc(sizeof(double) * N);
    double* b1 = (double*)malloc(sizeof(double) * N);
    double* b2 = (double*)malloc(sizeof(double) * N);
    int32_t* arg = (int32_t*)malloc(sizeof(int32_t) * N);
    int32_t* slot = (int32_t*)calloc((size_t)N, sizeof(int32_t));
    if (!s || !U || !C || !b1 || !b2 || !arg || !slot) return -1;
    double sc = (double)scale4(level);
    for (int64_t v = 0; v < N; ++v) {
        int32_t p = parent[v];
        s[v] = 0.0;
        if (p >= 0) {
            int64_t e;
            if (p == v - 1) e = 2 * (int64_t)p;
            else if (p == v + 1) e = 2 * v;
            else if (p == v - W) e = 2 * (int64_t)p + 1;
            else e = 2 * v + 1;
            s[v] = exp(-((double)w[e] / sc) / gamma);
        }
        b1[v] = INFINITY; b2[v] = INFINITY; arg[v] = -1;
    }
    for (int x = 0; x <= d_l; ++x) {
        for (int64_t v = 0; v < N; ++v)
            U[v] = set_has(tree_intv + ORC_WORDS * v, x)
                       ? orc_cost_m(L, gL, R, gR, W, level, (int)(v % W), (int)(v / W), x, alpha, tau_c, tau_g)
                       : 0.0;
        for (int64_t i = N - 1; i >= 0; --i) {      /* leaf to root */
            int32_t v = order[i];
            if (parent[v] >= 0 && set_has(tree_intv + ORC_WORDS * (int64_t)v, x))
                U[parent[v]] += s[v] * U[v];
        }
        for (int64_t i = 0; i < N; ++i) {           /* root to leaf */
            int32_t v = order[i];
            if (!set_has(tree_intv + ORC_WORDS * (int64_t)v, x)) continue;
            C[v] = parent[v] < 0 ? U[v] : s[v] * C[parent[v]] + (1.0 - s[v] * s[v]) * U[v];
        }
        for (int64_t v = 0; v < N; ++v) {
            if (!set_has(tree_intv + ORC_WORDS * v, x)) continue;
            if (C_out) C_out[row_off[v] + slot[v]] = C[v];
            slot[v]++;
            if (C[v] < b1[v]) { b2[v] = b1[v]; b1[v] = C[v]; arg[v] = x; }
            else if (C[v] < b2[v]) b2[v] = C[v];
        }
    }
    for (int64_t v = 0; v < N; ++v) {
        if (wta) wta[v] = arg[v];
        if (best) best[v] = b1[v];
        if (second) second[v] = b2[v];
    }
    free(s); free(U); free(C); free(b1); free(b2); free(arg); free(slot);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.1, prior P(D_l) by sampling.  G_l is cut into 5x5 squares; a
 * disparity is computed at each square's centre and kept if it passes a
 * left-right consistency check.  The paper defers the disparity method to a
 * citation without details; reading: the centre's disparity is the argmin of
 * the 5x5 box sum of the integer cost (ties to the lowest label), computed
 * for the left view at (cx, cy) and for the right view at (cx - dL, cy) (box
 * pixels clamped to the image); the centre is stable iff both agree and
 * cx - dL >= 0.  prior[j] = (number of stable centres with disparity j) + 1,
 * the +1 being a Laplace count so that no label has zero prior.             */
int orc_prior(const int32_t* L, const int32_t* gL, const int32_t* R, const int32_t* gR,
              int W, int H, int level, int d_l, int a20, int tc3, int tg6, int64_t* prior,
              int32_t* centres /* optional: per centre (b, a) row-major: dL, dR (-1 if no right match) */)
{
    for (int j = 0; j <= d_l; ++j) prior[j] = 1;
    for (int b = 0; b < H / 5; ++b)
        for (int a = 0; a < W / 5; ++a) {
            int cx = 5 * a + 2, cy = 5 * b + 2;
            int64_t bestL = INT64_MAX;
            int dL = 0;
            for (int x = 0; x <= d_l; ++x) {
                int64_t t = 0;
                for (int dy = -2; dy <= 2; ++dy)
                    for (int dx = -2; dx <= 2; ++dx)
                        t += orc_cost_mq(L, gL, R, gR, W, level, cx + dx, cy + dy, x, a20, tc3, tg6);
                if (t < bestL) { bestL = t; dL = x; }
            }
            int u = cx - dL;
            if (centres) { centres[2 * ((int64_t)b * (W / 5) + a)] = dL; centres[2 * ((int64_t)b * (W / 5) + a) + 1] = -1; }
            if (u < 0) continue;
            int64_t bestR = INT64_MAX;
            int dR = 0;
            for (int x = 0; x <= d_l; ++x) {
                int64_t t = 0;
                for (int dy = -2; dy <= 2; ++dy)
                    for (int dx = -2; dx <= 2; ++dx) {
                        int uu = u + dx;
                        if (uu < 0) uu = 0;
                        if (uu > W - 1) uu = W - 1;
                        t += cost_mq_right(L, gL, R, gR, W, level, uu, cy + dy, x, a20, tc3, tg6);
                    }
                if (t < bestR) { bestR = t; dR = x; }
            }
            if (centres) centres[2 * ((int64_t)b * (W / 5) + a) + 1] = dR;
            if (dR == dL) prior[dL] += 1;
        }
    return 0;
}

/* Sec. 2.2 + Sec. 3.1, pixel-wise interval prediction.
 * Likelihood P(D_{l+1} = i | D_l = j) = GMM_l(i - floor(j/2)), the mixture
 * density sum_k pi_k N(o | mu_k, sd_k) at the integer offset o (reading: the
 * density, not a bin integral).  Posterior row i (Eq. dpm) is proportional to
 * GMM_l(i - floor(j/2)) * prior[j]; the row normalisation does not change the
 * argmax or the ratio test, so it is left out.
 * Eq. crtr: start from the argmax of row i (ties to the lowest j), then take
 * the remaining labels by decreasing posterior (ties to the lower j) and add
 * j while P_j / (c + P_j) >= delta, written P_j * (1 - delta) >= delta * c,
 * c = sum of the posteriors already taken; stop at the first failure (the
 * ratio can only fall afterwards).  A row that is all zero (underflow) falls
 * back to {2i, 2i+1} clipped to [0, d_l].
 * masks: (d_up + 1) rows of 8 words.                                        */
typedef struct { double p; int j; } orc_pj;
static int cmp_pj(const void* A, const void* B)
{
    const orc_pj* a = (const orc_pj*)A;
    const orc_pj* b = (const orc_pj*)B;
    if (a->p != b->p) return a->p > b->p ? -1 : 1;
    return (a->j > b->j) - (a->j < b->j);
}

double orc_gmm_density(int K, const double* gmm, double o)
{
    const double inv_sqrt_2pi = 0.39894228040143267794;
    double acc = 0.0;
    for (int k = 0; k < K; ++k) {
        double pi = gmm[3 * k], mu = gmm[3 * k + 1], sd = gmm[3 * k + 2];
        double z = (o - mu) / sd;
        acc += pi * (inv_sqrt_2pi / sd) * exp(-0.5 * z * z);
    }
    return acc;
}

int orc_range_table(const int64_t* prior, int d_l, int d_up, int K, const double* gmm,
                    double delta, uint32_t* masks, double* post_out)
{
    orc_pj* row = (orc_pj*)malloc(sizeof(orc_pj) * (size_t)(d_l + 1));
    if (!row) return -1;
    memset(masks, 0, sizeof(uint32_t) * ORC_WORDS * (size_t)(d_up + 1));
    for (int i = 0; i <= d_up; ++i) {
        uint32_t* m = masks + ORC_WORDS * (size_t)i;
        double mx = 0.0;
        for (int j = 0; j <= d_l; ++j) {
            double p = orc_gmm_density(K, gmm, (double)(i - j / 2)) * (double)prior[j];
            row[j].p = p;
            row[j].j = j;
            if (post_out) post_out[(size_t)i * (d_l + 1) + j] = p;
            if (p > mx) mx = p;
        }
        if (!(mx > 0.0)) {
            for (int j = 2 * i; j <= 2 * i + 1 && j <= d_l; ++j) m[j >> 5] |= 1u << (j & 31);
            continue;
        }
        qsort(row, (size_t)(d_l + 1), sizeof(orc_pj), cmp_pj);
        double c = row[0].p;
        m[row[0].j >> 5] |= 1u << (row[0].j & 31);
        for (int t = 1; t <= d_l; ++t) {
            if (row[t].p * (1.0 - delta) >= delta * c) {
                c += row[t].p;
                m[row[t].j >> 5] |= 1u << (row[t].j & 31);
            } else {
                break;
            }
        }
    }
    free(row);
    return 0;
}

/* PixelIntv of every pixel of layer l from the disparities of layer l+1:
 * pixel (x, y) takes row D_{l+1}(floor(x/2), floor(y/2)) of the table.       */
int orc_pixel_intervals(int W, int H, const int32_t* d_up_map, int W_up,
                        const uint32_t* masks, uint32_t* pix_intv)
{
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int32_t i = d_up_map[(int64_t)(y / 2) * W_up + x / 2];
            memcpy(pix_intv + ORC_WORDS * ((int64_t)y * W + x), masks + ORC_WORDS * (int64_t)i,
                   sizeof(uint32_t) * ORC_WORDS);
        }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Eq. C for a given cost volume: C(p, x) = sum_q S(p, q) E(q, x) over the tree
 * of p, S = exp(-W/gamma), with the two-pass recurrences, every label defined.
 * s[v] = exp(-w(v, parent)/gamma) (0 for roots); E, C: [N][X].  Eup (optional)
 * receives the leaf-to-root pass U.                                         */
int orc_aggregate_given(int64_t N, int X, const int32_t* order, const int32_t* parent, const double* s,
                        const double* E, double* C, double* Eup)
{
    double* U = (double*)malloc(sizeof(double) * (size_t)N * X);
    if (!U) return -1;
    memcpy(U, E, sizeof(double) * (size_t)N * X);
    for (int64_t i = N - 1; i >= 0; --i) {
        int32_t v = order[i], p = parent[v];
        if (p < 0) continue;
        for (int x = 0; x < X; ++x) U[(size_t)p * X + x] += s[v] * U[(size_t)v * X + x];
    }
    for (int64_t i = 0; i < N; ++i) {
        int32_t v = order[i], p = parent[v];
        for (int x = 0; x < X; ++x)
            C[(size_t)v * X + x] = p < 0 ? U[(size_t)v * X + x]
                                         : s[v] * C[(size_t)p * X + x] + (1.0 - s[v] * s[v]) * U[(size_t)v * X + x];
    }
    if (Eup) memcpy(Eup, U, sizeof(double) * (size_t)N * X);
    free(U);
    return 0;
}

/* Adjoint of Eq. C with respect to the cost volume, the tree edge weights and
 * gamma, for L with g = dL/dC.  A(p, q) = exp(-W(p, q)/gamma) is symmetric, so
 * dL/dE = A g.  Tree edge e = (c, pi): the pairs whose path crosses e have one
 * end in the subtree of c; with up-pass values E^, g^ and full aggregates C, G,
 *   dL/dw_e = -(s_e/gamma) sum_x [ g^(c)(C(pi) - s_e E^(c)) + E^(c)(G(pi) - s_e g^(c)) ],
 *   dL/dgamma = -(1/gamma) sum_e w_e dL/dw_e   (W is linear in the weights).
 * w[v]: weight of the edge from v to its parent (real units; unused for roots).
 * Outputs gE [N][X], gw[v] per node (0 for roots), *ggamma.                  */
int orc_aggregate_adjoint(int64_t N, int X, const int32_t* order, const int32_t* parent, const double* w,
                          double gamma, const double* E, const double* g, double* gE, double* gw, double* ggamma)
{
    double* s = (double*)malloc(sizeof(double) * N);
    double* Eu = (double*)malloc(sizeof(double) * (size_t)N * X);
    double* Cf = (double*)malloc(sizeof(double) * (size_t)N * X);
    double* gu = (double*)malloc(sizeof(double) * (size_t)N * X);
    if (!s || !Eu || !Cf || !gu) return -1;
    for (int64_t v = 0; v < N; ++v) s[v] = parent[v] < 0 ? 0.0 : exp(-w[v] / gamma);
    orc_aggregate_given(N, X, order, parent, s, E, Cf, Eu);
    orc_aggregate_given(N, X, order, parent, s, g, gE, gu);
    double acc = 0.0;
    for (int64_t c = 0; c < N; ++c) {
        int32_t p = parent[c];
        gw[c] = 0.0;
        if (p < 0) continue;
        double t = 0.0;
        for (int x = 0; x < X; ++x) {
            size_t ic = (size_t)c * X + x, ip = (size_t)p * X + x;
            t += gu[ic] * (Cf[ip] - s[c] * Eu[ic]) + Eu[ic] * (gE[ip] - s[c] * gu[ic]);
        }
        gw[c] = -(s[c] / gamma) * t;
        acc += w[c] * gw[c];
    }
    *ggamma = -acc / gamma;
    free(s); free(Eu); free(Cf); free(gu);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* GMM_l by EM (Sec. 2.2).  The paper models the offset
 * o = D_{l+1} - floor(D_l / S) of a superpixel's disparity from the mode
 * given by each of its children, collects o over training pairs with ground
 * truth, and fits a Gaussian mixture to its distribution by EM.
 *
 * Ground truth per layer (reading; the paper does not say how the coarse
 * ground truth is formed): a map of integer labels, -1 where invalid
 * (occluded).  The superpixel of a square takes the mean of its valid
 * children divided by S = 2, rounded half up: floor((sum + n) / (2 n)) for n
 * valid children; no valid child gives -1.                                  */
int orc_gt_down(const int32_t* gt, int W, int H, int32_t* up)
{
    int Wu = (W + 1) / 2, Hu = (H + 1) / 2;
    for (int Y = 0; Y < Hu; ++Y)
        for (int X = 0; X < Wu; ++X) {
            int64_t sum = 0, n = 0;
            for (int dy = 0; dy < 2; ++dy)
                for (int dx = 0; dx < 2; ++dx) {
                    int x = 2 * X + dx, y = 2 * Y + dy;
                    if (x >= W || y >= H) continue;
                    int32_t v = gt[(size_t)y * W + x];
                    if (v < 0) continue;
                    sum += v;
                    n += 1;
                }
            up[(size_t)Y * Wu + X] = n ? (int32_t)((sum + n) / (2 * n)) : -1;
        }
    return 0;
}

/* Histogram of o = up(floor(x/2), floor(y/2)) - floor(lo(x, y) / 2) over the
 * pixels of layer l whose own and superpixel's labels are valid; bin
 * o + range for |o| <= range (other offsets are not counted).  Adds to hist. */
int orc_offset_hist(const int32_t* up, int Wu, const int32_t* lo, int W, int H, int range, int64_t* hist)
{
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int32_t a = lo[(size_t)y * W + x], b = up[(size_t)(y / 2) * Wu + x / 2];
            if (a < 0 || b < 0) continue;
            int o = b - a / 2;
            if (o < -range || o > range) continue;
            hist[o + range] += 1;
        }
    return 0;
}

/* EM for a K-component 1-D Gaussian mixture on histogram data: h[b] points
 * at o = b - range.  Standard EM (the GMM of Sec. 2.2, trained by the EM of
 * its citation):
 *   E-step  r_k(o) = pi_k N(o; mu_k, sd_k) / sum_j pi_j N(o; mu_j, sd_j)
 *   M-step  n_k = sum_o h(o) r_k(o);  pi_k = n_k / sum h;
 *           mu_k = sum_o h r_k o / n_k;  sd_k^2 = sum_o h r_k (o - mu_k)^2 / n_k
 * Readings: the data are integers, so a component could collapse onto one
 * value; sd_k is floored at sd_min (the constrained maximiser of the
 * M-step, so the likelihood still never decreases).  Start: every mu_k at
 * the data mean m, sd_k = max(s, sd_min) * 4^(k - (K-1)/2) with s the data's
 * standard deviation (a narrow core and wider tails), pi_k = 1/K.  A
 * component that loses all its points (n_k = 0) keeps its parameters with
 * pi_k = 0.  The responsibilities are evaluated in the log domain.  Runs
 * `iters` iterations; out: K rows of (pi, mu, sd); ll (optional, iters + 1
 * entries): the log-likelihood sum_o h(o) log sum_k pi_k N(o; mu_k, sd_k)
 * before the first and after every iteration.                           */
static double em_loglik(const int64_t* h, int range, int K, const double* g)
{
    double ll = 0.0;
    for (int b = 0; b <= 2 * range; ++b) {
        if (!h[b]) continue;
        double o = (double)(b - range), lmax = -INFINITY, acc = 0.0;
        double lp[64];
        for (int k = 0; k < K && k < 64; ++k) {
            double z = (o - g[3 * k + 1]) / g[3 * k + 2];
            lp[k] = g[3 * k] > 0.0 ? log(g[3 * k]) - log(g[3 * k + 2]) - 0.5 * z * z : -INFINITY;
            if (lp[k] > lmax) lmax = lp[k];
        }
        for (int k = 0; k < K && k < 64; ++k) acc += exp(lp[k] - lmax);
        ll += (double)h[b] * (lmax + log(acc) - 0.91893853320467274178);   /* - log sqrt(2 pi) */
    }
    return ll;
}

int orc_gmm_em(const int64_t* h, int range, int K, int iters, double sd_min, double* out, double* ll)
{
    const int nb = 2 * range + 1;
    double tot = 0.0, m = 0.0, s2 = 0.0;
    for (int b = 0; b < nb; ++b) { tot += (double)h[b]; m += (double)h[b] * (double)(b - range); }
    if (tot <= 0.0 || K < 1 || K > 64) return -1;
    m /= tot;
    for (int b = 0; b < nb; ++b) s2 += (double)h[b] * ((double)(b - range) - m) * ((double)(b - range) - m);
    double s = sqrt(s2 / tot);
    if (s < sd_min) s = sd_min;
    for (int k = 0; k < K; ++k) {
        out[3 * k] = 1.0 / K;
        out[3 * k + 1] = m;
        out[3 * k + 2] = s * pow(4.0, (double)k - 0.5 * (K - 1));
        if (out[3 * k + 2] < sd_min) out[3 * k + 2] = sd_min;
    }
    double* r = (double*)malloc(sizeof(double) * (size_t)nb * K);
    if (!r) return -1;
    if (ll) ll[0] = em_loglik(h, range, K, out);
    for (int it = 0; it < iters; ++it) {
        /* E-step */
        for (int b = 0; b < nb; ++b) {
            double o = (double)(b - range), lmax = -INFINITY;
            for (int k = 0; k < K; ++k) {
                double pi = out[3 * k], mu = out[3 * k + 1], sd = out[3 * k + 2];
                double z = (o - mu) / sd;
                double lp = pi > 0.0 ? log(pi) - log(sd) - 0.5 * z * z : -INFINITY;
                r[(size_t)b * K + k] = lp;
                if (lp > lmax) lmax = lp;
            }
            double den = 0.0;
            for (int k = 0; k < K; ++k) den += exp(r[(size_t)b * K + k] - lmax);
            for (int k = 0; k < K; ++k) r[(size_t)b * K + k] = exp(r[(size_t)b * K + k] - lmax) / den;
        }
        /* M-step: weights and means first, then spreads about the new means */
        for (int k = 0; k < K; ++k) {
            double nk = 0.0, sx = 0.0;
            for (int b = 0; b < nb; ++b) {
                double w = (double)h[b] * r[(size_t)b * K + k];
                nk += w;
                sx += w * (double)(b - range);
            }
            if (nk <= 0.0) { out[3 * k] = 0.0; continue; }
            double mu = sx / nk, sv = 0.0;
            for (int b = 0; b < nb; ++b) {
                double d = (double)(b - range) - mu;
                sv += (double)h[b] * r[(size_t)b * K + k] * d * d;
            }
            double sd = sqrt(sv / nk);
            out[3 * k] = nk / tot;
            out[3 * k + 1] = mu;
            out[3 * k + 2] = sd < sd_min ? sd_min : sd;
        }
        if (ll) ll[it + 1] = em_loglik(h, range, K, out);
    }
    free(r);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Tree-based refinement (Sec. 3.3, last paragraph: the refinement of the
 * cited MST/ST methods integrated at a layer).  Readings:
 *   - D_R, the disparity map of the right view, is the method run with the
 *     views' roles exchanged; a left pixel (x, y) with disparity D_L is
 *     stable iff x - D_L >= 0 and D_R(x - D_L, y) = D_L (left-right check);
 *     refD(p) = D_L(p) for a stable pixel, -1 otherwise.
 *   - The new cost is E'(p, x) = |x - D_L(p)| at a stable pixel and 0 at an
 *     unstable one, for x in TreeIntv(DT(p)); it is aggregated over the same
 *     forest (Eq. C, same two passes as orc_aggregate) and the refined map is
 *     its WTA (ties to the lowest label).                                     */
int orc_lr_check(const int32_t* DL, const int32_t* DR, int W, int H, int32_t* refD)
{
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int32_t d = DL[(size_t)y * W + x];
            int xr = x - d;
            refD[(size_t)y * W + x] = (xr >= 0 && DR[(size_t)y * W + xr] == d) ? d : -1;
        }
    return 0;
}

int orc_refine_aggregate(int W, int H, int level, int d_l, double gamma, const int32_t* order,
                         const int32_t* parent, const int64_t* w, const uint32_t* tree_intv, const int32_t* refD,
                         const int64_t* row_off, double* C_out, int32_t* wta, double* best, double* second)
{
    int64_t N = (int64_t)W * H;
    double* s = (double*)malloc(sizeof(double) * N);
    double* U = (double*)malloc(sizeof(double) * N);
    double* C = (double*)malloc(sizeof(double) * N);
    double* b1 = (double*)malloc(sizeof(double) * N);
    double* b2 = (double*)malloc(sizeof(double) * N);
    int32_t* arg = (int32_t*)malloc(sizeof(int32_t) * N);
    int32_t* slot = (int32_t*)calloc((size_t)N, sizeof(int32_t));
    if (!s || !U || !C || !b1 || !b2 || !arg || !slot) return -1;
    double sc = (double)scale4(level);
    for (int64_t v = 0; v < N; ++v) {
        int32_t p = parent[v];
        s[v] = 0.0;
        if (p >= 0) {
            int64_t e;
            if (p == v - 1) e = 2 * (int64_t)p;
            else if (p == v + 1) e = 2 * v;
            else if (p == v - W) e = 2 * (int64_t)p + 1;
            else e = 2 * v + 1;
            s[v] = exp(-((double)w[e] / sc) / gamma);
        }
        b1[v] = INFINITY; b2[v] = INFINITY; arg[v] = -1;
    }
    for (int x = 0; x <= d_l; ++x) {
        for (int64_t v = 0; v < N; ++v) {
            U[v] = 0.0;
            if (set_has(tree_intv + ORC_WORDS * v, x) && refD[v] >= 0) U[v] = fabs((double)(x - refD[v]));
        }
        for (int64_t i = N - 1; i >= 0; --i) {      /* leaf to root */
            int32_t v = order[i];
            if (parent[v] >= 0 && set_has(tree_intv + ORC_WORDS * (int64_t)v, x))
                U[parent[v]] += s[v] * U[v];
        }
        for (int64_t i = 0; i < N; ++i) {           /* root to leaf */
            int32_t v = order[i];
            if (!set_has(tree_intv + ORC_WORDS * (int64_t)v, x)) continue;
            C[v] = parent[v] < 0 ? U[v] : s[v] * C[parent[v]] + (1.0 - s[v] * s[v]) * U[v];
        }
        for (int64_t v = 0; v < N; ++v) {
            if (!set_has(tree_intv + ORC_WORDS * v, x)) continue;
            if (C_out) C_out[row_off[v] + slot[v]] = C[v];
            slot[v]++;
            if (C[v] < b1[v]) { b2[v] = b1[v]; b1[v] = C[v]; arg[v] = x; }
            else if (C[v] < b2[v]) b2[v] = C[v];
        }
    }
    for (int64_t v = 0; v < N; ++v) {
        if (wta) wta[v] = arg[v];
        if (best) best[v] = b1[v];
        if (second) second[v] = b2[v];
    }
    free(s); free(U); free(C); free(b1); free(b2); free(arg); free(slot);
    return 0;
}
