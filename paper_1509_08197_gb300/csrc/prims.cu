// Stable LSD radix sort and scans (see prims.cuh).
#include "prims.cuh"

// ------------------------------------------------------- one-sweep radix sort ---
// Stable LSD radix sort, 8-bit digits, one launch per digit pass (after one
// histogram launch per sort).  k_rs_ghist counts every pass's digits over all
// keys.  In k_rs_onesweep each block takes a tile of RS_TILE keys by an atomic
// ticket (so its predecessors are resident or done), counts the tile's digits
// per warp, and for each digit (one thread per digit) publishes the tile's
// count, walks back over the predecessors' published counts to the nearest
// inclusive prefix (decoupled look-back) and publishes its own inclusive
// prefix.  An item's position is the digit's global start, plus the items of
// that digit in earlier tiles, in earlier warps of the tile, in earlier chunks
// of the warp, then in lower lanes of the same chunk: the sort is stable.
#define RS_FLAG_AGG (1u << 30)
#define RS_FLAG_INC (2u << 30)
#define RS_COUNT ((1u << 30) - 1u)

__global__ void k_rs_ghist(const uint32_t* __restrict__ keys, const int* d_n, int first_bit, int npass, uint32_t* ghist)
{
    __shared__ uint32_t cnt[4 * 256];
    for (int i = threadIdx.x; i < 4 * 256; i += RS_THREADS) cnt[i] = 0;
    __syncthreads();
    const int n = *d_n;
    const long long base = (long long)blockIdx.x * RS_TILE;
    for (int c = 0; c < RS_TILE / RS_THREADS; ++c) {
        const long long idx = base + c * RS_THREADS + threadIdx.x;
        const bool valid = idx < n;
        const unsigned vmask = __ballot_sync(0xffffffffu, valid);
        if (!valid) continue;
        const uint32_t k = keys[idx];
        for (int p = 0; p < npass; ++p) {
            const unsigned d = (k >> (first_bit + 8 * p)) & 255u;
            const unsigned peers = __match_any_sync(vmask, d);   // one shared atomic per digit and warp
            if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&cnt[p * 256 + d], __popc(peers));
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < npass * 256; i += RS_THREADS)
        if (cnt[i]) atomicAdd(&ghist[i], cnt[i]);
}

__global__ void __launch_bounds__(RS_THREADS) k_rs_onesweep(const uint32_t* __restrict__ kin,
                                                            const uint32_t* __restrict__ vin, uint32_t* kout,
                                                            uint32_t* vout, const int* d_n, int shift,
                                                            const uint32_t* __restrict__ ghist, uint32_t* status,
                                                            unsigned* ticket, DevStatus* st)
{
    __shared__ uint32_t cnt[8][256];
    __shared__ uint32_t gbase[256];
    __shared__ uint32_t wsum[8];
    __shared__ int s_tile;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (t == 0) s_tile = (int)atomicAdd(ticket, 1u);
    for (int i = t; i < 8 * 256; i += RS_THREADS) (&cnt[0][0])[i] = 0;
    __syncthreads();
    const int tile = s_tile;
    const int n = *d_n;
    const int nt = (int)cdiv<long long>(n, RS_TILE);
    if (tile >= nt) return;   // the whole block
    const long long wbase = (long long)tile * RS_TILE + warp * 256;
    uint32_t key[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const long long idx = wbase + c * 32 + lane;
        const bool valid = idx < n;
        key[c] = valid ? kin[idx] : 0u;
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const long long idx = wbase + c * 32 + lane;
        const bool valid = idx < n;
        const unsigned vmask = __ballot_sync(0xffffffffu, valid);
        if (valid) {
            const unsigned d = (key[c] >> shift) & 255u;
            const unsigned peers = __match_any_sync(vmask, d);
            if (lane == __ffs(peers) - 1) cnt[warp][d] += __popc(peers);
        }
        __syncwarp();
    }
    __syncthreads();
    // thread t = digit t: offsets of the warps, the tile's count, then the look-back
    const int d = t;   // RS_THREADS == 256 digits
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        const uint32_t c = cnt[w][d];
        cnt[w][d] = run;
        run += c;
    }
    uint32_t prefix = 0;
    if (tile == 0) {
        atomicExch(status + d, RS_FLAG_INC | run);
    } else {
        atomicExch(status + (size_t)tile * 256 + d, RS_FLAG_AGG | run);
        const unsigned cap = spin_cap(st);
        unsigned it = 0;
        for (int j = tile - 1; j >= 0;) {
            const uint32_t w = *(volatile const uint32_t*)(status + (size_t)j * 256 + d);
            if (!(w & ~RS_COUNT)) {
                if (++it > cap || dev_err(st)) {
                    dev_fail(st, DEV_TIMEOUT, 64);
                    break;
                }
                __nanosleep(32);
                continue;
            }
            prefix += w & RS_COUNT;
            if ((w & ~RS_COUNT) == RS_FLAG_INC) break;
            --j;
        }
        atomicExch(status + (size_t)tile * 256 + d, RS_FLAG_INC | (prefix + run));
    }
    // the digit's global start: exclusive scan of the pass's digit counts
    uint32_t g = ghist[d], inc = g;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    uint32_t before = 0;
    for (int w = 0; w < warp; ++w) before += wsum[w];
    gbase[d] = before + inc - g + prefix;
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const long long idx = wbase + c * 32 + lane;
        const bool valid = idx < n;
        const unsigned vmask = __ballot_sync(0xffffffffu, valid);
        unsigned dd = 0, peers = 0;
        if (valid) {
            dd = (key[c] >> shift) & 255u;
            peers = __match_any_sync(vmask, dd);
            const uint32_t pos = gbase[dd] + cnt[warp][dd] + __popc(peers & lt);
            kout[pos] = key[c];
            if (vin) vout[pos] = vin[idx];
        }
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) cnt[warp][dd] += __popc(peers);
        __syncwarp();
    }
}

size_t scan_tmp_words(int n_max) { return (size_t)cdiv<long long>(n_max > 0 ? n_max : 1, SCAN_TILE) + 1; }

// one-sweep scratch: the digit counts of up to 4 passes, a ticket per pass,
// then the tiles' digit states of up to 4 passes
size_t radix_tmp_words(int n_max)
{
    size_t nb = (size_t)cdiv<long long>(n_max > 0 ? n_max : 1, RS_TILE);
    return 4 * 256 + 64 + 4 * 256 * nb;
}

__global__ void k_set_int(int* out, int v) { out[0] = v; }

// Decoupled look-back by one full warp: the 32 predecessors j0, j0-1, ...
// are read at once; the nearest inclusive prefix ends the walk, a window of
// aggregates only moves it back by 32.  Returns the exclusive prefix of
// `tile` on every lane.  Waits are bounded (DEV_TIMEOUT).
__device__ __forceinline__ uint32_t lookback_u32(const unsigned long long* stp, int tile, DevStatus* st, int where)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    uint32_t pre = 0;
    unsigned it = 0;
    const unsigned cap = spin_cap(st);
    for (int j0 = tile - 1; j0 >= 0;) {
        const int j = j0 - lane;
        const unsigned long long w = j >= 0 ? *(volatile const unsigned long long*)(stp + j) : (2ull << 32);
        const uint32_t f = (uint32_t)(w >> 32);
        const unsigned incl = __ballot_sync(FULL, f == 2u), none = __ballot_sync(FULL, f == 0u);
        const int k = incl ? __ffs(incl) - 1 : 31;
        const unsigned need = k == 31 ? FULL : (2u << k) - 1u;   // lanes 0..k
        if (none & need) {
            if (++it > cap || dev_err(st)) {
                if (lane == 0) dev_fail(st, DEV_TIMEOUT, where);
                break;
            }
            __nanosleep(32);
            continue;
        }
        uint32_t v = (need >> lane & 1u) ? (uint32_t)w : 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
        pre += v;
        if (incl) break;
        j0 -= 32;
    }
    return pre;
}

__device__ __forceinline__ I4 lookback_i4(const ScanStateI4& ss, int tile, int where)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    I4 pre = I4{0, 0, 0, 0};
    unsigned it = 0;
    const unsigned cap = spin_cap(ss.st);
    for (int j0 = tile - 1; j0 >= 0;) {
        const int j = j0 - lane;
        const unsigned f = j >= 0 ? *(volatile const unsigned*)(ss.flags + j) : 2u;
        const unsigned incl = __ballot_sync(FULL, f == 2u), none = __ballot_sync(FULL, f == 0u);
        const int k = incl ? __ffs(incl) - 1 : 31;
        const unsigned need = k == 31 ? FULL : (2u << k) - 1u;
        if (none & need) {
            if (++it > cap || dev_err(ss.st)) {
                if (lane == 0) dev_fail(ss.st, DEV_TIMEOUT, where);
                break;
            }
            __nanosleep(32);
            continue;
        }
        __threadfence();   // the value was written before its flag
        I4 v = I4{0, 0, 0, 0};
        if ((need >> lane & 1u) && j >= 0) {
            const I4* src = f == 2u ? ss.inclv : ss.aggv;
            v = I4{__ldcg(&src[j].x), __ldcg(&src[j].y), __ldcg(&src[j].z), __ldcg(&src[j].w)};
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            v.x += __shfl_xor_sync(FULL, v.x, o);
            v.y += __shfl_xor_sync(FULL, v.y, o);
            v.z += __shfl_xor_sync(FULL, v.z, o);
            v.w += __shfl_xor_sync(FULL, v.w, o);
        }
        pre = pre + v;
        if (incl) break;
        j0 -= 32;
    }
    return pre;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan1_u32(const uint32_t* in, uint32_t* out, const int* d_n,
                                                            int exclusive, ScanState ss, uint32_t* total)
{
    __shared__ uint32_t smem[33];
    __shared__ uint32_t stage[SCAN_TILE + SCAN_TILE / 32];
    __shared__ int s_tile;
    __shared__ uint32_t s_pre;
    __shared__ int s_last;
    const int t = threadIdx.x;
    if (t == 0) s_tile = (int)atomicAdd(ss.ctr, 1u);
    __syncthreads();
    const int tile = s_tile;
    const int n = *d_n;
    const int nt = (int)cdiv<long long>(n, SCAN_TILE);
    if (tile < nt && tile >= ss.max_tiles && t == 0) dev_fail(ss.st, DEV_BAD_INPUT, 61);   // scratch too small
    if (tile < nt && tile < ss.max_tiles) {
        const long long base = (long long)tile * SCAN_TILE;
        uint32_t v[SCAN_IPT], x[SCAN_IPT];
        // coalesced loads, transposed through shared memory (padded: no bank
        // conflicts) so that each thread scans SCAN_IPT consecutive items
#pragma unroll
        for (int i = 0; i < SCAN_IPT; ++i) {
            const int e = i * SCAN_THREADS + t;
            stage[e + (e >> 5)] = base + e < n ? in[base + e] : 0u;
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < SCAN_IPT; ++i) {
            const int e = t * SCAN_IPT + i;
            x[i] = stage[e + (e >> 5)];
            v[i] = x[i];
        }
        const uint32_t tot = block_scan_excl<uint32_t, OpSum>(v, 0u, OpSum(), smem);
        if (t < 32) {
            unsigned long long* stp = ss.state;
            uint32_t pre = 0;
            if (tile == 0) {
                if (t == 0) atomicExch(stp, (2ull << 32) | tot);
            } else {
                if (t == 0) atomicExch(stp + tile, (1ull << 32) | tot);
                pre = lookback_u32(stp, tile, ss.st, 60);
                if (t == 0) atomicExch(stp + tile, (2ull << 32) | (uint32_t)(pre + tot));
            }
            if (t == 0) {
                s_pre = pre;
                if (total && tile == nt - 1) *total = pre + tot;
            }
        }
        __syncthreads();
        const uint32_t pre = s_pre;
#pragma unroll
        for (int i = 0; i < SCAN_IPT; ++i) {
            const int e = t * SCAN_IPT + i;
            stage[e + (e >> 5)] = pre + v[i] + (exclusive ? 0u : x[i]);
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < SCAN_IPT; ++i) {
            const int e = i * SCAN_THREADS + t;
            if (base + e < n) out[base + e] = stage[e + (e >> 5)];
        }
    } else if (t == 0 && total && n == 0 && tile == 0) {
        *total = 0;
    }
    // the last block to finish clears the tile states and the counters
    __syncthreads();
    if (t == 0) {
        __threadfence();
        s_last = atomicAdd(ss.ctr + 1, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last) {
        const int m = min(nt, ss.max_tiles);
        for (int j = t; j < m; j += SCAN_THREADS) ss.state[j] = 0ull;
        __syncthreads();
        if (t == 0) {
            ss.ctr[0] = 0u;
            ss.ctr[1] = 0u;
            __threadfence();
        }
    }
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan1_i4(const I4* in, I4* out, const int* d_n, ScanStateI4 ss)
{
    __shared__ I4 smem[33];
    __shared__ I4 stage4[SCAN_TILE + SCAN_TILE / 8];
    __shared__ int s_tile;
    __shared__ I4 s_pre;
    __shared__ int s_last;
    const int t = threadIdx.x;
    if (t == 0) s_tile = (int)atomicAdd(ss.ctr, 1u);
    __syncthreads();
    const int tile = s_tile;
    const int n = *d_n;
    const int nt = (int)cdiv<long long>(n, SCAN_TILE);
    if (tile < nt && tile >= ss.max_tiles && t == 0) dev_fail(ss.st, DEV_BAD_INPUT, 62);   // scratch too small
    if (tile < nt && tile < ss.max_tiles) {
        const long long base = (long long)tile * SCAN_TILE;
        const I4 z = I4{0, 0, 0, 0};
        I4 v[SCAN_IPT], x[SCAN_IPT];
        // coalesced loads, transposed through shared memory (one pad per 8
        // items: no bank conflicts for 16-byte items)
#pragma unroll
        for (int i = 0; i < SCAN_IPT; ++i) {
            const int e = i * SCAN_THREADS + t;
            stage4[e + (e >> 3)] = base + e < n ? in[base + e] : z;
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < SCAN_IPT; ++i) {
            const int e = t * SCAN_IPT + i;
            x[i] = stage4[e + (e >> 3)];
            v[i] = x[i];
        }
        const I4 tot = block_scan_excl<I4, OpSum>(v, z, OpSum(), smem);
        if (t < 32) {
            I4 pre = z;
            if (tile > 0) {
                if (t == 0) {
                    ss.aggv[tile] = tot;
                    __threadfence();
                    atomicExch(ss.flags + tile, 1u);
                }
                pre = lookback_i4(ss, tile, 63);
            }
            if (t == 0) {
                ss.inclv[tile] = pre + tot;
                __threadfence();
                atomicExch(ss.flags + tile, 2u);
                s_pre = pre;
            }
        }
        __syncthreads();
        const I4 pre = s_pre;
#pragma unroll
        for (int i = 0; i < SCAN_IPT; ++i) {
            const int e = t * SCAN_IPT + i;
            stage4[e + (e >> 3)] = pre + v[i] + x[i];   // inclusive
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < SCAN_IPT; ++i) {
            const int e = i * SCAN_THREADS + t;
            if (base + e < n) out[base + e] = stage4[e + (e >> 3)];
        }
    }
    // the last block to finish clears the flags and the counters
    __syncthreads();
    if (t == 0) {
        __threadfence();
        s_last = atomicAdd(ss.ctr + 1, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last) {
        const int m = min(nt, ss.max_tiles);
        for (int j = t; j < m; j += SCAN_THREADS) ss.flags[j] = 0u;
        __syncthreads();
        if (t == 0) {
            ss.ctr[0] = 0u;
            ss.ctr[1] = 0u;
            __threadfence();
        }
    }
}

void scan_i4_inclusive(const I4* in, I4* out, const int* d_n, int n_max, const ScanStateI4& ss, cudaStream_t s)
{
    if (n_max <= 0) return;
    k_scan1_i4<<<(int)cdiv<long long>(n_max, SCAN_TILE), SCAN_THREADS, 0, s>>>(in, out, d_n, ss);
}

int scan_state_tiles(int n_max) { return (int)cdiv<long long>(n_max > 0 ? n_max : 1, SCAN_TILE) + 1; }

int radix_sort(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, const int* d_n, int n_max, int key_bits,
               uint32_t* tmp, const ScanState& ss, cudaStream_t s, int first_bit)
{
    if (n_max <= 0 || key_bits <= 0) return 0;
    const int nb = (int)cdiv<long long>(n_max, RS_TILE);
    const int npass = (key_bits + 7) / 8;   // at most 4 (32-bit keys)
    uint32_t* ghist = tmp;                        // [npass][256]
    unsigned* tickets = tmp + 4 * 256;            // [npass]
    uint32_t* status = tmp + 4 * 256 + 64;        // [npass][nb][256]
    // one clearing of the counts, tickets and tile states of every pass
    cudaMemsetAsync(tmp, 0, sizeof(uint32_t) * (4 * 256 + 64 + (size_t)npass * nb * 256), s);
    k_rs_ghist<<<nb, RS_THREADS, 0, s>>>(k0, d_n, first_bit, npass, ghist);
    int cur = 0;
    for (int p = 0; p < npass; ++p) {
        const uint32_t* ki = cur ? k1 : k0;
        const uint32_t* vi = cur ? v1 : v0;
        uint32_t* ko = cur ? k0 : k1;
        uint32_t* vo = cur ? v0 : v1;
        k_rs_onesweep<<<nb, RS_THREADS, 0, s>>>(ki, vi, ko, vo, d_n, first_bit + 8 * p, ghist + 256 * p,
                                                status + (size_t)p * nb * 256, tickets + p, ss.st);
        cur ^= 1;
    }
    return cur;
}

void scan_u32(const uint32_t* in, uint32_t* out, const int* d_n, int n_max, bool exclusive, const ScanState& ss,
              uint32_t* total, cudaStream_t s)
{
    if (n_max <= 0) return;
    const int nb = (int)cdiv<long long>(n_max, SCAN_TILE);
    k_scan1_u32<<<nb, SCAN_THREADS, 0, s>>>(in, out, d_n, exclusive ? 1 : 0, ss, total);
}

// ------------------------------------------------------ wait probes ---
// Drive one of the library's bounded waits into its limit on purpose: kind 0
// is a grid barrier that counts one block more than the grid has (the
// missing block never arrives), kind 1 a decoupled look-back on tile 1 whose
// predecessor's flag (zero[0], which nothing writes) never gets published.
// Both give up after st->spin_limit polls, record DEV_TIMEOUT and return;
// nothing is written but the status block.
__global__ void k_set_spin_limit(DevStatus* st, unsigned v) { st->spin_limit = v; }

__global__ void k_wait_probe(int kind, const unsigned long long* zero, DevStatus* st)
{
    if (kind == 0) {
        grid_sync(st, gridDim.x + 1);
    } else if (blockIdx.x == 0 && threadIdx.x < 32) {
        lookback_u32(zero, 1, st, 90);
    }
}

void launch_wait_probe(int kind, unsigned limit, const unsigned long long* zero, DevStatus* st, cudaStream_t s)
{
    k_set_spin_limit<<<1, 1, 0, s>>>(st, limit);
    k_wait_probe<<<kind == 0 ? 4 : 1, 32, 0, s>>>(kind, zero, st);
    k_set_spin_limit<<<1, 1, 0, s>>>(st, 0u);
}
