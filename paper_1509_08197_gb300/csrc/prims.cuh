// Device-wide primitives: tile scans and a stable LSD radix sort.
// Element counts may live in device memory (d_n) so that launches stay
// asynchronous; grids are sized by a host-side upper bound.
#pragma once
#include "common.cuh"

#define SCAN_THREADS 256
#define SCAN_IPT 8
#define SCAN_TILE (SCAN_THREADS * SCAN_IPT)

struct I4 {
    int x, y, z, w;
};
__host__ __device__ __forceinline__ I4 operator+(I4 a, I4 b) { return I4{a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w}; }

struct OpSum {
    template <typename T> __device__ __forceinline__ T operator()(T a, T b) const { return a + b; }
};
struct OpMin {
    template <typename T> __device__ __forceinline__ T operator()(T a, T b) const { return b < a ? b : a; }
};

__device__ __forceinline__ int shfl_up(int v, int d) { return __shfl_up_sync(0xffffffffu, v, d); }
__device__ __forceinline__ unsigned shfl_up(unsigned v, int d) { return __shfl_up_sync(0xffffffffu, v, d); }
__device__ __forceinline__ long long shfl_up(long long v, int d) { return __shfl_up_sync(0xffffffffu, v, d); }
__device__ __forceinline__ I4 shfl_up(I4 v, int d)
{
    return I4{__shfl_up_sync(0xffffffffu, v.x, d), __shfl_up_sync(0xffffffffu, v.y, d),
              __shfl_up_sync(0xffffffffu, v.z, d), __shfl_up_sync(0xffffffffu, v.w, d)};
}

// Exclusive block scan of SCAN_IPT items per thread (items contiguous per
// thread); returns the block total.  smem: at least 33 T.
template <typename T, typename Op>
__device__ __forceinline__ T block_scan_excl(T (&v)[SCAN_IPT], T ident, Op op, T* smem)
{
    T local = ident;
#pragma unroll
    for (int i = 0; i < SCAN_IPT; ++i) {
        T x = v[i];
        v[i] = local;
        local = op(local, x);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T incl = local;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        T o = shfl_up(incl, d);
        if (lane >= d) incl = op(o, incl);
    }
    if (lane == 31) smem[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        T w = lane < (SCAN_THREADS / 32) ? smem[lane] : ident;
        T wi = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            T o = shfl_up(wi, d);
            if (lane >= d) wi = op(o, wi);
        }
        T ex = shfl_up(wi, 1);
        if (lane == 0) ex = ident;
        if (lane < (SCAN_THREADS / 32)) smem[lane] = ex;
        if (lane == (SCAN_THREADS / 32) - 1) smem[32] = wi;
    }
    __syncthreads();
    T warp_pre = smem[warp];
    T thread_excl = shfl_up(incl, 1);
    if (lane == 0) thread_excl = ident;
    T pre = op(warp_pre, thread_excl);
#pragma unroll
    for (int i = 0; i < SCAN_IPT; ++i) v[i] = op(pre, v[i]);
    T total = smem[32];
    __syncthreads();
    return total;
}

template <typename T, typename Op>
__global__ void k_scan_reduce(const T* __restrict__ in, const int* d_n, T* block_sums, T ident, Op op, int reverse)
{
    __shared__ T smem[33];
    const int n = *d_n;
    const long long base = (long long)blockIdx.x * SCAN_TILE;
    T v[SCAN_IPT];
#pragma unroll
    for (int i = 0; i < SCAN_IPT; ++i) {
        long long idx = base + (long long)threadIdx.x * SCAN_IPT + i;
        v[i] = idx < n ? in[reverse ? (n - 1 - idx) : idx] : ident;
    }
    T tot = block_scan_excl<T, Op>(v, ident, op, smem);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

template <typename T, typename Op>
__global__ void k_scan_top(T* block_sums, const int* d_n, T ident, Op op, T* total)
{
    __shared__ T smem[33];
    const int n = *d_n;
    const int nb = (int)cdiv<long long>(n, SCAN_TILE);
    T carry = ident;
    for (int base = 0; base < nb; base += SCAN_TILE) {
        T v[SCAN_IPT];
#pragma unroll
        for (int i = 0; i < SCAN_IPT; ++i) {
            int idx = base + threadIdx.x * SCAN_IPT + i;
            v[i] = idx < nb ? block_sums[idx] : ident;
        }
        T tot = block_scan_excl<T, Op>(v, ident, op, smem);
#pragma unroll
        for (int i = 0; i < SCAN_IPT; ++i) {
            int idx = base + threadIdx.x * SCAN_IPT + i;
            if (idx < nb) block_sums[idx] = op(carry, v[i]);
        }
        carry = op(carry, tot);
        __syncthreads();
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

template <typename T, typename Op>
__global__ void k_scan_down(const T* __restrict__ in, T* out, const int* d_n, const T* block_pre, T ident, Op op,
                            int exclusive, int reverse)
{
    __shared__ T smem[33];
    const int n = *d_n;
    const long long base = (long long)blockIdx.x * SCAN_TILE;
    T v[SCAN_IPT], x[SCAN_IPT];
#pragma unroll
    for (int i = 0; i < SCAN_IPT; ++i) {
        long long idx = base + (long long)threadIdx.x * SCAN_IPT + i;
        x[i] = idx < n ? in[reverse ? (n - 1 - idx) : idx] : ident;
        v[i] = x[i];
    }
    block_scan_excl<T, Op>(v, ident, op, smem);
    const T pre = block_pre[blockIdx.x];
#pragma unroll
    for (int i = 0; i < SCAN_IPT; ++i) {
        long long idx = base + (long long)threadIdx.x * SCAN_IPT + i;
        if (idx < n) {
            T r = op(pre, v[i]);
            if (!exclusive) r = op(r, x[i]);
            out[reverse ? (n - 1 - idx) : idx] = r;
        }
    }
}

// Scan of d_n (<= n_max) elements.  tmp must hold cdiv(n_max, SCAN_TILE) T.
// total (optional, device) receives the reduction of all elements.
template <typename T, typename Op>
void device_scan(const T* in, T* out, const int* d_n, int n_max, T ident, Op op, bool exclusive, bool reverse,
                 T* tmp, T* total, cudaStream_t s)
{
    if (n_max <= 0) return;
    int nb = (int)cdiv<long long>(n_max, SCAN_TILE);
    k_scan_reduce<T, Op><<<nb, SCAN_THREADS, 0, s>>>(in, d_n, tmp, ident, op, reverse ? 1 : 0);
    k_scan_top<T, Op><<<1, SCAN_THREADS, 0, s>>>(tmp, d_n, ident, op, total);
    k_scan_down<T, Op><<<nb, SCAN_THREADS, 0, s>>>(in, out, d_n, tmp, ident, op, exclusive ? 1 : 0,
                                                    reverse ? 1 : 0);
}

// ------------------------------------------------- single-pass u32 scan ---
// Sum scan of unsigned ints in one launch: tiles take ids from an atomic
// ticket (so every tile's predecessors are resident), publish their
// aggregate, then walk back over published aggregates to the nearest
// inclusive prefix (decoupled look-back).  The last tile to finish resets the
// ticket and the tile states, so the scratch is ready for the next call
// without a clearing launch.  Waits are bounded (DEV_TIMEOUT).
struct ScanState {
    unsigned long long* state;   // per tile: flag << 32 | value (flag 1: aggregate, 2: inclusive prefix)
    unsigned int* ctr;           // [2]: ticket, tiles finished
    DevStatus* st;
    int max_tiles;
};

// The same for int4 sums (in place allowed).  A tile's aggregate and
// inclusive prefix live in separate arrays, written before flags 1 and 2, so a
// reader never mistakes one for the other.
struct ScanStateI4 {
    unsigned int* flags;   // per tile: 0, 1 (aggregate out), 2 (inclusive prefix out)
    I4* aggv;
    I4* inclv;
    unsigned int* ctr;     // [2]: ticket, tiles finished
    DevStatus* st;
    int max_tiles;
};
void scan_i4_inclusive(const I4* in, I4* out, const int* d_n, int n_max, const ScanStateI4& ss, cudaStream_t s);

// ------------------------------------------------------------ radix sort ---
#define RS_THREADS 256
#define RS_TILE 2048     // 8 warps x 256 items


// Stable LSD radix sort of (key, value) pairs on bits [first_bit, first_bit + key_bits).  vals may
// be null (keys only).  Buffers ping-pong between (k0, v0) and (k1, v1); the
// return value says where the result is: 0 -> (k0, v0), 1 -> (k1, v1).
// tmp: at least radix_tmp_words(n_max) uint32 (one-sweep digit counts and tile states).
int radix_sort(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, const int* d_n, int n_max, int key_bits,
               uint32_t* tmp, const ScanState& ss, cudaStream_t s, int first_bit = 0);
size_t radix_tmp_words(int n_max);

// Exclusive scans used across the library.
void scan_u32(const uint32_t* in, uint32_t* out, const int* d_n, int n_max, bool exclusive, const ScanState& ss,
              uint32_t* total, cudaStream_t s);
int scan_state_tiles(int n_max);
__global__ void k_set_int(int* out, int v);
// Enqueue a wait that is made to run out after `limit` polls (kind 0: grid
// barrier, 1: look-back); see prims.cu.  zero: a zeroed device word.
void launch_wait_probe(int kind, unsigned limit, const unsigned long long* zero, DevStatus* st, cudaStream_t s);
size_t scan_tmp_words(int n_max);
