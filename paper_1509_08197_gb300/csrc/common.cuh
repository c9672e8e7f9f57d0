// Shared device helpers of the HDP CUDA library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define HDP_WORDS 8                 // 256-bit label sets (labels 0..255)
#define HDP_END (-1)

// device-side error codes written into DevStatus::err
#define DEV_OK 0
#define DEV_TIMEOUT 1
#define DEV_BAD_INPUT 2

// Every spin-wait in this library gives up after this many polls (each poll
// sleeps ~100 ns, so roughly 2 s), records DEV_TIMEOUT and returns.
#define HDP_SPIN_LIMIT (1u << 24)

struct DevStatus {
    unsigned int bar_count;
    unsigned int bar_gen;
    int err;
    int where;
};

__device__ __forceinline__ int dev_err(const DevStatus* st) { return *(volatile const int*)&st->err; }

__device__ __forceinline__ void dev_fail(DevStatus* st, int code, int where)
{
    if (atomicCAS(&st->err, 0, code) == 0) st->where = where;
}

// Grid-wide barrier for cooperative launches (all blocks co-resident).  The
// wait is bounded: on timeout it records DEV_TIMEOUT and every caller returns
// false so the kernel can unwind.  Must be called by all threads of all blocks.
__device__ __forceinline__ bool grid_sync(DevStatus* st, unsigned nblocks)
{
    __syncthreads();
    if (nblocks > 1 && threadIdx.x == 0) {
        volatile unsigned* vgen = &st->bar_gen;
        unsigned g = *vgen;
        __threadfence();
        unsigned arrived = atomicAdd(&st->bar_count, 1u);
        if (arrived == nblocks - 1) {
            atomicExch(&st->bar_count, 0u);
            __threadfence();
            atomicAdd(&st->bar_gen, 1u);
        } else {
            unsigned it = 0;
            while (*vgen == g) {
                if (++it > HDP_SPIN_LIMIT || dev_err(st)) {
                    dev_fail(st, DEV_TIMEOUT, 1);
                    break;
                }
                if (it > 2048) __nanosleep(100);   // spin tight first: most barriers complete within microseconds
            }
        }
        __threadfence();
    }
    __syncthreads();
    return dev_err(st) == 0;
}

// Union-find root with path halving.  Loads bypass L1 (parents change across
// grid barriers while other SMs may hold stale L1 lines).
__device__ __forceinline__ int uf_find(int* parent, int v)
{
    for (int it = 0; it < (1 << 26); ++it) {
        int p = __ldcg(parent + v);
        if (p == v) return v;
        int gp = __ldcg(parent + p);
        if (gp == p) return p;
        __stcg(parent + v, gp);
        v = gp;
    }
    return v;
}

__device__ __forceinline__ int set_popc(const uint32_t* m)
{
    int n = 0;
#pragma unroll
    for (int i = 0; i < HDP_WORDS; ++i) n += __popc(m[i]);
    return n;
}

template <typename T>
__host__ __device__ __forceinline__ T cdiv(T a, T b) { return (a + b - 1) / b; }
