// Shared device helpers of the HDP CUDA library (sm_103a).
#pragma once
#include <cooperative_groups.h>
#include <cooperative_groups/reduce.h>
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
    // polls before a grid barrier or a look-back wait gives up; 0 means
    // HDP_SPIN_LIMIT.  Waits for bulk copies in flight keep HDP_SPIN_LIMIT.
    unsigned int spin_limit;
};

__device__ __forceinline__ int dev_err(const DevStatus* st) { return *(volatile const int*)&st->err; }

__device__ __forceinline__ unsigned spin_cap(const DevStatus* st)
{
    const unsigned c = *(volatile const unsigned*)&st->spin_limit;
    return c ? c : HDP_SPIN_LIMIT;
}

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
            const unsigned cap = spin_cap(st);
            unsigned it = 0;
            while (*vgen == g) {
                if (++it > cap || dev_err(st)) {
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

// A slot in a list or a count shared by the whole grid: one atomic per group
// of converged lanes instead of one per lane (the counter is one address, so
// per-lane atomics would serialise).
__device__ __forceinline__ int grid_ticket(int* ctr)
{
    namespace cg = cooperative_groups;
    cg::coalesced_group g = cg::coalesced_threads();
    int base = 0;
    if (g.thread_rank() == 0) base = atomicAdd(ctr, (int)g.size());
    return g.shfl(base, 0) + (int)g.thread_rank();
}

// Add 1 to cnt[key]: one atomic per distinct key among the converged lanes.
__device__ __forceinline__ void count_by_key(int* cnt, int key)
{
    namespace cg = cooperative_groups;
    cg::coalesced_group g = cg::coalesced_threads();
    cg::coalesced_group same = cg::labeled_partition(g, key);
    if (same.thread_rank() == 0) atomicAdd(cnt + key, (int)same.size());
}

// atomicMin(arr + key, v), one atomic per distinct key among the converged lanes.
__device__ __forceinline__ void min_by_key(int* arr, int key, int v)
{
    namespace cg = cooperative_groups;
    cg::coalesced_group g = cg::coalesced_threads();
    cg::coalesced_group same = cg::labeled_partition(g, key);
    const int m = cg::reduce(same, v, cg::less<int>());
    if (same.thread_rank() == 0) atomicMin(arr + key, m);
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
