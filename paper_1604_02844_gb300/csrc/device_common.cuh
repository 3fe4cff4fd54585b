// device_common.cuh -- device helpers shared by the BFS kernels: PTX
// wrappers, the bounded grid barrier, CTA prefix sums and cp.async.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.cuh"

namespace gbbfs {
namespace dev {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ uint64_t globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned ld_relaxed(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_relaxed64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Index check of the bounds-checking build (-DBFS_BOUNDS_CHECK): an index
// outside [0, bound) records the first violation, (site << 48) | index, in the
// control block's `bounds` word, sets ST_BOUNDS and is replaced by 0, so the
// access stays inside the array and the search ends with an error status
// (no trap, no assert).  Without the define GB_IX is the index itself.
#ifdef BFS_BOUNDS_CHECK
__device__ __forceinline__ int64_t bounds_checked(int64_t i, int64_t bound, int site, unsigned long long *first,
                                                  unsigned *status)
{
    if (i >= 0 && i < bound) return i;
    atomicCAS(first, 0ull, ((unsigned long long)site << 48) | ((unsigned long long)i & 0xFFFFFFFFFFFFull));
    atomicOr(status, ST_BOUNDS);
    return 0;
}
#define GB_IX(i, bound, site, ctrl) \
    ::gbbfs::dev::bounds_checked((int64_t)(i), (int64_t)(bound), (site), &(ctrl)->bounds, &(ctrl)->status)
#else
#define GB_IX(i, bound, site, ctrl) (i)
#endif

// 4-byte asynchronous global -> shared copy (no register staging).
__device__ __forceinline__ void cp_async4(void *smem_dst, const void *gmem_src)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem_src) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Bounded grid barrier for a cooperative (co-resident) grid.  `bar` points
// at {count, generation}; `status` collects ST_TIMEOUT.  A wait longer than
// timeout_ns (or 2^30 polls) sets ST_TIMEOUT and returns false; every later
// barrier also returns false, so all CTAs leave through their normal exit.
__device__ __forceinline__ bool grid_sync(unsigned *bar_count, unsigned *bar_gen, unsigned *status,
                                          unsigned nblocks, uint64_t timeout_ns, int *s_ok)
{
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned gen = ld_acquire(bar_gen);
        const unsigned arrived = atomicAdd(bar_count, 1u);
        if (arrived == nblocks - 1) {
            atomicExch(bar_count, 0u);
            __threadfence();
            st_release(bar_gen, gen + 1);
        } else {
            const uint64_t t0 = globaltimer();
            unsigned spins = 0;
            while (ld_acquire(bar_gen) == gen) {
                if (ld_relaxed(status) & ST_TIMEOUT) break;
                if (globaltimer() - t0 >= timeout_ns || ++spins > (1u << 30)) {
                    atomicOr(status, ST_TIMEOUT);
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        *s_ok = !(ld_relaxed(status) & ST_TIMEOUT);
    }
    __syncthreads();
    return *s_ok != 0;
}

// Exclusive prefix sum over the CTA; s_warp holds >= 33 ints.  Contains two
// __syncthreads; the caller must not reuse s_warp before another barrier.
template <int BLOCK>
__device__ __forceinline__ int block_exclusive_scan(int x, int *s_warp, int &total)
{
    constexpr int WARPS = BLOCK / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const int w = lane < WARPS ? s_warp[lane] : 0;
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, wi, o);
            if (lane >= o) wi += y;
        }
        s_warp[lane] = wi - w;
        if (lane == 31) s_warp[32] = wi;
    }
    __syncthreads();
    total = s_warp[32];
    return inc - x + s_warp[warp];
}

// Warp-aggregated reservation of `want` slots from a shared counter: one
// shared atomic per warp; returns this lane's first slot.  All 32 lanes call.
__device__ __forceinline__ int warp_reserve(int *s_counter, int want)
{
    const int lane = threadIdx.x & 31;
    int inc = want;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += y;
    }
    const int total = __shfl_sync(FULL, inc, 31);
    int base = 0;
    if (lane == 31 && total > 0) base = atomicAdd(s_counter, total);
    base = __shfl_sync(FULL, base, 31);
    return base + inc - want;
}

}  // namespace dev
}  // namespace gbbfs
