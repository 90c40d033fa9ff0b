// Small device helpers shared by the libgila kernels: warp/block scans and
// reductions with a fixed combination order (results do not depend on
// timing).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gila {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <class T>
__device__ __forceinline__ T warp_inclusive_scan(T v, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// Inclusive scan over a block of NT threads (NT a multiple of 32, <= 1024).
// `warp_tot` is shared scratch of NT/32 + 1 elements. Returns the inclusive
// prefix of this thread; *total receives the block total. Contains
// __syncthreads and must be reached by every thread of the block.
template <class T, int NT>
__device__ __forceinline__ T block_inclusive_scan(T v, T* warp_tot, T* total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = NT / 32;
    T incl = warp_inclusive_scan(v, lane);
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        T w = (lane < NW) ? warp_tot[lane] : T(0);
        T wi = warp_inclusive_scan(w, lane);
        if (lane < NW) warp_tot[lane] = wi - w;  // exclusive
        if (lane == NW - 1) warp_tot[NW] = wi;
    }
    __syncthreads();
    incl += warp_tot[warp];
    *total = warp_tot[NW];
    __syncthreads();
    return incl;
}

// Butterfly sum over `width` consecutive lanes (width a power of two <= 32).
template <class T>
__device__ __forceinline__ T group_sum(T v, int width)
{
    for (int o = width >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o, width);
    return v;
}

// ------------------------------------------------ bulk copies (TMA engine)
// One-dimensional cp.async.bulk copies from global to shared memory,
// completed through an mbarrier in shared memory. Every wait is bounded.

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Initialise an mbarrier expecting `count` arrivals and make the
// initialisation visible to the bulk-copy engine.
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Arrive once on `bar`, announcing `bytes` of bulk transfers to come.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// Copy `bytes` (a multiple of 16; both addresses 16-byte aligned) from
// global to shared memory; completion is signalled on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Ask the bulk-copy engine to bring [src, src + bytes) into L2 (a hint: no
// completion, no registers). src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// L2 prefetch of the 16-byte aligned part of [p, p + bytes) (the start
// rounded up, the end rounded down, so nothing outside the range is
// touched), in chunks of 16 KiB.
__device__ __forceinline__ void prefetch_l2_range(const void* p, size_t bytes)
{
    const uintptr_t s = ((uintptr_t)p + 15) & ~uintptr_t(15);
    const uintptr_t e = ((uintptr_t)p + bytes) & ~uintptr_t(15);
    for (uintptr_t a = s; a < e; a += 16384)
        bulk_prefetch_l2(reinterpret_cast<const void*>(a),
                         (uint32_t)((e - a < 16384) ? e - a : 16384));
}

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait until phase `parity` of `bar` has completed; gives up after
// `limit_ns` nanoseconds and returns false.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns)
{
    const uint32_t a = smem_addr(bar);
    const uint64_t t0 = globaltimer_ns();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n"
            ".reg .pred p;\n"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            "selp.u32 %0, 1, 0, p;\n"
            "}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if (globaltimer_ns() - t0 > limit_ns) return false;
    }
}

}  // namespace gila
