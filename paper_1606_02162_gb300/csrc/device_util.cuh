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

}  // namespace gila
