// gm_scan.cuh -- warp- and block-level prefix sums shared by the radix sort, the int64 prefix of
// the sampler counts and the allocation-free offsets entry point.
#pragma once

#include <cuda_runtime.h>

namespace {

// Inclusive prefix sum across the 32 lanes of a warp (all lanes active).
template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// Exclusive scan across the block of one value per thread; *total gets the block total. Every
// thread of the block must call it (it synchronises the block three times).
template <typename T, int NT>
__device__ __forceinline__ T block_excl_scan(T v, T* total) {
    static_assert(NT % 32 == 0 && NT <= 1024, "block size");
    __shared__ T warp_tot[NT / 32];
    __shared__ T tot_sh;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T inc = warp_incl_scan(v);
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T w = lane < NT / 32 ? warp_tot[lane] : T(0);
        T wi = warp_incl_scan(w);
        if (lane < NT / 32) warp_tot[lane] = wi - w;
        if (lane == NT / 32 - 1) tot_sh = wi;
    }
    __syncthreads();
    T res = warp_tot[warp] + inc - v;
    *total = tot_sh;
    __syncthreads();
    return res;
}

}  // namespace
