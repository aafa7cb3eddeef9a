// block.cuh -- block-wide scan helpers (warp shuffles + one shared-memory step).
#pragma once
#include <stdint.h>

namespace dnasa {

template <typename T>
__device__ __forceinline__ T warp_inclusive_sum(T x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

template <typename T>
__device__ __forceinline__ T warp_inclusive_max(T x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x = max(x, y);
    }
    return x;
}

// Exclusive prefix sum over the block in thread order; *total = block sum.
// `tmp` must hold THREADS/32 + 1 elements of shared memory.  All threads call.
template <int THREADS, typename T>
__device__ __forceinline__ T block_exclusive_sum(T v, T *tmp, T *total) {
    constexpr int W = THREADS / 32;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T inc = warp_inclusive_sum(v);
    if (lane == 31) tmp[w] = inc;
    __syncthreads();
    if (w == 0) {
        T s = lane < W ? tmp[lane] : T(0);
        T si = warp_inclusive_sum(s);
        if (lane < W) tmp[lane] = si - s;
        if (lane == W - 1) tmp[W] = si;
    }
    __syncthreads();
    T r = tmp[w] + inc - v;
    *total = tmp[W];
    __syncthreads();
    return r;
}

// Inclusive prefix max over the block in thread order; *total = block max.
template <int THREADS, typename T>
__device__ __forceinline__ T block_inclusive_max(T v, T *tmp, T *total, T identity) {
    constexpr int W = THREADS / 32;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T inc = warp_inclusive_max(v);
    if (lane == 31) tmp[w] = inc;
    __syncthreads();
    if (w == 0) {
        T s = lane < W ? tmp[lane] : identity;
        T si = warp_inclusive_max(s);
        // exclusive max of the warps before
        T ex = __shfl_up_sync(0xffffffffu, si, 1);
        if (lane == 0) ex = identity;
        if (lane < W) tmp[lane] = ex;
        if (lane == W - 1) tmp[W] = si;
    }
    __syncthreads();
    T r = max(tmp[w], inc);
    *total = tmp[W];
    __syncthreads();
    return r;
}

}  // namespace dnasa
