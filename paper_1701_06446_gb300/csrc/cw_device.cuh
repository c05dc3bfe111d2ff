// Small device helpers shared by several kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace cw {

// FP32 -> FP64 by re-encoding the bits on the integer pipe (the FP64 pipe,
// which a plain conversion would use, is the scarce one on this GPU).
// Subnormal inputs become signed zero; infinities and NaNs are kept.  Every
// kernel that folds FP32 tile sums into the FP64 running sums uses it, so a
// batch's sum converts identically when it enters and when it leaves.
__device__ __forceinline__ double f32_to_f64(float x)
{
    const uint32_t u = __float_as_uint(x);
    const uint32_t ex = (u >> 23) & 0xffu;
    const uint64_t sign = (uint64_t)(u & 0x80000000u) << 32;
    if (ex == 0) return __longlong_as_double((long long)sign);
    const uint64_t e64 = ex == 0xffu ? 0x7ffull : (uint64_t)ex + 896ull;
    return __longlong_as_double((long long)(sign | (e64 << 52) | ((uint64_t)(u & 0x7fffffu) << 29)));
}

// Sum the K-split partials of one workspace element: slice 2k holds the
// entering samples' partial k, slice 2k+1 the leaving samples' (stride
// `wslice` floats).  Loads are issued in groups of four so that several are
// in flight; the additions run in slice order, so every caller gets the same
// FP32 sums for the same partials.
__device__ __forceinline__ void sum_partials(const float* __restrict__ w, int64_t wslice, int ksplit,
                                             float& din, float& dout)
{
    din = 0.0f;
    dout = 0.0f;
    int k = 0;
    for (; k + 4 <= ksplit; k += 4) {
        float vi[4], vo[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            vi[j] = w[(int64_t)(2 * (k + j)) * wslice];
            vo[j] = w[(int64_t)(2 * (k + j) + 1) * wslice];
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            din += vi[j];
            dout += vo[j];
        }
    }
    for (; k < ksplit; ++k) {
        din += w[(int64_t)(2 * k) * wslice];
        dout += w[(int64_t)(2 * k + 1) * wslice];
    }
}

// The entering half only (slices 2k): the same additions in the same order as
// the `din` of sum_partials.
__device__ __forceinline__ float sum_in_partials(const float* __restrict__ w, int64_t wslice, int ksplit)
{
    float din = 0.0f;
    int k = 0;
    for (; k + 4 <= ksplit; k += 4) {
        float vi[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) vi[j] = w[(int64_t)(2 * (k + j)) * wslice];
#pragma unroll
        for (int j = 0; j < 4; ++j) din += vi[j];
    }
    for (; k < ksplit; ++k) din += w[(int64_t)(2 * k) * wslice];
    return din;
}

// Virtual CTAs of 256 threads.  A kernel of 256-thread CTAs uses its CTAs
// as they are (V = false); a kernel of 1024-thread CTAs (the single-launch
// batch shift) runs each quarter of a CTA as a virtual CTA (V = true) with its
// own named barrier (ids 1-4; id 0 is __syncthreads).
template <bool V>
__device__ __forceinline__ int vtid()
{
    return V ? (int)(threadIdx.x & 255u) : (int)threadIdx.x;
}

template <bool V>
__device__ __forceinline__ void vsync()
{
    if constexpr (V) {
        asm volatile("bar.sync %0, 256;" ::"r"(1 + (int)(threadIdx.x >> 8)) : "memory");
    } else {
        __syncthreads();
    }
}

}  // namespace cw
