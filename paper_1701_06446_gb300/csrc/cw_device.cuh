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

}  // namespace cw
