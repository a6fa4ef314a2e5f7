// Double-single arithmetic of the pair kernels (force.cu) and the fused
// block-step kernel (persist.cu).
#pragma once

#include <cuda_runtime.h>

namespace nb {

// ---------------------------------------------------------------------------
// Double-single accumulation (Knuth/Moller TwoSum + fast renormalisation).
// ---------------------------------------------------------------------------

__device__ __forceinline__ void ds_add(float &hi, float &lo, float x)
{
    const float s = hi + x;
    const float bb = s - hi;
    const float e = (hi - (s - bb)) + (x - bb);
    const float t = lo + e;
    hi = s + t;
    lo = t - (hi - s);
}

// A double-single value hi + lo (two FP32 numbers). On GB300 a warp-wide FP64
// instruction holds an SMSP's FP64 pipe for ~64 cycles, so partial sums are
// combined in double-single FP32 arithmetic and only final results are FP64.
struct dsf {
    float hi, lo;
};

// a += b for double-single values (TwoSum of the high parts, low parts added,
// renormalised).
__device__ __forceinline__ void ds_acc(dsf &a, dsf b)
{
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    float e = (a.hi - (s - bb)) + (b.hi - bb);
    e += a.lo + b.lo;
    a.hi = s + e;
    a.lo = e - (a.hi - s);
}

__device__ __forceinline__ dsf ds_shfl_xor(dsf a, int o)
{
    return dsf{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}

__device__ __forceinline__ double ds_to_double(dsf a) { return (double)a.hi + (double)a.lo; }

}  // namespace nb
