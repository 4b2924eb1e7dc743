// Storage types of the cell-ordered particle arrays.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mdpd {

struct __align__(32) D4 {
    double x, y, z, w;
};

template <typename T> struct Vec4;
template <> struct Vec4<float> { using type = float4; };
template <> struct Vec4<double> { using type = D4; };

// pos4.w carries the particle type and vel4.w the particle id.  In FP32 the
// words hold the integers' bits; in FP64 the integers' values (exact below 2^53).
__device__ __forceinline__ float pack_u32(float, uint32_t u) { return __uint_as_float(u); }
__device__ __forceinline__ double pack_u32(double, uint32_t u) { return (double)u; }
__device__ __forceinline__ uint32_t unpack_u32(float f) { return __float_as_uint(f); }
__device__ __forceinline__ uint32_t unpack_u32(double d) { return (uint32_t)d; }

__device__ __forceinline__ float4 make4(float x, float y, float z, float w)
{
    return make_float4(x, y, z, w);
}
__device__ __forceinline__ D4 make4(double x, double y, double z, double w)
{
    D4 r;
    r.x = x; r.y = y; r.z = z; r.w = w;
    return r;
}

}  // namespace mdpd
