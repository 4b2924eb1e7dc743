// Conversions between FP64 and FP32 / integers done in integer arithmetic.
//
// On this part the FP64 pipe runs at 1/64 of the FP32 rate and also executes
// the hardware conversions from and to FP64; in the binning kernels those
// conversions kept it the busiest unit.  These helpers work on the IEEE 754
// bit layouts (binary64: sign, 11 exponent bits with bias 1023, 52 fraction
// bits; binary32: sign, 8 exponent bits with bias 127, 23 fraction bits) and
// give the same bits as the correctly rounded conversions: the host-side test
// compares them with the compiler's conversions on random and edge inputs.
// Header-only and usable on the host too (for that test).
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>

#if defined(__CUDACC__)
#define MDPD_HD __host__ __device__ __forceinline__
#else
#define MDPD_HD inline
#endif

namespace mdpd {

MDPD_HD uint64_t f64_bits(double x)
{
    uint64_t b;
    std::memcpy(&b, &x, sizeof b);
    return b;
}

MDPD_HD double bits_f64(uint64_t b)
{
    double x;
    std::memcpy(&x, &b, sizeof x);
    return x;
}

MDPD_HD float bits_f32(uint32_t b)
{
    float x;
    std::memcpy(&x, &b, sizeof x);
    return x;
}

// x rounded to the nearest binary32, ties to even, when the result is a
// normal binary32 number, +-infinity by overflow of such a rounding, or +-0
// from x = +-0: *ok = true.  For every other x (|x| below 2^-126, so the
// result would be subnormal; |x| of 2^128 or more; inf; NaN) *ok = false and
// the caller converts in another way.
MDPD_HD float f64_to_f32_rn(double x, bool* ok)
{
    const uint64_t b = f64_bits(x);
    const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
    const uint32_t sign = hi & 0x80000000u;
    const uint32_t e = (hi >> 20) & 0x7FFu;            // biased binary64 exponent
    if (e - 897u <= 253u) {                             // 2^-126 <= |x| < 2^128
        // keep 23 fraction bits (20 from hi, 3 from lo), drop 29
        uint32_t f = ((e - 896u) << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29);
        const uint32_t rest = lo & 0x1FFFFFFFu, half = 0x10000000u;
        // a carry out of the fraction raises the exponent (up to infinity)
        f += (rest > half || (rest == half && (f & 1u))) ? 1u : 0u;
        *ok = true;
        return bits_f32(sign | f);
    }
    *ok = (hi & 0x7FFFFFFFu) == 0u && lo == 0u;
    return bits_f32(sign);
}

// x (binary32) as binary64, exactly, when x is normal or +-0: *ok = true;
// for subnormal, infinite or NaN x *ok = false.
MDPD_HD double f32_to_f64(float x, bool* ok)
{
    uint32_t b;
    std::memcpy(&b, &x, sizeof b);
    const uint64_t sign = (uint64_t)(b & 0x80000000u) << 32;
    const uint32_t e = (b >> 23) & 0xFFu;
    if (e - 1u < 254u) {
        *ok = true;
        return bits_f64(sign | ((uint64_t)(e + 896u) << 52) | ((uint64_t)(b & 0x7FFFFFu) << 29));
    }
    *ok = (b & 0x7FFFFFFFu) == 0u;
    return bits_f64(sign);
}

// x split as hi + lo in binary32: hi = x rounded to the nearest binary32
// (as f64_to_f32_rn), lo = x - hi (exact in binary64) rounded to binary32
// (zero when it is below 2^-126 * 2^29 * 2^-29 in scale, i.e. for |x| under
// about 2^-74).  Returns false where f64_to_f32_rn would.
MDPD_HD bool f64_split_f32(double x, float* hi, float* lo)
{
    const uint64_t b = f64_bits(x);
    const uint32_t h32 = (uint32_t)(b >> 32), l32 = (uint32_t)b;
    const uint32_t sign = h32 & 0x80000000u;
    const uint32_t e = (h32 >> 20) & 0x7FFu;
    if (e - 897u > 252u) return false;                  // keep hi finite: |x| < 2^127
    uint32_t f = ((e - 896u) << 23) | ((h32 & 0xFFFFFu) << 3) | (l32 >> 29);
    const uint32_t rest = l32 & 0x1FFFFFFFu, half = 0x10000000u;
    const bool up = rest > half || (rest == half && (f & 1u));
    f += up ? 1u : 0u;
    *hi = bits_f32(sign | f);
    // the rest in units of the last binary64 fraction bit, 2^(e - 1075)
    const int32_t r = (int32_t)rest - (up ? (int32_t)0x20000000 : 0);
    float l = 0.0f;
    if (e >= 949u) l = (float)r * bits_f32((e - 948u) << 23);
    *lo = sign ? -l : l;
    return true;
}

// Offset x - (c0 + q h) of a binary64 coordinate x from the centre of cell q
// along one axis, in binary32 arithmetic only: h = h_hi + h_lo and
// c0 = c0_hi + c0_lo are given as binary32 pairs, the centre is formed as a
// pair from an exact product (fma) and an error-free sum (Knuth's TwoSum),
// x is split by f64_split_f32, and the result is (x_hi - c_hi) + (x_lo - c_lo),
// within about one unit in the last place of the correctly rounded offset
// (the host-side test bounds it).  Requires 0 <= q < 2^24; returns false
// where f64_split_f32 does.
MDPD_HD bool cell_offset_f32(double x, int q, float h_hi, float h_lo, float c0_hi, float c0_lo,
                             float* off)
{
    float xh, xl;
    if (!f64_split_f32(x, &xh, &xl)) return false;
    const float qf = (float)q;
    const float p = qf * h_hi;
    const float pe = fmaf(qf, h_hi, -p);                // qf * h_hi - p, exactly
    const float pl = fmaf(qf, h_lo, pe);
    const float s = c0_hi + p;                          // TwoSum(c0_hi, p)
    const float bv = s - c0_hi;
    const float err = (c0_hi - (s - bv)) + (p - bv);
    const float cl = err + (c0_lo + pl);
    *off = (xh - s) + (xl - cl);
    return true;
}

// A signed 64-bit key that orders binary64 values as their comparison does
// (for everything but NaN; -0 and +0 get the same key): x < y exactly when
// f64_key(x) < f64_key(y).
MDPD_HD int64_t f64_key(double x)
{
    const int64_t b = (int64_t)f64_bits(x);
    if (b == (int64_t)0x8000000000000000ull) return 0;          // -0 orders as +0
    return b >= 0 ? b : (b ^ (int64_t)0x7FFFFFFFFFFFFFFFull);
}

MDPD_HD int clz32(uint32_t v)
{
#if defined(__CUDA_ARCH__)
    return __clz((int)v);
#else
    return v ? __builtin_clz(v) : 32;
#endif
}

// q as binary64 (exact for every 32-bit unsigned q).
MDPD_HD double u32_to_f64(uint32_t q)
{
    if (q == 0u) return 0.0;
    const int lz = clz32(q);
    // the leading 1 moves to bit 52 and is dropped; exponent 1023 + 31 - lz
    const uint64_t frac = ((uint64_t)q << (lz + 21)) & 0xFFFFFFFFFFFFFull;
    return bits_f64(((uint64_t)(1054 - lz) << 52) | frac);
}

#if defined(__CUDACC__)
// The same with the hardware conversion for the rare inputs the integer
// paths leave out.  The fallback sits behind a branch that a warp takes only
// when one of its active lanes needs it: written as a select, the hardware
// conversion (an FP64-pipe instruction) ran on every call and kept that pipe
// the busiest unit of the binning kernel.
// (The hardware conversions sit in functions that are not inlined, so the
// compiler cannot run them speculatively ahead of the branch.)
static __device__ __noinline__ float hw_f64_to_f32(double x) { return __double2float_rn(x); }
static __device__ __noinline__ double hw_f32_to_f64(float x) { return (double)x; }

__device__ __forceinline__ float to_f32(double x)
{
    bool ok;
    float f = f64_to_f32_rn(x, &ok);
    if (__any_sync(__activemask(), !ok)) {
        if (!ok) f = hw_f64_to_f32(x);
    }
    return f;
}
__device__ __forceinline__ double to_f64(float x)
{
    bool ok;
    double d = f32_to_f64(x, &ok);
    if (__any_sync(__activemask(), !ok)) {
        if (!ok) d = hw_f32_to_f64(x);
    }
    return d;
}
template <typename T>
__device__ __forceinline__ T to_t(double x);
template <>
__device__ __forceinline__ float to_t<float>(double x) { return to_f32(x); }
template <>
__device__ __forceinline__ double to_t<double>(double x) { return x; }
#endif

}  // namespace mdpd
