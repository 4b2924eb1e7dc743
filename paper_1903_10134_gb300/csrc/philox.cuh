// Counter-based Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) for device
// code, and the pair random variable xi_ij of the random force (Sec. 2.1).
#pragma once

#include <stdint.h>

namespace mdpd {

struct U4 {
    uint32_t x, y, z, w;
};

// Ten rounds; the key (k0, k1) advances by the Weyl increments between
// rounds.  Round: multiply words 0 and 2 by the two Philox multipliers, then
// mix the high halves with words 1 and 3 and the round key.
__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        U4 n;
        n.x = hi1 ^ c.y ^ k0;
        n.y = lo1;
        n.z = hi0 ^ c.w ^ k1;
        n.w = lo0;
        c = n;
    }
    return c;
}

// The same rounds with the round keys given (rk[r] = key + r * increments,
// prepared on the host): in a kernel whose Phys is a launch parameter the
// keys are read as constant operands, with no additions per round.  Each
// 32 x 32 -> 64-bit product is one widening multiply (both halves at once;
// 4 % faster force pass than separate low and high multiplies, measured).
__device__ __forceinline__ U4 philox4x32_10_rk(U4 c, const uint32_t (&rk)[10][2])
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
        const uint32_t lo0 = (uint32_t)p0, hi0 = (uint32_t)(p0 >> 32);
        const uint32_t lo1 = (uint32_t)p1, hi1 = (uint32_t)(p1 >> 32);
        U4 n;
        n.x = hi1 ^ c.y ^ rk[r][0];
        n.y = lo1;
        n.z = hi0 ^ c.w ^ rk[r][1];
        n.w = lo0;
        c = n;
    }
    return c;
}

// Round keys of the key (k0, k1), as philox4x32_10 forms them.
inline void philox_round_keys(uint32_t k0, uint32_t k1, uint32_t (&rk)[10][2])
{
    for (int r = 0; r < 10; ++r) {
        rk[r][0] = k0 + (uint32_t)r * 0x9E3779B9u;
        rk[r][1] = k1 + (uint32_t)r * 0xBB67AE85u;
    }
}

// Word 0 of the pair draw for the force evaluation of `step`; the counter
// holds (min id, max id, step) so both members of a pair see the same value.
__device__ __forceinline__ U4 pair_draw(uint32_t id_i, uint32_t id_j, uint64_t step,
                                        uint32_t k0, uint32_t k1)
{
    U4 c;
    c.x = min(id_i, id_j);
    c.y = max(id_i, id_j);
    c.z = (uint32_t)step;
    c.w = (uint32_t)(step >> 32);
    return philox4x32_10(c, k0, k1);
}

__device__ __forceinline__ U4 pair_draw_rk(uint32_t id_i, uint32_t id_j, uint64_t step,
                                           const uint32_t (&rk)[10][2])
{
    U4 c;
    c.x = min(id_i, id_j);
    c.y = max(id_i, id_j);
    c.z = (uint32_t)step;
    c.w = (uint32_t)(step >> 32);
    return philox4x32_10_rk(c, rk);
}

// Uniform xi with zero mean and unit variance: sqrt(3) * m * 2^-24 with the odd
// integer m = 2 (w >> 8) + 1 - 2^24, exact in FP32 and FP64 before the
// multiplication by sqrt(3).
template <typename T>
__device__ __forceinline__ T xi_uniform(uint32_t w)
{
    const int32_t m = (int32_t)((w >> 8) << 1) + 1 - (1 << 24);
    return (T)1.7320508075688772935274463415059 * ((T)m * (T)5.9604644775390625e-8);
}

// Standard normal xi by Box-Muller from words 0 and 1.
__device__ __forceinline__ float xi_gauss_f(uint32_t w0, uint32_t w1)
{
    const float u1 = ((float)(w0 >> 8) + 0.5f) * 5.9604644775390625e-8f;
    const float u2 = ((float)(w1 >> 8) + 0.5f) * 5.9604644775390625e-8f;
    return sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
}

__device__ __forceinline__ double xi_gauss_d(uint32_t w0, uint32_t w1)
{
    const double u1 = ((double)(w0 >> 8) + 0.5) * 5.9604644775390625e-8;
    const double u2 = ((double)(w1 >> 8) + 0.5) * 5.9604644775390625e-8;
    return sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
}

}  // namespace mdpd
