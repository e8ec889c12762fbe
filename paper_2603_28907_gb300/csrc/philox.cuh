// philox.cuh -- counter-based random numbers for the device.
//
// Philox4x32-10 as defined by Salmon, Moraes, Dror and Shaw ("Parallel random
// numbers: as easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64-bit
// multiplies (multipliers 0xD2511F53, 0xCD9E8D57) with a Weyl key schedule
// (0x9E3779B9, 0xBB67AE85).  Counter = {index, step, chain, stream},
// key = {seed lo, seed hi}.  Uniforms take the top 52 bits of a 64-bit word:
// u = (floor(r / 2^12) + 1/2) 2^-52, exact in FP64 and inside (0, 1).
#pragma once

#include <stdint.h>

namespace mt {

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ uint4 draw4(uint64_t seed, uint32_t stream, uint32_t chain,
                                       uint32_t step, uint32_t index)
{
    return philox4x32_10(make_uint4(index, step, chain, stream), (uint32_t)seed,
                         (uint32_t)(seed >> 32));
}

// (0,1) uniform from the 64-bit word hi:lo, exact in FP64.
__device__ __forceinline__ double u01_f64(uint32_t lo, uint32_t hi)
{
    const uint64_t r = ((uint64_t)hi << 32) | (uint64_t)lo;
    return __dmul_rn(__dadd_rn((double)(r >> 12), 0.5), 0x1p-52);
}

// The same uniform rounded to FP32 (relative precision kept near 0):
// (2 floor(r / 2^12) + 1) 2^-53 rounded once, from the integer, to FP32.
__device__ __forceinline__ float u01_to_f32(uint32_t lo, uint32_t hi)
{
    const uint64_t r = ((uint64_t)hi << 32) | (uint64_t)lo;
    return __ull2float_rn((r >> 11) | 1ull) * 0x1p-53f;
}

}  // namespace mt
