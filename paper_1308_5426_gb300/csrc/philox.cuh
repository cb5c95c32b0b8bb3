// Counter-based Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64-bit
// multiplies with the published multipliers and Weyl key increments.
// The job's random numbers are a pure function of (seed, counter); the counter
// layout is (site or pair, slot or stage, sweep or exchange index, tag).
#pragma once
#include <cstdint>

namespace plr {

enum : uint32_t { kTagInit = 0u, kTagMetro = 1u, kTagExch = 2u, kTagSite = 3u };

struct U4 {
    uint32_t x, y, z, w;
};

__host__ __device__ __forceinline__ void mul_hilo(uint32_t a, uint32_t b, uint32_t& hi, uint32_t& lo)
{
#ifdef __CUDA_ARCH__
    hi = __umulhi(a, b);
    lo = a * b;
#else
    const uint64_t p = (uint64_t)a * (uint64_t)b;
    hi = (uint32_t)(p >> 32);
    lo = (uint32_t)p;
#endif
}

__host__ __device__ __forceinline__ U4 philox10(U4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        uint32_t h0, l0, h1, l1;
        mul_hilo(0xD2511F53u, c.x, h0, l0);
        mul_hilo(0xCD9E8D57u, c.z, h1, l1);
        c = U4{h1 ^ c.y ^ k0, l1, h0 ^ c.w ^ k1, l0};
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// u in (0, 1] from 53 bits of (hi, lo): ((hi:lo >> 11) + 1) * 2^-53
__host__ __device__ __forceinline__ double unit53(uint32_t hi, uint32_t lo)
{
    const uint64_t bits = ((((uint64_t)hi) << 32) | (uint64_t)lo) >> 11;
    return (double)(bits + 1ull) * 0x1p-53;
}

// u in (0, 1] from 24 bits of hi (FP32 mode)
__host__ __device__ __forceinline__ float unit24(uint32_t hi)
{
    return (float)((hi >> 8) + 1u) * 0x1p-24f;
}

}  // namespace plr
