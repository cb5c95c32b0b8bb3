// Energy (Eq. 2) and magnetisation (Eq. 10) of one packed configuration,
// computed by one CTA of kAuxThreads threads -- the body shared by the
// handle's measure kernel and the allocation-free measure entry point.
//   N_r = #{i : s_i = s_{(i+r) mod L}}, r = 1..L/2  (N_{L-r} = N_r)
//   E = -(c/2) sum_{r=1}^{L-1} J*(r) N_r,  M = (q N_max / L - 1) / (q - 1)
// N_r is counted 8 sites at a time: the packed word of sites 8w..8w+7 is
// XORed with the word of sites 8w+r..8w+r+7 (a funnel shift of the doubled
// packed string held in shared memory) and the zero nibbles are counted.
// The FP64 sum over r runs in a fixed order (per thread, then a fixed tree),
// so the result is deterministic.
#pragma once
#include <cstdint>

#include "potts_internal.h"

namespace plr {

// dynamic shared memory of measure_body: doubled packed string + unpacked spins
inline size_t measure_smem_bytes(int L, int W) { return (size_t)(2 * W + 2) * 4 + (size_t)((L + 15) & ~15); }

__device__ __forceinline__ double block_sum_fixed(double v, double* red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double tot = 0.0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) tot += red[i];
        red[0] = tot;
    }
    __syncthreads();
    tot = red[0];
    __syncthreads();
    return tot;
}

// spins: packed words of one configuration (W = ceil(L/8) words, spin i at
// bits 4(i%8) of word i/8); J: J*(r) for r = 0..L/2 at least; smem: dynamic
// shared memory of measure_smem_bytes(L, W).  *E and *M are valid in thread 0.
__device__ __forceinline__ void measure_body(const uint32_t* __restrict__ spins, int L, int q, int W, int c,
                                             const double* __restrict__ J, unsigned char* smem, double* E,
                                             double* M)
{
    const int tid = threadIdx.x;
    const int nd = 2 * W + 2;  // doubled packed string, enough words for any shift
    uint32_t* dbl = (uint32_t*)smem;
    uint8_t* s = (uint8_t*)(dbl + nd);
    __shared__ int cnt[kMaxQ];
    __shared__ double red[kAuxThreads / 32];

    if (tid < kMaxQ) cnt[tid] = 0;
    for (int i = tid; i < L; i += kAuxThreads) s[i] = (uint8_t)((spins[i >> 3] >> (4 * (i & 7))) & 15u);
    __syncthreads();
    for (int m = tid; m < nd; m += kAuxThreads) {
        uint32_t word = 0;
        for (int b = 0; b < 8; ++b) word |= (uint32_t)s[(8 * m + b) % L] << (4 * b);
        dbl[m] = word;
    }
    for (int i = tid; i < L; i += kAuxThreads) atomicAdd(&cnt[s[i]], 1);
    __syncthreads();

    const int tail = L & 7;  // valid nibbles of the last word (0 = all 8)
    const uint32_t tail_bits = tail ? (0x11111111u & ((1u << (4 * tail)) - 1u)) : 0x11111111u;
    double part = 0.0;
    for (int r = 1 + tid; 2 * r <= L; r += kAuxThreads) {
        const int qo = r >> 3, sh = 4 * (r & 7);
        int Nr = 0;
        for (int w = 0; w < W; ++w) {
            const uint32_t lo = dbl[w + qo], hi = dbl[w + qo + 1];
            const uint32_t rot = __funnelshift_r(lo, hi, sh);
            uint32_t x = dbl[w] ^ rot;
            x |= x >> 1;
            x |= x >> 2;
            const uint32_t valid = (w == W - 1) ? tail_bits : 0x11111111u;
            Nr += __popc(valid) - __popc(x & valid);
        }
        const double wgt = (2 * r == L) ? 1.0 : 2.0;
        part += wgt * J[r] * (double)Nr;
    }
    const double tot = block_sum_fixed(part, red);
    if (tid == 0) {
        int nmax = 0;
        for (int x = 0; x < q; ++x) nmax = max(nmax, cnt[x]);
        *E = -0.5 * (double)c * tot;
        *M = ((double)q * (double)nmax / (double)L - 1.0) / (double)(q - 1);
    }
}

}  // namespace plr
