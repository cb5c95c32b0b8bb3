// Direct Metropolis sweep: the paper's own scheme (Sec. 4.2), kept as the
// baseline the local-field kernels are measured against.  No fields: every
// proposal's
//     dE = c sum_{j != k} J*(|k-j|) [delta(a, s_j) - delta(b, s_j)]   (Eq. 2, 8)
// is summed over all L sites.  One warp sweeps one slot (one warp per CTA,
// so the slots spread over all SMs): lane l takes the sites j = l, l + 32, ...
// (FP64 fused multiply-adds of J* by the +1 / 0 / -1 coefficient, four
// independent sums), an xor-shuffle tree gives every lane the same total, and
// every lane screens the FP64 rule of Eq. 8 in FP32 with a margin that covers
// the rounding of the screen; when the screen cannot tell, lane 0 applies the
// rule in FP64 (exp and log on one lane: each FP64 warp instruction occupies
// GB300's two-lane-per-SM FP64 pipe for many cycles) and broadcasts it.  The
// warp needs no barrier beyond its own shuffles.  The slot's spins sit in the
// warp's part of shared memory; J* is read through L1 from the doubled FP64
// table.
// The running energy accumulates dE in FP64 in attempt order.  With random
// sites, attempt k of a sweep goes to the site floor(x3 L / 2^32) of Philox
// counter (k, slot, sweep, 3) (the other reading of Sec. 4.2), with the
// proposal and u from the same block.
#include <cmath>

#include "sweep_common.cuh"

namespace plr {

namespace {

constexpr int kDirWarps = 1;  // slots per CTA, one warp each: few slots per CTA spread them over all SMs
constexpr int kDirThreads = 32 * kDirWarps;

// +1.0, -1.0 or 0.0 for s_j = a, s_j = b or neither (a != b), assembled from
// the bit patterns by integer selects: no int-to-double conversion, which
// would compete with the sum's FMAs for the FP64 pipe
__device__ __forceinline__ double coef(int sj, int a, int b)
{
    const long long bits = sj == a ? 0x3FF0000000000000ll : (sj == b ? (long long)0xBFF0000000000000ull : 0ll);
    return __longlong_as_double(bits);
}

__global__ void __launch_bounds__(kDirThreads) sweep_direct_kernel(const JobDev* __restrict__ jobs,
                                                                   const int2* __restrict__ work, int nwork,
                                                                   int nsweeps, int Lpad_max)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int item = blockIdx.x * kDirWarps + warp;
    if (item >= nwork) return;  // no CTA barrier below: idle warps may leave
    const int2 wk = work[item];
    const JobDev* jp = jobs + wk.x;
    const int t = wk.y;
    const int L = jp->L, q = jp->q, W = jp->W, c = jp->c;
    const int rep = jp->map[t];
    const double cb = jp->beta[t] * (double)c;
    uint32_t* __restrict__ spins = jp->spins + (size_t)rep * W;
    const double* __restrict__ J = jp->J64d;  // J[r] = J*(r mod L), r < 2L
    const float cb32 = (float)cb;
    uint8_t* s = smem + (size_t)warp * Lpad_max;

    for (int i = lane; i < L; i += 32) s[i] = (uint8_t)((spins[i >> 3] >> (4 * (i & 7))) & 15u);
    __syncwarp();

    const uint32_t n0 = jp->nsweep[t];
    const bool rs = jp->random_sites != 0;
    double E = jp->E[rep];
    unsigned long long nacc = 0, nnear = 0;
    for (int sw = 0; sw < nsweeps; ++sw) {
        for (int m = 0; m < L; ++m) {
            // every lane draws the same proposal (the same Philox block)
            int k = m, a, b;
            float nlu;
            uint32_t ux1, ux2;
            if (rs) {
                const U4 x = philox10(U4{(uint32_t)m, (uint32_t)t, n0 + (uint32_t)sw, kTagSite}, jp->key0,
                                      jp->key1);
                k = (int)__umulhi(x.w, (uint32_t)L);
                a = s[k];
                b = a + 1 + (int)__umulhi(x.x, (uint32_t)(q - 1));
                if (b >= q) b -= q;
                ux1 = x.y;
                ux2 = x.z;
                nlu = -logf((float)x.y * 0x1p-32f + (float)((x.z >> 11) + 1u) * 0x1p-53f);
            } else {
                a = s[k];
                draw_proposal<true>(k, t, n0 + (uint32_t)sw, jp->key0, jp->key1, q, a, b, nlu, ux1, ux2);
            }
            // dE / c over the lane's sites (j = k adds J*(0) = 0), four independent
            // sums, then the xor tree (the same sum in every lane)
            double part[4] = {0.0, 0.0, 0.0, 0.0};
            int j = lane;
            for (; j + 96 < L; j += 128) {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int jj = j + 32 * e;
                    const int sj = s[jj];
                    part[e] = fma(coef(sj, a, b), J[jj > k ? jj - k : k - jj], part[e]);
                }
            }
#pragma unroll
            for (int e = 0; e < 3; ++e) {  // the last sites: fewer than four per lane
                const int jj = j + 32 * e;
                if (jj < L) {
                    const int sj = s[jj];
                    part[e] = fma(coef(sj, a, b), J[jj > k ? jj - k : k - jj], part[e]);
                }
            }
            double d = (part[0] + part[1]) + (part[2] + part[3]);
            for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(kFullMask, d, o);
            // FP32 screen of the FP64 rule (margin covering the conversion of d
            // and the FP32 -ln u); only when it cannot tell does lane 0 apply the
            // rule in FP64
            const float d32 = (float)d;
            int st = decide_fp64_filter(d32, cb32, nlu, fabsf(d32) * 1e-6f + 1e-30f);
            if (st == kUnsure) {  // lane 0 applies the rule in FP64 and broadcasts it
                int acc = 0;
                if (lane == 0)
                    acc = decide_fp64_exact(d, cb, unit53(ux1, ux2), nnear,
                                            NearSink{jp->near_log, jp->near_log_n, t, n0 + (uint32_t)sw}, m)
                              ? 1
                              : 0;
                st = __shfl_sync(kFullMask, acc, 0) ? kAccept : kReject;
            }
            if (st == kAccept) {
                E += (double)c * d;
                ++nacc;
                __syncwarp();
                if (lane == 0) s[k] = (uint8_t)b;
                __syncwarp();
            }
        }
    }
    for (int w = lane; w < W; w += 32) {
        uint32_t word = 0;
        for (int i = 0; i < 8; ++i) {
            const int j = 8 * w + i;
            if (j < L) word |= (uint32_t)s[j] << (4 * i);
        }
        spins[w] = word;
    }
    if (lane == 0) {
        jp->E[rep] = E;
        jp->nsweep[t] = n0 + (uint32_t)nsweeps;
        if (nacc) atomicAdd(&jp->acc_flip[t], nacc);
        if (nnear) atomicAdd(&jp->near[0], nnear);
    }
}

}  // namespace

size_t direct_sweep_smem_bytes(int L, int Lpad)
{
    (void)L;
    return (size_t)kDirWarps * (size_t)Lpad;  // the spins of each warp's slot, one byte each
}

cudaError_t launch_sweep_direct(const JobDev* jobs_dev, const int2* work, int nwork, int nsweeps, size_t smem,
                                cudaStream_t st)
{
    if (nwork <= 0 || nsweeps <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(sweep_direct_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = (nwork + kDirWarps - 1) / kDirWarps;
    sweep_direct_kernel<<<grid, kDirThreads, smem, st>>>(jobs_dev, work, nwork, nsweeps, (int)(smem / kDirWarps));
    return cudaGetLastError();
}

}  // namespace plr
