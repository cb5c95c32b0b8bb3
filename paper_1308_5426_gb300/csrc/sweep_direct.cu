// Direct Metropolis sweep: the paper's own scheme (Sec. 4.2), kept as the
// baseline the local-field kernels are measured against.  No fields: every
// proposal's
//     dE = c sum_{j != k} J*(|k-j|) [delta(a, s_j) - delta(b, s_j)]   (Eq. 2, 8)
// is summed over all L sites by the whole CTA (each thread a strided share,
// then a warp-shuffle and shared-memory reduction), and one thread applies
// the FP64 rule of Eq. 8.  O(L) work and three CTA barriers per attempt.
// Spins and J* sit in shared memory; the running energy accumulates dE in
// FP64 in attempt order.  With random sites, attempt k of a sweep goes to the
// site floor(x3 L / 2^32) of Philox counter (k, slot, sweep, 3) (the other
// reading of Sec. 4.2), with the proposal and u from the same block.
#include <cmath>

#include "sweep_common.cuh"

namespace plr {

namespace {

constexpr int kDirThreads = 256;
constexpr int kDirWarps = kDirThreads / 32;

__global__ void __launch_bounds__(kDirThreads) sweep_direct_kernel(const JobDev* __restrict__ jobs,
                                                                   const int2* __restrict__ work, int nsweeps)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int2 wk = work[blockIdx.x];
    const JobDev* jp = jobs + wk.x;
    const int t = wk.y;
    const int L = jp->L, q = jp->q, Lpad = jp->Lpad, W = jp->W, c = jp->c;
    const int rep = jp->map[t];
    const double cb = jp->beta[t] * (double)c;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t* __restrict__ spins = jp->spins + (size_t)rep * W;

    double* J = (double*)smem;                       // J*(r), r = 0..L-1
    double* red = J + Lpad;                          // [kDirWarps]
    int* ab = (int*)(red + kDirWarps);               // proposal of the current site
    uint8_t* s = (uint8_t*)(ab + 4);
    for (int m = tid; m < L; m += kDirThreads) J[m] = jp->J64d[m];
    for (int i = tid; i < L; i += kDirThreads) s[i] = (uint8_t)((spins[i >> 3] >> (4 * (i & 7))) & 15u);
    __syncthreads();

    const uint32_t n0 = jp->nsweep[t];
    const bool rs = jp->random_sites != 0;
    double E = 0.0, u = 0.0;
    unsigned long long nacc = 0, nnear = 0;
    if (tid == 0) E = jp->E[rep];
    for (int sw = 0; sw < nsweeps; ++sw) {
        for (int k = 0; k < L; ++k) {
            if (tid == 0) {
                int b, site = k;
                if (rs) {  // attempt k at a uniformly drawn site (the proposal and u from the same block)
                    const U4 x = philox10(U4{(uint32_t)k, (uint32_t)t, n0 + (uint32_t)sw, kTagSite}, jp->key0,
                                          jp->key1);
                    site = (int)__umulhi(x.w, (uint32_t)L);
                    const int a = s[site];
                    b = a + 1 + (int)__umulhi(x.x, (uint32_t)(q - 1));
                    if (b >= q) b -= q;
                    u = unit53(x.y, x.z);
                    ab[0] = (a << 8) | b;
                } else {
                    float nlu;
                    uint32_t ux1, ux2;
                    const int a = s[k];
                    draw_proposal<true>(k, t, n0 + (uint32_t)sw, jp->key0, jp->key1, q, a, b, nlu, ux1, ux2);
                    u = unit53(ux1, ux2);
                    ab[0] = (a << 8) | b;
                }
                ab[1] = site;
            }
            __syncthreads();
            const int a = ab[0] >> 8, b = ab[0] & 255, kk = ab[1];
            double part = 0.0;
            for (int j = tid; j < L; j += kDirThreads) {
                const int w = (s[j] == a) - (s[j] == b);  // j = kk adds J*(0) = 0
                if (w) part += (double)w * J[j > kk ? j - kk : kk - j];
            }
            for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(kFullMask, part, o);
            if (lane == 0) red[warp] = part;
            __syncthreads();
            if (tid == 0) {
                double d = 0.0;
                for (int w = 0; w < kDirWarps; ++w) d += red[w];
                if (decide_fp64_exact(d, cb, u, nnear)) {
                    s[kk] = (uint8_t)b;
                    E += (double)c * d;
                    ++nacc;
                }
            }
            __syncthreads();
        }
    }
    for (int w = tid; w < W; w += kDirThreads) {
        uint32_t word = 0;
        for (int m = 0; m < 8; ++m) {
            const int i = 8 * w + m;
            if (i < L) word |= (uint32_t)s[i] << (4 * m);
        }
        spins[w] = word;
    }
    if (tid == 0) {
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
    return ((size_t)Lpad * sizeof(double) + kDirWarps * sizeof(double) + 16 + (size_t)Lpad + 15) & ~(size_t)15;
}

cudaError_t launch_sweep_direct(const JobDev* jobs_dev, const int2* work, int nwork, int nsweeps, size_t smem,
                                cudaStream_t st)
{
    if (nwork <= 0 || nsweeps <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(sweep_direct_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    sweep_direct_kernel<<<nwork, kDirThreads, smem, st>>>(jobs_dev, work, nsweeps);
    return cudaGetLastError();
}

}  // namespace plr
