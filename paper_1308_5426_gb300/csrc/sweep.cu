// Metropolis sweep of the long-range Potts chain (Eq. 8, Sec. 4.2 of the paper)
// with local fields h[x][i] = sum_{j != i} J*(|i-j|) delta(x, s_j).
//
// One CTA per temperature slot.  The slot's spins (and, when they fit, its
// fields and the doubled coupling table) are staged in shared memory.  Sites
// are processed in blocks of 32:
//   1. warp 0, lane l owns site k = k0 + l: draws its Philox numbers, proposes
//      b, and reads d_l = h[a][k] - h[b][k] from the fields, which are current
//      up to the previous block;
//   2. the 32 decisions are then taken in site order; after an accepted flip
//      j -> (a_j -> b_j) every later lane l corrects its d_l by
//      J*(l - j) ([a_l = b_j] - [a_l = a_j] - [b_l = b_j] + [b_l = a_j]),
//      which is exactly the change the rank-1 field update of flip j makes at
//      site k_l -- so each decision sees the same dE as a strictly sequential
//      sweep (dE = c (h[a][k] - h[b][k]), Eq. 2 and 8);
//   3. all threads apply the block's accepted flips to the fields:
//      h[a_j][i] -= J*(|i-k_j|), h[b_j][i] += J*(|i-k_j|), in flip order.
// The periodic distance is read from the doubled table J*((i - k) mod L).
#include <cmath>

#include "philox.cuh"
#include "potts_internal.h"

namespace plr {

namespace {

constexpr unsigned kFull = 0xffffffffu;

// FP64-mode decision: the exact FP64 rule "dE <= 0 or u < exp(-beta dE)".
// It is decided in FP32 when the FP32 margin is far wider than the rounding of
// the FP32 evaluation (|x - (-ln u)| > 1e-6 + 1e-5 max(x, -ln u); the FP32
// errors of x and -ln u are below 1e-6 relative), else in FP64.  A decision
// with |beta dE + ln u| < 1e-9 is counted as a near tie.
__device__ __forceinline__ bool decide64(double d, double cb, double c, double u, float nlu,
                                         unsigned long long& near)
{
    const double dE = c * d;
    if (dE <= 0.0) return true;
    const double x = cb * d;  // beta * c * d
    const float xf = (float)x;
    const float m = 1e-6f + 1e-5f * fmaxf(xf, nlu);
    if (xf < nlu - m) return true;
    if (xf > nlu + m) return false;
    const bool acc = u < exp(-x);
    if (fabs(x + log(u)) < 1e-9) ++near;
    return acc;
}

// FP32-mode decision: dE <= 0 or beta dE < -ln u, in FP32.
__device__ __forceinline__ bool decide32(float d, float cb, float nlu)
{
    if (d <= 0.0f) return true;
    return cb * d < nlu;
}

template <typename T>
__global__ void __launch_bounds__(kSweepThreads) sweep_kernel(const JobDev* __restrict__ jobs,
                                                              const int2* __restrict__ work, int nsweeps)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int2 wk = work[blockIdx.x];
    const JobDev& jb = jobs[wk.x];
    const int t = wk.y;
    const int L = jb.L, q = jb.q, Lpad = jb.Lpad, W = jb.W;
    const int rep = jb.map[t];
    const double beta = jb.beta[t];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    const T* Jg = (sizeof(T) == 8) ? (const T*)(const void*)jb.J64d : (const T*)(const void*)jb.J32d;
    T* hg = (T*)jb.fields + (size_t)rep * q * Lpad;
    uint32_t* spins = jb.spins + (size_t)rep * W;

    // shared-memory carve-up (must match sweep_smem_bytes)
    size_t off = 0;
    const T* Jd = Jg;
    if (jb.j_smem) {
        T* p = (T*)(smem + off);
        for (int m = tid; m < 2 * L; m += kSweepThreads) p[m] = Jg[m];
        Jd = p;
        off += (size_t)2 * Lpad * sizeof(T);
    }
    T* h = hg;
    if (jb.h_smem) {
        h = (T*)(smem + off);
        const size_t n = (size_t)q * Lpad;
        for (size_t e = tid; e < n; e += kSweepThreads) h[e] = hg[e];
        off += n * sizeof(T);
    }
    uint8_t* s = smem + off;
    off += (size_t)Lpad;
    int* fk = (int*)(smem + off);   // flip sites of the current block
    int* fab = fk + kSiteBlock;     // (a << 8) | b
    int* nfl = fab + kSiteBlock;    // number of flips

    for (int i = tid; i < L; i += kSweepThreads) s[i] = (uint8_t)((spins[i >> 3] >> (4 * (i & 7))) & 15u);
    __syncthreads();

    const uint32_t n0 = jb.nsweep[t];
    const int c = jb.c;
    const double cb64 = beta * (double)c;
    const float cb32 = (float)cb64;
    double dE_sum = 0.0;               // per lane of warp 0
    unsigned long long nacc = 0, nnear = 0;

    for (int it = 0; it < nsweeps; ++it) {
        const uint32_t n = n0 + (uint32_t)it;
        for (int k0 = 0; k0 < L; k0 += kSiteBlock) {
            if (warp == 0) {
                const int k = k0 + lane;
                const int nv = min(kSiteBlock, L - k0);
                const bool valid = lane < nv;
                int a = 0, b = 0;
                double u = 1.0;
                float nlu = 0.0f;
                T d = (T)0;
                if (valid) {
                    a = s[k];
                    const U4 x = philox10(U4{(uint32_t)k, (uint32_t)t, n, kTagMetro}, jb.key0, jb.key1);
                    b = a + 1 + (int)__umulhi(x.x, (uint32_t)(q - 1));
                    if (b >= q) b -= q;
                    if (sizeof(T) == 8) {
                        u = unit53(x.y, x.z);
                        nlu = -logf((float)u);
                    } else {
                        nlu = -logf(unit24(x.y));
                    }
                    d = h[(size_t)a * Lpad + k] - h[(size_t)b * Lpad + k];
                }
                bool mine = false;
                for (int j = 0; j < nv; ++j) {
                    bool dec = false;
                    if (lane == j) {
                        if (sizeof(T) == 8)
                            dec = decide64((double)d, cb64, (double)c, u, nlu, nnear);
                        else
                            dec = decide32((float)d, cb32, nlu);
                        if (dec) {
                            mine = true;
                            dE_sum += (double)c * (double)d;
                        }
                    }
                    if (__ballot_sync(kFull, dec)) {
                        const int aj = __shfl_sync(kFull, a, j);
                        const int bj = __shfl_sync(kFull, b, j);
                        if (lane > j && valid) {
                            const int coef = (a == bj) - (a == aj) - (b == bj) + (b == aj);
                            if (coef) d += (T)coef * Jd[lane - j];
                        }
                    }
                }
                const unsigned mask = __ballot_sync(kFull, mine);
                if (mine) {
                    const int pos = __popc(mask & ((1u << lane) - 1u));
                    fk[pos] = k;
                    fab[pos] = (a << 8) | b;
                    s[k] = (uint8_t)b;
                }
                if (lane == 0) {
                    *nfl = __popc(mask);
                    nacc += (unsigned long long)__popc(mask);
                }
            }
            __syncthreads();
            const int nf = *nfl;
            for (int f = 0; f < nf; ++f) {
                const int kf = fk[f], af = fab[f] >> 8, bf = fab[f] & 255;
                T* ha = h + (size_t)af * Lpad;
                T* hb = h + (size_t)bf * Lpad;
                const T* Jc = Jd + (L - kf);  // Jc[i] = J*((i - kf) mod L)
                for (int i = tid; i < L; i += kSweepThreads) {
                    const T v = Jc[i];
                    ha[i] -= v;
                    hb[i] += v;
                }
            }
            __syncthreads();
        }
    }

    // write back
    for (int w = tid; w < W; w += kSweepThreads) {
        uint32_t word = 0;
        for (int m = 0; m < 8; ++m) {
            const int i = 8 * w + m;
            if (i < L) word |= (uint32_t)s[i] << (4 * m);
        }
        spins[w] = word;
    }
    if (jb.h_smem) {
        const size_t ne = (size_t)q * Lpad;
        for (size_t e = tid; e < ne; e += kSweepThreads) hg[e] = h[e];
    }
    if (warp == 0) {
        for (int o = 16; o > 0; o >>= 1) {
            dE_sum += __shfl_xor_sync(kFull, dE_sum, o);
            nnear += __shfl_xor_sync(kFull, nnear, o);
        }
        if (lane == 0) {
            jb.E[rep] += dE_sum;
            jb.nsweep[t] = n0 + (uint32_t)nsweeps;
            if (nacc) atomicAdd(&jb.acc_flip[t], nacc);
            if (nnear) atomicAdd(&jb.near[0], nnear);
        }
    }
}

}  // namespace

size_t sweep_smem_bytes(const JobDev& j)
{
    const size_t w = j.precision == 0 ? 8 : 4;
    size_t b = 0;
    if (j.j_smem) b += (size_t)2 * j.Lpad * w;
    if (j.h_smem) b += (size_t)j.q * j.Lpad * w;
    b += (size_t)j.Lpad;
    b += 3 * kSiteBlock * sizeof(int);
    return b;
}

cudaError_t launch_sweep(const JobDev* jobs_dev, const int2* work, int nwork, int nsweeps, int precision,
                         size_t smem_bytes, cudaStream_t st)
{
    if (nwork <= 0 || nsweeps <= 0) return cudaSuccess;
    if (precision == 0) {
        cudaError_t e = cudaFuncSetAttribute(sweep_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem_bytes);
        if (e != cudaSuccess) return e;
        sweep_kernel<double><<<nwork, kSweepThreads, smem_bytes, st>>>(jobs_dev, work, nsweeps);
    } else {
        cudaError_t e = cudaFuncSetAttribute(sweep_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem_bytes);
        if (e != cudaSuccess) return e;
        sweep_kernel<float><<<nwork, kSweepThreads, smem_bytes, st>>>(jobs_dev, work, nsweeps);
    }
    return cudaGetLastError();
}

}  // namespace plr
