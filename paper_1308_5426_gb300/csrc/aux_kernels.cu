// Initial spins, energy/magnetisation measurement, replica exchange and the
// FP64 direct field rebuild of the long-range Potts chain.
#include <cmath>

#include "measure_body.cuh"
#include "philox.cuh"
#include "potts_internal.h"

namespace plr {

namespace {

constexpr unsigned kFull = 0xffffffffu;

// s_{r,i} = floor(x0 q / 2^32), x = Philox(i, r, 0, init): one thread per packed word.
__global__ void init_spins_kernel(const JobDev* __restrict__ jobs, int job)
{
    const JobDev& jb = jobs[job];
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (w >= jb.W) return;
    uint32_t word = 0;
    for (int m = 0; m < 8; ++m) {
        const int i = 8 * w + m;
        if (i >= jb.L) break;
        const U4 x = philox10(U4{(uint32_t)i, (uint32_t)r, 0u, kTagInit}, jb.key0, jb.key1);
        word |= (uint32_t)__umulhi(x.x, (uint32_t)jb.q) << (4 * m);
    }
    jb.spins[(size_t)r * jb.W + w] = word;
}

// Energy and magnetisation of one slot per CTA (see measure_body.cuh).
__global__ void __launch_bounds__(kAuxThreads) measure_kernel(const JobDev* __restrict__ jobs,
                                                              const int2* __restrict__ work, int anchor, int cond)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int2 wk = work[blockIdx.x];
    const JobDev& jb = jobs[wk.x];
    if (cond && !rebuild_due(jb)) return;
    const int t = wk.y;
    const int rep = jb.map[t];
    double E, M;
    measure_body(jb.spins + (size_t)rep * jb.W, jb.L, jb.q, jb.W, jb.c, jb.J64d, smem, &E, &M);
    if (threadIdx.x == 0) {
        jb.meas_E[t] = E;
        jb.meas_M[t] = M;
        if (anchor) jb.E[rep] = E;
    }
}

// One exchange step of one job per CTA (Eq. 9, Sec. 4.2): stage 0 pairs
// (t, t+1) with t even, then stage 1 with t odd.  Configurations move by
// swapping the slot -> replica map; energies travel with their replica.
__global__ void __launch_bounds__(kAuxThreads) exchange_kernel(const JobDev* __restrict__ jobs)
{
    const JobDev& jb = jobs[blockIdx.x];
    const uint32_t m = *jb.nexch;
    const int R = jb.R;
    unsigned long long near = 0;
    for (int stage = 0; stage < 2; ++stage) {
        for (int t = stage + 2 * (int)threadIdx.x; t + 1 < R; t += 2 * kAuxThreads) {
            const U4 x = philox10(U4{(uint32_t)t, (uint32_t)stage, m, kTagExch}, jb.key0, jb.key1);
            const double u = unit53(x.y, x.z);
            const int ra = jb.map[t], rb = jb.map[t + 1];
            const double D = (jb.beta[t] - jb.beta[t + 1]) * (jb.E[ra] - jb.E[rb]);
            const bool acc = (D >= 0.0) || (u < exp(D));
            if (D > -40.0 && fabs(D - log(u)) < 1e-9) ++near;
            if (acc) {
                jb.map[t] = rb;
                jb.map[t + 1] = ra;
                jb.acc_swap[t] += 1ull;
            }
        }
        __syncthreads();
    }
    if (near) atomicAdd(&jb.near[1], near);
    if (threadIdx.x == 0) *jb.nexch = m + 1u;
}

// FP64 direct fields of one replica, element tile per CTA:
//   h[x][i] = sum_{j : s_j = x} J*((i - j) mod L)   (J*(0) = 0 drops j = i),
// summed over the positions of state x in ascending j.  mode 0 stores the
// result (as double or float); mode 1 compares it with the stored fields.
__global__ void __launch_bounds__(kAuxThreads) fields_direct_kernel(const JobDev* __restrict__ job, int mode,
                                                                    int cond)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const JobDev& jb = *job;
    if (cond && !rebuild_due(jb)) return;
    const int L = jb.L, q = jb.q, Lpad = jb.Lpad, W = jb.W;
    const int rep = blockIdx.y;
    const uint32_t* spins = jb.spins + (size_t)rep * W;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int kWarps = kAuxThreads / 32;

    uint16_t* pos = (uint16_t*)smem;             // L positions grouped by state (L <= 65536)
    __shared__ int offs[kMaxQ + 1];
    __shared__ int wcount[kMaxQ];

    // positions of state x in ascending order: warp x (mod kWarps) compacts state x
    for (int x = warp; x < q; x += kWarps) {
        int c = 0;
        for (int j0 = 0; j0 < L; j0 += 32) {
            const int j = j0 + lane;
            const bool hit = j < L && (int)((spins[j >> 3] >> (4 * (j & 7))) & 15u) == x;
            c += __popc(__ballot_sync(kFull, hit));
        }
        if (lane == 0) wcount[x] = c;
    }
    __syncthreads();
    if (tid == 0) {
        offs[0] = 0;
        for (int x = 0; x < q; ++x) offs[x + 1] = offs[x] + wcount[x];
    }
    __syncthreads();
    for (int x = warp; x < q; x += kWarps) {
        int base = offs[x];
        for (int j0 = 0; j0 < L; j0 += 32) {
            const int j = j0 + lane;
            const bool hit = j < L && (int)((spins[j >> 3] >> (4 * (j & 7))) & 15u) == x;
            const unsigned bal = __ballot_sync(kFull, hit);
            if (hit) pos[base + __popc(bal & ((1u << lane) - 1u))] = (uint16_t)j;
            base += __popc(bal);
        }
    }
    __syncthreads();

    const int i = blockIdx.x * blockDim.x + tid;
    if (i >= L) return;
    const double* Jc = jb.J64d + (L + i);  // Jc[-j] = J*((i - j) mod L)
    double err = 0.0;
    for (int x = 0; x < q; ++x) {
        double acc = 0.0;
        for (int p = offs[x]; p < offs[x + 1]; ++p) acc += Jc[-pos[p]];
        const size_t e = ((size_t)rep * q + x) * Lpad + i;
        if (mode == 0) {
            if (jb.precision == 0) ((double*)jb.fields)[e] = acc;
            else ((float*)jb.fields)[e] = (float)acc;
        } else {
            const double cur = jb.precision == 0 ? ((const double*)jb.fields)[e] : (double)((const float*)jb.fields)[e];
            err = fmax(err, fabs(cur - acc));
        }
    }
    if (mode == 1) {
        const double rel = err / jb.jtot;  // non-negative: bit order equals value order
        atomicMax(jb.err_bits, (unsigned long long)__double_as_longlong(rel));
    }
}

__global__ void rebuild_policy_kernel(const JobDev* __restrict__ jobs, const int* __restrict__ idx, int njobs,
                                      int cond)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= njobs) return;
    const JobDev& jb = jobs[idx ? idx[i] : i];
    if (cond && !rebuild_due(jb)) return;
    const double d = __longlong_as_double((long long)*jb.drift_bits);
    int k = jb.sched[0];
    if (d > kDriftHigh) k = max(1, k / 2);
    else if (d < kDriftLow) k = min(max(jb.recompute_every, 1), 2 * k);
    jb.sched[0] = k;
    jb.sched[1] = (int)(jb.nsweep[0] + (uint32_t)k);
    *jb.drift_bits = 0ull;
}

}  // namespace

cudaError_t launch_rebuild_policy(const JobDev* jobs_dev, const int* idx, int njobs, int cond, cudaStream_t st)
{
    if (njobs <= 0) return cudaSuccess;
    rebuild_policy_kernel<<<(njobs + 127) / 128, 128, 0, st>>>(jobs_dev, idx, njobs, cond);
    return cudaGetLastError();
}

size_t direct_smem_bytes(int L, int q) { (void)q; return (size_t)((L + 7) & ~7) * sizeof(uint16_t); }

cudaError_t launch_init_spins(const JobDev* jobs_dev, int job, int L, int W, int R, cudaStream_t st)
{
    (void)L;
    dim3 grid((W + kAuxThreads - 1) / kAuxThreads, R);
    init_spins_kernel<<<grid, kAuxThreads, 0, st>>>(jobs_dev, job);
    return cudaGetLastError();
}

cudaError_t launch_measure(const JobDev* jobs_dev, const int2* work, int nwork, int anchor, int cond,
                           size_t smem_bytes, cudaStream_t st)
{
    if (nwork <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(measure_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
    if (e != cudaSuccess) return e;
    measure_kernel<<<nwork, kAuxThreads, smem_bytes, st>>>(jobs_dev, work, anchor, cond);
    return cudaGetLastError();
}

cudaError_t launch_exchange(const JobDev* jobs_dev, int njobs, cudaStream_t st)
{
    if (njobs <= 0) return cudaSuccess;
    exchange_kernel<<<njobs, kAuxThreads, 0, st>>>(jobs_dev);
    return cudaGetLastError();
}

cudaError_t launch_fields_direct(const JobDev* job_dev, int L, int R, int mode, int cond, size_t smem_bytes,
                                 cudaStream_t st)
{
    cudaError_t e = cudaFuncSetAttribute(fields_direct_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_bytes);
    if (e != cudaSuccess) return e;
    dim3 grid((L + kAuxThreads - 1) / kAuxThreads, R);
    fields_direct_kernel<<<grid, kAuxThreads, smem_bytes, st>>>(job_dev, mode, cond);
    return cudaGetLastError();
}

}  // namespace plr
