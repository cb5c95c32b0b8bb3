// Initial spins, energy/magnetisation measurement, replica exchange and the
// FP64 direct field rebuild of the long-range Potts chain.
#include <cmath>

#include "measure_body.cuh"
#include "near_tie.cuh"
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

// Energy (Eq. 2) and magnetisation (Eq. 10) of one slot, from its packed spins
// (the bit-plane count of measure_body.cuh):
//   N_r = #{i : s_i = s_{(i+r) mod L}}, r = 1..L/2  (N_{L-r} = N_r),
//   E = -(c/2) sum_{r=1}^{L-1} J*(r) N_r,  M = (q N_max / L - 1) / (q - 1).
// The sum over (r, w) is cut into the jb.meas_parts tiles of meas_geom(L), one
// CTA each (blockIdx.x = item * max_parts + part; CTAs past the job's part
// count return at once).  A CTA builds the bit planes of the string words its
// tile reads and sums J*(r) N_r over the tile in a fixed order (per thread,
// then a fixed tree).  The CTA that finishes last (a per-slot ticket) adds the
// tiles' sums in tile order, counts the states and writes E and M, so the
// result does not depend on which CTA ends first.
__global__ void __launch_bounds__(kAuxThreads) measure_kernel(const JobDev* __restrict__ jobs,
                                                              const int2* __restrict__ work, int max_parts,
                                                              int anchor, int cond)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int cnt[kMaxQ];
    __shared__ double red[kAuxThreads / 32];
    __shared__ int last;
    const int item = blockIdx.x / max_parts, part = blockIdx.x - item * max_parts;
    const int2 wk = work[item];
    const JobDev& jb = jobs[wk.x];
    const int np = jb.meas_parts;
    if (part >= np || (cond && !rebuild_due(jb))) return;
    if (anchor && cond && !anchor_due(jb)) return;  // a scheduled rebuild between energy anchors
    const int t = wk.y;
    const int rep = jb.map[t];
    const int L = jb.L, tid = threadIdx.x;
    const uint32_t* __restrict__ spins = jb.spins + (size_t)rep * jb.W;
    const MeasGeom g = meas_geom(L);
    const int P = meas_planes(jb.q), ws = meas_window_words(g);
    const int rt = part / g.nwt, wt = part - rt * g.nwt;
    int w_lo, w_hi, nwin;
    tile_words(g, rt, wt, &w_lo, &w_hi, &nwin);
    uint32_t* win = (uint32_t*)smem;
    build_planes(spins, L, P, w_lo, nwin, win, ws);
    __syncthreads();
    const double tot = block_sum_fixed(measure_tile_any(P, win, ws, w_lo, g, L, rt, w_lo, w_hi, jb.J64d), red);
    if (tid == 0) {
        jb.meas_part[(size_t)t * kMeasMaxParts + part] = tot;
        __threadfence();
        last = atomicAdd(&jb.meas_ticket[t], 1) == np - 1;
    }
    if (tid < kMaxQ) cnt[tid] = 0;
    __syncthreads();
    if (!last) return;
    count_states(spins, L, jb.q, cnt);
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        double sum = 0.0;
        for (int p = 0; p < np; ++p) sum += __ldcg(&jb.meas_part[(size_t)t * kMeasMaxParts + p]);
        int nmax = 0;
        for (int x = 0; x < jb.q; ++x) nmax = max(nmax, cnt[x]);
        const double E = -0.5 * (double)jb.c * sum;
        jb.meas_E[t] = E;
        jb.meas_M[t] = ((double)jb.q * (double)nmax / (double)L - 1.0) / (double)(jb.q - 1);
        if (anchor) jb.E[rep] = E;
        jb.meas_ticket[t] = 0;  // ready for the next launch
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
            if (D > -40.0 && fabs(D - log(u)) < kNearTie) {  // a near tie: counted and logged
                ++near;
                near_tie_log(jb.near_log, jb.near_log_n, 1, t, m, stage, acc);
            }
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
// result (as double or float; FX64 mode: the same sum of the rounded integer
// couplings, exact in any order); mode 1 compares the stored fields (FX64:
// converted from field units) with the FP64 sum.
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
    if (mode == 0 && jb.precision == kPrecFX64) {
        const long long* Jx = jb.Jfxd + (L + i);
        for (int x = 0; x < q; ++x) {
            long long acc = 0;
            for (int p = offs[x]; p < offs[x + 1]; ++p) acc += Jx[-pos[p]];
            ((long long*)jb.fields)[((size_t)rep * q + x) * Lpad + i] = acc;
        }
        return;
    }
    for (int x = 0; x < q; ++x) {
        double acc = 0.0;
        for (int p = offs[x]; p < offs[x + 1]; ++p) acc += Jc[-pos[p]];
        const size_t e = ((size_t)rep * q + x) * Lpad + i;
        if (mode == 0) {
            if (jb.precision == kPrecFP64) ((double*)jb.fields)[e] = acc;
            else ((float*)jb.fields)[e] = (float)acc;
        } else {
            const double cur = jb.precision == kPrecFP64   ? ((const double*)jb.fields)[e]
                               : jb.precision == kPrecFX64 ? (double)((const long long*)jb.fields)[e] * jb.fx_scale
                                                           : (double)((const float*)jb.fields)[e];
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
    const double d = __longlong_as_double((long long)jb.drift_bits[0]);
    int k = jb.sched[0];
    if (d > kDriftHigh) k = max(1, k / 2);
    else if (d < kDriftLow) k = min(max(jb.recompute_every, 1), 2 * k);
    if (!cond || anchor_due(jb)) jb.sched[3] = (int)jb.nsweep[0];  // this rebuild re-anchored the energy
    jb.sched[0] = k;
    jb.sched[1] = (int)(jb.nsweep[0] + (uint32_t)k);
    jb.sched[2] += 1;                    // rebuilds done
    jb.drift_bits[1] = jb.drift_bits[0];  // the drift of the period just closed
    jb.drift_bits[0] = 0ull;
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

int measure_parts(int L)
{
    const MeasGeom g = meas_geom(L);
    return g.nrt * g.nwt;
}

cudaError_t launch_measure(const JobDev* jobs_dev, const int2* work, int nwork, int anchor, int cond,
                           size_t smem_bytes, int max_parts, cudaStream_t st)
{
    if (nwork <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(measure_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
    if (e != cudaSuccess) return e;
    measure_kernel<<<nwork * max_parts, kAuxThreads, smem_bytes, st>>>(jobs_dev, work, max_parts, anchor, cond);
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
