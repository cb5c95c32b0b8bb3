// Metropolis sweep with a slot's fields spread over the shared memory of a
// thread-block cluster (Eq. 8, Sec. 4.2; the local-field scheme of sweep.cu),
// for FP32 fields (T = float), FP64 fields (T = double) and FX64 fields
// (T = long long: 64-bit integers in units of 2^-F).
//
// Fields of a long chain (q L words: 320 KB at L = 16384, q = 5 in FP32,
// 640 KB in FP64 or FX64) fit no single CTA's shared memory; one CTA working
// on them in global memory waits on L2 round trips and leaves most SMs idle
// when a job has fewer slots than the GPU has SMs.  Here the C CTAs of a
// cluster (C = 2, 4 or 8) share one slot: CTA r holds the fields h[x][i] of
// every state x for the sites of blocks [r P, (r + 1) P) (P = ceil(nblk / C)
// blocks of 32 sites), and its spins.  Per block g of the sweep:
// - the CTA owning the block decides it with warp 0, exactly as the
//   single-CTA kernel does (corrections for block g-1's flips, in-order scan;
//   FP64 and FX64: the FP64 rule, screened in FP32, exact where unsure),
//   writes the accepted flips (site, a, b) into every CTA's flip list through
//   distributed shared memory, and brings its own 32 sites up to date;
// - meanwhile every CTA's update warps apply block g-1's flips to the sites it
//   holds (all but the block being decided);
// - one cluster barrier (release / acquire) ends the step.
// Each field element receives the same updates in the same order as in the
// single-CTA kernels, and the decisions are the same, so spins and fields are
// bit-identical to theirs.  The FP32 energy change is accumulated per lane of
// the deciding warp in block order; the 32 lane sums move to the next owner's
// shared memory when a block's owner changes, so the final energy is
// bit-identical too.  FP64 and FX64 energies are recomputed from the fields
// after the sweep by CTA 0, from the fields and spins the cluster wrote back:
// FP64 summed over the same 256 fixed strands as the single-CTA kernel, FX64
// exactly in 128-bit integers, so they are bit-identical as well.
#include <cooperative_groups.h>
#include <type_traits>

#include "sweep_common.cuh"

namespace cg = cooperative_groups;

namespace plr {

namespace {

constexpr int kClThreads = 512;  // warp 0 decides, warps 1..15 update

// all threads of the cluster: writes before (local and distributed shared
// memory) visible to every thread after
__device__ __forceinline__ void cluster_barrier()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

struct ClLayout {
    // carve-up of the dynamic shared memory (must match the kernel); w: bytes
    // of a field word
    int Lp;        // local row stride: P * 32 sites
    size_t o_dacc, o_lk, o_lab, o_lcnt, o_jn, o_h, o_s, bytes;
    __host__ __device__ ClLayout(int L, int q, int C, int w = 4)
    {
        const int nblk = (L + kSiteBlock - 1) / kSiteBlock;
        const int P = (nblk + C - 1) / C;
        Lp = P * kSiteBlock;
        size_t o = 0;
        o_dacc = o;  // [32] double: the lane energy sums handed to the next owner
        o += 32 * sizeof(double);
        o_lk = o;    // [2][32] flip sites
        o += 2 * kSiteBlock * sizeof(int);
        o_lab = o;   // [2][32] (a << 8) | b
        o += 2 * kSiteBlock * sizeof(int);
        o_lcnt = o;  // [2] flip counts (+ padding)
        o += 16;
        o_jn = o;    // J*(r), r < 64, FP32
        o += kNearTable * sizeof(float);
        o_h = o;     // [q][Lp] fields of this CTA's sites
        o += (size_t)q * Lp * w;
        o_s = o;     // [Lp] spins of this CTA's sites
        o += (size_t)Lp;
        bytes = (o + 15) & ~(size_t)15;
    }
};

// Rank-1 updates of the flips (pk, pab)[0..nf) on this CTA's sites: local
// element j (site lo + j), j in [0, n) except [x0, x0 + nx):
// h[a][j] -= J*((lo + j - k) mod L), h[b][j] += J*((lo + j - k) mod L).
// One site per thread with consecutive threads on consecutive sites (the
// field rows and the coupling table are read without bank conflicts or
// misaligned vectors), four sites in flight per thread (stride nw), all flips
// applied to those four before moving on.  J is the doubled table (J[m] =
// J*(m mod L), m < 2L).
template <typename T>
__device__ __forceinline__ void apply_flips_part(T* __restrict__ h, int Lp, int lo, int n, const T* __restrict__ J,
                                                 int L, const int* pk, const int* pab, int nf, int x0, int nx, int u)
{
    constexpr int nw = kClThreads - 32;
    constexpr int G = 4;
    const int m = n - nx;
    int j = u;
    for (; j + (G - 1) * nw < m; j += G * nw) {
        int idx[G], r0[G];
#pragma unroll
        for (int e = 0; e < G; ++e) {
            const int jj = j + e * nw;
            idx[e] = jj < x0 ? jj : jj + nx;
            r0[e] = lo + idx[e] + L;  // J[r0 - k] = J*((lo + idx - k) mod L): the table runs to 2L
        }
        for (int f = 0; f < nf; ++f) {
            const int kf = pk[f], af = pab[f] >> 8, bf = pab[f] & 255;
            T* __restrict__ ha = h + (size_t)af * Lp;
            T* __restrict__ hb = h + (size_t)bf * Lp;
            T v[G], xa[G], xb[G];
#pragma unroll
            for (int e = 0; e < G; ++e) {
                v[e] = J[r0[e] - kf];
                xa[e] = ha[idx[e]];
                xb[e] = hb[idx[e]];
            }
#pragma unroll
            for (int e = 0; e < G; ++e) {
                ha[idx[e]] = xa[e] - v[e];
                hb[idx[e]] = xb[e] + v[e];
            }
        }
    }
    for (; j < m; j += nw) {
        const int i = j < x0 ? j : j + nx;
        for (int f = 0; f < nf; ++f) {
            const int kf = pk[f], af = pab[f] >> 8, bf = pab[f] & 255;
            int r = lo + i - kf;
            r += r < 0 ? L : 0;
            const T v = J[r];
            h[(size_t)af * Lp + i] -= v;
            h[(size_t)bf * Lp + i] += v;
        }
    }
}

// One cluster of C CTAs per work item (blockIdx.x / C); nsweeps sweeps.
template <typename T, int C>
__global__ void __launch_bounds__(kClThreads, 1) sweep_cluster_kernel(const JobDev* __restrict__ jobs,
                                                                      const int2* __restrict__ work, int nsweeps)
{
    constexpr bool kFP64 = sizeof(T) == 8;  // the FP64 rule (FP64 and FX64 fields)
    constexpr bool kFX = kFP64 && !std::is_floating_point<T>::value;
    constexpr int kMode = kFX ? 2 : (kFP64 ? 1 : 0);
    extern __shared__ __align__(16) unsigned char smem[];
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int2 wk = work[blockIdx.x / C];
    const JobDev* jp = jobs + wk.x;
    const int t = wk.y;
    const int L = jp->L, q = jp->q, Lpad = jp->Lpad, W = jp->W, c = jp->c;
    const uint32_t key0 = jp->key0, key1 = jp->key1;
    const int rep = jp->map[t];
    const double beta = jp->beta[t];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const ClLayout lay(L, q, C, (int)sizeof(T));
    const int Lp = lay.Lp, P = Lp / kSiteBlock;
    const int lo = rank * Lp;
    const int n = max(0, min(L, lo + Lp) - lo);  // sites held here

    // the doubled coupling table of the field type (J[m] = J*(m mod L), m < 2L)
    const T* __restrict__ J = kFX     ? (const T*)(const void*)jp->Jfxd
                              : kFP64 ? (const T*)(const void*)jp->J64d
                                      : (const T*)(const void*)jp->J32d;
    T* __restrict__ hg = (T*)jp->fields + (size_t)rep * q * Lpad;
    uint32_t* __restrict__ spins = jp->spins + (size_t)rep * W;
    double* dacc = (double*)(smem + lay.o_dacc);
    int* lk = (int*)(smem + lay.o_lk);
    int* lab = (int*)(smem + lay.o_lab);
    int* lcnt = (int*)(smem + lay.o_lcnt);
    float* Jn = (float*)(smem + lay.o_jn);
    T* h = (T*)(smem + lay.o_h);
    uint8_t* s = smem + lay.o_s;

    for (int x = 0; x < q; ++x)
        for (int j = tid; j < n; j += kClThreads) h[(size_t)x * Lp + j] = hg[(size_t)x * Lpad + lo + j];
    for (int j = tid; j < n; j += kClThreads) {
        const int i = lo + j;
        s[j] = (uint8_t)((spins[i >> 3] >> (4 * (i & 7))) & 15u);
    }
    if (tid < kNearTable) Jn[tid] = tid < L ? (float)jp->J64d[tid] : 0.0f;
    if (tid < 2) lcnt[tid] = 0;
    // every CTA initialised before any flip list arrives from another
    cluster_barrier();

    const uint32_t n0 = jp->nsweep[t];
    const double cb64 = beta * (double)c;
    const float cb32 = (float)cb64;
    const float errd = kFP64 ? (float)(2.4e-5 * jp->jtot) : 0.0f;  // FP32 screen margin of the FP64 rule
    const double fxs = kFX ? jp->fx_scale : 1.0;                    // FX64: value of one field unit
    const float fxs32 = (float)fxs;                                 // a power of two: exact
    const int nblk = (L + kSiteBlock - 1) / kSiteBlock;
    const int total = nsweeps * nblk;
    double dE_acc = 0.0;  // FP32: warp 0 of the owning CTA: energy change of this lane's flips, in block order
    unsigned long long nacc = 0;
    unsigned long long nnear = 0;

    for (int g = 0; g <= total; ++g) {
        const int pb = (g + 1) & 1;  // list of block g-1 (pending)
        const int npend = g > 0 ? lcnt[pb] : 0;
        const int* pk = lk + pb * kSiteBlock;
        const int* pab = lab + pb * kSiteBlock;
        const int blk = g < total ? g % nblk : 0;
        const int owner = g < total ? blk / P : -1;
        const int k0 = blk * kSiteBlock;
        const int nv = g < total ? min(kSiteBlock, L - k0) : 0;

        if (warp == 0) {
            if (owner == rank) {
                // the lane sums arrive with the first block this CTA owns in a run
                if (!kFP64 && g > 0 && ((g - 1) % nblk) / P != rank) dE_acc = dacc[lane];
                const int k = k0 + lane;
                const int kl = k - lo;
                const bool valid = lane < nv;
                const uint32_t nsw = n0 + (uint32_t)(g / nblk);
                int a = 0, b = 0;
                float nlu = 0.0f, d32 = 0.0f;
                double base = 0.0;
                long long basefx = 0;
                uint32_t ux1 = 0, ux2 = 0;
                if (valid) {
                    a = s[kl];
                    draw_proposal<kFP64>(k, t, nsw, key0, key1, q, a, b, nlu, ux1, ux2);
                    const T dd = h[(size_t)a * Lp + kl] - h[(size_t)b * Lp + kl];
                    if constexpr (kFX) {
                        basefx = (long long)dd;
                        d32 = (float)dd * fxs32;
                    } else {
                        base = (double)dd;
                        d32 = (float)dd;
                    }
                }
                const int cbuf = g & 1;
                int* ck = lk + cbuf * kSiteBlock;
                int* cab = lab + cbuf * kSiteBlock;
                bool mine;
                float dmine;
                const int nf = decide_block<kMode>(lane, nv, k, L, a, b, nlu, ux1, ux2, d32, base, pk, pab, npend,
                                                   cb32, cb64, errd, Jn,
                                                   kMode == 1 ? (const double*)(const void*)J : nullptr, ck, cab,
                                                   mine, dmine, nnear, basefx,
                                                   kFX ? (const long long*)(const void*)J : nullptr, fxs,
                                                   NearSink{jp->near_log, jp->near_log_n, t, nsw});
                if (mine) {
                    s[kl] = (uint8_t)b;
                    if constexpr (!kFP64) dE_acc += (double)((float)c * dmine);
                }
                if (lane == 0) {
                    lcnt[cbuf] = nf;
                    nacc += (unsigned long long)nf;
                }
                // the block's flips to every other CTA of the cluster
                for (int r = 0; r < C; ++r) {
                    if (r == rank) continue;
                    int* rk = cl.map_shared_rank(ck, r);
                    int* rab = cl.map_shared_rank(cab, r);
                    if (lane < nf) {
                        rk[lane] = ck[lane];
                        rab[lane] = cab[lane];
                    }
                    if (lane == 0) cl.map_shared_rank(lcnt, r)[cbuf] = nf;
                }
                // FP32: hand the lane sums on when the next block belongs to another CTA
                if (!kFP64 && g + 1 < total && ((g + 1) % nblk) / P != rank)
                    cl.map_shared_rank(dacc, ((g + 1) % nblk) / P)[lane] = dE_acc;
                // bring the block's own sites up to date with block g-1's flips
                if (valid) {
                    for (int f = 0; f < npend; ++f) {
                        const int kf = pk[f], af = pab[f] >> 8, bf = pab[f] & 255;
                        int r = k - kf;
                        r += r < 0 ? L : 0;
                        const T v = J[r];
                        h[(size_t)af * Lp + kl] -= v;
                        h[(size_t)bf * Lp + kl] += v;
                    }
                }
            }
        } else if (npend > 0) {
            // block g-1's flips on this CTA's sites, except the block being decided here
            const bool here = owner == rank;
            apply_flips_part<T>(h, Lp, lo, n, J, L, pk, pab, npend, here ? k0 - lo : 0, here ? nv : 0, tid - 32);
        }
        cluster_barrier();
    }

    // write back this CTA's sites (whole packed words: lo is a multiple of 32)
    for (int w = tid; w < (n + 7) / 8; w += kClThreads) {
        uint32_t word = 0;
        for (int m = 0; m < 8; ++m) {
            const int j = 8 * w + m;
            if (j < n) word |= (uint32_t)s[j] << (4 * m);
        }
        spins[lo / 8 + w] = word;
    }
    for (int x = 0; x < q; ++x)
        for (int j = tid; j < n; j += kClThreads) hg[(size_t)x * Lpad + lo + j] = h[(size_t)x * Lp + j];
    if constexpr (!kFP64) {
        if (warp == 0 && total > 0 && (nblk - 1) / P == rank) {
            // this CTA decided the last block: it holds the lane sums
            for (int o = 16; o > 0; o >>= 1) dE_acc += __shfl_xor_sync(kFullMask, dE_acc, o);
            if (lane == 0) jp->E[rep] += dE_acc;
        }
    }
    if (tid == 0) {
        if (rank == 0) jp->nsweep[t] = n0 + (uint32_t)nsweeps;
        if (nacc) atomicAdd(&jp->acc_flip[t], nacc);
        if (nnear) atomicAdd(&jp->near[0], nnear);
    }
    if constexpr (kFP64) {
        // E = -(c/2) sum_i h[s_i][i] over the whole chain, by CTA 0 from what
        // the cluster wrote back: the same strands and order as the single-CTA
        // kernel (FP64), or exact (FX64)
        __threadfence();
        cluster_barrier();
        if (rank == 0) {
            const uint32_t* sp = spins;
            double* red = (double*)(smem + lay.o_dacc);  // 32 words, free now
            if constexpr (kFX) {
                unsigned long long lo2 = 0, hi2 = 0;
                for (int i = tid; i < L; i += kClThreads) {
                    const int si = (int)((__ldcg(sp + (i >> 3)) >> (4 * (i & 7))) & 15u);
                    u128_add(lo2, hi2, (unsigned long long)__ldcg(hg + (size_t)si * Lpad + i));
                }
                const double Efx = block_sum_u128(lo2, hi2, (unsigned long long*)red);
                if (tid == 0) jp->E[rep] = -0.5 * (double)c * Efx * fxs;
            } else {
                double part = 0.0;
                if (tid < kSweepThreads)
                    for (int i = tid; i < L; i += kSweepThreads) {
                        const int si = (int)((__ldcg(sp + (i >> 3)) >> (4 * (i & 7))) & 15u);
                        part += (double)__ldcg(hg + (size_t)si * Lpad + i);
                    }
                for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(kFullMask, part, o);
                if (lane == 0 && warp < kSweepThreads / 32) red[warp] = part;
                __syncthreads();
                if (tid == 0) {
                    double tot = 0.0;
                    for (int w = 0; w < kSweepThreads / 32; ++w) tot += red[w];
                    jp->E[rep] = -0.5 * (double)c * tot;
                }
            }
        }
    }
}

template <typename T, int C>
cudaError_t launch_c(const JobDev* jobs_dev, const int2* work, int nwork, int nsweeps, size_t smem,
                     const SweepSched* sched, cudaStream_t st)
{
    auto k = sweep_cluster_kernel<T, C>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(nwork * C));
    cfg.blockDim = dim3(kClThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const int2* items = work;
    if ((e = cluster_plan((const void*)k, cfg, nwork, sched, jobs_dev, work, &items, st)) != cudaSuccess) return e;
    return cudaLaunchKernelEx(&cfg, k, jobs_dev, items, nsweeps);
}

template <typename T>
cudaError_t launch_t(int C, const JobDev* jobs_dev, const int2* work, int nwork, int nsweeps, size_t smem,
                     const SweepSched* sched, cudaStream_t st)
{
    switch (C) {
    case 2: return launch_c<T, 2>(jobs_dev, work, nwork, nsweeps, smem, sched, st);
    case 4: return launch_c<T, 4>(jobs_dev, work, nwork, nsweeps, smem, sched, st);
    case 8: return launch_c<T, 8>(jobs_dev, work, nwork, nsweeps, smem, sched, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

size_t cluster_sweep_smem(int L, int q, int C, int precision)
{
    return ClLayout(L, q, C, precision == kPrecFP32 ? 4 : 8).bytes;
}

int cluster_size_for(int L, int q, size_t budget, int precision)
{
    for (int C = 2; C <= 8; C *= 2)
        if (cluster_sweep_smem(L, q, C, precision) <= budget) return C;
    return 0;
}

cudaError_t launch_sweep_cluster(int C, int precision, const JobDev* jobs_dev, const int2* work, int nwork,
                                 int nsweeps, size_t smem, const SweepSched* sched, cudaStream_t st)
{
    if (nwork <= 0 || nsweeps <= 0) return cudaSuccess;
    switch (precision) {
    case kPrecFP32: return launch_t<float>(C, jobs_dev, work, nwork, nsweeps, smem, sched, st);
    case kPrecFP64: return launch_t<double>(C, jobs_dev, work, nwork, nsweeps, smem, sched, st);
    case kPrecFX64: return launch_t<long long>(C, jobs_dev, work, nwork, nsweeps, smem, sched, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace plr
