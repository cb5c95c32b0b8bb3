// Register-resident Metropolis sweep of a long chain over a thread-block
// cluster (Eq. 8, Sec. 4.2): the fields of one slot held in the registers of
// the update warps of C CTAs (C = 2, 4 or 8), FP32 (T = float) or FX64
// (T = long long, the FP64 rule's decisions).
//
// It joins the two designs beside it.  As in the register sweep
// (sweep_rf.cuh), update thread u of a CTA keeps the fields of its E sites for
// all Q states in registers and applies a flip a -> b with two warp-uniform
// switches, and a dedicated decision warp decides the 32 sites of a block
// from field values published by the block's owner warp one phase earlier
// (the block's pending flips added as corrections).  As in the shared-memory
// cluster sweep (sweep_cluster.cu), CTA r holds the contiguous sites
// [r S, (r + 1) S), S = 32 E NU, the CTA holding a block decides it, and the
// accepted flips travel to every CTA's flip list through distributed shared
// memory; one cluster barrier ends each block.  The register form costs an
// update thread one coupling load and two adds per site and flip, where the
// shared-memory form pays loads and stores of both field rows as well.
//
// Phase g: the decision warp of the CTA holding block g decides it and sends
// its flips; the update warps of every CTA apply block g-1's flips to their
// registers; the warp holding block g+1 publishes that block's field values
// (not yet holding block g's flips) and draws its proposals.  The FP32
// energy change is accumulated per lane of the deciding warps in block order
// and handed to the next holder's shared memory when a block's holder
// changes; FX64 energies are recomputed after the sweep, exactly, from what
// the cluster wrote back.  Every field element receives the same updates in
// the same order as in the other kernels of its precision, and the decisions
// and energies are the same, so results are bit-identical to theirs.
#pragma once
#include <cooperative_groups.h>

#include "sweep_rf.cuh"

namespace plr {
namespace rfc {

namespace cg = cooperative_groups;

constexpr int NU = 15;                  // update warps per CTA; warp NU decides
constexpr int kThreads = 32 * (NU + 1);
constexpr int NUT = 32 * NU;

__device__ __forceinline__ void cluster_sync_all()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// FP32 clusters of 2 or 4 CTAs keep their shifted coupling table as pairs
// (J*((lo + y) mod L), J*((lo + y + NUT) mod L)) -- see rf::rf_pair_table;
// at 8 CTAs (L above 4 x 4320) the pairs would not fit
template <typename T, int E, int C>
__host__ __device__ constexpr bool rfc_pair_table()
{
    return rf::rf_paired<T, E, NU>() && C <= 4;
}

// carve-up of the dynamic shared memory (must match the kernel)
template <typename T, int Q, int E, int C>
struct RfcLayout {
    size_t o_j, o_s, o_lk, o_lab, o_lcnt, o_jn, o_del, o_dacc, o_hv, o_pab, o_pnlu, o_pux, bytes;
    __host__ __device__ RfcLayout(int L)
    {
        size_t o = 0;
        o_j = o;     // J*((lo + y) mod L), y < E NUT + L (pairs: rfc_pair_table)
        o += (size_t)(E * NUT + L) * (rfc_pair_table<T, E, C>() ? 8 : sizeof(T));
        o = (o + 15) & ~(size_t)15;
        o_s = o;     // spins of this CTA's sites
        o += (size_t)E * NUT;
        o = (o + 15) & ~(size_t)15;
        o_lk = o;    // [2][32] flip sites
        o += 2 * kSiteBlock * sizeof(int);
        o_lab = o;   // [2][32] (a << 8) | b
        o += 2 * kSiteBlock * sizeof(int);
        o_lcnt = o;  // [2] flip counts (+ padding)
        o += 16;
        o_jn = o;    // J*(r), r < 64, FP32
        o += kNearTable * sizeof(float);
        o_del = o;   // [32] double: lane energy sums of this CTA's decisions
        o += 32 * sizeof(double);
        o_dacc = o;  // [32] double: lane sums handed over by the previous holder
        o += 32 * sizeof(double);
        o_hv = o;    // [2][Q][32] published field values
        o += 2 * Q * kSiteBlock * sizeof(T);
        o_pab = o;   // [2][32] proposals
        o += 2 * kSiteBlock * sizeof(int);
        o_pnlu = o;  // [2][32] -ln u
        o += 2 * kSiteBlock * sizeof(float);
        o_pux = o;   // [2][2][32] the words of u (FP64 rule)
        o += 4 * kSiteBlock * sizeof(uint32_t);
        bytes = (o + 15) & ~(size_t)15;
    }
};

// One cluster of C CTAs per work item (blockIdx.x / C); nsweeps sweeps.
template <typename T, int Q, int E, int C>
__global__ void __launch_bounds__(kThreads, 1) sweep_rfc_kernel(const JobDev* __restrict__ jobs,
                                                                const int2* __restrict__ work, int nsweeps)
{
    constexpr bool kFX = sizeof(T) == 8;  // FX64 fields: the FP64 rule
    constexpr int S = E * NUT;            // sites per CTA
    constexpr int PB = E * NU;            // blocks per CTA
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
    const bool decider = warp == NU;
    const int lo = rank * S;
    const int n = max(0, min(L, lo + S) - lo);  // sites held here

    constexpr bool PT = rfc_pair_table<T, E, C>();
    const RfcLayout<T, Q, E, C> lay(L);
    T* J2 = (T*)(smem + lay.o_j);
    uint8_t* s = smem + lay.o_s;
    int* lk = (int*)(smem + lay.o_lk);
    int* lab = (int*)(smem + lay.o_lab);
    int* lcnt = (int*)(smem + lay.o_lcnt);
    float* Jn = (float*)(smem + lay.o_jn);
    double* dEl = (double*)(smem + lay.o_del);
    double* dacc = (double*)(smem + lay.o_dacc);
    T* hv = (T*)(smem + lay.o_hv);
    int* pab = (int*)(smem + lay.o_pab);
    float* pnlu = (float*)(smem + lay.o_pnlu);
    uint32_t* pux = (uint32_t*)(smem + lay.o_pux);

    T* __restrict__ hg = (T*)jp->fields + (size_t)rep * q * Lpad;
    uint32_t* __restrict__ spins = jp->spins + (size_t)rep * W;
    const T* __restrict__ Jsrc = kFX ? (const T*)(const void*)jp->Jfxd : (const T*)(const void*)jp->J32d;

    // the coupling of local site y (site lo + y) to a flip at k is
    // J2[y - k + L] = J*((lo + y - k) mod L): a table shifted by lo
    if constexpr (PT) {
        float2* JP = reinterpret_cast<float2*>(J2);
        for (int m = tid; m < S + L; m += kThreads)
            JP[m] = make_float2(Jsrc[(lo + m) % L], Jsrc[(lo + m + NUT) % L]);
    } else {
        for (int m = tid; m < S + L; m += kThreads) J2[m] = Jsrc[(lo + m) % L];
    }
    for (int y = tid; y < S; y += kThreads) {
        const int i = lo + y;
        s[y] = y < n ? (uint8_t)((spins[i >> 3] >> (4 * (i & 7))) & 15u) : (uint8_t)0;
    }
    if (tid < kNearTable) Jn[tid] = tid < L ? (float)jp->J64d[tid] : 0.0f;
    if (tid < 32) dEl[tid] = 0.0;
    if (tid < 2) lcnt[tid] = 0;
    T h[E][Q];
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const int y = m * NUT + tid;
#pragma unroll
        for (int x = 0; x < Q; ++x) h[m][x] = (!decider && y < n) ? hg[(size_t)x * Lpad + lo + y] : (T)0;
    }

    const uint32_t n0 = jp->nsweep[t];
    const double cb64 = beta * (double)c;
    const float cb32 = (float)cb64;
    const float errd = kFX ? (float)(2.4e-5 * jp->jtot) : 0.0f;  // FP32 screen margin of the FP64 rule
    const double fxs = kFX ? jp->fx_scale : 1.0;
    const float fxs32 = (float)fxs;
    unsigned long long nacc = 0, nnear = 0;
    const int nblk = (L + kSiteBlock - 1) / kSiteBlock;  // >= 2 (the host checks)
    const int total = nsweeps * nblk;

    // block g of the sweep sequence: its holder, local block, global first site
    auto holder = [&](int g) { return (g % nblk) / PB; };
    // proposals of block g (held here) into buffer g & 1 (one warp)
    auto draw_block = [&](int g) {
        const int blk = g % nblk;
        const int k = blk * kSiteBlock + lane;
        const int kl = k - lo;
        int a = 0, b = 0;
        float nlu = 0.0f;
        uint32_t ux1 = 0, ux2 = 0;
        if (k < L) {
            a = s[kl];
            draw_proposal<kFX>(k, t, n0 + (uint32_t)(g / nblk), key0, key1, q, a, b, nlu, ux1, ux2);
        }
        pab[(g & 1) * kSiteBlock + lane] = (a << 8) | b;
        pnlu[(g & 1) * kSiteBlock + lane] = nlu;
        if constexpr (kFX) {
            pux[(g & 1) * 2 * kSiteBlock + lane] = ux1;
            pux[(g & 1) * 2 * kSiteBlock + kSiteBlock + lane] = ux2;
        }
    };
    // field values and proposals of block g into buffer g & 1 (its owner warp, here)
    auto publish_block = [&](int g) {
        const int lb = g % nblk - rank * PB;
        if (warp == lb % NU) {
            rf::publish_row<T, Q, E>(h, lb / NU, hv + (g & 1) * Q * kSiteBlock, lane);
            draw_block(g);
        }
    };

    if (total > 0 && !decider && holder(0) == rank) publish_block(0);
    // every CTA initialised before any flip list arrives from another
    cluster_sync_all();

    for (int g = 0; g <= total; ++g) {
        const int pb = (g + 1) & 1;  // block g-1's list
        const int npend = g > 0 ? lcnt[pb] : 0;
        const int* pk = lk + pb * kSiteBlock;
        const int* pl = lab + pb * kSiteBlock;
        if (decider) {
            if (g < total && holder(g) == rank) {
                const int cb = g & 1;
                const int k0 = (g % nblk) * kSiteBlock;
                const int nv = min(kSiteBlock, L - k0);
                const int k = k0 + lane;
                const bool valid = lane < nv;
                // FP32: the lane sums arrive with the first block this CTA holds in a run
                if (!kFX && g > 0 && holder(g - 1) != rank) dEl[lane] = dacc[lane];
                const int ab = pab[cb * kSiteBlock + lane];
                const int a = ab >> 8, b = ab & 255;
                const float nlu = pnlu[cb * kSiteBlock + lane];
                float d32 = 0.0f;
                long long dfx = 0;
                if (valid) {
                    const T* hvb = hv + cb * Q * kSiteBlock;
                    const T dd = hvb[a * kSiteBlock + lane] - hvb[b * kSiteBlock + lane];
                    if constexpr (kFX) {
                        dfx = (long long)dd;
                        d32 = (float)dd * fxs32;
                    } else {
                        d32 = (float)dd;
                    }
                }
                int* ck = lk + cb * kSiteBlock;
                int* cab = lab + cb * kSiteBlock;
                bool mine;
                float dmine;
                int nf;
                if constexpr (kFX) {
                    const uint32_t ux1 = pux[cb * 2 * kSiteBlock + lane];
                    const uint32_t ux2 = pux[cb * 2 * kSiteBlock + kSiteBlock + lane];
                    // the exact path's couplings by distance, from the global doubled table
                    nf = decide_block<2>(lane, nv, k, L, a, b, nlu, ux1, ux2, d32, 0.0, pk, pl, npend, cb32, cb64,
                                         errd, Jn, nullptr, ck, cab, mine, dmine, nnear, dfx, jp->Jfxd, fxs,
                                         NearSink{jp->near_log, jp->near_log_n, t, n0 + (uint32_t)(g / nblk)});
                } else {
                    nf = decide_block<0>(lane, nv, k, L, a, b, nlu, 0u, 0u, d32, 0.0, pk, pl, npend, cb32, cb64,
                                         0.0f, Jn, nullptr, ck, cab, mine, dmine, nnear);
                }
                if (mine) {
                    s[k - lo] = (uint8_t)b;
                    if constexpr (!kFX) dEl[lane] += (double)((float)c * dmine);
                }
                if (lane == 0) {
                    lcnt[cb] = nf;
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
                    if (lane == 0) cl.map_shared_rank(lcnt, r)[cb] = nf;
                }
                // FP32: hand the lane sums on when the next block is held elsewhere
                if (!kFX && g + 1 < total && holder(g + 1) != rank)
                    cl.map_shared_rank(dacc, holder(g + 1))[lane] = dEl[lane];
            }
        } else {
            rf::apply_rows<T, Q, E, NU, PT>(h, J2, tid, L, pk, pl, npend);
            if (g + 1 < total && holder(g + 1) == rank) publish_block(g + 1);
        }
        cluster_sync_all();
    }

    // write back this CTA's sites (whole packed words: lo is a multiple of 32)
    for (int w = tid; w < (n + 7) / 8; w += kThreads) {
        uint32_t word = 0;
        for (int m = 0; m < 8; ++m) {
            const int y = 8 * w + m;
            if (y < n) word |= (uint32_t)s[y] << (4 * m);
        }
        spins[lo / 8 + w] = word;
    }
    if (!decider) {
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int y = m * NUT + tid;
            if (y < n) {
#pragma unroll
                for (int x = 0; x < Q; ++x) hg[(size_t)x * Lpad + lo + y] = h[m][x];
            }
        }
    }
    if (decider) {
        for (int o = 16; o > 0; o >>= 1) nnear += __shfl_xor_sync(kFullMask, nnear, o);
        if (lane == 0) {
            if (nacc) atomicAdd(&jp->acc_flip[t], nacc);
            if (nnear) atomicAdd(&jp->near[0], nnear);
        }
        if constexpr (!kFX) {
            // the CTA that decided the last block holds the lane sums
            if (total > 0 && holder(total - 1) == rank) {
                double dE = dEl[lane];
                for (int o = 16; o > 0; o >>= 1) dE += __shfl_xor_sync(kFullMask, dE, o);
                if (lane == 0) jp->E[rep] += dE;
            }
        }
    }
    if (tid == 0 && rank == 0) jp->nsweep[t] = n0 + (uint32_t)nsweeps;
    if constexpr (kFX) {
        // E = -(c/2) sum_i h[s_i][i], exactly, by CTA 0 from what the cluster wrote back
        __threadfence();
        cluster_sync_all();
        if (rank == 0) {
            unsigned long long lo2 = 0, hi2 = 0;
            for (int i = tid; i < L; i += kThreads) {
                const int si = (int)((__ldcg(spins + (i >> 3)) >> (4 * (i & 7))) & 15u);
                u128_add(lo2, hi2, (unsigned long long)__ldcg(hg + (size_t)si * Lpad + i));
            }
            const double Efx = block_sum_u128(lo2, hi2, (unsigned long long*)dEl);
            if (tid == 0) jp->E[rep] = -0.5 * (double)c * Efx * fxs;
        }
    }
}

template <typename T, int Q, int E, int C>
cudaError_t launch_rfc(const JobDev* jobs_dev, const int2* work, int nwork, int nsweeps, size_t smem,
                       const SweepSched* sched, cudaStream_t st)
{
    auto k = sweep_rfc_kernel<T, Q, E, C>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(nwork * C));
    cfg.blockDim = dim3(kThreads);
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

// dispatch over Q (QMIN..QMAX, within 2..12) and C (2, 4, 8) for one field type and E
template <typename T, int E, int QMIN, int QMAX>
cudaError_t launch_rfc_qc(int q, int C, const JobDev* jobs_dev, const int2* work, int nwork, int nsweeps,
                          size_t smem, const SweepSched* sched, cudaStream_t st)
{
    switch (q * 16 + C) {
#define PLR_RFC(Qv, Cv)                                                                             \
    case Qv * 16 + Cv:                                                                              \
        if constexpr (Qv >= QMIN && Qv <= QMAX)                                                     \
            return launch_rfc<T, Qv, E, Cv>(jobs_dev, work, nwork, nsweeps, smem, sched, st);        \
        break;
#define PLR_RFC_Q(Qv) PLR_RFC(Qv, 2) PLR_RFC(Qv, 4) PLR_RFC(Qv, 8)
        PLR_RFC_Q(2) PLR_RFC_Q(3) PLR_RFC_Q(4) PLR_RFC_Q(5) PLR_RFC_Q(6) PLR_RFC_Q(7) PLR_RFC_Q(8)
        PLR_RFC_Q(9) PLR_RFC_Q(10) PLR_RFC_Q(11) PLR_RFC_Q(12)
#undef PLR_RFC_Q
#undef PLR_RFC
    default: break;
    }
    return cudaErrorNotSupported;
}

template <typename T, int E, int QMIN, int QMAX>
size_t rfc_smem_q(int q, int C, int L)
{
    switch (q * 16 + C) {
#define PLR_RFC_S(Qv, Cv) \
    case Qv * 16 + Cv: return (Qv >= QMIN && Qv <= QMAX) ? RfcLayout<T, Qv, E, Cv>(L).bytes : 0;
#define PLR_RFC_SQ(Qv) PLR_RFC_S(Qv, 2) PLR_RFC_S(Qv, 4) PLR_RFC_S(Qv, 8)
        PLR_RFC_SQ(2) PLR_RFC_SQ(3) PLR_RFC_SQ(4) PLR_RFC_SQ(5) PLR_RFC_SQ(6) PLR_RFC_SQ(7) PLR_RFC_SQ(8)
        PLR_RFC_SQ(9) PLR_RFC_SQ(10) PLR_RFC_SQ(11) PLR_RFC_SQ(12)
#undef PLR_RFC_SQ
#undef PLR_RFC_S
    default: return 0;
    }
}

}  // namespace rfc
}  // namespace plr
