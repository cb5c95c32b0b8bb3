// Register-resident Metropolis sweep (Eq. 8, Sec. 4.2 of the paper), FP32
// fields (T = float) or FX64 fields (T = long long: 64-bit integers in units
// of 2^-F, exact integer updates, the FP64 rule's decisions).
//
// One CTA sweeps one temperature slot at a time: NU update warps hold the local fields
// h[x][i] of their sites in registers, one decision warp holds none.  Update
// thread u (0 <= u < 32 NU) keeps sites i = m 32 NU + u (m = 0..E-1) for all Q
// states, so an accepted flip (a -> b at site k) costs it two warp-uniform
// switches, h[a][i] -= J*((i-k) mod L) and h[b][i] += J*(...), and one
// shared-memory read of J* per site; the fields never travel through shared
// memory.  Sites are decided in blocks of 32 (block g: sites 32 g .. 32 g + 31,
// held by update warp g mod NU in register row g / NU).  In phase g:
//   - the decision warp reads block g's proposals and field values (published
//     during phase g-1, not yet holding block g-1's flips), decides block g with
//     the in-order scan of sweep_common.cuh (which adds block g-1's flips as
//     corrections) and publishes the accepted flips;
//   - every update warp applies block g-1's flips to its registers; the owner
//     of block g+1 then publishes that block's field values and draws its
//     proposals.
// One CTA barrier per block; deciding and updating overlap.
//
// The arithmetic is that of the shared-memory kernel -- the same values J*,
// the same subtractions and additions in flip order, the same decisions and
// (FP32) the same grouping of the energy sum, (FX64) the same exact integer
// energy sum -- so both give identical results.  FX64 decisions take the FP64
// rule through decide_block<2>: the FP32 screen, and where it cannot tell,
// the exact integer difference converted to FP64 once.
#pragma once
#include "sweep_common.cuh"
#include "sweep_sched.cuh"

namespace plr {
namespace rf {

// FP32 fields in 512-thread CTAs apply flips to pairs of a thread's sites
// (m, m+1) with packed two-lane adds (measured faster there; the 256-thread
// configurations have no registers to spare for the packing) ...
template <typename T, int E, int NU>
__host__ __device__ constexpr bool rf_paired()
{
    return sizeof(T) == 4 && NU >= 15 && E >= 2;
}
// ... and, where it fits beside the rest of the shared memory (up to 26
// sites per thread), take both couplings of a pair in one 64-bit load from a
// table of pairs (J*(i), J*(i + 32 NU)): sites m and m+1 of a thread lie 32 NU
// apart, so the pair's index is that of site m.
template <typename T, int E, int NU>
__host__ __device__ constexpr bool rf_pair_table()
{
    return rf_paired<T, E, NU>() && E <= 26;
}

template <typename T, int NU, int E, int Q>
struct RfSmem {
    // J*(m mod L), m < E 32 NU + L (as pairs with J*((m + 32 NU) mod L) when
    // rf_pair_table); the kernel's carve-up takes its size from here too
    __host__ __device__ static size_t table_bytes(int L)
    {
        return (size_t)(E * 32 * NU + L) * (rf_pair_table<T, E, NU>() ? 8 : sizeof(T));
    }
    static size_t bytes(int L, int Lpad)
    {
        size_t b = table_bytes(L);
        b += (size_t)Lpad;                                   // spins
        b = (b + 15) & ~(size_t)15;
        b += 2 * 2 * kSiteBlock * sizeof(int);   // double-buffered flip lists
        b += kNearTable * sizeof(float);         // J*(r), r < 64
        b += 32 * sizeof(double);                // per-lane energy change
        b += 2 * Q * kSiteBlock * sizeof(T);     // published field values, double-buffered
        b += 2 * kSiteBlock * sizeof(int);       // proposals (a << 8 | b), double-buffered
        b += 2 * kSiteBlock * sizeof(float);     // -ln u, double-buffered
        b += 2 * 2 * kSiteBlock * sizeof(uint32_t);  // the words u is made of (FP64 rule), double-buffered
        b += 16;                                 // flip counts
        return (b + 15) & ~(size_t)15;
    }
};

#define PLR_RF_CASE(c, OP)                                                              \
    case c:                                                                             \
        if constexpr ((c) < Q) {                                                        \
            _Pragma("unroll") for (int m = 0; m < E; ++m) h[m][c] OP v[m];              \
        }                                                                               \
        break;

// Two FP32 values in one 64-bit register, for the packed two-lane adds of
// sm_100-class GPUs (add/sub.rn.f32x2: each half rounds as a scalar add).
__device__ __forceinline__ unsigned long long pack_f32x2(float lo, float hi)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void unpack_f32x2(unsigned long long p, float& lo, float& hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(p));
}

// FP32 rows, sites m and m+1 of the thread paired: one packed add or subtract
// applies a flip to both (an odd last site takes a scalar one)
#define PLR_RF2_CASE(c, PTX, OP)                                                       \
    case c:                                                                            \
        if constexpr ((c) < Q) {                                                       \
            _Pragma("unroll") for (int m = 0; m + 1 < E; m += 2) {                     \
                unsigned long long hp = pack_f32x2(h[m][c], h[m + 1][c]);              \
                asm(PTX " %0, %0, %1;" : "+l"(hp) : "l"(vv[m / 2]));                    \
                unpack_f32x2(hp, h[m][c], h[m + 1][c]);                                \
            }                                                                          \
            if constexpr (E & 1) h[E - 1][c] OP vl;                                    \
        }                                                                              \
        break;
#define PLR_RF2_SWITCH(s, PTX, OP)                                                                          \
    switch (s) {                                                                                            \
        PLR_RF2_CASE(0, PTX, OP) PLR_RF2_CASE(1, PTX, OP) PLR_RF2_CASE(2, PTX, OP) PLR_RF2_CASE(3, PTX, OP)     \
        PLR_RF2_CASE(4, PTX, OP) PLR_RF2_CASE(5, PTX, OP) PLR_RF2_CASE(6, PTX, OP) PLR_RF2_CASE(7, PTX, OP)     \
        PLR_RF2_CASE(8, PTX, OP) PLR_RF2_CASE(9, PTX, OP) PLR_RF2_CASE(10, PTX, OP) PLR_RF2_CASE(11, PTX, OP)   \
        PLR_RF2_CASE(12, PTX, OP) PLR_RF2_CASE(13, PTX, OP) PLR_RF2_CASE(14, PTX, OP) PLR_RF2_CASE(15, PTX, OP) \
        default: break;                                                                                     \
    }

// PT: J2 is the table of pairs (rf_pair_table), else the plain shifted table
template <int Q, int E, int NU, bool PT>
__device__ __forceinline__ void apply_rows_paired(float (&h)[E][Q], const float* __restrict__ J2, int u, int L,
                                                  const int* pk, const int* pab, int nf)
{
    for (int f = 0; f < nf; ++f) {
        const int kf = pk[f], af = pab[f] >> 8, bf = pab[f] & 255;
        const int i0 = u - kf + L;  // the index of this thread's site 0
        unsigned long long vv[E / 2];
        float vl = 0.0f;  // the odd last site's coupling
        if constexpr (PT) {
            const float2* JP = reinterpret_cast<const float2*>(J2);
#pragma unroll
            for (int m = 0; m + 1 < E; m += 2) {
                const float2 p = JP[m * 32 * NU + i0];
                vv[m / 2] = pack_f32x2(p.x, p.y);
            }
            if constexpr (E & 1) vl = J2[2 * ((E - 1) * 32 * NU + i0)];
        } else {
#pragma unroll
            for (int m = 0; m + 1 < E; m += 2)
                vv[m / 2] = pack_f32x2(J2[m * 32 * NU + i0], J2[(m + 1) * 32 * NU + i0]);
            if constexpr (E & 1) vl = J2[(E - 1) * 32 * NU + i0];
        }
        PLR_RF2_SWITCH(af, "sub.rn.f32x2", -=)
        PLR_RF2_SWITCH(bf, "add.rn.f32x2", +=)
    }
}

#undef PLR_RF2_SWITCH
#undef PLR_RF2_CASE

// apply flips (pk, pab)[0..nf) to all register rows of update thread u; PT:
// J2 is the table of pairs (rf_pair_table)
template <typename T, int Q, int E, int NU, bool PT>
__device__ __forceinline__ void apply_rows(T (&h)[E][Q], const T* __restrict__ J2, int u, int L, const int* pk,
                                           const int* pab, int nf)
{
    if constexpr (rf_paired<T, E, NU>()) {
        apply_rows_paired<Q, E, NU, PT>(h, J2, u, L, pk, pab, nf);
    } else {
        for (int f = 0; f < nf; ++f) {
            const int kf = pk[f], af = pab[f] >> 8, bf = pab[f] & 255;
            T v[E];
    #pragma unroll
            for (int m = 0; m < E; ++m) v[m] = J2[m * 32 * NU + u - kf + L];
            switch (af) {
                PLR_RF_CASE(0, -=) PLR_RF_CASE(1, -=) PLR_RF_CASE(2, -=) PLR_RF_CASE(3, -=)
                PLR_RF_CASE(4, -=) PLR_RF_CASE(5, -=) PLR_RF_CASE(6, -=) PLR_RF_CASE(7, -=)
                PLR_RF_CASE(8, -=) PLR_RF_CASE(9, -=) PLR_RF_CASE(10, -=) PLR_RF_CASE(11, -=)
                PLR_RF_CASE(12, -=) PLR_RF_CASE(13, -=) PLR_RF_CASE(14, -=) PLR_RF_CASE(15, -=)
                default: break;
            }
            switch (bf) {
                PLR_RF_CASE(0, +=) PLR_RF_CASE(1, +=) PLR_RF_CASE(2, +=) PLR_RF_CASE(3, +=)
                PLR_RF_CASE(4, +=) PLR_RF_CASE(5, +=) PLR_RF_CASE(6, +=) PLR_RF_CASE(7, +=)
                PLR_RF_CASE(8, +=) PLR_RF_CASE(9, +=) PLR_RF_CASE(10, +=) PLR_RF_CASE(11, +=)
                PLR_RF_CASE(12, +=) PLR_RF_CASE(13, +=) PLR_RF_CASE(14, +=) PLR_RF_CASE(15, +=)
                default: break;
            }
        }
    }
}

#undef PLR_RF_CASE

// publish register row M (all states) of this lane: hv[x][lane] = h[M][x]
template <typename T, int Q, int E>
__device__ __forceinline__ void publish_row(const T (&h)[E][Q], int M, T* hv, int lane)
{
#pragma unroll
    for (int m = 0; m < E; ++m)
        if (m == M) {
#pragma unroll
            for (int x = 0; x < Q; ++x) hv[x * kSiteBlock + lane] = h[m][x];
        }
}

// CTAs per SM to aim for, holding the compiler to the matching register budget
template <typename T, int Q, int E, int NU>
constexpr int rf_min_blocks()
{
    constexpr int w = sizeof(T) / 4;  // registers per field value
    const int threads = 32 * (NU + 1);
    if (w * Q * E <= 25 && threads <= 256) return 4;  // fits 64 registers
    const int need = threads * (w * (Q * E + E) + 48);
    const int b = 65536 / need;
    return b < 1 ? 1 : (b > 4 ? 4 : b);
}

// nsweeps sweeps of one work item wk = (job, slot) by the whole CTA
template <typename T, int Q, int E, int NU>
__device__ __forceinline__ void rf_item(const JobDev* __restrict__ jobs, const int2 wk, int nsweeps,
                                        unsigned char* __restrict__ smem)
{
    constexpr bool kFX = sizeof(T) == 8;  // FX64 fields: the FP64 rule
    constexpr int NUT = 32 * NU;          // update threads
    const JobDev* jp = jobs + wk.x;
    const int t = wk.y;
    const int L = jp->L, q = jp->q, Lpad = jp->Lpad, W = jp->W, c = jp->c;
    const uint32_t key0 = jp->key0, key1 = jp->key1;
    const int rep = jp->map[t];
    const double beta = jp->beta[t];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool decider = warp == NU;
    T* __restrict__ hg = (T*)jp->fields + (size_t)rep * q * Lpad;
    uint32_t* __restrict__ spins = jp->spins + (size_t)rep * W;
    const T* __restrict__ Jsrc = kFX ? (const T*)(const void*)jp->Jfxd : (const T*)(const void*)jp->J32d;

    constexpr bool PT = rf_pair_table<T, E, NU>();
    T* J2 = (T*)smem;
    size_t off = RfSmem<T, NU, E, Q>::table_bytes(L);
    uint8_t* s = smem + off;
    off = (off + (size_t)Lpad + 15) & ~(size_t)15;
    int* lk = (int*)(smem + off);
    int* lab = lk + 2 * kSiteBlock;
    float* Jn = (float*)(lab + 2 * kSiteBlock);
    double* dEl = (double*)(Jn + kNearTable);
    T* hv = (T*)(dEl + 32);                 // [2][Q][32] published field values
    int* pab = (int*)(hv + 2 * Q * kSiteBlock);  // [2][32] proposals
    float* pnlu = (float*)(pab + 2 * kSiteBlock);
    uint32_t* pux = (uint32_t*)(pnlu + 2 * kSiteBlock);  // [2][2][32] words of u (FP64 rule)
    int* lcnt = (int*)(pux + 4 * kSiteBlock);

    if constexpr (PT) {
        float2* JP = reinterpret_cast<float2*>(J2);
        for (int m = tid; m < E * NUT + L; m += blockDim.x) JP[m] = make_float2(Jsrc[m % L], Jsrc[(m + NUT) % L]);
    } else {
        for (int m = tid; m < E * NUT + L; m += blockDim.x) J2[m] = Jsrc[m % L];
    }
    for (int i = tid; i < L; i += blockDim.x) s[i] = (uint8_t)((spins[i >> 3] >> (4 * (i & 7))) & 15u);
    if (tid < kNearTable) Jn[tid] = tid < L ? (float)jp->J64d[tid] : 0.0f;
    if (tid < 32) dEl[tid] = 0.0;
    if (tid < 2) lcnt[tid] = 0;
    T h[E][Q];
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const int i = m * NUT + tid;
#pragma unroll
        for (int x = 0; x < Q; ++x) h[m][x] = (!decider && i < L) ? hg[(size_t)x * Lpad + i] : (T)0;
    }
    __syncthreads();

    const uint32_t n0 = jp->nsweep[t];
    const double cb64 = beta * (double)c;
    const float cb32 = (float)cb64;
    const float errd = kFX ? (float)(2.4e-5 * jp->jtot) : 0.0f;  // FP32 screen margin of the FP64 rule
    const double fxs = kFX ? jp->fx_scale : 1.0;                  // value of one field unit
    const float fxs32 = (float)fxs;                               // a power of two: exact
    unsigned long long nacc = 0, nnear = 0;
    const int nblk = (L + kSiteBlock - 1) / kSiteBlock;
    const int total = nsweeps * nblk;

    // proposals of block g into buffer g & 1 (one warp)
    auto draw_block = [&](int g) {
        const int k = (g % nblk) * kSiteBlock + lane;
        int a = 0, b = 0;
        float nlu = 0.0f;
        uint32_t ux1 = 0, ux2 = 0;
        if (k < L) {
            a = s[k];
            draw_proposal<kFX>(k, t, n0 + (uint32_t)(g / nblk), key0, key1, q, a, b, nlu, ux1, ux2);
        }
        pab[(g & 1) * kSiteBlock + lane] = (a << 8) | b;
        pnlu[(g & 1) * kSiteBlock + lane] = nlu;
        if constexpr (kFX) {
            pux[(g & 1) * 2 * kSiteBlock + lane] = ux1;
            pux[(g & 1) * 2 * kSiteBlock + kSiteBlock + lane] = ux2;
        }
    };
    // field values and proposals of block g into buffer g & 1 (its owner warp)
    auto publish_block = [&](int g) {
        const int gb = g % nblk;
        if (warp == gb % NU) {
            publish_row<T, Q, E>(h, gb / NU, hv + (g & 1) * Q * kSiteBlock, lane);
            if (nblk > 1 || g == 0) draw_block(g);
        }
    };

    if (total > 0 && !decider) publish_block(0);
    __syncthreads();

    for (int g = 0; g <= total; ++g) {
        const int pb = (g + 1) & 1;  // block g-1's list
        const int npend = g > 0 ? lcnt[pb] : 0;
        const int* pk = lk + pb * kSiteBlock;
        const int* pl = lab + pb * kSiteBlock;
        if (decider) {
            if (g < total) {
                const int cb = g & 1;
                const int k0 = (g % nblk) * kSiteBlock;
                const int nv = min(kSiteBlock, L - k0);
                const int k = k0 + lane;
                const bool valid = lane < nv;
                if (nblk == 1 && g > 0) {  // one block per sweep: its proposals could not be drawn early
                    __syncwarp();
                    draw_block(g);
                    __syncwarp();
                }
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
                    const uint32_t ux1 = pux[cb * 2 * kSiteBlock + lane], ux2 = pux[cb * 2 * kSiteBlock + kSiteBlock + lane];
                    nf = decide_block<2>(lane, nv, k, L, a, b, nlu, ux1, ux2, d32, 0.0, pk, pl, npend, cb32, cb64,
                                         errd, Jn, nullptr, ck, cab, mine, dmine, nnear, dfx,
                                         (const long long*)(const void*)J2, fxs,
                                         NearSink{jp->near_log, jp->near_log_n, t, n0 + (uint32_t)(g / nblk)});
                } else {
                    nf = decide_block<0>(lane, nv, k, L, a, b, nlu, 0u, 0u, d32, 0.0, pk, pl, npend, cb32, cb64,
                                         0.0f, Jn, nullptr, ck, cab, mine, dmine, nnear);
                }
                if (mine) {
                    s[k] = (uint8_t)b;
                    if constexpr (!kFX) dEl[lane] += (double)((float)c * dmine);
                }
                if (lane == 0) {
                    lcnt[cb] = nf;
                    nacc += (unsigned long long)nf;
                }
            }
        } else {
            apply_rows<T, Q, E, NU, PT>(h, J2, tid, L, pk, pl, npend);
            if (g + 1 < total) publish_block(g + 1);
        }
        __syncthreads();
    }

    // write back
    for (int w = tid; w < W; w += blockDim.x) {
        uint32_t word = 0;
        for (int m = 0; m < 8; ++m) {
            const int i = 8 * w + m;
            if (i < L) word |= (uint32_t)s[i] << (4 * m);
        }
        spins[w] = word;
    }
    if (!decider) {
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int i = m * NUT + tid;
            if (i < L) {
#pragma unroll
                for (int x = 0; x < Q; ++x) hg[(size_t)x * Lpad + i] = h[m][x];
            }
        }
    }
    if constexpr (kFX) {
        // E = -(c/2) sum_i h[s_i][i], the sum exact in 128-bit integers (every
        // FX64 variant then rounds it alike), counted once per launch
        unsigned long long lo = 0, hi = 0;
        if (!decider) {
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const int i = m * NUT + tid;
                if (i < L) {
                    const int si = s[i];
                    long long v = 0;
#pragma unroll
                    for (int x = 0; x < Q; ++x) v = x == si ? h[m][x] : v;
                    u128_add(lo, hi, (unsigned long long)v);
                }
            }
        }
        // scratch: the per-lane energy buffer (unused in FX64 mode), 32 words
        const double Efx = block_sum_u128(lo, hi, (unsigned long long*)dEl);
        if (tid == 0) jp->E[rep] = -0.5 * (double)c * Efx * fxs;  // fxs: a power of two
        if (decider) {  // the counts live in the decision warp
            for (int o = 16; o > 0; o >>= 1) nnear += __shfl_xor_sync(kFullMask, nnear, o);
            if (lane == 0) {
                jp->nsweep[t] = n0 + (uint32_t)nsweeps;
                if (nacc) atomicAdd(&jp->acc_flip[t], nacc);
                if (nnear) atomicAdd(&jp->near[0], nnear);
            }
        }
    } else if (decider) {
        double dE = dEl[lane];
        for (int o = 16; o > 0; o >>= 1) dE += __shfl_xor_sync(kFullMask, dE, o);
        if (lane == 0) {
            jp->E[rep] += dE;
            jp->nsweep[t] = n0 + (uint32_t)nsweeps;
            if (nacc) atomicAdd(&jp->acc_flip[t], nacc);
        }
    }
}

// One item per CTA (sc.n == 0), or persistent CTAs placed by a SweepSched plan.
template <typename T, int Q, int E, int NU>
__global__ void __launch_bounds__(32 * (NU + 1), rf_min_blocks<T, Q, E, NU>())
    sweep_rf_kernel(const JobDev* __restrict__ jobs, const int2* __restrict__ work, int nsweeps, const SweepSched sc)
{
    extern __shared__ __align__(16) unsigned char smem[];
    if (sc.n == 0) {
        rf_item<T, Q, E, NU>(jobs, work[blockIdx.x], nsweeps, smem);
        return;
    }
    __shared__ int s_item;
    bool waited = false;  // thread 0's
    if (threadIdx.x == 0) s_item = sched_claim_home(sc);
    __syncthreads();
    for (;;) {
        const int item = s_item;
        if (item >= 0) rf_item<T, Q, E, NU>(jobs, work[item], nsweeps, smem);
        __syncthreads();
        if (threadIdx.x == 0) s_item = sched_claim_next(sc, waited);
        __syncthreads();
        if (s_item < 0) break;
    }
}

template <typename T, int Q, int E, int NU>
cudaError_t launch_rf(const JobDev* jobs_dev, const int2* work, int nwork, int nsweeps, size_t smem,
                      const SweepSched* sched, cudaStream_t st)
{
    auto k = sweep_rf_kernel<T, Q, E, NU>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    SweepSched sc{};
    int grid = nwork;
    if (sched && sched->nsm > 0 && nwork > sched->nsm) {
        int occ = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, 32 * (NU + 1), smem);
        if (e != cudaSuccess) return e;
        if (occ > 0) {
            sc = *sched;
            sc.n = nwork;
            sc.occ = occ < kSchedMaxOcc ? occ : kSchedMaxOcc;
            grid = sc.nsm * sc.occ;
            if ((e = launch_sweep_plan(jobs_dev, work, sc, st)) != cudaSuccess) return e;
        }
    }
    k<<<grid, 32 * (NU + 1), smem, st>>>(jobs_dev, work, nsweeps, sc);
    return cudaGetLastError();
}

// dispatch over Q for one (field type, E, NU) configuration
template <typename T, int E, int NU, int QMAX>
cudaError_t launch_rf_q(int q, const JobDev* jobs_dev, const int2* work, int nwork, int nsweeps, size_t smem,
                        const SweepSched* sched, cudaStream_t st)
{
    switch (q) {
#define PLR_RF_Q(Qv) \
    case Qv:         \
        if constexpr (Qv <= QMAX) return launch_rf<T, Qv, E, NU>(jobs_dev, work, nwork, nsweeps, smem, sched, st); \
        break;
        PLR_RF_Q(2) PLR_RF_Q(3) PLR_RF_Q(4) PLR_RF_Q(5) PLR_RF_Q(6) PLR_RF_Q(7) PLR_RF_Q(8) PLR_RF_Q(9)
        PLR_RF_Q(10) PLR_RF_Q(11) PLR_RF_Q(12) PLR_RF_Q(13) PLR_RF_Q(14) PLR_RF_Q(15) PLR_RF_Q(16)
#undef PLR_RF_Q
    default: break;
    }
    return cudaErrorNotSupported;
}

// smem bytes for one (field type, E, NU) configuration (depends on q through
// the published values)
template <typename T, int E, int NU>
size_t rf_smem_q(int q, int L, int Lpad)
{
    switch (q) {
#define PLR_RF_S(Qv) \
    case Qv: return RfSmem<T, NU, E, Qv>::bytes(L, Lpad);
        PLR_RF_S(2) PLR_RF_S(3) PLR_RF_S(4) PLR_RF_S(5) PLR_RF_S(6) PLR_RF_S(7) PLR_RF_S(8) PLR_RF_S(9)
        PLR_RF_S(10) PLR_RF_S(11) PLR_RF_S(12) PLR_RF_S(13) PLR_RF_S(14) PLR_RF_S(15) PLR_RF_S(16)
#undef PLR_RF_S
    default: return 0;
    }
}

}  // namespace rf
}  // namespace plr
