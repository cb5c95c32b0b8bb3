// Metropolis sweep of the long-range Potts chain (Eq. 8, Sec. 4.2 of the paper)
// with local fields h[x][i] = sum_{j != i} J*(|i-j|) delta(x, s_j).
//
// One CTA sweeps one temperature slot at a time (see SweepSched for which
// CTA takes which slot); 8 warps.  Sites are taken in blocks of 32 in
// order k = 0..L-1.  Warp 0 decides a block; warps 1..7 meanwhile apply the
// previous block's accepted flips to the fields (the rank-1 updates
// h[a][i] -= J*(|i-k|), h[b][i] += J*(|i-k|)), except at the 32 sites of the
// block being decided, which warp 0 brings up to date itself first.  One CTA
// barrier per block.
//
// Deciding a block of 32 sites exactly as a sequential sweep would: lane l
// holds site k0 + l, its proposal b_l, -ln u_l and d_l = h[a_l][k] - h[b_l][k]
// (dE = c d, Eq. 2/8).  All undecided lanes evaluate their rule at once; the
// first lane that accepts is then certain to accept (nothing before it
// changed), every lane before it is certain to reject.  After an accepted flip
// j, each later lane corrects d_l by J*(l-j)([a_l=b_j]-[a_l=a_j]-[b_l=b_j]+[b_l=a_j])
// -- the change flip j makes to h at site k_l -- and the scan continues after j.
// So a block costs one round per accepted flip, not one per site.
//
// FP64 mode decides in FP32 with a margin that bounds every FP32 rounding
// (|d32 - d64| <= 1.2e-5 Jtot, see decide_fp64_filter); only when the margin is
// too small does the lane rebuild d in FP64 and apply the FP64 rule
// u < exp(-beta dE) itself.  FP32 mode decides in FP32.
//
// FX64 mode (T = long long) keeps the fields as integers in units of 2^-F,
// built from the couplings rounded to that grid: every update is an exact
// integer add (two 32-bit integer instructions, on pipes 64 times wider than
// GB300's FP64 pipe), so the fields hold the exact local fields of the
// rounded couplings whatever the order of the updates.  Decisions are those
// of FP64 mode, the exact difference converted to FP64 once.
#include <cmath>
#include <type_traits>

#include "sweep_common.cuh"
#include "sweep_sched.cuh"

namespace plr {

namespace {

#ifndef PLR_GLOBAL_THREADS
#define PLR_GLOBAL_THREADS 512
#endif
// threads of a sweep CTA: 256 with the fields in shared memory (several CTAs
// per SM), more with the fields in global memory, where the update's round
// trips to L2 want more warps in flight per slot
template <bool HS>
constexpr int sweep_threads()
{
    return HS ? kSweepThreads : PLR_GLOBAL_THREADS;
}
constexpr int kWarpsMax = 1024 / 32;

template <typename T>
struct SweepSmem {
    // carve-up of the dynamic shared memory (must match the kernel)
    static size_t bytes(int L, int Lpad, int q, bool hs, bool js)
    {
        (void)L;
        size_t b = 0;
        if (js) b += ((size_t)Lpad + 4) * sizeof(T);  // J*(m mod L), m < Lpad + 4
        if (hs) b += (size_t)q * Lpad * sizeof(T);
        b += (size_t)Lpad;                       // spins
        b += 2 * 2 * kSiteBlock * sizeof(int);   // double-buffered flip lists
        b += kNearTable * sizeof(float);         // J* at distances 0..63 in FP32
        b += kWarpsMax * sizeof(double) + 16;    // reduction scratch, counts
        return (b + 15) & ~(size_t)15;
    }
};

// Rank-1 updates of the flips (pk, pab)[0..nf), in flip order, on every
// element except [x0, x0 + nx): h[a][i] -= J*((i-k) mod L), h[b][i] += J*((i-k) mod L).
// The elements form one index space j = 0..L-nx-1 (i = j, or j + nx past x0);
// worker u of nw = NT - 32 takes j = u + nw m (stride 1 across a
// warp: conflict-free shared-memory access) four at a time, and applies all
// flips to those four before moving on, so four independent read-modify-write
// chains are in flight and the flip list is read once per four elements.
template <typename T, int NT>
__device__ __forceinline__ void apply_flips(T* __restrict__ h, const T* __restrict__ J, int L, int Lpad,
                                            const int* pk, const int* pab, int nf, int x0, int nx, int u)
{
    constexpr int nw = NT - 32;
    const int n = L - nx;
    int j = u;
    for (; j + 3 * nw < n; j += 4 * nw) {
        int idx[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int jj = j + e * nw;
            idx[e] = jj < x0 ? jj : jj + nx;
        }
        for (int f = 0; f < nf; ++f) {
            const int kf = pk[f], af = pab[f] >> 8, bf = pab[f] & 255;
            T* __restrict__ ha = h + (size_t)af * Lpad;
            T* __restrict__ hb = h + (size_t)bf * Lpad;
            T v[4], xa[4], xb[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                int r = idx[e] - kf;
                r += r < 0 ? L : 0;
                v[e] = J[r];
                xa[e] = ha[idx[e]];
                xb[e] = hb[idx[e]];
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                ha[idx[e]] = xa[e] - v[e];
                hb[idx[e]] = xb[e] + v[e];
            }
        }
    }
    for (; j < n; j += nw) {
        const int i = j < x0 ? j : j + nx;
        for (int f = 0; f < nf; ++f) {
            const int kf = pk[f], af = pab[f] >> 8, bf = pab[f] & 255;
            int r = i - kf;
            r += r < 0 ? L : 0;
            const T v = J[r];
            h[(size_t)af * Lpad + i] -= v;
            h[(size_t)bf * Lpad + i] += v;
        }
    }
}

// FP32 form of apply_flips: the same updates in the same order, each thread
// taking four consecutive sites at a time with 16-byte loads and stores of
// the two field rows (two such groups in flight), the coupling of site i0 + e
// read as J[r + e], r = (i0 - k) mod L, from a table that runs four entries
// past L (J[m] = J*(m mod L)).  Groups that overlap the block being decided,
// [x0, x0 + nx), are left to the deciding warp (its sites) or untouched
// (padding past L).
template <int NT>
__device__ __forceinline__ void apply_flips_vec4(float* __restrict__ h, const float* __restrict__ J, int L, int Lpad,
                                                 const int* pk, const int* pab, int nf, int x0, int nx, int u)
{
    constexpr int nw = NT - 32;
    const int ng = (L + 3) >> 2;                        // groups holding sites < L
    const int g0 = x0 >> 2, g1 = (x0 + nx + 3) >> 2;    // groups of the decided block (x0 % 32 == 0)
    const int n = ng - (g1 - g0);
    for (int jg = u; jg < n; jg += 2 * nw) {
        int i0[2];
        bool ok[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int gg = jg + e * nw;
            ok[e] = gg < n;
            i0[e] = 4 * ((ok[e] ? gg : jg) < g0 ? (ok[e] ? gg : jg) : (ok[e] ? gg : jg) + (g1 - g0));
        }
        for (int f = 0; f < nf; ++f) {
            const int kf = pk[f], af = pab[f] >> 8, bf = pab[f] & 255;
            float4 xa[2], xb[2], v[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                int r = i0[e] - kf;
                r += r < 0 ? L : 0;
                v[e] = make_float4(J[r], J[r + 1], J[r + 2], J[r + 3]);
                xa[e] = *(const float4*)(h + (size_t)af * Lpad + i0[e]);
                xb[e] = *(const float4*)(h + (size_t)bf * Lpad + i0[e]);
            }
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                if (!ok[e]) continue;
                xa[e].x -= v[e].x; xa[e].y -= v[e].y; xa[e].z -= v[e].z; xa[e].w -= v[e].w;
                xb[e].x += v[e].x; xb[e].y += v[e].y; xb[e].z += v[e].z; xb[e].w += v[e].w;
                *(float4*)(h + (size_t)af * Lpad + i0[e]) = xa[e];
                *(float4*)(h + (size_t)bf * Lpad + i0[e]) = xb[e];
            }
        }
    }
}

// nsweeps sweeps of one work item wk = (job, slot) by the whole CTA
template <typename T, bool HS, bool JS>
__device__ __forceinline__ void sweep_item(const JobDev* __restrict__ jobs, const int2 wk, int nsweeps,
                                           unsigned char* __restrict__ smem)
{
    constexpr bool kFP64 = sizeof(T) == 8;  // FP64 rule (FP64 and FX64 modes)
    constexpr bool kFX = std::is_same<T, long long>::value;
    constexpr int kMode = kFX ? 2 : (kFP64 ? 1 : 0);
    constexpr int NT = sweep_threads<HS>();
    const JobDev* jp = jobs + wk.x;
    const int t = wk.y;
    const int L = jp->L, q = jp->q, Lpad = jp->Lpad, W = jp->W, c = jp->c;
    const uint32_t key0 = jp->key0, key1 = jp->key1;
    const int rep = jp->map[t];
    const double beta = jp->beta[t];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    const T* __restrict__ Jg = kFX     ? (const T*)(const void*)jp->Jfxd
                               : kFP64 ? (const T*)(const void*)jp->J64d
                                       : (const T*)(const void*)jp->J32d;
    T* __restrict__ hg = (T*)jp->fields + (size_t)rep * q * Lpad;
    uint32_t* __restrict__ spins = jp->spins + (size_t)rep * W;

    size_t off = 0;
    T* Js = nullptr;
    if constexpr (JS) {
        Js = (T*)(smem + off);
        off += ((size_t)Lpad + 4) * sizeof(T);
    }
    T* hs = nullptr;
    if constexpr (HS) {
        hs = (T*)(smem + off);
        off += (size_t)q * Lpad * sizeof(T);
    }
    uint8_t* s = smem + off;
    off += (size_t)Lpad;
    int* lk = (int*)(smem + off);      // [2][32] flip sites
    int* lab = lk + 2 * kSiteBlock;    // [2][32] (a << 8) | b
    float* Jn = (float*)(lab + 2 * kSiteBlock);  // J*(r), r < 64, FP32
    double* red = (double*)(((uintptr_t)(Jn + kNearTable) + 7) & ~(uintptr_t)7);
    int* lcnt = (int*)(red + kWarpsMax);  // [2] flip counts

    if constexpr (JS)
        for (int m = tid; m < Lpad + 4; m += NT) Js[m] = Jg[m % L];
    if constexpr (HS) {
        const int n = q * Lpad;
        for (int e = tid; e < n; e += NT) hs[e] = hg[e];
    }
    for (int i = tid; i < L; i += NT) s[i] = (uint8_t)((spins[i >> 3] >> (4 * (i & 7))) & 15u);
    if (tid < kNearTable) Jn[tid] = tid < L ? (float)jp->J64d[tid] : 0.0f;
    if (tid < 2) lcnt[tid] = 0;
    __syncthreads();

    T* __restrict__ h = HS ? hs : hg;
    const T* __restrict__ J = JS ? (const T*)Js : Jg;  // J[r], r = 0..L-1 (J[0] = 0)

    const uint32_t n0 = jp->nsweep[t];
    const double cb64 = beta * (double)c;
    const float cb32 = (float)cb64;
    const float errd = (float)(2.4e-5 * jp->jtot);
    const double fxs = kFX ? jp->fx_scale : 1.0;  // value of one field unit
    const float fxs32 = (float)fxs;                // a power of two: exact
    const int nblk = (L + kSiteBlock - 1) / kSiteBlock;
    const int total = nsweeps * nblk;

    double dE_acc = 0.0;                 // FP32 mode: running energy change (lane-local)
    unsigned long long nacc = 0, nnear = 0;

    for (int g = 0; g <= total; ++g) {
        const int pb = (g + 1) & 1;                // list of block g-1 (pending)
        const int npend = g > 0 ? lcnt[pb] : 0;
        const int* pk = lk + pb * kSiteBlock;
        const int* pab = lab + pb * kSiteBlock;
        const int k0 = g < total ? (g % nblk) * kSiteBlock : 0;
        const int nv = g < total ? min(kSiteBlock, L - k0) : 0;

        if (warp == 0) {
            if (g < total) {
                const int k = k0 + lane;
                const bool valid = lane < nv;
                const uint32_t n = n0 + (uint32_t)(g / nblk);
                // the block's sites do not hold block g-1's flips yet: decide with
                // corrections, then bring them up to date
                int a = 0, b = 0;
                float nlu = 0.0f, d32 = 0.0f;
                double base = 0.0;
                long long basefx = 0;
                uint32_t ux1 = 0, ux2 = 0;
                if (valid) {
                    a = s[k];
                    draw_proposal<kFP64>(k, t, n, key0, key1, q, a, b, nlu, ux1, ux2);
                    const T dd = h[(size_t)a * Lpad + k] - h[(size_t)b * Lpad + k];
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
                                                   NearSink{jp->near_log, jp->near_log_n, t, n});
                if (mine) {
                    s[k] = (uint8_t)b;
                    if constexpr (!kFP64) dE_acc += (double)((float)c * dmine);
                }
                if (lane == 0) {
                    lcnt[cbuf] = nf;
                    nacc += (unsigned long long)nf;
                }
                if (valid) {
                    for (int f = 0; f < npend; ++f) {
                        const int kf = pk[f], af = pab[f] >> 8, bf = pab[f] & 255;
                        int r = k - kf;
                        r += r < 0 ? L : 0;
                        const T v = J[r];
                        h[(size_t)af * Lpad + k] -= v;
                        h[(size_t)bf * Lpad + k] += v;
                    }
                }
            }
        } else if (npend > 0) {
            // apply block g-1's flips everywhere except at the sites warp 0 owns
            // now: ranges [0, k0) and [k0 + nv, L)
            // FP32 with fields or table in global memory: four sites per thread
            // (with both in shared memory, the table reads four sites apart
            // conflict in the banks and the one-site form is faster)
            if constexpr (kFP64 || (HS && JS)) apply_flips<T, NT>(h, J, L, Lpad, pk, pab, npend, k0, nv, tid - 32);
            else apply_flips_vec4<NT>(h, J, L, Lpad, pk, pab, npend, k0, nv, tid - 32);
        }
        __syncthreads();
    }

    // write back
    for (int w = tid; w < W; w += NT) {
        uint32_t word = 0;
        for (int m = 0; m < 8; ++m) {
            const int i = 8 * w + m;
            if (i < L) word |= (uint32_t)s[i] << (4 * m);
        }
        spins[w] = word;
    }
    if constexpr (HS) {
        const int n = q * Lpad;
        for (int e = tid; e < n; e += NT) hg[e] = hs[e];
    }
    double Efx = 0.0;
    if constexpr (kFX) {
        // E = -(c/2) sum_i h[s_i][i] from the integer fields, the sum exact in
        // 128 bits, so that every FX64 kernel variant gets the same value
        unsigned long long lo = 0, hi = 0;
        for (int i = tid; i < L; i += NT) u128_add(lo, hi, (unsigned long long)h[(size_t)s[i] * Lpad + i]);
        Efx = block_sum_u128(lo, hi, (unsigned long long*)red);
    } else if constexpr (kFP64) {
        // E = -(c/2) sum_i h[s_i][i] from the FP64 fields (Eq. 2 through the
        // fields), summed over 256 fixed strands whatever the CTA size, so
        // that every kernel variant rounds the sum alike
        double part = 0.0;
        if (tid < kSweepThreads)
            for (int i = tid; i < L; i += kSweepThreads) part += (double)h[(size_t)s[i] * Lpad + i];
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(kFullMask, part, o);
        if (lane == 0 && warp < kSweepThreads / 32) red[warp] = part;
    }
    if (warp == 0) {
        for (int o = 16; o > 0; o >>= 1) {
            dE_acc += __shfl_xor_sync(kFullMask, dE_acc, o);
            nnear += __shfl_xor_sync(kFullMask, nnear, o);
        }
    }
    __syncthreads();
    if (tid == 0) {
        if constexpr (kFX) {
            jp->E[rep] = -0.5 * (double)c * Efx * fxs;  // fxs: FX64 field units (a power of two)
        } else if constexpr (kFP64) {
            double tot = 0.0;
            for (int w = 0; w < kSweepThreads / 32; ++w) tot += red[w];
            jp->E[rep] = -0.5 * (double)c * tot;
        } else {
            jp->E[rep] += dE_acc;
        }
        jp->nsweep[t] = n0 + (uint32_t)nsweeps;
        if (nacc) atomicAdd(&jp->acc_flip[t], nacc);
        if (nnear) atomicAdd(&jp->near[0], nnear);
    }
}

// Without a plan (sc.n == 0) CTA b sweeps item b.  With one, the grid is
// persistent: each CTA takes the item dealt to its place on its SM, then
// further items from the ordered list until none is left.
template <typename T, bool HS, bool JS>
__global__ void __launch_bounds__(sweep_threads<HS>(), HS ? 4 : 1) sweep_kernel(const JobDev* __restrict__ jobs,
                                                              const int2* __restrict__ work, int nsweeps,
                                                              const SweepSched sc)
{
    extern __shared__ __align__(16) unsigned char smem[];
    if (sc.n == 0) {
        sweep_item<T, HS, JS>(jobs, work[blockIdx.x], nsweeps, smem);
        return;
    }
    __shared__ int s_item;
    bool waited = false;  // thread 0's
    if (threadIdx.x == 0) s_item = sched_claim_home(sc);
    __syncthreads();
    for (;;) {
        const int item = s_item;
        if (item >= 0) sweep_item<T, HS, JS>(jobs, work[item], nsweeps, smem);
        __syncthreads();
        if (threadIdx.x == 0) s_item = sched_claim_next(sc, waited);
        __syncthreads();
        if (s_item < 0) break;
    }
}

template <typename T, bool HS, bool JS>
cudaError_t launch_variant(const JobDev* jobs_dev, const int2* work, int nwork, int nsweeps, size_t smem,
                           const SweepSched* sched, cudaStream_t st)
{
    auto k = sweep_kernel<T, HS, JS>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    SweepSched sc{};
    int grid = nwork;
    // a plan pays when there are more items than SMs (fewer: the hardware
    // already gives each its own SM)
    if (sched && sched->nsm > 0 && nwork > sched->nsm) {
        int occ = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, sweep_threads<HS>(), smem);
        if (e != cudaSuccess) return e;
        if (occ > 0) {
            sc = *sched;
            sc.n = nwork;
            sc.occ = occ < kSchedMaxOcc ? occ : kSchedMaxOcc;
            grid = sc.nsm * sc.occ;
            if ((e = launch_sweep_plan(jobs_dev, work, sc, st)) != cudaSuccess) return e;
        }
    }
    k<<<grid, sweep_threads<HS>(), smem, st>>>(jobs_dev, work, nsweeps, sc);
    return cudaGetLastError();
}

}  // namespace

size_t sweep_smem_bytes(const JobDev& j)
{
    return sweep_smem_bytes_for(j.precision, j.L, j.Lpad, j.q, j.h_smem, j.j_smem);
}

size_t sweep_smem_bytes_for(int precision, int L, int Lpad, int q, int h_smem, int j_smem)
{
    if (precision == kPrecFP32) return SweepSmem<float>::bytes(L, Lpad, q, h_smem, j_smem);
    return SweepSmem<double>::bytes(L, Lpad, q, h_smem, j_smem);  // FP64 or FX64: 8-byte words
}

cudaError_t launch_sweep(const JobDev* jobs_dev, const int2* work, int nwork, int nsweeps, int precision,
                         int h_smem, int j_smem, size_t smem, const SweepSched* sched, cudaStream_t st)
{
    if (nwork <= 0 || nsweeps <= 0) return cudaSuccess;
    const int v = precision * 4 + (h_smem ? 2 : 0) + (j_smem ? 1 : 0);
    switch (v) {
    case 0: return launch_variant<double, false, false>(jobs_dev, work, nwork, nsweeps, smem, sched, st);
    case 1: return launch_variant<double, false, true>(jobs_dev, work, nwork, nsweeps, smem, sched, st);
    case 2: return launch_variant<double, true, false>(jobs_dev, work, nwork, nsweeps, smem, sched, st);
    case 3: return launch_variant<double, true, true>(jobs_dev, work, nwork, nsweeps, smem, sched, st);
    case 4: return launch_variant<float, false, false>(jobs_dev, work, nwork, nsweeps, smem, sched, st);
    case 5: return launch_variant<float, false, true>(jobs_dev, work, nwork, nsweeps, smem, sched, st);
    case 6: return launch_variant<float, true, false>(jobs_dev, work, nwork, nsweeps, smem, sched, st);
    case 7: return launch_variant<float, true, true>(jobs_dev, work, nwork, nsweeps, smem, sched, st);
    case 8: return launch_variant<long long, false, false>(jobs_dev, work, nwork, nsweeps, smem, sched, st);
    case 9: return launch_variant<long long, false, true>(jobs_dev, work, nwork, nsweeps, smem, sched, st);
    case 10: return launch_variant<long long, true, false>(jobs_dev, work, nwork, nsweeps, smem, sched, st);
    case 11: return launch_variant<long long, true, true>(jobs_dev, work, nwork, nsweeps, smem, sched, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace plr
