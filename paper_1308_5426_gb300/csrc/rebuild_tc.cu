// FP32-mode field rebuild on the tensor cores:
//   H[i][n] = sum_j C[i][j] X[j][n],   C[i][j] = J*((i - j) mod L)   (J*(0) = 0),
//   X[j][n] = delta(x_n, s_{r_n, j}),  n = r q + x  (replica r, state x),
// so H[i][r q + x] = h_r[x][i], the local fields of every replica at once (the
// fields are sums over sites of the coupling to the site's state, Eq. 2).
//
// tcgen05.mma kind::f16 with BF16 operands and FP32 accumulation in tensor
// memory.  X is exact in BF16 (0 or 1); C is carried as three BF16 parts
// hi + mid + lo of the FP64 J* (representation error ~2^-25 J*), each part one
// MMA per K-step.  One CTA computes a 128 x TN tile of H (TN = 64 or 128) over
// all of K in chunks of kChunk = 128 sites: eight warps build the operand tiles in
// shared memory from the split table and the packed spins, one thread issues
// the 24 MMAs of the chunk (8 K-steps x 3 parts) and commits them to the
// mbarrier of the chunk's stage; two stages alternate, so chunk t + 1 is
// built while the MMAs of chunk t run.  The tensor core's FP32 accumulation rounds every MMA's sum into
// the accumulator, so the accumulation chains are kept short: the hi parts of
// successive chunks rotate over 512 / TN - 1 accumulators (seven or three),
// and the small mid + lo parts go to one of their own (their rounding is then
// relative to their own small size); together they fill the 512 TMEM columns.
// The epilogue adds them in FP64 and stores FP32 fields.
//
// Operand layout (both K-major, no swizzle): 8-row x 16-byte core matrices.
// B: core matrix (row group g, K group c) at byte (c G + g) 128 (leading (K)
// byte offset 128 G, stride (row-group) byte offset 128; K-step s at 256 G s).
// A: the chunk's sites are taken in reverse order (as in B), which makes the
// circulant tile Hankel: core matrix (g, c) = core matrix g + c of a strip of
// 31, so both byte offsets are 128 and K-step s starts at 256 s.
#include <cstdint>
#include <vector>

#include "potts_internal.h"

namespace plr {

namespace {

constexpr int kTcThreads = 256;      // 8 warps build the tiles; warps w and w + 4 share TMEM lanes 32 (w % 4) ..
constexpr int kTileM = 128;

constexpr int kChunk = 128;          // K sites per chunk
constexpr int kHank = kTileM / 8 + kChunk / 8 - 1;  // distinct core matrices of an A tile (Hankel form)
constexpr int kTileBytes = kHank * 128;            // 3968 B per A tile of one split
constexpr int kSplit = 3;
constexpr int kTmemCols = 512;       // all of the SM's tensor memory: accumulators of TN columns each
// per tile width TN (64 or 128 output columns): accumulators, B tile, stage
template <int TN>
struct TcShape {
    static constexpr int kAcc = kTmemCols / TN;      // 8 or 4 accumulators
    static constexpr int kAccHi = kAcc - 1;          // rotating accumulators of the hi parts; the last takes mid + lo
    static constexpr int kTileBytesB = TN * kChunk * 2;  // TN x kChunk BF16 B tile
    static constexpr int kGB = TN / 8;               // row groups of the B tile
    static constexpr int kStageBytes = kSplit * kTileBytes + kTileBytesB;  // three A tiles + the B tile
};
constexpr int kStages = 2;           // chunk t + 1 is built while the MMAs of chunk t run
constexpr long long kWaitLimit = 1ll << 26;  // bounded mbarrier wait (iterations)
constexpr size_t kTcMinSmem = 120 * 1024;   // forces one CTA per SM (owner of all 512 columns)

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= 1ull << 46;  // descriptor version for tcgen05; layout type 0 = no swizzle
    return d;
}

// kind::f16 instruction descriptor: D = F32, A = B = BF16, both K-major, M x N.
__host__ __device__ constexpr uint32_t make_idesc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    for (long long it = 0; it < kWaitLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ uint16_t bf16_one() { return 0x3F80u; }

// (i - k) mod L for i < L + 128 and k < L + kChunk (tile and chunk padding past L
// only meet zero operands, so any in-range index serves there)
__device__ __forceinline__ int circ(int d, int L)
{
    d += d < 0 ? L : 0;
    d -= d >= L ? L : 0;
    return (d < 0 || d >= L) ? 0 : d;
}

template <int TN>
__global__ void __launch_bounds__(kTcThreads, 1) fields_tc_kernel(const JobDev* __restrict__ jobs,
                                                                  const int4* __restrict__ tiles, int ntiles,
                                                                  int cond)
{
    constexpr int kTileN = TN;
    constexpr int kAcc = TcShape<TN>::kAcc, kAccHi = TcShape<TN>::kAccHi;
    constexpr int kGB = TcShape<TN>::kGB, kStageBytes = TcShape<TN>::kStageBytes;
    constexpr int kHB = kGB / (kTcThreads / 32);  // B row groups per build warp
    static_assert(kAcc * TN == kTmemCols, "accumulators fill the tensor memory");
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int kWarps = kTcThreads / 32;
    static_assert(kHB * kWarps == kGB, "whole B row groups per build warp");

    // stage b: A tiles at b * kStageBytes, then its B tile
    uint64_t* mbar = (uint64_t*)(smem + kStages * kStageBytes);  // one per stage
    uint32_t* tmem_slot = (uint32_t*)(mbar + kStages);
    uint16_t* tab = (uint16_t*)(smem + kStages * kStageBytes + 64);  // split table [3][Lpad], if staged

    // skip the whole CTA when none of its tiles is due (no tensor memory taken)
    bool any = false;
    for (int ti = blockIdx.x; ti < ntiles && !any; ti += gridDim.x) any = !cond || rebuild_due(jobs[tiles[ti].x]);
    if (!any) return;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int b = 0; b < kStages; ++b)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar + b)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    // this thread's place in a core matrix: row rr = lane / 4, sites 2 (lane % 4), +1
    const int rr = lane >> 2, kp = (lane & 3) * 2;
    const uint32_t idesc = make_idesc(kTileM, kTileN);
    bool ok = true;
    uint32_t parity[kStages] = {0u, 0u};  // phase of each stage's barrier that is awaited next
    int pending[kStages] = {0, 0};        // commits on each stage's barrier not yet awaited
    const JobDev* staged = nullptr;       // job whose split table is in shared memory

    for (int ti = blockIdx.x; ti < ntiles && ok; ti += gridDim.x) {
    const int4 tile = tiles[ti];
    const JobDev& jb = jobs[tile.x];
    if (cond && !rebuild_due(jb)) continue;
    const int L = jb.L, q = jb.q, Lpad = jb.Lpad, W = jb.W;
    const int N = q * jb.R;
    const int m0 = tile.y, n0 = tile.z;
    const bool tab_smem = jb.tc_tab_smem != 0;
    const uint16_t* gtab = jb.Jsplit;
    if (tab_smem && staged != &jb) {
        __syncthreads();  // previous tile done with the old table
        for (int m = tid; m < kSplit * Lpad; m += kTcThreads) tab[m] = gtab[m];
        __syncthreads();
        staged = &jb;
    }
    const uint16_t* T = tab_smem ? tab : gtab;
    const int nchunks = (L + kChunk - 1) / kChunk;
    // this thread's rows of the B tile: n = n0 + 8 (warp + 8 hb) + rr, hb < kHB, fixed over the tile
    int bx[kHB];
    bool nvalid[kHB];
    const uint32_t* bsp[kHB];
#pragma unroll
    for (int hb = 0; hb < kHB; ++hb) {
        const int nb = n0 + 8 * (warp + kWarps * hb) + rr;
        nvalid[hb] = nb < N;
        const int brep = nvalid[hb] ? nb / q : 0;
        bx[hb] = nvalid[hb] ? nb - brep * q : 0;
        bsp[hb] = jb.spins + (size_t)brep * W;
    }
    const int bshift = 4 * (6 - kp);  // nibble of site k0 + kChunk - 2 - 8 kc - kp within its word

    // chunk order: decreasing circular distance from the chunk holding the tile's
    // centre, so the large near-diagonal couplings are added last and the many
    // small far-field sums accumulate while the accumulators are still small
    const int cc = ((m0 + kTileM / 2) / kChunk) % nchunks;
    auto chunk_of = [&](int t) {
        const int kk = nchunks - 1 - t;  // rank in increasing distance: 0, +1, -1, +2, -2, ...
        const int o = kk == 0 ? 0 : ((kk & 1) ? (kk + 1) / 2 : -(kk / 2));
        int c = cc + o;  // |o| <= nchunks / 2
        c += c < 0 ? nchunks : 0;
        c -= c >= nchunks ? nchunks : 0;
        return c;
    };
    // the spin words of this thread's B rows for a chunk (word (kChunk / 8) (c + 1) - 1 - kc
    // holds K group kc)
    uint32_t wnext[kHB][kChunk / 8];
    auto load_words = [&](int c) {
#pragma unroll
        for (int hb = 0; hb < kHB; ++hb)
#pragma unroll
            for (int kc = 0; kc < kChunk / 8; ++kc) {
                const int wi = (kChunk / 8) * (c + 1) - 1 - kc;
                wnext[hb][kc] = (nvalid[hb] && wi < W) ? bsp[hb][wi] : 0u;
            }
    };
    load_words(chunk_of(0));
    for (int t = 0; t < nchunks; ++t) {
        const int c = chunk_of(t);
        const int k0 = c * kChunk;
        uint32_t words[kHB][kChunk / 8];
#pragma unroll
        for (int hb = 0; hb < kHB; ++hb)
#pragma unroll
            for (int kc = 0; kc < kChunk / 8; ++kc) words[hb][kc] = wnext[hb][kc];
        if (t + 1 < nchunks) load_words(chunk_of(t + 1));  // in flight during this chunk
        const int b = t % kStages;
        unsigned char* tileA = smem + b * kStageBytes;
        unsigned char* tileB = tileA + kSplit * kTileBytes;
        // the MMAs that last read this stage (chunk t - kStages) must be done:
        // warp 0 waits, the barrier tells the others
        if (pending[b]) {
            if (warp == 0 && !mbar_wait(smem_u32(mbar + b), parity[b])) ok = false;
            parity[b] ^= 1u;
            pending[b] = 0;
            if (!__syncthreads_and(ok)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        }
        // The chunk's K sites are taken in reverse, k = k0 + kChunk - 1 - k', so A[i][k'] =
        // J*((i - k) mod L) depends on i + k' only: core matrix (g, c) is core
        // matrix h = g + c of a Hankel strip of kHank = 31, which the MMA reads with
        // row-group and K-group strides both 128 bytes.  Element (rr, e) of
        // core matrix h is J*((m0 - k0 - kChunk + 1 + 8 h + rr + e) mod L).
        for (int h = warp; h < kHank; h += kWarps) {
            const int r0 = circ(m0 - k0 - (kChunk - 1) + 8 * h + rr + kp, L);
            const int r1 = r0 + 1 == L ? 0 : r0 + 1;
            const uint32_t off = (uint32_t)(h * 128 + rr * 16 + kp * 2);
#pragma unroll
            for (int sp = 0; sp < kSplit; ++sp) {
                const uint32_t v = (uint32_t)T[sp * Lpad + r0] | ((uint32_t)T[sp * Lpad + r1] << 16);
                *(uint32_t*)(tileA + sp * kTileBytes + off) = v;
            }
        }
        // B tile: row n = (replica, state), X = 1 where the replica's spin at site
        // k = k0 + kChunk - 1 - k' is that state (K reversed as for A)
        // (warp w holds row groups w + 8 hb: the core matrices (g, kc), kc < kChunk / 8;
        // spin word (k0 + kChunk) / 8 - 1 - kc holds the sites of K group kc)
#pragma unroll
        for (int hb = 0; hb < kHB; ++hb)
#pragma unroll
            for (int kc = 0; kc < kChunk / 8; ++kc) {
                const int ka = k0 + (kChunk - 1) - (8 * kc + kp);  // site of k' = 8 kc + kp; k' + 1 is ka - 1
                const uint32_t off = (uint32_t)((kc * kGB + warp + kWarps * hb) * 128 + rr * 16 + kp * 2);
                uint32_t v = 0;
                if (nvalid[hb] && ka - 1 < L) {
                    const uint32_t word = words[hb][kc] >> bshift;
                    if (ka < L && (int)((word >> 4) & 15u) == bx[hb]) v |= bf16_one();  // next nibble: site ka
                    if ((int)(word & 15u) == bx[hb]) v |= (uint32_t)bf16_one() << 16;
                }
                *(uint32_t*)(tileB + off) = v;
            }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (!__syncthreads_and(ok)) {
            ok = false;
            break;
        }
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t dhi = tmem + (uint32_t)((t % kAccHi) * kTileN);
            const uint32_t dsmall = tmem + (uint32_t)(kAccHi * kTileN);
#pragma unroll
            for (int s = 0; s < kChunk / 16; ++s) {
                const uint64_t bdesc = make_desc(smem_u32(tileB) + s * 256 * kGB, 128 * kGB, 128);
#pragma unroll
                for (int sp = 0; sp < kSplit; ++sp) {
                    const uint64_t adesc = make_desc(smem_u32(tileA + sp * kTileBytes) + s * 256, 128, 128);
                    const uint32_t dcol = sp == 0 ? dhi : dsmall;
                    const bool first = s == 0 && (sp == 0 ? t < kAccHi : (t == 0 && sp == 1));
                    const uint32_t accumulate = first ? 0u : 1u;
                    asm volatile(
                        "{\n\t.reg .pred p;\n\t"
                        "setp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dcol),
                        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
                        : "memory");
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(mbar + b))
                         : "memory");
        }
        pending[b] = 1;
    }
    // all of the tile's MMAs done before its accumulators are read
    for (int b = 0; b < kStages; ++b)
        if (pending[b]) {
            if (warp == 0 && !mbar_wait(smem_u32(mbar + b), parity[b])) ok = false;
            parity[b] ^= 1u;
            pending[b] = 0;
        }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!__syncthreads_and(ok)) ok = false;

    if (ok) {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 = rows m0 + 32 (w % 4) + lane,
        // columns half (w / 4) of the tile
        const int quad = warp & 3;
        const int i = m0 + 32 * quad + lane;
        const int nhi = nchunks < kAccHi ? nchunks : kAccHi;
        float* F = (float*)jb.fields;
        double dmax = 0.0;
        constexpr int kCols = kTileN / (kWarps / 4);
        for (int cb = (warp >> 2) * kCols; cb < (warp >> 2) * kCols + kCols; cb += 8) {
            double sum[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) sum[e] = 0.0;
            for (int a = 0; a <= nhi; ++a) {
                const int col = a < nhi ? a : kAccHi;  // the used hi accumulators, then mid + lo
                uint32_t v[8];
                const uint32_t taddr = tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)(col * kTileN + cb);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                    : "r"(taddr)
                    : "memory");
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int e = 0; e < 8; ++e) sum[e] += (double)__uint_as_float(v[e]);
            }
            if (i < L) {
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int n = n0 + cb + e;
                    if (n < N) {
                        const size_t idx = (size_t)n * Lpad + i;
                        dmax = fmax(dmax, fabs((double)F[idx] - sum[e]));  // drift of the ending period
                        F[idx] = (float)sum[e];
                    }
                }
            }
        }
        for (int o = 16; o > 0; o >>= 1) dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
        if (lane == 0 && dmax > 0.0)
            atomicMax(jb.drift_bits, (unsigned long long)__double_as_longlong(dmax / jb.jtot));
        // the tensor-memory reads above are complete before the next tile's MMAs
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    } else if (tid == 0) {
        atomicExch(jb.status, 1);  // a bounded wait expired; the host reports ETIMEOUT
    }
    }  // tiles
    // no MMA may still write tensor memory when it is freed (after an expired
    // wait, give the outstanding commits a bounded chance to land)
    if (warp == 0)
        for (int b = 0; b < kStages; ++b)
            if (pending[b]) mbar_wait(smem_u32(mbar + b), parity[b]);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

}  // namespace

size_t tc_smem_bytes(int Lpad, int tab_smem)
{
    // sized for the wider tile, so either width fits
    size_t b = (size_t)kStages * TcShape<128>::kStageBytes + 64 + (tab_smem ? (size_t)kSplit * Lpad * 2 : 0);
    b = (b + 127) & ~(size_t)127;
    return b < kTcMinSmem ? kTcMinSmem : b;
}

int tc_table_in_smem(int Lpad)
{
    return (size_t)kStages * TcShape<128>::kStageBytes + 64 + (size_t)kSplit * Lpad * 2 <= 200 * 1024;
}

int tc_tile_width(long long tiles64, long long tiles128, int nsm)
{
    // persistent CTAs walk the tiles; a 128-wide tile costs about 1.4 times a
    // 64-wide one (half the MMA instructions per output), so the wider tile
    // pays unless it leaves the SMs idler
    if (nsm <= 0) return 64;
    const double w64 = (double)((tiles64 + nsm - 1) / nsm), w128 = (double)((tiles128 + nsm - 1) / nsm);
    return 1.4 * w128 < w64 ? 128 : 64;
}

cudaError_t launch_fields_tc(const JobDev* jobs_dev, const int4* tiles, int ntiles, int any_tab_smem_Lpad,
                             int cond, int tn, cudaStream_t st)
{
    if (ntiles <= 0) return cudaSuccess;
    const size_t smem = tc_smem_bytes(any_tab_smem_Lpad, any_tab_smem_Lpad > 0);
    auto k = tn == 128 ? fields_tc_kernel<128> : fields_tc_kernel<64>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = ntiles < sms ? ntiles : sms;  // persistent: one CTA per SM walks the tile table
    k<<<grid, kTcThreads, smem, st>>>(jobs_dev, tiles, ntiles, cond);
    return cudaGetLastError();
}

void tc_tiles(int job, int L, int q, int R, int tn, std::vector<int4>& out)
{
    for (int m = 0; m < L; m += kTileM)
        for (int n = 0; n < q * R; n += tn) out.push_back(make_int4(job, m, n, 0));
}

long long tc_tile_count(int L, int q, int R, int tn)
{
    return (long long)((L + kTileM - 1) / kTileM) * ((q * R + tn - 1) / tn);
}

}  // namespace plr
