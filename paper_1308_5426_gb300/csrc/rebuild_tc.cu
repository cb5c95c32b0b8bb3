// FP32-mode field rebuild on the tensor cores:
//   H[i][n] = sum_j C[i][j] X[j][n],   C[i][j] = J*((i - j) mod L)   (J*(0) = 0),
//   X[j][n] = delta(x_n, s_{r_n, j}),  n = r q + x  (replica r, state x),
// so H[i][r q + x] = h_r[x][i], the local fields of every replica at once (the
// fields are sums over sites of the coupling to the site's state, Eq. 2).
//
// tcgen05.mma kind::f16 with BF16 operands and FP32 accumulation in tensor
// memory.  X is exact in BF16 (0 or 1); C is carried as three BF16 parts
// hi + mid + lo of the FP64 J* (representation error ~2^-25 J*), each part one
// MMA per K-step (a job may ask for hi + mid only: two MMAs per K-step).  One CTA computes a 128 x TN tile of H (TN = 64 or 128) over
// all of K in chunks of kChunk = 128 sites.
//
// Both operands come from device memory, ready in the MMA's shared-memory
// layout, by bulk asynchronous copies (cp.async.bulk, completion counted on an
// mbarrier), so no thread builds operand tiles:
// - A: the chunk's K sites are taken in reverse order, which makes the
//   circulant tile Hankel: core matrix (g, c) is core matrix g + c of a strip
//   of kHank = 31, and the strip of tile row m0 and chunk k0 depends on
//   m0 - k0 only.  A per-job table (built once at job creation) holds, for
//   every such offset, the strip's core matrices back to back; one A tile is
//   one 3968-byte copy per BF16 part.
// - B: a one-hot kernel writes X before the rebuild, per chunk and 8-row group
//   the 16 core matrices of the chunk's K groups (2 KB); a TN-row tile of a
//   chunk is one contiguous copy of TN x 256 bytes.
// Warp 0 issues the copies into a ring of stages (4 or 7), warp 1 issues the
// MMAs of each chunk part by part (8 K-steps each, 2 or 3 parts) and commits
// them to the stage's "empty" barrier, warps 2..9 read the accumulators.  The FP32 accumulation
// rounds every MMA's sum into the accumulator, so the chains are kept short:
// the hi parts of successive chunks rotate over 512 / TN - 1 accumulators
// (seven or three), and the small mid + lo parts go to one of their own
// (their rounding is then relative to their own small size); together they
// fill the 512 TMEM columns.  The epilogue adds them in FP32 with error-free
// (TwoSum) compensation -- as accurate, for the FP32 fields it stores, as an
// FP64 sum, at a 64th of the cost on GB300's narrow FP64 pipe -- and the old
// values (for the drift) are read from global memory a group of columns ahead,
// which leaves the shared memory to the copy ring.
//
// Operand layout (both K-major, no swizzle): 8-row x 16-byte core matrices.
// A: core matrix h of the strip at byte 128 h; leading (K) and stride (row
// group) byte offsets both 128; K-step s starts at byte 256 s.
// B: core matrix (row group g, K group kc) at byte (16 g + kc) 128; leading
// byte offset 128, stride byte offset 2048; K-step s starts at byte 256 s.
//
// Every wait is bounded (a timer): a pipeline wait that expires (after the
// job's tc_wait_ns, 4 s unless set otherwise) raises a shared abort flag that
// ends the other roles' loops, the job's status word is set, and the CTA
// still drains its own copies and MMAs (waits bounded by 4 s, which such
// waits never approach) before it frees the tensor memory.
#include <algorithm>
#include <cstdint>
#include <vector>

#include "potts_internal.h"

namespace plr {

namespace {

constexpr int kEpiWarps = 8;                       // warps 2..9: two per TMEM lane quarter
constexpr int kTcThreads = 32 * (2 + kEpiWarps);   // + the copy warp and the MMA warp
constexpr int kTileM = 128;
constexpr int kSplit = 3;
constexpr int kHank = kTileM / 8 + kChunk / 8 - 1;  // distinct core matrices of an A tile (Hankel form)
constexpr int kTileBytes = kHank * 128;            // 3968 B per A tile of one part
constexpr int kTmemCols = 512;       // all of the SM's tensor memory: accumulators of TN columns each
constexpr int kOnehotThreads = 256;
constexpr unsigned long long kDrainWaitNs = kTcWaitNs;  // the waits for the CTA's own copies and MMAs at exit
constexpr size_t kTcMinSmem = 120 * 1024;   // forces one CTA per SM (owner of all 512 columns)

// per tile width TN (64 or 128 output columns): accumulators, B tile, stage
template <int TN>
struct TcShape {
    static constexpr int kAcc = kTmemCols / TN;      // 8 or 4 accumulators
    static constexpr int kAccHi = kAcc - 1;          // rotating accumulators of the hi parts; the last takes mid + lo
    static constexpr int kTileBytesB = TN * kChunk * 2;  // TN x kChunk BF16 B tile
    static constexpr int kStageBytes = kSplit * kTileBytes + kTileBytesB;  // three A tiles + the B tile
    // copies run up to kStages - 1 chunks ahead of the MMAs (179 KB of stages
    // at TN = 128, 198 KB at TN = 64)
    static constexpr int kStages = TN == 128 ? 4 : 7;
};
constexpr int kBarBytes = 256;  // full[kStages], empty[kStages], tfull, tempty, drain; TMEM slot; abort flag

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

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Wait for the phase of the given parity to complete; false if the abort
// flag is raised meanwhile (abort may be null: no early exit) or limit_ns
// passes (which raises the flag).  sleep_ns: back-off between polls.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort, uint32_t sleep_ns = 0,
                                          unsigned long long limit_ns = kDrainWaitNs)
{
    unsigned long long t0 = 0;
    for (uint32_t it = 0;; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (abort && *abort) return false;
        // the clock is read at every poll: a try_wait may itself suspend the
        // thread for a while, so polls are few and a read is cheap beside one
        const unsigned long long t = global_ns();
        if (it == 0) t0 = t;
        else if (t - t0 > limit_ns) {
            if (abort) *abort = 1;
            return false;
        }
        if (sleep_ns) __nanosleep(sleep_ns);
    }
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// bulk copy global -> this CTA's shared memory, completion counted on bar
// (addresses 16-byte aligned, bytes a multiple of 16)
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// chunk order of a tile: decreasing circular distance from the chunk holding
// the tile's centre, so the large near-diagonal couplings are added last and
// the many small far-field sums accumulate while the accumulators are still
// small
__device__ __forceinline__ int chunk_of(int t, int m0, int nchunks)
{
    const int cc = ((m0 + kTileM / 2) / kChunk) % nchunks;
    const int kk = nchunks - 1 - t;  // rank in increasing distance: 0, +1, -1, +2, -2, ...
    const int o = kk == 0 ? 0 : ((kk & 1) ? (kk + 1) / 2 : -(kk / 2));
    int c = cc + o;  // |o| <= nchunks / 2
    c += c < 0 ? nchunks : 0;
    c -= c >= nchunks ? nchunks : 0;
    return c;
}

__device__ __forceinline__ bool tile_live(const JobDev& jb, int cond) { return !cond || rebuild_due(jb); }

// output columns of a tile: TN, or 64 for the half-width last column tile of a
// job whose remaining columns are at most 64 (tile.w == 64, only with TN = 128)
template <int TN>
__device__ __forceinline__ int tile_width(const int4& tile)
{
    return (TN == 128 && tile.w == 64) ? 64 : TN;
}

// One-hot B operand of the jobs due for a rebuild (blockIdx.y: entry of the
// job list).  Thread u writes the 16-byte row rr of core matrix (row group G,
// K group kc) of chunk c, u = ((c NG + G) 16 + kc) 8 + rr: element e is 1 when
// replica r_n of row n = 8 G + rr has state x_n at site
// k = 128 c + 127 - 8 kc - e (K reversed within the chunk), else 0.
__global__ void __launch_bounds__(kOnehotThreads) onehot_kernel(const JobDev* __restrict__ jobs,
                                                                const int* __restrict__ idx, int cond)
{
    const JobDev& jb = jobs[idx ? idx[blockIdx.y] : (int)blockIdx.y];
    if (!tile_live(jb, cond)) return;
    const int L = jb.L, q = jb.q, W = jb.W, NG = jb.NG;
    const int N = q * jb.R;
    const long long total = (long long)((L + kChunk - 1) / kChunk) * NG * 128;
    uint4* __restrict__ X = (uint4*)jb.Xoh;
    const long long stride = (long long)gridDim.x * kOnehotThreads;
    for (long long u = (long long)blockIdx.x * kOnehotThreads + threadIdx.x; u < total; u += stride) {
        const int rr = (int)(u & 7), kc = (int)((u >> 3) & 15);
        const long long cg = u >> 7;
        const int c = (int)(cg / NG), G = (int)(cg - (long long)c * NG);
        const int n = 8 * G + rr;
        uint32_t v[4] = {0u, 0u, 0u, 0u};
        if (n < N) {
            const int r = n / q, x = n - r * q;
            const int wi = 16 * c + 15 - kc;  // word of sites 8 wi .. 8 wi + 7: element e is nibble 7 - e
            const uint32_t word = wi < W ? jb.spins[(size_t)r * W + wi] : 0u;
            const int k0 = 128 * c + 127 - 8 * kc;
#pragma unroll
            for (int e = 0; e < 8; ++e)
                if (k0 - e < L && (int)((word >> (4 * (7 - e))) & 15u) == x) v[e >> 1] |= 0x3F80u << (16 * (e & 1));
        }
        X[u] = make_uint4(v[0], v[1], v[2], v[3]);
    }
}

template <int TN>
__global__ void __launch_bounds__(kTcThreads, 1) fields_tc_kernel(const JobDev* __restrict__ jobs,
                                                                  const int4* __restrict__ tiles, int ntiles,
                                                                  int cond)
{
    using S = TcShape<TN>;
    constexpr int kAcc = S::kAcc, kAccHi = S::kAccHi, kStageBytes = S::kStageBytes, kStages = S::kStages;
    static_assert(kAcc * TN == kTmemCols, "accumulators fill the tensor memory");
    static_assert(kStageBytes % 128 == 0, "stages stay 128-byte aligned");
    static_assert((2 * kStages + 3) * 8 + 8 <= kBarBytes, "barriers, TMEM slot and abort flag fit their area");
    static_assert(kStages * kStageBytes + kBarBytes <= 227 * 1024, "one CTA's shared memory");
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    uint64_t* full = (uint64_t*)(smem + kStages * kStageBytes);  // copies of stage b landed
    uint64_t* empty = full + kStages;                              // MMAs reading stage b done
    uint64_t* tfull = empty + kStages;                             // a tile's MMAs done
    uint64_t* tempty = tfull + 1;                                  // its accumulators read
    uint64_t* drain = tfull + 2;                                   // every MMA of the CTA done
    uint32_t* tmem_slot = (uint32_t*)(drain + 1);
    volatile int* abort = (volatile int*)(tmem_slot + 1);

    // skip the whole CTA when none of its tiles is due (no tensor memory taken)
    bool any = false;
    for (int ti = blockIdx.x; ti < ntiles && !any; ti += gridDim.x) any = tile_live(jobs[tiles[ti].x], cond);
    if (!any) return;
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int b = 0; b < kStages; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(full + b)) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(empty + b)) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(tfull)) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(tempty)), "r"(kEpiWarps) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(drain)) : "memory");
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    int failed_job = -1;  // job of the tile at which this thread's wait expired
    uint32_t issued = 0;  // chunks whose copies the copy thread started

    if (warp == 0) {
        // ---- copies: A strips (three parts) and the B tile of each chunk into the stage ring
        if (lane == 0) {
            for (int ti = blockIdx.x; ti < ntiles && failed_job < 0 && !*abort; ti += gridDim.x) {
                const int4 tile = tiles[ti];
                const JobDev& jb = jobs[tile.x];
                if (!tile_live(jb, cond)) continue;
                const int nchunks = (jb.L + kChunk - 1) / kChunk;
                const int m0 = tile.y, n0 = tile.z;
                const unsigned char* hank = (const unsigned char*)jb.Jhank;
                const size_t hank_part = (size_t)jb.hank_cores * 128;
                const unsigned char* xb = (const unsigned char*)jb.Xoh + (size_t)(n0 / 8) * 2048;
                const size_t xchunk = (size_t)jb.NG * 2048;
                for (int t = 0; t < nchunks; ++t) {
                    const uint32_t b = issued % kStages;
                    if (issued >= kStages &&
                        !mbar_wait(smem_u32(empty + b), ((issued / kStages) - 1) & 1u, abort, 0, jb.tc_wait_ns)) {
                        failed_job = tile.x;
                        break;
                    }
                    const int c = chunk_of(t, m0, nchunks);
                    const int j0 = (m0 - c * kChunk) / 8 + 16 * nchunks - 16;  // first core matrix of the strip
                    const uint32_t st = smem_u32(smem + b * kStageBytes);
                    const uint32_t fb = smem_u32(full + b);
                    // a half-width tile (tile.w == 64) copies the first 64 rows of the B tile
                    const uint32_t bbytes = tile_width<TN>(tile) * kChunk * 2;
                    mbar_expect_tx(fb, (uint32_t)(kSplit * kTileBytes) + bbytes);
#pragma unroll
                    for (int sp = 0; sp < kSplit; ++sp)
                        bulk_g2s(st + sp * kTileBytes, hank + sp * hank_part + (size_t)j0 * 128, kTileBytes, fb);
                    bulk_g2s(st + kSplit * kTileBytes, xb + (size_t)c * xchunk, bbytes, fb);
                    ++issued;
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---- MMAs: one thread issues the chunk's MMAs (8 K-steps x 2 or 3 parts) and commits them
        if (lane == 0) {
            const uint32_t idesc_full = make_idesc(kTileM, TN), idesc_half = make_idesc(kTileM, 64);
            uint32_t used = 0, ntile = 0;
            for (int ti = blockIdx.x; ti < ntiles && failed_job < 0 && !*abort; ti += gridDim.x) {
                const int4 tile = tiles[ti];
                const JobDev& jb = jobs[tile.x];
                if (!tile_live(jb, cond)) continue;
                const int nchunks = (jb.L + kChunk - 1) / kChunk;
                const int parts = rebuild_parts(jb);
                const uint32_t idesc = tile_width<TN>(tile) == TN ? idesc_full : idesc_half;
                // the accumulators of the previous tile have been read
                if (ntile > 0 && !mbar_wait(smem_u32(tempty), (ntile - 1) & 1u, abort, 0, jb.tc_wait_ns)) {
                    failed_job = tile.x;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                for (int t = 0; t < nchunks; ++t) {
                    const uint32_t b = used % kStages;
                    if (!mbar_wait(smem_u32(full + b), (used / kStages) & 1u, abort, 0, jb.tc_wait_ns)) {
                        failed_job = tile.x;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t sa = smem_u32(smem + b * kStageBytes);
                    const uint32_t sb = sa + kSplit * kTileBytes;
                    const uint32_t dhi = tmem + (uint32_t)((t % kAccHi) * TN);
                    const uint32_t dsmall = tmem + (uint32_t)(kAccHi * TN);
                    // The descriptors of the chunk's MMAs differ from the stage's
                    // first ones only in the address field (byte address / 16,
                    // 14 bits), and shared-memory addresses stay below 256 KB, so
                    // desc(addr + off) = desc(addr) + off / 16: one add per MMA
                    // instead of a full descriptor build in this single issuing
                    // thread (checked on the host for every stage address)
                    const uint64_t a0 = make_desc(sa, 128, 128), b0 = make_desc(sb, 128, 2048);
                    const bool first_hi = t < kAccHi, first_small = t == 0;
                    // part by part, each over the chunk's 8 K-steps into one
                    // accumulator: issued K-step by K-step with the parts
                    // interleaved (accumulators alternating), every K-step took
                    // about 250 cycles whether it held 2 or 3 MMAs; this order
                    // runs near the tensor cores' rate (measured)
#pragma unroll
                    for (int sp = 0; sp < kSplit; ++sp) {
                        if (sp >= parts) break;  // two parts: hi + mid only
#pragma unroll
                        for (int s = 0; s < kChunk / 16; ++s) {
                            const uint64_t bdesc = b0 + (uint64_t)((s * 256) >> 4);
                            const uint64_t adesc = a0 + (uint64_t)((sp * kTileBytes + s * 256) >> 4);
                            const uint32_t dcol = sp == 0 ? dhi : dsmall;
                            const bool first = s == 0 && (sp == 0 ? first_hi : (first_small && sp == 1));
                            const uint32_t accumulate = first ? 0u : 1u;
                            asm volatile(
                                "{\n\t.reg .pred p;\n\t"
                                "setp.ne.b32 p, %4, 0;\n\t"
                                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dcol),
                                "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
                                : "memory");
                        }
                    }
                    tc_commit(smem_u32(empty + b));  // stage b free once these MMAs have read it
                    ++used;
                }
                if (failed_job >= 0) break;
                tc_commit(smem_u32(tfull));  // the tile's accumulators complete
                ++ntile;
            }
            // every MMA issued by this thread complete before the tensor memory is freed
            tc_commit(smem_u32(drain));
            mbar_wait(smem_u32(drain), 0u, nullptr);
        }
        __syncwarp();
    } else {
        // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 = rows
        // m0 + 32 (w % 4) + lane, columns half (w - 2) / 4 of the tile
        const int quad = warp & 3;
        constexpr int kCols = TN / 2;
        const int cb0 = ((warp - 2) >> 2) * kCols;
        uint32_t ntile = 0;
        for (int ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
            // warp-uniform exit (the accumulator reads below are warp-collective)
            if (__any_sync(0xffffffffu, *abort != 0)) break;
            const int4 tile = tiles[ti];
            const JobDev& jb = jobs[tile.x];
            if (!tile_live(jb, cond)) continue;
            const int L = jb.L, Lpad = jb.Lpad, N = jb.q * jb.R;
            const int nchunks = (L + kChunk - 1) / kChunk;
            const int m0 = tile.y, n0 = tile.z;
            const int i = m0 + 32 * quad + lane;
            float* F = (float*)jb.fields;
            // the fields being replaced (for the drift), read by this thread
            // alone before it writes them: a group of 8 columns one group ahead
            // of its use (the shared memory goes to the copy ring)
            auto load_old = [&](int cb, float (&o)[8]) {
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const bool in = i < L && n0 + cb0 + cb + e < N;
                    o[e] = in ? __ldcg(F + (size_t)(n0 + cb0 + cb + e) * Lpad + i) : 0.0f;
                }
            };
            float onext[8];
            load_old(0, onext);
            // lane 0 polls (backing off: the wait spans the tile's main loop, and
            // polls compete with the copies and MMAs for shared memory); then
            // every lane observes the completed phase itself
            bool got = true;
            if (lane == 0) got = mbar_wait(smem_u32(tfull), ntile & 1u, abort, 256, jb.tc_wait_ns);
            if (!__shfl_sync(0xffffffffu, got, 0)) {
                failed_job = tile.x;
                break;
            }
            mbar_wait(smem_u32(tfull), ntile & 1u, nullptr);
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int nhi = nchunks < kAccHi ? nchunks : kAccHi;
            float dmaxf = 0.0f;
#pragma unroll
            for (int cb = 0; cb < kCols; cb += 8) {
                float ocur[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) ocur[e] = onext[e];
                if (cb + 8 < kCols) load_old(cb + 8, onext);
                uint32_t v[kAcc][8];
#pragma unroll
                for (int a = 0; a < kAcc; ++a) {
                    if (a < nhi || a == kAccHi) {  // the used hi accumulators, and mid + lo
                        const uint32_t taddr = tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)(a * TN + cb0 + cb);
                        asm volatile(
                            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                            : "=r"(v[a][0]), "=r"(v[a][1]), "=r"(v[a][2]), "=r"(v[a][3]), "=r"(v[a][4]),
                              "=r"(v[a][5]), "=r"(v[a][6]), "=r"(v[a][7])
                            : "r"(taddr)
                            : "memory");
                    }
                }
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                // the accumulators summed in FP32 with error-free (TwoSum)
                // compensation, mid + lo first, then the hi parts in order: FP64
                // adds would occupy GB300's two-lane FP64 pipe for most of the tile
                float fs[8], fc[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    fs[e] = __uint_as_float(v[kAccHi][e]);
                    fc[e] = 0.0f;
                }
#pragma unroll
                for (int a = 0; a < kAccHi; ++a)
                    if (a < nhi)
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            const float x = __uint_as_float(v[a][e]);
                            const float t = fs[e] + x;
                            const float bb = t - fs[e];
                            fc[e] += (fs[e] - (t - bb)) + (x - bb);
                            fs[e] = t;
                        }
                if (i < L) {
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const int n = n0 + cb0 + cb + e;
                        if (n < N) {
                            const float r = fs[e] + fc[e];
                            dmaxf = fmaxf(dmaxf, fabsf(ocur[e] - r));  // drift of the ending period
                            F[(size_t)n * Lpad + i] = r;
                        }
                    }
                }
            }
            double dmax = (double)dmaxf;
            for (int o = 16; o > 0; o >>= 1) dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
            if (lane == 0 && dmax > 0.0)
                atomicMax(jb.drift_bits, (unsigned long long)__double_as_longlong(dmax / jb.jtot));
            // the accumulator reads above are complete before the next tile's MMAs
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(tempty));
            ++ntile;
        }
    }
    if (failed_job >= 0) atomicExch(jobs[failed_job].status, 1);  // the host reports ETIMEOUT
    __syncthreads();
    // no copy may still write this CTA's shared memory when it exits: the last
    // phase started on each stage's "full" barrier has completed (immediate
    // when the MMAs consumed it)
    if (tid == 0)
        for (uint32_t g = issued > kStages ? issued - kStages : 0; g < issued; ++g)
            mbar_wait(smem_u32(full + g % kStages), (g / kStages) & 1u, nullptr);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

template <int TN>
size_t tc_smem_bytes()
{
    using S = TcShape<TN>;
    const size_t b = (size_t)S::kStages * S::kStageBytes + kBarBytes;
    return b < kTcMinSmem ? kTcMinSmem : b;
}

}  // namespace

int tc_ng(int q, int R) { return ((q * R + 127) / 128) * 16; }

long long tc_hank_cores(int L) { return (long long)((L + kChunk - 1) / kChunk) * (kChunk / 4) - 1; }

size_t tc_hank_bytes(int L) { return (size_t)kSplit * (size_t)tc_hank_cores(L) * 128; }

size_t tc_onehot_bytes(int L, int q, int R)
{
    return (size_t)((L + kChunk - 1) / kChunk) * (size_t)tc_ng(q, R) * 2048;
}

void tc_hank_table(const std::vector<double>& J, const uint16_t* split, int Lpad, std::vector<uint16_t>& out)
{
    // core matrix j of part sp, row rr, element e: part sp of J*(u mod L),
    // u = 8 j + rr + e + 1 - Lc (the strip of tile row m0 and chunk k0 starts
    // at j0 = (m0 - k0) / 8 + Lc / 8 - 16)
    const int L = (int)J.size();
    const long long ncores = tc_hank_cores(L);
    const long long Lc = (long long)((L + kChunk - 1) / kChunk) * kChunk;
    out.assign((size_t)kSplit * (size_t)ncores * 64, 0);
    for (int sp = 0; sp < kSplit; ++sp)
        for (long long j = 0; j < ncores; ++j)
            for (int rr = 0; rr < 8; ++rr)
                for (int e = 0; e < 8; ++e) {
                    const long long u = 8 * j + rr + e + 1 - Lc;
                    const int r = (int)(((u % L) + L) % L);
                    out[((size_t)sp * ncores + j) * 64 + rr * 8 + e] = split[(size_t)sp * Lpad + r];
                }
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

int tc_onehot_blocks(int L, int q, int R)
{
    const long long rows = (long long)((L + kChunk - 1) / kChunk) * tc_ng(q, R) * 128;
    const long long b = (rows + kOnehotThreads - 1) / kOnehotThreads;
    return (int)(b < 4096 ? b : 4096);
}

cudaError_t launch_fields_tc(const JobDev* jobs_dev, const int* idx, int njobs, int onehot_blocks,
                             const int4* tiles, int ntiles, int cond, int tn, cudaStream_t st)
{
    if (ntiles <= 0 || njobs <= 0) return cudaSuccess;
    onehot_kernel<<<dim3(onehot_blocks > 0 ? onehot_blocks : 1, njobs), kOnehotThreads, 0, st>>>(jobs_dev, idx, cond);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    auto k = tn == 128 ? fields_tc_kernel<128> : fields_tc_kernel<64>;
    const size_t smem = tn == 128 ? tc_smem_bytes<128>() : tc_smem_bytes<64>();
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int sms = device_sm_count() > 0 ? device_sm_count() : 148;
    const int grid = ntiles < sms ? ntiles : sms;  // persistent: one CTA per SM walks the tile table
    k<<<grid, kTcThreads, smem, st>>>(jobs_dev, tiles, ntiles, cond);
    return cudaGetLastError();
}

void tc_tiles(int job, int L, int q, int R, int tn, std::vector<int4>& out)
{
    // at TN = 128 a last column tile with at most 64 columns left runs at
    // half width (w = 64): half the MMA work and B copies
    const int N = q * R;
    for (int m = 0; m < L; m += kTileM)
        for (int n = 0; n < N; n += tn) out.push_back(make_int4(job, m, n, tn == 128 && N - n <= 64 ? 64 : 0));
}

void tc_order_tiles(std::vector<int4>& tiles)
{
    // full-width tiles first: the persistent CTAs take tiles round-robin, so the
    // half-width ones fill the last round
    std::stable_partition(tiles.begin(), tiles.end(), [](const int4& t) { return t.w == 0; });
}

long long tc_tile_count(int L, int q, int R, int tn)
{
    return (long long)((L + kTileM - 1) / kTileM) * ((q * R + tn - 1) / tn);
}

}  // namespace plr
