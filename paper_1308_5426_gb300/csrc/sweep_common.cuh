// Pieces shared by the sweep kernels: the proposal draw of one site and the
// exact in-order decision of a block of 32 sites by one warp (Eq. 8, Sec. 4.2).
#pragma once
#include <cmath>
#include <cstdint>

#include "near_tie.cuh"
#include "philox.cuh"
#include "potts_internal.h"

namespace plr {

constexpr unsigned kFullMask = 0xffffffffu;
constexpr int kNearTable = 64;  // J* in FP32 for distances < 64 (corrections within two blocks)
enum : int { kReject = 0, kAccept = 1, kUnsure = 2 };

// (lo, hi) += v: 128-bit unsigned accumulation
__device__ __forceinline__ void u128_add(unsigned long long& lo, unsigned long long& hi, unsigned long long v)
{
    lo += v;
    hi += lo < v ? 1ull : 0ull;
}

// Exact sum over the CTA of every thread's 128-bit (lo, hi), returned to every
// thread as hi 2^64 + lo in FP64 by one fixed formula -- the same value
// whatever the order of the terms (FX64 energies, from non-negative integer
// fields).  scratch: shared memory of 2 words per warp of the CTA.
__device__ __forceinline__ double block_sum_u128(unsigned long long lo, unsigned long long hi,
                                                 unsigned long long* scratch)
{
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long l2 = __shfl_xor_sync(kFullMask, lo, o);
        const unsigned long long h2 = __shfl_xor_sync(kFullMask, hi, o);
        u128_add(lo, hi, l2);
        hi += h2;
    }
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();  // the scratch may have been read by an earlier step
    if ((threadIdx.x & 31) == 0) {
        scratch[2 * warp] = lo;
        scratch[2 * warp + 1] = hi;
    }
    __syncthreads();
    unsigned long long L0 = 0, H0 = 0;
    for (int w = 0; w < nw; ++w) {
        u128_add(L0, H0, scratch[2 * w]);
        H0 += scratch[2 * w + 1];
    }
    __syncthreads();
    return (double)H0 * 0x1p64 + (double)L0;
}

// FP64 rule, evaluated exactly: dE <= 0 or u < exp(-beta dE).  A decision
// with |beta dE + ln u| < 1e-9 (on either branch) is a near tie: counted, and
// logged as attempt `attempt` of slot ns.t at sweep ns.n.
__device__ __forceinline__ bool decide_fp64_exact(double d, double cb, double u, unsigned long long& near,
                                                  const NearSink& ns, int attempt)
{
    const double x = cb * d;  // beta * c * d
    const bool acc = d <= 0.0 || u < exp(-x);
    if (x < 40.0 && fabs(x + log(u)) < kNearTie) {
        ++near;
        near_tie_log(ns.log, ns.count, 0, ns.t, ns.n, attempt, acc);
    }
    return acc;
}

// FP32 filter of the FP64 rule.  d32 is within errd of the FP64 d: errd =
// 2.4e-5 Jtot bounds the conversion and up to 64 FP32 corrections of
// magnitude <= 3 Jtot, each rounded to 2^-24, with a factor 2 to spare; x and
// -ln u are within 2.4e-7 relative of their FP64 values.
__device__ __forceinline__ int decide_fp64_filter(float d, float cb, float nlu, float errd)
{
    if (d <= -errd) return kAccept;
    if (d < errd) return kUnsure;
    const float x = cb * d;
    const float m = cb * errd + 1e-6f * (x + nlu + 1.0f);
    if (x < nlu - m) return kAccept;
    if (x > nlu + m) return kReject;
    return kUnsure;
}

// The same screen in threshold form, fixed per lane for a block: a lane
// accepts for sure if d <= -errd or errd <= d < dA, rejects for sure if
// d > dR (always > errd), and is unsure otherwise, with
//   dA = (nlu (1 - 2e-6) - cb errd - 2e-6) / (cb (1 + 2e-6)),
//   dR = (nlu (1 + 2e-6) + cb errd + 2e-6) / (cb (1 - 2e-6)):
// the margins of decide_fp64_filter doubled, which also covers the rounding
// of the division (each bound is formed with a reciprocal and products that
// move it towards the unsure band).  Within a block's scan the verdict is
// then one compare (d <= dR) and the unsure test runs beside it.
struct Screen {
    float dAe;  // max(dA, errd): sure accepts below, from errd up
    float dR;
};
__device__ __forceinline__ Screen fp64_screen(float cb, float nlu, float errd)
{
    const float r = 1.0f / cb;
    const float dA = (nlu * (1.0f - 2e-6f) - cb * errd - 2e-6f) * r * (1.0f - 2e-6f);
    const float dR = (nlu * (1.0f + 2e-6f) + cb * errd + 2e-6f) * r * (1.0f + 2e-6f);
    return Screen{fmaxf(dA, errd), dR};
}

// Proposal of site k of slot t at sweep n: b uniform over the other q-1 states
// and nlu = -ln u in FP32.  (ux1, ux2) are the words u is made of: FP64 mode's
// u = ((ux1:ux2 >> 11) + 1) 2^-53 is formed only when the exact rule runs; its
// FP32 value here is within 2^-23 relative.  FP32 mode: u = ((ux1 >> 8) + 1) 2^-24.
template <bool kFP64>
__device__ __forceinline__ void draw_proposal(int k, int t, uint32_t n, uint32_t key0, uint32_t key1, int q, int a,
                                              int& b, float& nlu, uint32_t& ux1, uint32_t& ux2)
{
    const U4 x = philox10(U4{(uint32_t)k, (uint32_t)t, n, kTagMetro}, key0, key1);
    b = a + 1 + (int)__umulhi(x.x, (uint32_t)(q - 1));
    if (b >= q) b -= q;
    ux1 = x.y;
    ux2 = x.z;
    if constexpr (kFP64) {
        const float uf = (float)x.y * 0x1p-32f + (float)((x.z >> 11) + 1u) * 0x1p-53f;
        nlu = -logf(uf);
    } else {
        nlu = -logf(unit24(x.y));
    }
}

// Decide the nv sites of a block in site order, exactly as a sequential sweep
// would.  Lane l holds site k = k0 + l (valid if l < nv) with spin a, proposal
// b, nlu = -ln u, and d32 = h[a][k] - h[b][k] read from fields that do not yet
// hold the flips (pk, pab)[0..npend) of the previous block (base64: the same
// difference in FP64 mode).  First those flips are added as corrections; then
// all undecided lanes evaluate the rule at once: the first lane that accepts
// is certain to accept, every lane before it to reject.  After accepted flip j
// every later lane corrects d32 by J*(l-j)([a=b_j]-[a=a_j]-[b=b_j]+[b=a_j]) --
// the change flip j makes to h at site k_l -- and the scan continues after j,
// one round per accepted flip.  Accepted flips are appended to (ck, cab) in
// site order; returns their number.  Jn: J*(r) in FP32 for r < 64; J64: the
// FP64 table (for the exact rule in FP64 mode).
// kMode: 0 = FP32 rule; 1 = FP64 rule (FP32 filter, exact FP64 difference
// where the filter is unsure); 2 = FX64: the FP64 rule with the exact
// difference kept in fixed point -- basefx = h[a][k] - h[b][k] in field
// units, Jfx the rounded integer table, fxs = 2^-F the value of one unit; the
// corrections are integer adds, so the difference is exact before its one
// conversion to FP64.
// Lanes j whose proposal shares a state with this lane's, from the bit planes
// of the block's states (q <= 16): bit j of m_ab is [a == b_j], of m_aa
// [a == a_j], of m_bb [b == b_j], of m_ba [b == a_j].  The whole warp calls it.
__device__ __forceinline__ void state_masks(int a, int b, unsigned& m_ab, unsigned& m_aa, unsigned& m_bb,
                                            unsigned& m_ba)
{
    m_ab = m_aa = m_bb = m_ba = kFullMask;
#pragma unroll
    for (int bit = 0; bit < 4; ++bit) {
        const unsigned pa = __ballot_sync(kFullMask, (a >> bit) & 1);
        const unsigned pb = __ballot_sync(kFullMask, (b >> bit) & 1);
        const bool ia = (a >> bit) & 1, ib = (b >> bit) & 1;
        m_ab &= ia ? pb : ~pb;
        m_aa &= ia ? pa : ~pa;
        m_bb &= ib ? pb : ~pb;
        m_ba &= ib ? pa : ~pa;
    }
}

// The FP64 rule for lane j of a block, where the FP32 screen is unsure: lane
// j rebuilds its FP64 difference from the previous block's flips and this
// block's accepted ones before j (written to ck, cab here), in FX64 fields
// exactly in integers (kMode 2) or in FP64 (kMode 1).  The whole warp calls
// it; returns the decision (bit 0, every lane) and lane j's near-tie count
// (bit 1).
template <int kMode>
__device__ __noinline__ int decide_exact_lane(int lane, int j, unsigned accmask, int k, int L, int a, int b, int ab,
                                              uint32_t ux1, uint32_t ux2, double base64, const int* pk,
                                              const int* pab, int npend, double cb64, const double* J64, int* ck,
                                              int* cab, long long basefx, const long long* Jfx, double fxs,
                                              NearSink ns)
{
    const unsigned before = accmask & ((1u << j) - 1u);
    if (accmask & (1u << lane)) {
        const int pos = __popc(accmask & ((1u << lane) - 1u));
        ck[pos] = k;
        cab[pos] = ab;
    }
    __syncwarp();
    bool dec = false;
    unsigned long long near = 0;
    if (lane == j) {
        double d64;
        const int nb = __popc(before);
        if constexpr (kMode == 2) {
            long long dx = basefx;
            for (int g = 0; g < npend; ++g) {
                const int kf = pk[g], af = pab[g] >> 8, bf = pab[g] & 255;
                int r = k - kf;
                r += r < 0 ? L : 0;
                const int coef = (a == bf) - (a == af) - (b == bf) + (b == af);
                if (coef) dx += (long long)coef * Jfx[r];
            }
            for (int g = 0; g < nb; ++g) {
                const int kf = ck[g], af = cab[g] >> 8, bf = cab[g] & 255;
                const int coef = (a == bf) - (a == af) - (b == bf) + (b == af);
                if (coef) dx += (long long)coef * Jfx[k - kf];
            }
            d64 = (double)dx * fxs;
        } else {
            d64 = base64;
            for (int g = 0; g < npend; ++g) {
                const int kf = pk[g], af = pab[g] >> 8, bf = pab[g] & 255;
                int r = k - kf;
                r += r < 0 ? L : 0;
                const int coef = (a == bf) - (a == af) - (b == bf) + (b == af);
                if (coef) d64 += (double)coef * J64[r];
            }
            for (int g = 0; g < nb; ++g) {
                const int kf = ck[g], af = cab[g] >> 8, bf = cab[g] & 255;
                const int coef = (a == bf) - (a == af) - (b == bf) + (b == af);
                if (coef) d64 += (double)coef * J64[k - kf];
            }
        }
        dec = decide_fp64_exact(d64, cb64, unit53(ux1, ux2), near, ns, k);
    }
    const bool acc = __shfl_sync(kFullMask, dec, j);
    __syncwarp();
    return (acc ? 1 : 0) | (int)(near << 1);
}

template <int kMode>
__device__ __forceinline__ int decide_block(int lane, int nv, int k, int L, int a, int b, float nlu, uint32_t ux1,
                                            uint32_t ux2, float d32, double base64, const int* pk, const int* pab,
                                            int npend, float cb32, double cb64, float errd, const float* Jn,
                                            const double* J64, int* ck, int* cab, bool& mine, float& dmine,
                                            unsigned long long& nnear, long long basefx = 0,
                                            const long long* Jfx = nullptr, double fxs = 0.0,
                                            const NearSink& ns = NearSink{nullptr, nullptr, 0, 0u})
{
    constexpr bool kFP64 = kMode != 0;
    const bool valid = lane < nv;
    // The state masks (state_masks) give the change of this lane's difference
    // by a flip at j of this block: ([a == b_j] - [a == a_j] - [b == b_j] +
    // [b == a_j]) J*(lane - j).  They are made at the block's first accepted
    // flip, so that blocks without flips do not pay for them.
    unsigned m_ab = 0u, m_aa = 0u, m_bb = 0u, m_ba = 0u;
    bool masks = false;
    // corrections for the previous block's flips, eight independent loads at a time
    int f = 0;
    for (; f + 8 <= npend; f += 8) {
        float jv[8];
        int cf[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int kf = pk[f + e], af = pab[f + e] >> 8, bf = pab[f + e] & 255;
            int r = k - kf;
            r += r < 0 ? L : 0;  // 1..63 for valid lanes
            jv[e] = Jn[r & (kNearTable - 1)];
            cf[e] = (a == bf) - (a == af) - (b == bf) + (b == af);
        }
#pragma unroll
        for (int e = 0; e < 8; ++e) d32 = fmaf((float)cf[e], jv[e], d32);
    }
    for (; f < npend; ++f) {
        const int kf = pk[f], af = pab[f] >> 8, bf = pab[f] & 255;
        int r = k - kf;
        r += r < 0 ? L : 0;
        const int coef = (a == bf) - (a == af) - (b == bf) + (b == af);
        d32 = fmaf((float)coef, Jn[r & (kNearTable - 1)], d32);
    }
    const int ab = (a << 8) | b;
    unsigned accmask = 0;  // lanes whose flip was accepted
    dmine = 0.0f;
    // One round per accepted flip; the loop ends on an empty ballot (lanes at
    // or past nv never vote), with no separate test of p on the round's chain.
    Screen scr{0.0f, 0.0f};
    if constexpr (kFP64) scr = fp64_screen(cb32, nlu, errd);
    int p = 0;
    while (true) {
        bool vote, unsure_l = false;
        if constexpr (kFP64) {
            vote = d32 <= scr.dR;
            unsure_l = (d32 > -errd && d32 < errd) || (d32 >= scr.dAe && d32 <= scr.dR);
        } else {
            vote = d32 <= 0.0f || cb32 * d32 < nlu;
        }
        const bool live = valid && lane >= p;
        const unsigned hit = __ballot_sync(kFullMask, vote && live);
        // FP64 rule: the lanes the FP32 screen left unsure, from a ballot beside
        // the first (a bit test of lane j, no shuffle on the round's chain)
        const unsigned unsure = kFP64 ? __ballot_sync(kFullMask, unsure_l && live) : 0u;
        if (!hit) break;
        const int j = __ffs(hit) - 1;
        bool acc = true;
        if constexpr (kFP64) {
            if ((unsure >> j) & 1u) {
                // rare: lane j applies the FP64 rule to the FP64 difference (out of
                // line, so that the common round carries none of its code)
                const int r = decide_exact_lane<kMode>(lane, j, accmask, k, L, a, b, ab, ux1, ux2, base64, pk, pab,
                                                       npend, cb64, J64, ck, cab, basefx, Jfx, fxs, ns);
                acc = r & 1;
                nnear += (unsigned long long)(r >> 1);
            }
        }
        if (acc) {
            if (!masks) {  // warp-uniform
                masks = true;
                state_masks(a, b, m_ab, m_aa, m_bb, m_ba);
            }
            const float jd = Jn[(lane - j) & 31];
            const unsigned bj = 1u << j;
            accmask |= bj;
            dmine = lane == j ? d32 : dmine;
            // coefficient x J*, exact (a multiple of jd by -2..2), then one rounding
            const float t = (((m_ab & bj) ? jd : 0.0f) + ((m_ba & bj) ? jd : 0.0f)) -
                            (((m_aa & bj) ? jd : 0.0f) + ((m_bb & bj) ? jd : 0.0f));
            d32 += (lane > j) ? t : 0.0f;  // lanes past nv: never read
        }
        p = j + 1;
    }
    // the accepted flips, in site order
    mine = (accmask >> lane) & 1u;
    if (mine) {
        const int pos = __popc(accmask & ((1u << lane) - 1u));
        ck[pos] = k;
        cab[pos] = ab;
    }
    __syncwarp();
    return __popc(accmask);
}

}  // namespace plr
