// Energy (Eq. 2) and magnetisation (Eq. 10) of one packed configuration:
//   N_r = #{i : s_i = s_{(i+r) mod L}}, r = 1..L/2  (N_{L-r} = N_r)
//   E = -(c/2) sum_{r=1}^{L-1} J*(r) N_r,  M = (q N_max / L - 1) / (q - 1)
// -- the pieces shared by the handle's measure kernel (one CTA per tile of a
// slot's sum) and the allocation-free measure entry point (one CTA per
// configuration, all tiles in turn).
//
// N_r is counted 32 sites at a time on bit planes: plane p of the doubled
// string holds, at bit b of word m, bit p of s_{(32m + b) mod L}, for the
// P = ceil(log2 q) planes a spin needs.  Sites i and i+r hold equal spins iff
// all P planes agree, so the mismatches of the word of sites 32w..32w+31 with
// sites 32w+r..32w+r+31 are popc(OR_p a_p ^ b_p), b_p a funnel shift of two
// plane words.  A thread takes 8 consecutive distances r = 8k+1..8k+8 (they
// share the two words of each plane they shift) over a strided range of words
// w; the sum over (r, w) is cut into tiles of 8*ngp distances by Wt words.
// Each tile sums J*(r) N_r in a fixed order (per thread, then a fixed tree)
// and the tiles are added in tile order, so the result is deterministic and
// depends on L (the tiling) but not on the launch.
#pragma once
#include <cstdint>

#include "potts_internal.h"

namespace plr {

// Tiling of one configuration's sum over (r, w); a function of L alone.
struct MeasGeom {
    int nr;    // L/2 pair distances
    int ng;    // groups of 8 distances: r = 8k+1 .. 8k+8, k < ng
    int W32;   // 32-site words of the configuration (the last may be partial)
    int ngp;   // groups per tile (a power of two <= kAuxThreads)
    int nsub;  // threads per group within a tile (kAuxThreads / ngp), striding over w
    int nrt;   // tiles along r
    int nwt;   // tiles along w
    int Wt;    // words per w tile
};

__host__ __device__ inline MeasGeom meas_geom(int L)
{
    MeasGeom g;
    g.nr = L / 2;
    g.ng = (g.nr + 7) / 8;
    g.W32 = (L + 31) / 32;
    int p = 1;
    while (p < g.ng && p < kAuxThreads) p <<= 1;
    g.ngp = p;
    g.nsub = kAuxThreads / p;
    g.nrt = (g.ng + p - 1) / p;
    // about 64 words per thread; at most kMeasMaxParts tiles in all
    int nwt = g.W32 / (g.nsub * 64);
    const int cap = kMeasMaxParts / g.nrt;
    if (nwt > cap) nwt = cap;
    if (nwt < 1) nwt = 1;
    g.nwt = nwt;
    g.Wt = (g.W32 + nwt - 1) / nwt;
    return g;
}

// bit planes a spin of q states needs
__host__ __device__ inline int meas_planes(int q) { return q <= 2 ? 1 : q <= 4 ? 2 : q <= 8 ? 3 : 4; }

// plane words of the window of any tile: Wt words of the tile plus the
// largest word offset of a distance, plus one
__host__ __device__ inline int meas_window_words(const MeasGeom& g) { return g.Wt + ((8 * (g.ng - 1) + 1) >> 5) + 2; }

// dynamic shared memory of one measuring CTA (every plane of one window)
inline size_t measure_smem_bytes(int L, int q)
{
    const MeasGeom g = meas_geom(L);
    return (size_t)meas_planes(q) * (size_t)meas_window_words(g) * 4;
}

__device__ __forceinline__ double block_sum_fixed(double v, double* red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double tot = 0.0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) tot += red[i];
        red[0] = tot;
    }
    __syncthreads();
    tot = red[0];
    __syncthreads();
    return tot;
}

// bits 0, 4, .., 28 of x gathered into bits 0..7
__device__ __forceinline__ uint32_t gather_nibble_bits(uint32_t x)
{
    x &= 0x11111111u;
    x = (x | (x >> 3)) & 0x03030303u;
    x = (x | (x >> 6)) & 0x000f000fu;
    return (x | (x >> 12)) & 0xffu;
}

// Plane words of string words m0 .. m0+nwin-1 into win[p * ws + j], j = m - m0,
// by the whole CTA.  spins: packed words of the configuration (spin i at bits
// 4(i%8) of word i/8).
__device__ __forceinline__ void build_planes(const uint32_t* __restrict__ spins, int L, int P, int m0, int nwin,
                                             uint32_t* win, int ws)
{
    const int W32 = (L + 31) / 32;
    for (int j = threadIdx.x; j < nwin; j += kAuxThreads) {
        const int m = m0 + j;
        uint32_t pl[4] = {0u, 0u, 0u, 0u};
        if ((L & 31) == 0) {  // sites 32m..32m+31 (mod L) are four whole packed words
            const int mm = m % W32;
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const uint32_t v = spins[4 * mm + h];
#pragma unroll
                for (int p = 0; p < 4; ++p)
                    if (p < P) pl[p] |= gather_nibble_bits(v >> p) << (8 * h);
            }
        } else {
            int pos = (int)(((long long)m * 32) % L);
            for (int b = 0; b < 32; ++b) {
                const uint32_t nib = (spins[pos >> 3] >> (4 * (pos & 7))) & 15u;
#pragma unroll
                for (int p = 0; p < 4; ++p) pl[p] |= ((nib >> p) & 1u) << b;
                if (++pos == L) pos = 0;
            }
        }
#pragma unroll
        for (int p = 0; p < 4; ++p)
            if (p < P) win[p * ws + j] = pl[p];
    }
}

// One thread's share of tile (rt, wt): sum over its group k = rt*ngp + tid%ngp
// and its words w = w_lo + tid/ngp, step nsub, below w_hi, of
// wgt(r) J*(r) N_r(those words) (wgt = 1 at r = L/2 for even L, else 2).
// win holds plane words of string words m0 ..; w_lo >= m0.
template <int P>
__device__ __forceinline__ double measure_tile(const uint32_t* win, int ws, int m0, const MeasGeom& g, int L,
                                               int rt, int w_lo, int w_hi, const double* __restrict__ J)
{
    const int kk = threadIdx.x % g.ngp, ss = threadIdx.x / g.ngp;
    const int k = rt * g.ngp + kk;
    if (k >= g.ng) return 0.0;
    const int rb = 8 * k + 1, qo = rb >> 5, sh0 = rb & 31;  // shifts sh0 + j lie in [1, 32]
    const int full_hi = min(w_hi, L >> 5);                  // words below this hold 32 sites
    int mism[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) mism[j] = 0;
    int sites = 0;
    int w = w_lo + ss;
    for (; w < full_hi; w += g.nsub) {
        uint32_t a[P], lo[P], hi[P];
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const uint32_t* pw = win + p * ws - m0;
            a[p] = pw[w];
            lo[p] = pw[w + qo];
            hi[p] = pw[w + qo + 1];
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            uint32_t x = a[0] ^ __funnelshift_rc(lo[0], hi[0], sh0 + j);
#pragma unroll
            for (int p = 1; p < P; ++p) x |= a[p] ^ __funnelshift_rc(lo[p], hi[p], sh0 + j);
            mism[j] += __popc(x);
        }
        sites += 32;
    }
    if (w < w_hi) {  // the partial last word, w = W32 - 1
        const uint32_t valid = (1u << (L & 31)) - 1u;
        uint32_t a[P], lo[P], hi[P];
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const uint32_t* pw = win + p * ws - m0;
            a[p] = pw[w];
            lo[p] = pw[w + qo];
            hi[p] = pw[w + qo + 1];
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            uint32_t x = a[0] ^ __funnelshift_rc(lo[0], hi[0], sh0 + j);
#pragma unroll
            for (int p = 1; p < P; ++p) x |= a[p] ^ __funnelshift_rc(lo[p], hi[p], sh0 + j);
            mism[j] += __popc(x & valid);
        }
        sites += L & 31;
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int r = rb + j;
        if (r <= g.nr) s += ((2 * r == L) ? 1.0 : 2.0) * J[r] * (double)(sites - mism[j]);
    }
    return s;
}

__device__ __forceinline__ double measure_tile_any(int P, const uint32_t* win, int ws, int m0, const MeasGeom& g,
                                                   int L, int rt, int w_lo, int w_hi, const double* __restrict__ J)
{
    switch (P) {
        case 1: return measure_tile<1>(win, ws, m0, g, L, rt, w_lo, w_hi, J);
        case 2: return measure_tile<2>(win, ws, m0, g, L, rt, w_lo, w_hi, J);
        case 3: return measure_tile<3>(win, ws, m0, g, L, rt, w_lo, w_hi, J);
        default: return measure_tile<4>(win, ws, m0, g, L, rt, w_lo, w_hi, J);
    }
}

// words [w_lo, w_hi) of w tile wt, and the string words its window spans
__device__ __forceinline__ void tile_words(const MeasGeom& g, int rt, int wt, int* w_lo, int* w_hi, int* nwin)
{
    *w_lo = min(g.W32, wt * g.Wt);
    *w_hi = min(g.W32, *w_lo + g.Wt);
    const int kmax = min(g.ng, (rt + 1) * g.ngp) - 1;
    *nwin = (*w_hi - *w_lo) + ((8 * kmax + 1) >> 5) + 2;
}

// Spin counts of one packed configuration (W = ceil(L/8) words) added into
// cnt[0..q-1] by the whole CTA: nibbles equal to x counted per word.
__device__ __forceinline__ void count_states(const uint32_t* __restrict__ spins, int L, int q, int* cnt)
{
    const int W = (L + 7) / 8;
    int own[kMaxQ];
#pragma unroll
    for (int x = 0; x < kMaxQ; ++x) own[x] = 0;
    for (int w = threadIdx.x; w < W; w += kAuxThreads) {
        const uint32_t v = spins[w];
        const int nn = (w == W - 1 && (L & 7)) ? (L & 7) : 8;
        const uint32_t bit3 = nn == 8 ? 0x88888888u : (0x88888888u & ((1u << (4 * nn)) - 1u));
#pragma unroll
        for (int x = 0; x < kMaxQ; ++x) {
            const uint32_t y = v ^ (0x11111111u * (uint32_t)x);
            // bit 3 of a nibble set iff the nibble of y is nonzero
            const uint32_t nz = (((y & 0x77777777u) + 0x77777777u) | y) & bit3;
            own[x] += nn - __popc(nz);
        }
    }
#pragma unroll
    for (int x = 0; x < kMaxQ; ++x)
        if (x < q && own[x]) atomicAdd(&cnt[x], own[x]);
}

// One configuration by one CTA, all tiles in turn.  spins: W = ceil(L/8)
// packed words; J: J*(r) for r = 0..L/2 at least; smem: dynamic shared memory
// of measure_smem_bytes(L, q).  *E and *M are valid in thread 0.
__device__ __forceinline__ void measure_body(const uint32_t* __restrict__ spins, int L, int q, int c,
                                             const double* __restrict__ J, unsigned char* smem, double* E,
                                             double* M)
{
    __shared__ int cnt[kMaxQ];
    __shared__ double red[kAuxThreads / 32];
    const MeasGeom g = meas_geom(L);
    const int P = meas_planes(q), ws = meas_window_words(g);
    uint32_t* win = (uint32_t*)smem;
    if (threadIdx.x < kMaxQ) cnt[threadIdx.x] = 0;
    double part = 0.0;
    for (int rt = 0; rt < g.nrt; ++rt)
        for (int wt = 0; wt < g.nwt; ++wt) {
            int w_lo, w_hi, nwin;
            tile_words(g, rt, wt, &w_lo, &w_hi, &nwin);
            __syncthreads();  // the previous tile's window is no longer read
            build_planes(spins, L, P, w_lo, nwin, win, ws);
            __syncthreads();
            part += measure_tile_any(P, win, ws, w_lo, g, L, rt, w_lo, w_hi, J);
        }
    count_states(spins, L, q, cnt);
    const double tot = block_sum_fixed(part, red);  // its barriers also order the counts
    if (threadIdx.x == 0) {
        int nmax = 0;
        for (int x = 0; x < q; ++x) nmax = max(nmax, cnt[x]);
        *E = -0.5 * (double)c * tot;
        *M = ((double)q * (double)nmax / (double)L - 1.0) / (double)(q - 1);
    }
}

}  // namespace plr
