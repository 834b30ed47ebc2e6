// enum_core.cuh -- the per-tile body of the level enumerators (single-unit kernel and
// batched kernel share it).
//
// A tile of a product block (i-subsets of one half of the rows times (g-i)-subsets
// of the other half) is 32 * XP lane-side subset sums held in registers (XP per lane,
// consecutive colex ranks) times YL walk-side sums staged in the warp's shared-memory
// buffer.  The walk visits every pair: per walk step one broadcast of y, and per lane
// entry the codeword x ^ y.
#pragma once

#include <climits>
#include <cstdint>

#include "combinatorics.cuh"
#include "internal.h"

namespace mdist {

template <int NW>
__device__ __forceinline__ void xor_rows(uint32_t (&x)[NW], const uint32_t *__restrict__ rows, uint32_t mask) {
    while (mask) {
        const int b = __ffs(mask) - 1;
        mask &= mask - 1;
        const uint32_t *r = rows + b * NW;
#pragma unroll
        for (int w = 0; w < NW; ++w) x[w] ^= r[w];
    }
}

// x[p] = sum of the rows of lane-side subset e0 + p (colex ranks), p < nvalid; entries
// past nvalid repeat the previous one (same codewords again, never counted).
template <int NW, int XP>
__device__ __forceinline__ void build_lane_entries(uint32_t (&x)[XP][NW], const uint32_t *__restrict__ bn,
                                                   const uint32_t *__restrict__ rows, int kh, int t, uint32_t e0,
                                                   int nvalid) {
    uint32_t m = unrank_colex(bn, kh, t, e0);
#pragma unroll
    for (int w = 0; w < NW; ++w) x[0][w] = 0;
    xor_rows<NW>(x[0], rows, m);
#pragma unroll
    for (int p = 1; p < XP; ++p) {
#pragma unroll
        for (int w = 0; w < NW; ++w) x[p][w] = x[p - 1][w];
        if (p < nvalid) {
            const uint32_t nm = next_colex(m);
            xor_rows<NW>(x[p], rows, m ^ nm);
            m = nm;
        }
    }
}

// wbuf[s] = sum of the rows of walk-side subset w_first + s, s < walk_len, entries
// walk_stride(NW) words apart (16-byte aligned); lane l builds entries
// [l * per, (l + 1) * per).
template <int NW>
__device__ __forceinline__ void stage_walk(uint32_t *__restrict__ wbuf, const uint32_t *__restrict__ bn,
                                           const uint32_t *__restrict__ rows, int kh, int t,
                                           unsigned long long w_first, int walk_len, int per, int lane) {
    const int s0 = lane * per;
    if (s0 >= walk_len) return;
    uint32_t wm = unrank_colex(bn, kh, t, (uint32_t)(w_first + s0));
    uint32_t y[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) y[w] = 0;
    constexpr int SW = walk_stride(NW);
    xor_rows<NW>(y, rows, wm);
#pragma unroll
    for (int w = 0; w < NW; ++w) wbuf[s0 * SW + w] = y[w];
    for (int q = 1; q < per && s0 + q < walk_len; ++q) {
        const uint32_t nm = next_colex(wm);
        xor_rows<NW>(y, rows, wm ^ nm);
        wm = nm;
#pragma unroll
        for (int w = 0; w < NW; ++w) wbuf[(s0 + q) * SW + w] = y[w];
    }
}

// Lower bound of the weight of x ^ y: sum over groups of G consecutive words of the
// popcount of the OR of the group's XORed words.
template <int NW, int G>
__device__ __forceinline__ int or_bound(const uint32_t (&x)[NW], const uint32_t (&y)[NW]) {
    int lb = 0;
#pragma unroll
    for (int q = 0; q < NW; q += G) {
        uint32_t o = 0;
#pragma unroll
        for (int w = q; w < q + G && w < NW; ++w) o |= x[w] ^ y[w];
        lb += __popc(o);
    }
    return lb;
}

// The walk over one tile.  GS = 0: exact weight of every codeword (XOR, POPC per
// word, sum, running min, one compare per step).  GS = 2, 3, 4: a lower bound first,
// the popcount of the OR of each group of GS XORed words (weight >= bound), and the
// exact weights only in the walk steps where the bound reaches the threshold.  `thr`
// is the largest reduced weight still a candidate; `cand(p, s, reduced_weight)`
// handles a candidate and may lower thr.  HIST adds every valid codeword's weight to s_hist.
template <int NW, int XP, int GS, bool HIST, class Cand>
__device__ __forceinline__ void walk_tile(const uint32_t (&x)[XP][NW], const uint32_t *__restrict__ wbuf,
                                          int walk_len, int nvalid, int &thr, unsigned int *s_hist, int base,
                                          Cand &&cand) {
    constexpr int SW = walk_stride(NW);
    for (int s = 0; s < walk_len; ++s) {
        uint32_t y[NW];
        {  // one broadcast 128-bit shared load per 4 words
            const uint4 *v = reinterpret_cast<const uint4 *>(wbuf + s * SW);
#pragma unroll
            for (int q = 0; q < SW / 4; ++q) {
                const uint4 t = v[q];
                if (4 * q + 0 < NW) y[4 * q + 0] = t.x;
                if (4 * q + 1 < NW) y[4 * q + 1] = t.y;
                if (4 * q + 2 < NW) y[4 * q + 2] = t.z;
                if (4 * q + 3 < NW) y[4 * q + 3] = t.w;
            }
        }
        if (GS == 0) {
            int mn = INT_MAX;
#pragma unroll
            for (int p = 0; p < XP; ++p) {
                int acc = 0;
#pragma unroll
                for (int w = 0; w < NW; ++w) acc += __popc(x[p][w] ^ y[w]);
                mn = acc < mn ? acc : mn;
                if (HIST && p < nvalid) atomicAdd(&s_hist[acc + base], 1u);
            }
            if (mn <= thr) {
#pragma unroll
                for (int p = 0; p < XP; ++p) {
                    int acc = 0;
#pragma unroll
                    for (int w = 0; w < NW; ++w) acc += __popc(x[p][w] ^ y[w]);
                    if (p < nvalid && acc <= thr) cand(p, s, acc);
                }
            }
        } else {
            // lower bound first (weight >= sum over groups of G1 words of the popcount of
            // their OR), minimum over the lane's entries, one branch per step; GS = 5
            // takes groups of 4 first and, in the steps that pass, groups of 2; the exact
            // weights are computed only in steps where the last bound reaches the threshold
            constexpr int G1 = GS == 5 ? 4 : GS;
            int mn = INT_MAX;
#pragma unroll
            for (int p = 0; p < XP; ++p) {
                const int lb = or_bound<NW, G1>(x[p], y);
                mn = lb < mn ? lb : mn;
            }
            if (GS == 5 && mn <= thr) {
                mn = INT_MAX;
#pragma unroll
                for (int p = 0; p < XP; ++p) {
                    const int lb = or_bound<NW, 2>(x[p], y);
                    mn = lb < mn ? lb : mn;
                }
            }
            if (mn <= thr) {
#pragma unroll
                for (int p = 0; p < XP; ++p) {
                    int acc = 0;
#pragma unroll
                    for (int w = 0; w < NW; ++w) acc += __popc(x[p][w] ^ y[w]);
                    if (p < nvalid && acc <= thr) cand(p, s, acc);
                }
            }
        }
    }
}

}  // namespace mdist
