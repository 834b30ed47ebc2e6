// enum_kernel.cuh -- the level enumerator (hot path) for sm_103a.
//
// One launch enumerates one (g, j) unit of Alg. 1 (§2): every c in F2^k with
// wt(c) = g, the codeword c * Gamma_j and its weight, keeping the least
// (weight, lexicographic rank) among codewords of weight <= U.
//
// Work decomposition (a GPU form of the left/right join of Alg. 5, §3.4):
// the k rows are cut into two disjoint halves H1 = rows [0, k1), H2 = rows [k1, k).
// A g-subset is uniquely an i-subset of H1 joined with a (g-i)-subset of H2, so a
// level is the union over i of full Cartesian products X_i x Y_{g-i}; unlike the
// paper's join (right part must start after the left part's last element) every
// pair is valid, which keeps all 32 lanes of a warp on the same control path.
// For each product block the larger side is the "lane side": every lane builds XP
// consecutive lane-side sums in registers (combinatorial-number-system unranking of
// the first, then colex successors, each one XOR of the changed rows).  The warp
// stages YL consecutive walk-side sums in shared memory the same way, then walks
// them: each step is one shared-memory broadcast of y and, per lane entry, the
// XOR x ^ y, POPC per 32-bit word, a running minimum, and one compare against the
// threshold.  Codewords at or below the threshold (rare) take a side path that
// recovers their combination, its lexicographic rank, and updates the per-thread
// best key and the unit's U (atomicMin) so every warp prunes with the newest U.
// Warps take tiles (lane chunk x walk chunk) from a global counter (persistent
// grid); at the end the warp's best key is reduced with __reduce_min_sync and one
// atomicMin per warp publishes it.
#pragma once

#include <climits>
#include <cstdint>

#include "combinatorics.cuh"
#include "enum_core.cuh"
#include "internal.h"

namespace mdist {

static __constant__ BinomTable64 c_binom = make_binom_table64();

struct DeviceBinom {
    __device__ __forceinline__ unsigned long long operator()(int a, int b) const { return c_binom.v[a][b]; }
};

// Side path for a codeword at or below the threshold: rebuild its combination,
// compute the key, publish the weight.  Kept out of line so the hot loop stays small.
static __device__ __forceinline__ unsigned long long candidate_key(const EnumParams &P, const ProductBlock &B,
                                                         const uint32_t *bn, uint32_t lane_rank, uint32_t walk_rank,
                                                         int weight) {
    const int lane_kh = B.lane_half ? P.k2 : P.k1;
    const int walk_kh = B.lane_half ? P.k1 : P.k2;
    const uint32_t lm = unrank_colex(bn, lane_kh, (int)B.lane_t, lane_rank);
    const uint32_t wm = unrank_colex(bn, walk_kh, (int)B.walk_t, walk_rank);
    const unsigned long long h1 = B.lane_half ? wm : lm;
    const unsigned long long h2 = B.lane_half ? lm : wm;
    const unsigned long long full = h1 | (h2 << P.k1);
    const unsigned long long rank = lexrank64(full, P.k, P.g, DeviceBinom{});
    atomicMin(P.U, (unsigned int)weight);
    return ((unsigned long long)weight << kKeyRankBits) | rank;
}

template <int NW>
struct EnumCfg {
    static constexpr int XP = lane_entries_per_thread(NW);  // lane-side entries per thread
    static constexpr int YL = walk_len_for(NW);             // walk-side entries per tile
};

template <int NW, int GS, bool HIST>
__global__ void __launch_bounds__(kCtaThreads, MDIST_ENUM_MIN_BLOCKS) enum_unit_kernel(const __grid_constant__ EnumParams P) {
    constexpr int XP = EnumCfg<NW>::XP;
    constexpr int YL = EnumCfg<NW>::YL;
    constexpr int PER = YL / 32;
    constexpr int SW = walk_stride(NW);
    extern __shared__ __align__(16) uint32_t smem[];
    uint32_t *s_walk = smem;                             // warps x YL x SW (16-byte entries)
    uint32_t *s_rows = s_walk + kWarpsPerCta * YL * SW;  // k x NW
    uint32_t *s_bn = s_rows + P.k * NW;                  // 33 x 33
    unsigned int *s_hist = s_bn + kBn * kBn;             // histogram mode: n+1 bins

    // bits past n_bits are cleared while staging, so that no weight exceeds n_bits (the
    // histogram index stays inside s_hist) whatever the caller's padding holds
    for (int i = threadIdx.x; i < P.k * NW; i += blockDim.x) {
        const int vb = P.n_bits - 32 * (i % NW);
        const uint32_t valid = vb >= 32 ? 0xFFFFFFFFu : (vb <= 0 ? 0u : (1u << vb) - 1u);
        s_rows[i] = P.rows[i] & valid;
    }
    for (int i = threadIdx.x; i < kBn * kBn; i += blockDim.x) {
        const unsigned long long v = c_binom.v[i / kBn][i % kBn];
        s_bn[i] = (uint32_t)v;  // C(a, b) <= C(32, 16) < 2^32
    }
    if (HIST)
        for (int i = threadIdx.x; i <= P.n_bits + P.base; i += blockDim.x) s_hist[i] = 0;
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    uint32_t *wbuf = s_walk + warp * YL * SW;
    UnitSlot *slot = P.slot;
    int thr = (int)(*(volatile unsigned int *)P.U) - P.base;  // candidates: reduced weight <= thr
    unsigned long long best = kNoKey;
    unsigned long long cnt = 0;

    for (;;) {
        unsigned long long tile = 0;
        if (lane == 0) tile = P.tile_lo + atomicAdd(&slot->tile_next, 1ull);
        tile = __shfl_sync(0xffffffffu, tile, 0);
        if (tile >= P.total_tiles) break;
        int b = 0;
        while (b + 1 < P.nblocks && tile >= P.blocks[b + 1].tile_begin) ++b;
        const ProductBlock &B = P.blocks[b];
        const unsigned long long t = tile - B.tile_begin;
        const unsigned long long lane_chunk = t / B.walk_chunks;
        const unsigned long long walk_chunk = t - lane_chunk * B.walk_chunks;
        const int lane_kh = B.lane_half ? P.k2 : P.k1;
        const int walk_kh = B.lane_half ? P.k1 : P.k2;
        const uint32_t *lane_rows = s_rows + (B.lane_half ? P.k1 : 0) * NW;
        const uint32_t *walk_rows = s_rows + (B.lane_half ? 0 : P.k1) * NW;

        {  // newest U from the other warps
            const int gU = (int)(*(volatile unsigned int *)P.U) - P.base;
            thr = gU < thr ? gU : thr;
        }

        // ---- lane side: XP consecutive entries per lane, in registers ----
        const unsigned long long chunk_first = lane_chunk * (unsigned long long)(32 * XP);
        const unsigned long long e_first = chunk_first + (unsigned long long)lane * XP;
        const long long left = (long long)B.lane_n - (long long)e_first;
        const int nvalid = left <= 0 ? 0 : (left >= XP ? XP : (int)left);
        const uint32_t e0 = (uint32_t)(e_first < B.lane_n ? e_first : B.lane_n - 1);
        uint32_t x[XP][NW];
        build_lane_entries<NW, XP>(x, s_bn, lane_rows, lane_kh, (int)B.lane_t, e0, nvalid);

        // ---- walk side: YL consecutive entries staged in this warp's buffer ----
        const unsigned long long w_first = walk_chunk * (unsigned long long)YL;
        const unsigned long long wleft = B.walk_n - w_first;
        const int walk_len = wleft >= (unsigned long long)YL ? YL : (int)wleft;
        stage_walk<NW>(wbuf, s_bn, walk_rows, walk_kh, (int)B.walk_t, w_first, walk_len, PER, lane);
        __syncwarp();

        // ---- the walk ----
        walk_tile<NW, XP, GS, HIST>(x, wbuf, walk_len, nvalid, thr, s_hist, P.base, [&](int p, int s, int acc) {
            const unsigned long long key =
                candidate_key(P, B, s_bn, e0 + (uint32_t)p, (uint32_t)(w_first + s), acc + P.base);
            best = key < best ? key : best;
            thr = acc;
        });
        if (lane == 0) {
            const unsigned long long in_chunk = B.lane_n - chunk_first;
            const unsigned long long lanes_valid = in_chunk < (unsigned long long)(32 * XP) ? in_chunk : 32 * XP;
            cnt += lanes_valid * (unsigned long long)walk_len;
        }
        __syncwarp();
    }

    // ---- publish: warp min of the 64-bit keys (two 32-bit reductions), counters ----
    const unsigned int hi = (unsigned int)(best >> 32);
    const unsigned int mhi = __reduce_min_sync(0xffffffffu, hi);
    const unsigned int lo = hi == mhi ? (unsigned int)best : 0xffffffffu;
    const unsigned int mlo = __reduce_min_sync(0xffffffffu, lo);
    if (lane == 0) {
        const unsigned long long wbest = ((unsigned long long)mhi << 32) | mlo;
        if (wbest != kNoKey) atomicMin(&slot->key, wbest);
        if (cnt) atomicAdd(&slot->count, cnt);
    }
    if (HIST) {
        __syncthreads();
        for (int i = threadIdx.x; i <= P.n_bits + P.base; i += blockDim.x)
            if (s_hist[i]) atomicAdd(&P.hist[i], (unsigned long long)s_hist[i]);
    }
}

inline size_t enum_smem_bytes_nw(int k, int nw, int hist_bins) {
    const int yl = walk_len_for(nw);
    return sizeof(uint32_t) *
           ((size_t)k * nw + kBn * kBn + (size_t)kWarpsPerCta * yl * walk_stride(nw) + (size_t)hist_bins);
}

template <int NW, int GS, bool HIST>
cudaError_t launch_variant(const EnumParams &p, int sm_count, int blocks_per_sm, cudaStream_t stream) {
    const int hist_bins = HIST ? p.n_bits + p.base + 1 : 0;
    const size_t smem = enum_smem_bytes_nw(p.k, NW, hist_bins);
    auto kern = enum_unit_kernel<NW, GS, HIST>;
    cudaError_t e = allow_dynamic_smem((const void *)kern, smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = mdist::blocks_per_sm((const void *)kern, kCtaThreads, smem, &occ);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const int per_sm = blocks_per_sm > 0 && blocks_per_sm < occ ? blocks_per_sm : occ;
    unsigned long long want = (p.total_tiles - p.tile_lo + kWarpsPerCta - 1) / kWarpsPerCta;
    unsigned long long grid = (unsigned long long)sm_count * (unsigned long long)per_sm;
    if (want < grid) grid = want;
    if (grid < 1) grid = 1;
    kern<<<(unsigned int)grid, kCtaThreads, smem, stream>>>(p);
    return cudaGetLastError();
}

// group: 0 = exact count for every codeword; 2, 3, 4 = OR-group lower bound first;
// 5 = groups of 4, then groups of 2, then exact
template <int NW>
cudaError_t launch_nw(const EnumParams &p, int group, bool hist_mode, int sm_count, int blocks_per_sm,
                      cudaStream_t stream) {
    if (hist_mode) return launch_variant<NW, 0, true>(p, sm_count, blocks_per_sm, stream);
    switch (group) {
        case 0: return launch_variant<NW, 0, false>(p, sm_count, blocks_per_sm, stream);
        case 2: return launch_variant<NW, 2, false>(p, sm_count, blocks_per_sm, stream);
        case 3: return launch_variant<NW, 3, false>(p, sm_count, blocks_per_sm, stream);
        case 4: return launch_variant<NW, 4, false>(p, sm_count, blocks_per_sm, stream);
        case 5: return launch_variant<NW, 5, false>(p, sm_count, blocks_per_sm, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace mdist
