// enum_launch.cu -- level planning (product blocks and tiles) and the dispatch of
// the enumerator instantiations by row width.
#include "internal.h"

namespace mdist {

template <int NW>
cudaError_t launch_nw(const EnumParams &, bool, int, int, cudaStream_t);

unsigned long long binom_host(int a, int b) {
    static unsigned long long tab[kMaxK + 1][kMaxK + 1];
    static bool ready = false;
    if (!ready) {
        for (int x = 0; x <= kMaxK; ++x) {
            for (int y = 0; y <= kMaxK; ++y) tab[x][y] = 0;
            tab[x][0] = 1;
            for (int y = 1; y <= x; ++y) tab[x][y] = tab[x - 1][y - 1] + tab[x - 1][y];
        }
        ready = true;
    }
    if (a < 0 || b < 0 || b > a || a > kMaxK) return 0;
    return tab[a][b];
}

// A level g of a k-row matrix is the disjoint union over i of
// (i-subsets of H1 = rows [0, k1)) x ((g-i)-subsets of H2 = rows [k1, k)).
// Blocks are laid out one after the other in tile space; a tile is
// (32 * XP lane-side entries) x (YL walk-side entries).
bool plan_level(int k, int g, int nwords, EnumParams &p) {
    if (k < 1 || k > kMaxK || g < 1 || g > k) return false;
    if (binom_host(k, g) >= (1ull << kKeyRankBits)) return false;
    const int k1 = (k + 1) / 2;
    const int k2 = k - k1;
    const unsigned long long lane_chunk = 32ull * (unsigned long long)lane_entries_per_thread(nwords);
    const unsigned long long walk_chunk = (unsigned long long)walk_len_for(nwords);
    p.k = k;
    p.k1 = k1;
    p.k2 = k2;
    p.g = g;
    int nb = 0;
    unsigned long long tiles = 0;
    const int ilo = g - k2 > 0 ? g - k2 : 0;
    const int ihi = g < k1 ? g : k1;
    for (int i = ilo; i <= ihi; ++i) {
        const unsigned long long n1 = binom_host(k1, i);
        const unsigned long long n2 = binom_host(k2, g - i);
        ProductBlock &b = p.blocks[nb++];
        if (n1 >= n2) {
            b.lane_half = 0; b.lane_t = (unsigned)i; b.walk_t = (unsigned)(g - i); b.lane_n = n1; b.walk_n = n2;
        } else {
            b.lane_half = 1; b.lane_t = (unsigned)(g - i); b.walk_t = (unsigned)i; b.lane_n = n2; b.walk_n = n1;
        }
        b.pad = 0;
        const unsigned long long lc = (b.lane_n + lane_chunk - 1) / lane_chunk;
        b.walk_chunks = (b.walk_n + walk_chunk - 1) / walk_chunk;
        b.tile_begin = tiles;
        tiles += lc * b.walk_chunks;
    }
    p.nblocks = nb;
    p.total_tiles = tiles;
    return true;
}

size_t enum_smem_bytes(int k, int nwords) {
    return sizeof(uint32_t) * ((size_t)k * nwords + 33 * 33 + (size_t)kWarpsPerCta * walk_len_for(nwords) * nwords);
}

cudaError_t launch_enum_unit(const EnumParams &p, int nwords, bool hist_mode, int sm_count, int blocks_per_sm,
                             cudaStream_t stream) {
    switch (nwords) {
        case 1: return launch_nw<1>(p, hist_mode, sm_count, blocks_per_sm, stream);
        case 2: return launch_nw<2>(p, hist_mode, sm_count, blocks_per_sm, stream);
        case 3: return launch_nw<3>(p, hist_mode, sm_count, blocks_per_sm, stream);
        case 4: return launch_nw<4>(p, hist_mode, sm_count, blocks_per_sm, stream);
        case 5: return launch_nw<5>(p, hist_mode, sm_count, blocks_per_sm, stream);
        case 6: return launch_nw<6>(p, hist_mode, sm_count, blocks_per_sm, stream);
        case 7: return launch_nw<7>(p, hist_mode, sm_count, blocks_per_sm, stream);
        case 8: return launch_nw<8>(p, hist_mode, sm_count, blocks_per_sm, stream);
        case 9: return launch_nw<9>(p, hist_mode, sm_count, blocks_per_sm, stream);
        case 10: return launch_nw<10>(p, hist_mode, sm_count, blocks_per_sm, stream);
        case 11: return launch_nw<11>(p, hist_mode, sm_count, blocks_per_sm, stream);
        case 12: return launch_nw<12>(p, hist_mode, sm_count, blocks_per_sm, stream);
        case 13: return launch_nw<13>(p, hist_mode, sm_count, blocks_per_sm, stream);
        case 14: return launch_nw<14>(p, hist_mode, sm_count, blocks_per_sm, stream);
        case 15: return launch_nw<15>(p, hist_mode, sm_count, blocks_per_sm, stream);
        case 16: return launch_nw<16>(p, hist_mode, sm_count, blocks_per_sm, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace mdist
