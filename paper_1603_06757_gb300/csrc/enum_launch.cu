// enum_launch.cu -- level planning (product blocks and tiles) and the dispatch of
// the enumerator instantiations by row width.
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "internal.h"

namespace mdist {

template <int NW>
cudaError_t launch_nw(const EnumParams &, int, bool, int, int, cudaStream_t);

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

// Distribution of the OR-group lower bound for a codeword with iid Bernoulli(1/2)
// bits (what the rows of a random code give): a bit position of a group is 1 in the
// OR with probability 1 - 2^-c, c = words of the group that store that position.
// Returned as the CDF over 0..n_bits, cached per (nwords, n_bits, group).
static const std::vector<double> &lower_bound_cdf(int nwords, int n_bits, int gs) {
    static std::mutex mu;
    static std::map<std::tuple<int, int, int>, std::vector<double>> cache;
    std::lock_guard<std::mutex> lock(mu);
    auto key = std::make_tuple(nwords, n_bits, gs);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    std::vector<double> dist(1, 1.0);
    for (int q = 0; q < nwords; q += gs) {
        for (int pos = 0; pos < 32; ++pos) {
            int c = 0;
            for (int w = q; w < q + gs && w < nwords; ++w)
                if (w * 32 + pos < n_bits) ++c;
            if (c == 0) continue;
            const double p1 = 1.0 - std::ldexp(1.0, -c);
            std::vector<double> nd(dist.size() + 1, 0.0);
            for (size_t v = 0; v < dist.size(); ++v) {
                nd[v] += dist[v] * (1.0 - p1);
                nd[v + 1] += dist[v] * p1;
            }
            dist.swap(nd);
        }
    }
    for (size_t v = 1; v < dist.size(); ++v) dist[v] += dist[v - 1];
    return cache.emplace(key, std::move(dist)).first->second;
}

// Expected SM clocks per codeword: POPC retire at 16 per SM-clock, issue at 128 per
// SM-clock (4 schedulers x 32 lanes).  Exact variant: nwords XOR + nwords POPC +
// ~nwords adds/min.  Group variant: nwords fused XOR/OR (LOP3) + one POPC and one
// add/min per group; a walk step (32 lanes x XP entries) whose minimum bound reaches
// the threshold also pays the exact count of all its entries.
int choose_filter_group(int nwords, int n_bits, int thr) {
    const double exact = std::fmax(nwords / 16.0, 3.0 * nwords / 128.0);
    if (thr >= n_bits) return 0;
    const double step_cw = 32.0 * lane_entries_per_thread(nwords);
    auto pstep = [&](int gs) {
        if (thr < 0) return 0.0;
        const std::vector<double> &cdf = lower_bound_cdf(nwords, n_bits, gs);
        const double p = cdf[(size_t)(thr < (int)cdf.size() ? thr : (int)cdf.size() - 1)];
        return 1.0 - std::pow(1.0 - p, step_cw);
    };
    double best_cost = exact;
    int best = 0;
    for (int gs = 2; gs <= 4; ++gs) {
        if (gs > nwords) break;
        const int ng = (nwords + gs - 1) / gs;
        const double ps = pstep(gs);
        const double popc = ng + ps * nwords;
        const double instr = nwords + 2.0 * ng + ps * (3.0 * nwords + 3.0);
        const double cost = std::fmax(popc / 16.0, instr / 128.0);
        if (cost < best_cost * 0.98) {
            best_cost = cost;
            best = gs;
        }
    }
    if (nwords >= 4) {  // two levels: groups of 4, then groups of 2 where the first passes
        const int ng4 = (nwords + 3) / 4, ng2 = (nwords + 1) / 2;
        const double p4 = pstep(4), p2 = pstep(2);
        const double popc = ng4 + p4 * ng2 + p2 * nwords;
        const double instr = nwords + 2.0 * ng4 + p4 * (nwords + 2.0 * ng2 + 2.0) + p2 * (3.0 * nwords + 3.0);
        const double cost = std::fmax(popc / 16.0, instr / 128.0);
        if (cost < best_cost * 0.98) {
            best_cost = cost;
            best = 5;
        }
    }
    return best;
}

size_t enum_smem_bytes(int k, int nwords) {
    return sizeof(uint32_t) *
           ((size_t)k * nwords + 33 * 33 + (size_t)kWarpsPerCta * walk_len_for(nwords) * walk_stride(nwords));
}

// One unit: the tensor-core blocks, then the product blocks they do not cover on the
// ALU kernel.  Both launches share the threshold word, key, count and status of `p`.
cudaError_t launch_unit_split(const EnumParams &p, int nwords, int group, bool hist_mode, int sm_count,
                              int blocks_per_sm, const GramBlockSpec *gblocks, int ngblocks, const bool *covered,
                              cudaStream_t stream, cudaEvent_t tc_ev0, cudaEvent_t tc_ev1,
                              unsigned long long *tc_combos, int *kernels, int part, int nparts) {
    if (nparts < 1 || part < 0 || part >= nparts) return cudaErrorInvalidValue;
    if (hist_mode) {
        ngblocks = 0;
        covered = nullptr;
    }
    unsigned long long combos = 0;
    for (int i = 0; i < ngblocks; ++i) combos += gblocks[i].a.n * gblocks[i].b.n;
    if (tc_combos) *tc_combos = nparts == 1 ? combos : (unsigned long long)((double)combos / nparts);
    if (kernels) *kernels = 0;
    if (ngblocks > 0) {
        if (tc_ev0 && cudaEventRecord(tc_ev0, stream) != cudaSuccess) return cudaErrorUnknown;
        const cudaError_t e = launch_gram_unit(p, gblocks, ngblocks, p.U, p.slot,
                                               reinterpret_cast<int *>(&p.slot->status), sm_count, stream, part,
                                               nparts);
        if (e != cudaSuccess) return e;
        if (tc_ev1 && cudaEventRecord(tc_ev1, stream) != cudaSuccess) return cudaErrorUnknown;
        if (kernels) *kernels += 1;
    }
    EnumParams q = p;
    const unsigned long long lane_chunk = 32ull * (unsigned long long)lane_entries_per_thread(nwords);
    int nb = 0;
    unsigned long long tiles = 0;
    for (int b = 0; b < p.nblocks; ++b) {
        if (covered && covered[b]) continue;
        ProductBlock B = p.blocks[b];
        B.tile_begin = tiles;
        tiles += ((B.lane_n + lane_chunk - 1) / lane_chunk) * B.walk_chunks;
        q.blocks[nb++] = B;
    }
    if (nb == 0) return cudaSuccess;
    q.nblocks = nb;
    q.tile_lo = tiles * (unsigned long long)part / (unsigned long long)nparts;
    q.total_tiles = tiles * (unsigned long long)(part + 1) / (unsigned long long)nparts;
    if (q.total_tiles <= q.tile_lo) return cudaSuccess;
    const cudaError_t e = launch_enum_unit(q, nwords, group, hist_mode, sm_count, blocks_per_sm, stream);
    if (e == cudaSuccess && kernels) *kernels += 1;
    return e;
}

cudaError_t launch_enum_unit(const EnumParams &p, int nwords, int group, bool hist_mode, int sm_count,
                             int blocks_per_sm, cudaStream_t stream) {
    switch (nwords) {
        case 1: return launch_nw<1>(p, group, hist_mode, sm_count, blocks_per_sm, stream);
        case 2: return launch_nw<2>(p, group, hist_mode, sm_count, blocks_per_sm, stream);
        case 3: return launch_nw<3>(p, group, hist_mode, sm_count, blocks_per_sm, stream);
        case 4: return launch_nw<4>(p, group, hist_mode, sm_count, blocks_per_sm, stream);
        case 5: return launch_nw<5>(p, group, hist_mode, sm_count, blocks_per_sm, stream);
        case 6: return launch_nw<6>(p, group, hist_mode, sm_count, blocks_per_sm, stream);
        case 7: return launch_nw<7>(p, group, hist_mode, sm_count, blocks_per_sm, stream);
        case 8: return launch_nw<8>(p, group, hist_mode, sm_count, blocks_per_sm, stream);
        case 9: return launch_nw<9>(p, group, hist_mode, sm_count, blocks_per_sm, stream);
        case 10: return launch_nw<10>(p, group, hist_mode, sm_count, blocks_per_sm, stream);
        case 11: return launch_nw<11>(p, group, hist_mode, sm_count, blocks_per_sm, stream);
        case 12: return launch_nw<12>(p, group, hist_mode, sm_count, blocks_per_sm, stream);
        case 13: return launch_nw<13>(p, group, hist_mode, sm_count, blocks_per_sm, stream);
        case 14: return launch_nw<14>(p, group, hist_mode, sm_count, blocks_per_sm, stream);
        case 15: return launch_nw<15>(p, group, hist_mode, sm_count, blocks_per_sm, stream);
        case 16: return launch_nw<16>(p, group, hist_mode, sm_count, blocks_per_sm, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace mdist
