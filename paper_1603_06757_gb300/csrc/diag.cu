// diag.cu -- host-only entry points (no CUDA calls): the information-set partition
// alone, and the exact combinatorics / level planning / row layout the enumerator
// uses, so that a machine without a GPU can test them.
#include <cstring>
#include <vector>

#include "combinatorics.cuh"
#include "internal.h"
#include "prep.h"
#include "../../include/mdist_debug.h"

namespace {

struct HostBinom {
    unsigned long long operator()(int a, int b) const { return mdist::binom_host(a, b); }
};

const uint32_t *host_bn32() {
    static uint32_t tab[mdist::kBn * mdist::kBn];
    static bool ready = false;
    if (!ready) {
        for (int a = 0; a < mdist::kBn; ++a)
            for (int b = 0; b < mdist::kBn; ++b) tab[a * mdist::kBn + b] = (uint32_t)mdist::binom_host(a, b);
        ready = true;
    }
    return tab;
}

}  // namespace

extern "C" {

int mdist_partition_host(const uint64_t *G, int n, int k, int words_per_row, int max_sets, int *m, int *ranks,
                         int32_t *pivcols, uint64_t *gammas, uint64_t *transforms) {
    if (!G || !m || k < 1 || k > MDIST_MAX_K || n <= k || n > MDIST_MAX_N || words_per_row < (n + 63) / 64)
        return MDIST_EINVAL;
    if (max_sets <= 0 || max_sets > MDIST_MAX_SETS) max_sets = MDIST_MAX_SETS;
    mdist::Partition p;
    const int rc = mdist::partition_info_sets(G, n, k, words_per_row, max_sets, p);
    if (rc != MDIST_OK) return rc;
    *m = (int)p.sets.size();
    for (int j = 0; j < *m; ++j) {
        const mdist::InfoSet &s = p.sets[(size_t)j];
        if (ranks) ranks[j] = s.rank;
        if (pivcols)
            for (int i = 0; i < k; ++i) pivcols[(size_t)j * k + i] = i < s.rank ? s.pivcols[(size_t)i] : -1;
        if (gammas) std::memcpy(gammas + (size_t)j * k * words_per_row, s.gamma.data(), sizeof(uint64_t) * s.gamma.size());
        if (transforms) std::memcpy(transforms + (size_t)j * k, s.transform.data(), sizeof(uint64_t) * k);
    }
    return MDIST_OK;
}

int mdist_partition_overlap_host(const uint64_t *G, int n, int k, int words_per_row, int msets, int *ranks,
                                 int32_t *pivcols, uint64_t *gammas, uint64_t *transforms, int32_t *cover) {
    if (!G || k < 1 || k > MDIST_MAX_K || n <= k || n > MDIST_MAX_N || words_per_row < (n + 63) / 64 ||
        msets < 1 || msets > MDIST_MAX_SETS)
        return MDIST_EINVAL;
    mdist::Partition p;
    const int rc = mdist::partition_overlapping_sets(G, n, k, words_per_row, msets, p);
    if (rc != MDIST_OK) return rc;
    for (int j = 0; j < msets; ++j) {
        const mdist::InfoSet &s = p.sets[(size_t)j];
        if (ranks) ranks[j] = s.bound_rank;
        if (pivcols)
            for (int i = 0; i < k; ++i) pivcols[(size_t)j * k + i] = s.pivcols[(size_t)i];
        if (gammas) std::memcpy(gammas + (size_t)j * k * words_per_row, s.gamma.data(), sizeof(uint64_t) * s.gamma.size());
        if (transforms) std::memcpy(transforms + (size_t)j * k, s.transform.data(), sizeof(uint64_t) * k);
    }
    if (cover) {
        for (int c = 0; c < n; ++c) cover[c] = 0;
        for (const mdist::InfoSet &s : p.sets)
            for (int c : s.pivcols) ++cover[c];
    }
    return MDIST_OK;
}

int mdist_overlap_bound_host(const uint64_t *G, int n, int k, int words_per_row, int msets, const int *levels,
                             int *L) {
    if (!G || !levels || !L || k < 1 || k > MDIST_MAX_K || n <= k || n > MDIST_MAX_N ||
        words_per_row < (n + 63) / 64 || msets < 1 || msets > MDIST_MAX_SETS)
        return MDIST_EINVAL;
    mdist::Partition p;
    const int rc = mdist::partition_overlapping_sets(G, n, k, words_per_row, msets, p);
    if (rc != MDIST_OK) return rc;
    *L = mdist::lower_bound(p, levels);
    return MDIST_OK;
}

int mdist_debug_set_rows(const uint64_t *G, int n, int k, int words_per_row, int j, int *full_rank, int *n_bits,
                         int *nwords, uint32_t *words /* k * 16 */) {
    if (!G || !full_rank || !n_bits || !nwords || !words) return MDIST_EINVAL;
    mdist::Partition p;
    const int rc = mdist::partition_info_sets(G, n, k, words_per_row, MDIST_MAX_SETS, p);
    if (rc != MDIST_OK) return rc;
    if (j < 0 || j >= (int)p.sets.size()) return MDIST_EINVAL;
    mdist::DeviceRows dr;
    mdist::build_rows(p, j, dr);
    *full_rank = dr.full_rank ? 1 : 0;
    *n_bits = dr.n_bits;
    *nwords = dr.nwords;
    std::memcpy(words, dr.words.data(), dr.words.size() * sizeof(uint32_t));
    return MDIST_OK;
}

int mdist_debug_unrank_colex(int kh, int t, uint32_t rank, uint32_t *mask) {
    if (!mask || kh < 0 || kh > 32 || t < 0 || t > kh || rank >= mdist::binom_host(kh, t)) return MDIST_EINVAL;
    *mask = mdist::unrank_colex(host_bn32(), kh, t, rank);
    return MDIST_OK;
}

int mdist_debug_next_colex(uint32_t m, uint32_t *next) {
    if (!next || m == 0) return MDIST_EINVAL;
    *next = mdist::next_colex(m);
    return MDIST_OK;
}

int mdist_debug_lexrank(uint64_t mask, int k, int g, uint64_t *rank) {
    if (!rank || k < 1 || k > 64 || g < 1 || g > k || __builtin_popcountll(mask) != g) return MDIST_EINVAL;
    if (k < 64 && (mask >> k)) return MDIST_EINVAL;
    *rank = mdist::lexrank64(mask, k, g, HostBinom{});
    return MDIST_OK;
}

int mdist_debug_filter_choice(int nwords, int n_bits, int thr, int *group) {
    if (!group || nwords < 1 || nwords > 16 || n_bits < 1 || n_bits > 32 * nwords) return MDIST_EINVAL;
    *group = mdist::choose_filter_group(nwords, n_bits, thr);
    return MDIST_OK;
}

int mdist_debug_level_plan(int k, int g, int nwords, int *nblocks, uint64_t *blocks /* 34 * 7 */,
                           uint64_t *total_tiles, int *lane_chunk, int *walk_chunk) {
    if (!nblocks || !blocks || !total_tiles || nwords < 1 || nwords > 16) return MDIST_EINVAL;
    mdist::EnumParams p{};
    if (!mdist::plan_level(k, g, nwords, p)) return MDIST_ERANGE;
    *nblocks = p.nblocks;
    for (int b = 0; b < p.nblocks; ++b) {
        const mdist::ProductBlock &B = p.blocks[b];
        uint64_t *o = blocks + 7 * b;
        o[0] = B.lane_half; o[1] = B.lane_t; o[2] = B.walk_t; o[3] = B.lane_n; o[4] = B.walk_n;
        o[5] = B.walk_chunks; o[6] = B.tile_begin;
    }
    *total_tiles = p.total_tiles;
    if (lane_chunk) *lane_chunk = 32 * mdist::lane_entries_per_thread(nwords);
    if (walk_chunk) *walk_chunk = mdist::walk_len_for(nwords);
    return MDIST_OK;
}

}  // extern "C"
