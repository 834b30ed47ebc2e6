// prep.cpp -- host preparation of a code (§8 step "info-set partition"):
// disjoint information sets S_1..S_m of the generator matrix and the systematic
// matrices Gamma_j = T_j * G (§2), then the per-set row layout the enumerator reads.
//
// Reading of §2 used here (the paper assumes the sets "can be found" and fixes no
// procedure): set j is built by Gauss-Jordan elimination on a fresh copy of the
// ORIGINAL G, scanning the columns not taken by earlier sets in ascending order.  A
// column becomes the next pivot iff some row at or below the current pivot position
// has a 1 in it (i.e. it is independent of this set's earlier pivots); the lowest
// such row is swapped up and the column is cleared in every other row.  Scanning
// stops at rank k or when the columns run out.  Sets are formed while unused columns
// remain and have nonzero rank (and at most max_sets of them).
#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.h"
#include "prep.h"

namespace mdist {

namespace {

inline bool bit_at(const uint64_t *row, int col) { return (row[col >> 6] >> (col & 63)) & 1ull; }

}  // namespace

int partition_info_sets(const uint64_t *G, int n, int k, int W, int max_sets, Partition &out) {
    out = Partition{};
    out.n = n;
    out.k = k;
    out.W = W;
    std::vector<char> taken((size_t)n, 0);
    std::vector<uint64_t> work((size_t)k * W);
    std::vector<uint64_t> tr((size_t)k);
    for (int set = 0; set < max_sets; ++set) {
        bool free_cols = false;
        for (int c = 0; c < n && !free_cols; ++c) free_cols = !taken[(size_t)c];
        if (!free_cols) break;
        std::memcpy(work.data(), G, sizeof(uint64_t) * (size_t)k * W);
        for (int r = 0; r < k; ++r) tr[(size_t)r] = 1ull << r;
        std::vector<int> pivots;
        pivots.reserve((size_t)k);
        for (int col = 0; col < n && (int)pivots.size() < k; ++col) {
            if (taken[(size_t)col]) continue;
            const int pos = (int)pivots.size();
            int src = -1;
            for (int r = pos; r < k; ++r)
                if (bit_at(&work[(size_t)r * W], col)) { src = r; break; }
            if (src < 0) continue;
            if (src != pos) {
                for (int w = 0; w < W; ++w) std::swap(work[(size_t)src * W + w], work[(size_t)pos * W + w]);
                std::swap(tr[(size_t)src], tr[(size_t)pos]);
            }
            const uint64_t *prow = &work[(size_t)pos * W];
            for (int r = 0; r < k; ++r) {
                if (r == pos || !bit_at(&work[(size_t)r * W], col)) continue;
                uint64_t *dst = &work[(size_t)r * W];
                for (int w = 0; w < W; ++w) dst[w] ^= prow[w];
                tr[(size_t)r] ^= tr[(size_t)pos];
            }
            pivots.push_back(col);
        }
        const int rank = (int)pivots.size();
        if (set == 0 && rank < k) return MDIST_ERANK;
        if (rank == 0) break;
        InfoSet s;
        s.rank = rank;
        s.bound_rank = rank;
        s.pivcols = pivots;
        s.gamma = work;
        s.transform = tr;
        for (int c : pivots) taken[(size_t)c] = 1;
        out.sets.push_back(std::move(s));
    }
    return MDIST_OK;
}

// Overlapping sets (the non-disjoint case of §2, for which the paper gives the bound
// only by citation).  Set j: Gauss-Jordan on a fresh copy of the original G over all n
// columns, scanned in the order (number of earlier sets holding the column, column
// index) ascending, with the same pivot rule as above, until rank k (every set is a
// full information set, so Gamma_j = (I | A_j) on its k positions).  Its relative rank
// is the number of its pivots that no earlier set holds.
int partition_overlapping_sets(const uint64_t *G, int n, int k, int W, int msets, Partition &out) {
    out = Partition{};
    out.n = n;
    out.k = k;
    out.W = W;
    out.overlapping = true;
    std::vector<int> cover((size_t)n, 0);
    std::vector<uint64_t> work((size_t)k * W);
    std::vector<uint64_t> tr((size_t)k);
    std::vector<int> order;
    for (int set = 0; set < msets; ++set) {
        order.clear();
        for (int cv = 0; cv <= set; ++cv)
            for (int c = 0; c < n; ++c)
                if (cover[(size_t)c] == cv) order.push_back(c);
        std::memcpy(work.data(), G, sizeof(uint64_t) * (size_t)k * W);
        for (int r = 0; r < k; ++r) tr[(size_t)r] = 1ull << r;
        std::vector<int> pivots;
        pivots.reserve((size_t)k);
        for (size_t q = 0; q < order.size() && (int)pivots.size() < k; ++q) {
            const int col = order[q];
            const int pos = (int)pivots.size();
            int src = -1;
            for (int r = pos; r < k; ++r)
                if (bit_at(&work[(size_t)r * W], col)) { src = r; break; }
            if (src < 0) continue;
            if (src != pos) {
                for (int w = 0; w < W; ++w) std::swap(work[(size_t)src * W + w], work[(size_t)pos * W + w]);
                std::swap(tr[(size_t)src], tr[(size_t)pos]);
            }
            const uint64_t *prow = &work[(size_t)pos * W];
            for (int r = 0; r < k; ++r) {
                if (r == pos || !bit_at(&work[(size_t)r * W], col)) continue;
                uint64_t *dst = &work[(size_t)r * W];
                for (int w = 0; w < W; ++w) dst[w] ^= prow[w];
                tr[(size_t)r] ^= tr[(size_t)pos];
            }
            pivots.push_back(col);
        }
        if ((int)pivots.size() < k) return MDIST_ERANK;
        InfoSet s;
        s.rank = k;
        s.bound_rank = 0;
        for (int c : pivots) s.bound_rank += cover[(size_t)c] == 0;
        s.pivcols = pivots;
        s.gamma = work;
        s.transform = tr;
        for (int c : pivots) ++cover[(size_t)c];
        out.sets.push_back(std::move(s));
    }
    out.cover_desc = cover;
    std::sort(out.cover_desc.begin(), out.cover_desc.end(), [](int a, int b) { return a > b; });
    return MDIST_OK;
}

// Disjoint sets: sum_j max(0, h_j + 1 - (k - r_j)) (Alg. 1, line 7, for sets of any
// ranks).  Overlapping full information sets: a codeword not yet enumerated has at least
// h_j + 1 ones inside S_j for every j, which gives two bounds, and the larger is used:
// the same sum over the relative ranks (the ones of S_j outside its new positions number
// at most k - rho_j, and the new positions of different sets are disjoint), and the
// coverage bound (the support's cover counts add up to sum_j |supp & S_j| >=
// sum_j (h_j + 1), so the weight is at least the least w whose w largest cover counts
// reach that sum).
int lower_bound(const Partition &p, const int *h) {
    int L = 0;
    long demand = 0;
    for (size_t j = 0; j < p.sets.size(); ++j) {
        const int v = h[j] + 1 - (p.k - p.sets[j].bound_rank);
        L += v > 0 ? v : 0;
        demand += h[j] + 1;
    }
    if (!p.overlapping) return L;
    int w = 0;
    long sum = 0;
    while (sum < demand && w < (int)p.cover_desc.size() && p.cover_desc[(size_t)w] > 0) sum += p.cover_desc[(size_t)w++];
    const int Lcov = sum >= demand ? w : p.n + 1;
    return Lcov > L ? Lcov : L;
}

double estimated_work(int n, int k, const Partition &p, int wstar) {
    const int m = (int)p.sets.size();
    int w = wstar;
    if (w < 1) {
        std::vector<int> ranks((size_t)m);
        for (int j = 0; j < m; ++j) ranks[(size_t)j] = p.sets[(size_t)j].bound_rank;
        int d_gv = 0;
        if (m < 1 || mdist_gv_estimate(n, k, m, ranks.data(), &d_gv, &w) != MDIST_OK) w = k;
    }
    double work = 0;
    for (int g = 1; g <= w && g <= k; ++g) work += (double)binom_host(k, g);
    return work * m;
}

// Row layout read by the enumerator for set j.  For a full-rank set every codeword
// c * Gamma_j carries exactly wt(c) = g ones on the pivot columns (identity block),
// so only the n - k other columns are stored and `base` adds g back.  A set of rank
// r < k has rows r..k-1 that are zero on its pivots, so the pivot-column weight
// depends on c; those sets store all n columns and base = 0.
void build_rows(const Partition &p, int j, DeviceRows &out) {
    const InfoSet &s = p.sets[(size_t)j];
    const bool full = s.rank == p.k;
    std::vector<int> cols;
    if (full) {
        std::vector<char> piv((size_t)p.n, 0);
        for (int c : s.pivcols) piv[(size_t)c] = 1;
        for (int c = 0; c < p.n; ++c)
            if (!piv[(size_t)c]) cols.push_back(c);
    } else {
        for (int c = 0; c < p.n; ++c) cols.push_back(c);
    }
    out.full_rank = full;
    out.n_bits = (int)cols.size();
    out.nwords = out.n_bits == 0 ? 1 : (out.n_bits + 31) / 32;
    out.words.assign((size_t)p.k * out.nwords, 0u);
    for (int r = 0; r < p.k; ++r) {
        const uint64_t *row = &s.gamma[(size_t)r * p.W];
        for (int t = 0; t < out.n_bits; ++t)
            if (bit_at(row, cols[(size_t)t])) out.words[(size_t)r * out.nwords + (t >> 5)] |= 1u << (t & 31);
    }
}

}  // namespace mdist
