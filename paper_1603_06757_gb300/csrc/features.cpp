// features.cpp -- input features of the termination-level / distance predictor and
// the analytic Gilbert-Varshamov fallback.  Host only; used to size and order work,
// never to decide a result.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"
#include "prep.h"

namespace {

inline bool bit_at(const uint64_t *row, int col) { return (row[col >> 6] >> (col & 63)) & 1ull; }

inline int row_weight(const uint64_t *r, int W) {
    int w = 0;
    for (int t = 0; t < W; ++t) w += __builtin_popcountll(r[t]);
    return w;
}

int set_bound(int h, int k, int r) {
    const int v = h + 1 - (k - r);
    return v > 0 ? v : 0;
}

// least w with sum_{i<=w} C(n, i) >= 2^(n-k) (sphere-covering / GV radius), in logs
int gv_distance(int n, int k) {
    const double target = (double)(n - k) * std::log(2.0);
    double acc = -INFINITY;  // log of the partial sum
    for (int w = 0; w <= n; ++w) {
        const double lt = std::lgamma(n + 1.0) - std::lgamma(w + 1.0) - std::lgamma(n - w + 1.0);
        acc = acc == -INFINITY ? lt : std::max(acc, lt) + std::log1p(std::exp(-std::fabs(acc - lt)));
        if (acc >= target - 1e-12) return w;
    }
    return n;
}

}  // namespace

extern "C" {

// Gilbert-Varshamov estimate of d and the level where the bound L(g) first reaches it
// (L(g) = sum_j max(0, g + 1 - (k - r_j)) over the code's information sets).
int mdist_gv_estimate(int n, int k, int m, const int *ranks, int *d_gv, int *wstar_gv) {
    if (n <= k || k < 1 || m < 1 || !ranks) return MDIST_EINVAL;
    const int d = gv_distance(n, k);
    if (d_gv) *d_gv = d;
    if (wstar_gv) {
        int g = 1;
        for (; g <= k; ++g) {
            int L = 0;
            for (int j = 0; j < m; ++j) L += set_bound(g, k, ranks[j]);
            if (L >= d) break;
        }
        *wstar_gv = g > k ? k : g;
    }
    return MDIST_OK;
}

// Feature vector (MDIST_NFEATURES floats, each roughly in [0, 1]):
//  0 n/512, 1 k/64, 2 k/n, 3 m/16, 4..7 ranks of the first four sets / k,
//  8 GV distance / n, 9 GV termination level / k,
//  10 least weight over level 1 of every set / n, 11 same over levels <= 2 / n,
//  12 level the bound needs to pass the level-2 weight / k,
//  13..20 histogram of the column weights of A_j (relative to k, 8 bins) over the
//  full-rank sets, as fractions, 21 mean relative column weight, 22 its spread,
//  23 fraction of columns of weight <= 2.
int mdist_features(const uint64_t *G, int n, int k, int words_per_row, float *f) {
    if (!G || !f || k < 1 || k > MDIST_MAX_K || n <= k || n > MDIST_MAX_N || words_per_row < (n + 63) / 64)
        return MDIST_EINVAL;
    mdist::Partition p;
    const int rc = mdist::partition_info_sets(G, n, k, words_per_row, MDIST_MAX_SETS, p);
    if (rc != MDIST_OK) return rc;
    const int W = words_per_row;
    const int m = (int)p.sets.size();
    std::memset(f, 0, sizeof(float) * MDIST_NFEATURES);
    f[0] = n / 512.0f;
    f[1] = k / 64.0f;
    f[2] = (float)k / (float)n;
    f[3] = m / 16.0f;
    for (int j = 0; j < 4 && j < m; ++j) f[4 + j] = (float)p.sets[(size_t)j].rank / (float)k;
    std::vector<int> ranks((size_t)m);
    for (int j = 0; j < m; ++j) ranks[(size_t)j] = p.sets[(size_t)j].rank;
    int dgv = 0, wgv = 0;
    mdist_gv_estimate(n, k, m, ranks.data(), &dgv, &wgv);
    f[8] = (float)dgv / (float)n;
    f[9] = (float)wgv / (float)k;
    // least weights at levels 1 and 2 (all sets)
    int w1 = n, w2 = n;
    std::vector<uint64_t> tmp((size_t)W);
    for (int j = 0; j < m; ++j) {
        const std::vector<uint64_t> &g = p.sets[(size_t)j].gamma;
        for (int a = 0; a < k; ++a) {
            w1 = std::min(w1, row_weight(&g[(size_t)a * W], W));
            for (int b2 = a + 1; b2 < k; ++b2) {
                for (int t = 0; t < W; ++t) tmp[(size_t)t] = g[(size_t)a * W + t] ^ g[(size_t)b2 * W + t];
                w2 = std::min(w2, row_weight(tmp.data(), W));
            }
        }
    }
    w2 = std::min(w1, w2);
    f[10] = (float)w1 / (float)n;
    f[11] = (float)w2 / (float)n;
    int gneed = 1;
    for (; gneed <= k; ++gneed) {
        int L = 0;
        for (int j = 0; j < m; ++j) L += set_bound(gneed, k, ranks[(size_t)j]);
        if (L >= w2) break;
    }
    f[12] = (float)std::min(gneed, k) / (float)k;
    // column weights of A_j (non-pivot columns) in the full-rank sets
    double sum = 0, sum2 = 0, low = 0, cnt = 0;
    float hist[8] = {};
    for (int j = 0; j < m; ++j) {
        const mdist::InfoSet &s = p.sets[(size_t)j];
        if (s.rank != k) continue;
        std::vector<char> piv((size_t)n, 0);
        for (int c : s.pivcols) piv[(size_t)c] = 1;
        for (int c = 0; c < n; ++c) {
            if (piv[(size_t)c]) continue;
            int cw = 0;
            for (int r = 0; r < k; ++r) cw += bit_at(&s.gamma[(size_t)r * W], c);
            const double rel = (double)cw / (double)k;
            int bin = (int)(rel * 8.0);
            if (bin > 7) bin = 7;
            hist[bin] += 1.0f;
            sum += rel;
            sum2 += rel * rel;
            low += cw <= 2 ? 1.0 : 0.0;
            cnt += 1.0;
        }
    }
    if (cnt > 0) {
        for (int b = 0; b < 8; ++b) f[13 + b] = hist[b] / (float)cnt;
        const double mean = sum / cnt;
        f[21] = (float)mean;
        f[22] = (float)std::sqrt(std::max(0.0, sum2 / cnt - mean * mean));
        f[23] = (float)(low / cnt);
    }
    return MDIST_OK;
}

}  // extern "C"
