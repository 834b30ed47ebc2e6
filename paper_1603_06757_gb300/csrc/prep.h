// prep.h -- host preparation of a code: information sets and enumerator row layout.
#pragma once

#include <cstdint>
#include <vector>

namespace mdist {

struct InfoSet {
    int rank = 0;                   // rank of Gamma_j on S_j (k for a full information set)
    int bound_rank = 0;             // rank entering the lower bound: rank, or for an
                                    // overlapping set its relative rank (new positions)
    std::vector<int> pivcols;       // rank entries
    std::vector<uint64_t> gamma;    // k x W words: Gamma_j = T_j * G
    std::vector<uint64_t> transform;// k entries: row r of T_j as a mask over G's rows
};

struct Partition {
    int n = 0, k = 0, W = 0;
    bool overlapping = false;       // full information sets that may share positions
    std::vector<InfoSet> sets;
    std::vector<int> cover_desc;    // overlapping: per position the number of sets holding
                                    // it, in decreasing order
};

// Returns MDIST_OK or MDIST_ERANK.
int partition_info_sets(const uint64_t *G, int n, int k, int W, int max_sets, Partition &out);

// `msets` overlapping full information sets (every Gamma_j systematic on k positions).
// Returns MDIST_OK or MDIST_ERANK.
int partition_overlapping_sets(const uint64_t *G, int n, int k, int W, int msets, Partition &out);

// Estimated codewords of a whole run: every set up to the predicted termination level
// (wstar > 0), else up to the level at which the bound reaches the Gilbert-Varshamov
// estimate of d.  Sizing and routing only.
double estimated_work(int n, int k, const Partition &p, int wstar);

// Codes whose estimated work reaches this run on the single-code path with the
// tensor-core enumerator when the batched engine or the serving loop gets them
// (mdist_options.route_work_log10 = 0; otherwise 10^route_work_log10).
constexpr double kTensorPathWork = 1e9;
inline double tensor_path_work(int route_work_log10) {
    if (route_work_log10 <= 0) return kTensorPathWork;
    double w = 1.0;
    for (int i = 0; i < route_work_log10; ++i) w *= 10.0;
    return w;
}

// Lower bound on the weight of every codeword not yet enumerated, once set j has all of
// its units of levels <= h[j] done (h[j] = 0: none).
int lower_bound(const Partition &p, const int *h);

struct DeviceRows {
    bool full_rank = false;
    int n_bits = 0;                 // bits per stored row
    int nwords = 0;                 // 32-bit words per stored row
    std::vector<uint32_t> words;    // k x nwords
};

void build_rows(const Partition &p, int j, DeviceRows &out);

}  // namespace mdist
