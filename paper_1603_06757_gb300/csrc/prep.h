// prep.h -- host preparation of a code: information sets and enumerator row layout.
#pragma once

#include <cstdint>
#include <vector>

namespace mdist {

struct InfoSet {
    int rank = 0;
    std::vector<int> pivcols;       // rank entries
    std::vector<uint64_t> gamma;    // k x W words: Gamma_j = T_j * G
    std::vector<uint64_t> transform;// k entries: row r of T_j as a mask over G's rows
};

struct Partition {
    int n = 0, k = 0, W = 0;
    std::vector<InfoSet> sets;
};

// Returns MDIST_OK or MDIST_ERANK.
int partition_info_sets(const uint64_t *G, int n, int k, int W, int max_sets, Partition &out);

struct DeviceRows {
    bool full_rank = false;
    int n_bits = 0;                 // bits per stored row
    int nwords = 0;                 // 32-bit words per stored row
    std::vector<uint32_t> words;    // k x nwords
};

void build_rows(const Partition &p, int j, DeviceRows &out);

}  // namespace mdist
