// batch_kernels.cuh -- device side of the batched engine: many codes of different
// n, k advance through Alg. 1 together.
//
// The work is organised in rounds.  In a round every active code enumerates its next
// level(s): all m units (g, j) of each level (several levels in the first round when a
// predicted termination level is given).  A round is four kinds of launch:
//   batch_round_begin -- clears the round's counters;
//   batch_prep        -- one thread per code: picks the levels, appends one item per
//                        unit, plans its product blocks and claims a tile range in
//                        the bucket of its row width (one enumerator instantiation
//                        per width);
//   batch_enum<NW>    -- per bucket, a persistent grid of warps taking tiles; each tile
//                        is one product-block tile of one unit of one code (rows
//                        staged per warp), walked with the single-unit kernel's core;
//   batch_update      -- one thread per code: folds the units' results in (g, j) order
//                        exactly as the single-code driver does (U, key, L, counters,
//                        termination).
// Units of one code run concurrently and keep ties (weight <= the code's U).  The
// in-order fold then gives the same d, key, last unit and counters as the one-unit-
// at-a-time driver: a codeword first met past the termination level weighs at least
// L >= U, so pruning with it never drops the unit that holds the final U.
#pragma once

#include "enum_core.cuh"
#include "internal.h"

namespace mdist {

constexpr int kBatchMaxPlan = 34;            // product blocks per level (<= 33)
constexpr int kBatchBuckets = kMaxWords32;   // one bucket per row width (1..16 words)
constexpr int kTileBits = 44;                // bucket_packed = items << 44 | tiles

struct BatchUnit {               // one (code, set), fixed for the run
    unsigned int rows_off;       // first 32-bit word of its rows in the rows buffer
    unsigned int gs_off;         // filter choice: gs_table[gs_off + thr + 1], thr in [-1, n_bits]
    int k, k1, k2, nwords, n_bits, full_rank, rank, code;
};

struct BatchCode {               // per-code Alg. 1 state, on the device
    int n, k, m, unit0;
    int active, status;
    int g_next, spec;            // next level; levels to take in the next round
    int U, L;
    int have_key, key_w, key_g, key_j;
    unsigned long long key_rank;
    int g_final, j_final;
    int item0, nitems;           // this round's items: contiguous, (g, j) order
    int per_matrix, rounds;
    unsigned long long counts_off;   // counts[counts_off + g * m + j]
    unsigned long long combos;       // combinations enumerated up to termination
};

struct BatchItem {               // one unit of one round
    int unit, code, g, nblocks;
    unsigned long long tiles;
};

struct BucketEntry {             // an item of a bucket and its first tile in the bucket
    unsigned long long tile_begin;
    int item, pad;
};

struct ItemSlot {
    unsigned long long key;      // weight << 54 | rank, or kNoKey
    unsigned long long count;
};

struct BatchDev {                // what the kernels share (passed by value)
    const uint32_t *rows;
    const BatchUnit *units;
    const unsigned char *gs_table;
    BatchCode *codes;
    unsigned long long *counts;
    BatchItem *items;
    ItemSlot *slots;
    unsigned long long *plans;          // item * kBatchMaxPlan: first tile of each product block
    BucketEntry *bucket_items;          // bucket * item_cap + index
    unsigned long long *bucket_packed;  // per bucket, claimed atomically
    unsigned long long *tile_ctr;       // per bucket: work counter of batch_enum
    unsigned int *codeU;                // per code: candidate threshold shared by its units
    int *item_ctr;
    int *active_ctr;                    // codes still active after the last update
    int ncodes;
    int item_cap;
};

// Grid of the enumerator of each present bucket (SMs x CTAs per SM).
cudaError_t batch_bucket_grids(const bool present[kBatchBuckets], int sm_count, int blocks_per_sm,
                               int grid[kBatchBuckets]);
// One round: clear counters, prepare items, enumerate every present bucket, fold.
void batch_launch_round(const BatchDev &D, const bool present[kBatchBuckets], const int grid[kBatchBuckets],
                        cudaStream_t st);

}  // namespace mdist
