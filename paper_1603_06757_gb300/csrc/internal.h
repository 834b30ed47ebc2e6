// internal.h -- structures shared by the library's translation units (host prep,
// enumerator kernels, C-ABI).  Not part of the public ABI (include/mdist.h).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/mdist.h"

namespace mdist {

constexpr int kMaxK = MDIST_MAX_K;
constexpr int kMaxN = MDIST_MAX_N;
constexpr int kMaxSets = MDIST_MAX_SETS;
constexpr int kMaxWords32 = kMaxN / 32;  // 32-bit words of a reduced row
constexpr int kMaxBlocks = 34;           // product blocks per level: i in [0, 32] (+1 spare)
constexpr int kWarpsPerCta = 8;
constexpr int kCtaThreads = 32 * kWarpsPerCta;
// CTAs per SM the enumerator kernels are compiled for (register budget 65536 / (256 x this))
#ifndef MDIST_ENUM_MIN_BLOCKS
#define MDIST_ENUM_MIN_BLOCKS 2
#endif
constexpr int kKeyRankBits = 54;         // device key = weight << 54 | lexicographic rank
constexpr uint64_t kNoKey = ~0ull;

// Device-side result slot of one (g, j) unit.
struct UnitSlot {
    unsigned int U;              // threshold word for launches that own their slot
    unsigned int status;         // nonzero: a bounded device wait ran out
    unsigned long long key;      // least (weight << 54 | rank) among candidates, or kNoKey
    unsigned long long count;    // combinations enumerated
    unsigned long long tile_next;// work counter of the persistent grid
    unsigned long long tc_cand;  // pairs the tensor-core filter passed to the exact recheck
    unsigned long long pad[3];
};
static_assert(sizeof(UnitSlot) == 64, "slot layout");

// One product block of a level: all i-subsets of the first half H1 of the rows,
// times all (g-i)-subsets of the second half H2.  The larger side is spread over
// the lanes of a warp ("lane side"); the warp walks the smaller side ("walk side").
struct ProductBlock {
    unsigned int lane_half;      // 0: lane side = H1 subsets, 1: lane side = H2 subsets
    unsigned int lane_t;         // subset size on the lane side
    unsigned int walk_t;         // subset size on the walk side
    unsigned int pad;
    unsigned long long lane_n;   // C(k_lane_half, lane_t)
    unsigned long long walk_n;   // C(k_walk_half, walk_t)
    unsigned long long walk_chunks;
    unsigned long long tile_begin;
};

// Parameters of one enumerator launch (one unit).
struct EnumParams {
    const uint32_t *rows;        // k reduced rows of nwords 32-bit words each (row-major)
    unsigned int *U;             // candidate threshold (weight <= *U), shared by the units of a wave
    UnitSlot *slot;              // this unit's key, count and work counter
    unsigned long long *hist;    // n_bits+1 bins (histogram mode only)
    int k, k1, k2, g;            // rows, half sizes (k1 = ceil(k/2)), level
    int nwords;                  // 32-bit words per reduced row
    int base;                    // weight every codeword carries outside the reduced row
    int n_bits;                  // bits per reduced row
    int nblocks;
    long long wait_polls;        // tensor-core enumerator: polls per bounded wait, 0 = default
    unsigned long long tile_lo;  // first tile of this launch (a slice of the unit: [tile_lo, total_tiles))
    unsigned long long total_tiles;
    ProductBlock blocks[kMaxBlocks];
};

// Kernel tile geometry per word count (lanes x XP lane entries, YL walk entries).
__host__ __device__ constexpr int lane_entries_per_thread(int nwords) { return nwords <= 4 ? 16 : (nwords <= 8 ? 8 : 4); }
__host__ __device__ constexpr int walk_len_for(int nwords) { return nwords <= 8 ? 256 : 128; }

// Launch one unit's enumerator (enum_launch.cu).  hist == nullptr for the normal path.
cudaError_t launch_enum_unit(const EnumParams &p, int nwords, int group, bool hist_mode, int sm_count,
                             int blocks_per_sm, cudaStream_t stream);

// Tensor-core (tcgen05) enumerator for the large product blocks of a unit (gram.cu).
// A block goes there directly when both of its sides hold at least kGramMinSide
// entries and the stored rows are at most kGramMaxWords words; a large block with a
// smaller side is split into sub-blocks over the two quarters of its large side's half
// (gram_block_parts in api.cpp), which gives every sub-block two larger sides.
constexpr int kGramMinSide = 128;
constexpr int kGramMaxWords = 8;
constexpr int kMaxGramBlocks = 128;
bool gram_eligible(int nwords);

// One side of a tensor-core block: per entry the sum of one subset of the rows.  The
// subset is the union of one or two components; component c is a t[c]-subset of the
// kc[c] rows starting at row off[c] (kc[c] <= 32), and entry e has colex rank e % cnt0
// in component 0 and e / cnt0 in component 1.
struct GramSide {
    uint8_t nc, off[2], kc[2], t[2], pad;
    uint32_t cnt0;               // C(kc[0], t[0])
    unsigned long long n;        // entries: cnt0 (x C(kc[1], t[1]))
};

// A block of the tensor-core enumerator: every pair (A entry, B entry), with the
// device tables of both sides' sums (packed, nwords words per entry, entry order) and
// the B side expanded to operand tiles (gram_expanded_bytes).
struct GramBlockSpec {
    GramSide a, b;
    const uint32_t *a_tab = nullptr;
    const uint32_t *b_tab = nullptr;
    const uint8_t *b_exp = nullptr;
};
// part / nparts: enumerate the part-th of nparts near-equal contiguous slices of the
// launch's work units (a unit split over several ranks)
cudaError_t launch_gram_unit(const EnumParams &ep, const GramBlockSpec *blocks, int nblocks, unsigned int *U,
                             UnitSlot *slot, int *status, int sm_count, cudaStream_t stream, int part = 0,
                             int nparts = 1);
// Tables built together (one launch each for the packed sums and for the expansions).
constexpr int kMaxTableJobs = 128;
// for i < n: outs[i][e * nwords ..] = the sum of the rows (rows: all k rows of the set)
// of entry e of sides[i]; outs[i] 16-byte aligned (entries of 2 and 4 words are stored
// as vectors).  lows (may be null) / lows[i] non-null: the finished table of the
// one-component side (off0, kc0, low_t[i]) of sides[i]'s component 0 on the same rows
// (0 < low_t[i] < t0, 16-byte aligned, written by an earlier launch on the stream), read
// instead of building the low-subset sums in shared memory.
cudaError_t launch_side_tables(const uint32_t *rows, int k, int nwords, const GramSide *sides, uint32_t *const *outs,
                               const uint32_t *const *lows, const int *low_t, int n, int sm_count,
                               cudaStream_t stream);
// bytes of the expanded operand tiles of a packed table of `count` entries
size_t gram_expanded_bytes(int nwords, unsigned long long count);
// for i < n: outs[i] = the operand tiles of packed[i] (counts[i] entries)
cudaError_t launch_expand_tables(int nwords, int n_bits, const uint32_t *const *packed,
                                 const unsigned long long *counts, uint8_t *const *outs, int n, int sm_count,
                                 cudaStream_t stream);
// A unit: the tensor-core blocks (may be none), then the product blocks of `p` not
// marked in `covered` (null: none covered) on the ALU kernel.  When the tensor-core
// kernel is launched and tc_ev0 / tc_ev1 are given they are recorded around it,
// *tc_combos (may be null) receives the combinations it enumerates (else 0) and
// *kernels (may be null) the number of kernels launched (0 to 2).
// part / nparts: only the part-th of nparts near-equal contiguous slices of each kernel's
// work (tensor-core work units, ALU tiles); the slices of a unit partition its
// combinations.  *tc_combos is then the slice's share of the tensor-core combinations.
cudaError_t launch_unit_split(const EnumParams &p, int nwords, int group, bool hist_mode, int sm_count,
                              int blocks_per_sm, const GramBlockSpec *gblocks, int ngblocks, const bool *covered,
                              cudaStream_t stream, cudaEvent_t tc_ev0 = nullptr, cudaEvent_t tc_ev1 = nullptr,
                              unsigned long long *tc_combos = nullptr, int *kernels = nullptr, int part = 0,
                              int nparts = 1);

// Filter variant for a unit: 0 (exact count for every codeword) or the OR-group size
// 2, 3, 4 whose expected cost is least for this row width and threshold.
int choose_filter_group(int nwords, int n_bits, int thr);

// Variant codes: 0 exact; 2..4 one level of OR groups (group size <= nwords);
// 5 groups of 4 then of 2 (nwords >= 4).
inline bool filter_group_valid(int group, int nwords) {
    return group == 0 || (group >= 2 && group <= 4 && group <= nwords) || (group == 5 && nwords >= 4);
}

// Stride in 32-bit words of a staged walk entry: padded to whole 16-byte vectors.
__host__ __device__ constexpr int walk_stride(int nwords) { return (nwords + 3) & ~3; }
size_t enum_smem_bytes(int k, int nwords);

// Host-side binomial coefficients C(a, b), a <= 64 (enum_launch.cu).
unsigned long long binom_host(int a, int b);

// Unique id of the CUDA context current on the calling thread: MDIST_OK, kNoContext when
// no context is current yet, MDIST_ECUDA when the driver cannot be asked.
constexpr int kNoContext = 1;
int current_context_id(unsigned long long *id);

// Kernel launch settings shared by all threads, per CUDA context: raise `func`'s
// dynamic shared-memory limit to at least `bytes` (never lowered), and its blocks per SM
// at `threads` threads and `smem` bytes (remembered).
cudaError_t allow_dynamic_smem(const void *func, size_t bytes);
cudaError_t blocks_per_sm(const void *func, int threads, size_t smem, int *occ);

// Fill the product-block table of a level; false if C(k, g) >= 2^54.
bool plan_level(int k, int g, int nwords, EnumParams &p);

}  // namespace mdist
