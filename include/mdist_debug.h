/*
 * mdist_debug.h -- host-only inspection entry points of libmdist.so: the row layout
 * the enumerators read and the combination indexing and work plans they run, evaluated
 * on the host (no CUDA call; usable without a GPU).  The tests check them against
 * independent computations; mdist_enumerate_unit_noalloc callers use
 * mdist_debug_set_rows to lay out a set's rows.  One entry point, mdist_debug_side_tables,
 * runs on the device: the table kernel of the tensor-core enumerator, so that the GPU
 * tests can check its tables entry by entry.  Conventions as in mdist.h.
 */
#ifndef MDIST_DEBUG_H
#define MDIST_DEBUG_H

#include "mdist.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Row layout the enumerator reads for set j (0-based): a full-rank set stores its
 * n - k non-pivot columns (every codeword of a weight-g combination has exactly g
 * ones on the pivots, §2's identity block); a set of rank < k stores all n columns.
 * words[k * *nwords] receives the rows as 32-bit words (capacity k * 16). */
int mdist_debug_set_rows(const uint64_t *G, int n, int k, int words_per_row, int j, int *full_rank, int *n_bits,
                         int *nwords, uint32_t *words);

/* The combination indexing the kernels run, evaluated on the host:
 *  unrank_colex: t-subset of {0..kh-1} (kh <= 32) with colex rank `rank`, as a mask;
 *  next_colex:   the next subset of the same size in colex order;
 *  lexrank:      lexicographic rank (§3.1 order) of a g-subset of {0..k-1}. */
int mdist_debug_unrank_colex(int kh, int t, uint32_t rank, uint32_t *mask);
int mdist_debug_next_colex(uint32_t m, uint32_t *next);
int mdist_debug_lexrank(uint64_t mask, int k, int g, uint64_t *rank);

/* Enumerator variant the library picks for a unit (mdist_options.filter_group = 0):
 * 0 = exact count, 2..4 = OR-group size; nwords 32-bit words of n_bits stored bits,
 * thr = largest reduced weight that is still a candidate. */
int mdist_debug_filter_choice(int nwords, int n_bits, int thr, int *group);

/* Work plan of one level (k rows, level g, nwords 32-bit words per row): the product
 * blocks (i-subsets of rows [0, ceil(k/2)) times (g-i)-subsets of the rest), 7 values
 * per block in blocks[]: lane_half, lane_t, walk_t, lane_n, walk_n, walk_chunks,
 * tile_begin (capacity 34 blocks); the tile count and the tile shape.  MDIST_ERANGE
 * if C(k, g) >= 2^54. */
int mdist_debug_level_plan(int k, int g, int nwords, int *nblocks, uint64_t *blocks, uint64_t *total_tiles,
                           int *lane_chunk, int *walk_chunk);

/* Tensor-core plan of one level (same k, g, nwords as mdist_debug_level_plan) under
 * mdist_options.tensor_cores = tensor_cores, before any table is built: the parts the
 * tensor-core enumerator takes, each a product A x B of two sides, and which product
 * blocks of the level plan they cover.  A side is the set of sums of one t0-subset of
 * rows [off0, off0 + kc0) and, when it has two components, one t1-subset of rows
 * [off1, off1 + kc1).  parts[15 * i ..]: block, then for A and for B in turn off0,
 * kc0, t0, off1, kc1, t1 (-1 for an absent second component) and the component count;
 * sizes[2 * i ..]: the entry counts of A and B; covered[b] (34 entries): 1 if block b
 * is split into parts, 0 if it stays on the ALU kernel.  Capacity 128 parts.  The
 * library swaps A and B when B is the larger side; this reports them unswapped.
 * MDIST_EINVAL on a null pointer or a mode outside 0..3, MDIST_ERANGE if
 * C(k, g) >= 2^54.  Host only, no CUDA calls. */
int mdist_debug_gram_plan(int k, int g, int nwords, int tensor_cores, int *nparts, int *parts, uint64_t *sizes,
                          int *covered);

/* The subset-sum tables of tensor-core sides (the one device entry point here; it
 * launches the kernel the enumerator uses).  rows: device pointer to k rows of nwords
 * 32-bit words (4-byte aligned; a set's layout as mdist_debug_set_rows gives it).
 * sides[6 * i ..] for i < n: off0, kc0, t0, off1, kc1, t1 as in mdist_debug_gram_plan
 * (t1 = -1: one component).  outs[i]: device buffer, 16-byte aligned, of
 * C(kc0, t0) x C(kc1, t1) x nwords words; entry e, whose component-0 subset has colex
 * rank e mod C(kc0, t0) and component-1 subset colex rank e div C(kc0, t0), receives
 * the XOR of the rows of both subsets (component c: rows off_c + its elements) at
 * words e * nwords ...  lows (may be NULL) and low_t: where lows[i] is not NULL it is
 * the finished table (from an earlier call, 16-byte aligned) of the one-component side
 * (off0, kc0, low_t[i]) on the same rows, 0 < low_t[i] < t0, which the kernel reads
 * instead of building the low-subset sums in shared memory (the library passes the
 * tables of earlier levels this way).  The caller owns every buffer.  Queued on `stream`
 * (a cudaStream_t; NULL: the legacy default stream); the call returns without waiting.
 * MDIST_EINVAL on a null or misaligned pointer, n outside 1..128, nwords outside 1..8,
 * k outside 1..64, a component of 0 or more than 32 rows, past row k or with t > kc,
 * two components that share a row, or a low_t[i] outside (0, t0); MDIST_ECUDA if the
 * launch fails. */
int mdist_debug_side_tables(const uint32_t *rows, int k, int nwords, int n, const int *sides, uint32_t *const *outs,
                            const uint32_t *const *lows, const int *low_t, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MDIST_DEBUG_H */
