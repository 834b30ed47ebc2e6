/*
 * mdist.h -- C-ABI of the GB300 minimum-distance library (libmdist.so).
 *
 * Computes the minimum distance d of a binary linear [n, k] code by the
 * Brouwer-Zimmerman enumeration (Hernando, Igual, Quintana-Orti, arXiv:1603.06757,
 * §2 and Alg. 1): the generator matrix G is split into disjoint information sets
 * S_1..S_m with matrices Gamma_j = (I | A_j) (the last ones possibly of rank
 * r_j < k); for g = 1, 2, ... every c in F2^k with wt(c) = g is expanded to the
 * codeword c * Gamma_j and weighed, the upper bound U is the least weight seen and
 * the lower bound is L(g) = sum_j max(0, g + 1 - (k - r_j)); the run stops when
 * L >= U and then d = U.  The enumeration runs in hand-written sm_103a CUDA kernels.
 *
 * Conventions (all entry points):
 *  - Bit matrices are rows of uint64 words, LSB first: bit i of a row is bit (i & 63)
 *    of word (i >> 6).  Bits at columns >= n must be zero.
 *  - Set indices j are 0-based (the paper counts from 1).  Combination ranks are
 *    lexicographic over the rows of Gamma_j, 0-based (§3.1-§3.2 order).
 *  - Host pointers are read or written only during the call; the caller keeps
 *    ownership.  Everything behind an mdist_code handle is owned by the library and
 *    released by mdist_free().
 *  - Device memory: the library allocates through opts->dev_alloc / dev_free when
 *    given (e.g. a PyTorch caching allocator), else with cudaMalloc / cudaFree.
 *    dev_alloc must return memory aligned to at least 16 bytes (cudaMalloc and
 *    PyTorch's allocator give 256 or more) or NULL when it cannot.
 *  - Work is issued on the stream given to mdist_prepare (NULL = legacy default
 *    stream).  Calls return after their results are on the host.
 *  - Return value: MDIST_OK (0) or a negative MDIST_E* code; no exception or signal
 *    crosses the ABI.  mdist_strerror() names a code.
 *  - Limits: 1 <= k <= 64, k < n <= 512, at most MDIST_MAX_SETS information sets
 *    (set formation stops there; fewer sets only weaken L, never the result).
 *  - A handle is not thread-safe: one call at a time per handle.
 */
#ifndef MDIST_H
#define MDIST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MDIST_MAX_K 64
#define MDIST_MAX_N 512
#define MDIST_MAX_SETS 64

enum {
    MDIST_OK = 0,
    MDIST_EINVAL = -1,     /* bad argument or shape (n <= k, k > 64, n > 512, bad W, bits past n) */
    MDIST_ERANK = -2,      /* rank(G) < k */
    MDIST_ENOMEM = -3,     /* host or device allocation failed */
    MDIST_ECUDA = -4,      /* a CUDA runtime call failed (no device, launch error, ...) */
    MDIST_ETIMEOUT = -5,   /* a bounded device wait ran out */
    MDIST_ECANCELLED = -6, /* request cancelled */
    MDIST_ERANGE = -7,     /* C(k, g) >= 2^54: the level is beyond the device key range */
    MDIST_ESTATE = -8,     /* state blob does not belong to this code / is corrupt */
    MDIST_EAGAIN = -9      /* resource busy (serving queue full) */
};

typedef void *(*mdist_alloc_fn)(size_t bytes, void *ctx);
typedef void (*mdist_free_fn)(void *ptr, void *ctx);

/* Options; a zeroed struct (or NULL) means defaults. */
typedef struct {
    int check_per_matrix;    /* 0: check L >= U after each level (Alg. 1, line 7);
                                1: after each (g, j) unit, with
                                L = sum_{i<=j} t_i(g) + sum_{i>j} t_i(g-1),
                                t_i(h) = max(0, h + 1 - (k - r_i)) (the bound rises
                                "one after each Gamma_j", §2). */
    int max_sets;            /* 0 = MDIST_MAX_SETS */
    int blocks_per_sm;       /* enumerator CTAs per SM; 0 = occupancy limit */
    int filter_group;        /* enumerator variant: 0 = chosen per unit from the threshold,
                                1 = exact weight of every codeword, 2..4 = first a lower
                                bound (popcount of the OR of each group of that many
                                32-bit words), exact weight only where the bound does not
                                already exceed the threshold, 5 = groups of 4, then of 2,
                                then exact.  Results are identical. */
    long long timeout_cycles;/* bound of the tensor-core enumerator's pipeline waits, in polls
                                of an mbarrier (each poll may suspend for a hardware-chosen
                                time); 0 = default (2e8).  A wait that runs out ends the launch
                                early (after its own copies and MMAs have drained, which
                                get at least the default bound) and the call returns
                                MDIST_ETIMEOUT; the handle stays usable.  Negative: EINVAL. */
    mdist_alloc_fn dev_alloc;/* optional device allocator */
    mdist_free_fn dev_free;
    void *alloc_ctx;
    int wstar_hint;          /* > 1: predicted termination level; mdist_run then launches
                                levels 1 .. wstar_hint-1 as one wave (one host
                                synchronisation).  Sizing only: results never depend on it. */
    int tensor_cores;        /* product blocks on the tensor cores (tcgen05 Gram-matrix
                                enumerator, stored rows of at most 8 words): 0 = blocks
                                whose two sides hold >= 128 subsets each, and blocks of
                                >= 2^24 codewords with a smaller side split into parts
                                whose sides are large (the large side's half cut in two
                                quarters), or, on a code whose Gilbert-Varshamov work
                                estimate (mdist_gv_estimate's level w*: m * sum over
                                g <= w* of C(k, g)) reaches 10^7 codewords, as 3;
                                1 = none; 2 = every block as it is; 3 = as 0 with every
                                block that has a side under 128 subsets split, whatever
                                its size.  Results are identical. */
    int skip_idle_sets;      /* 1: at level g leave out the sets whose bound term
                                max(0, g+1-(k-r_j)) is still 0; a set enumerates the
                                levels it skipped when its term first becomes positive;
                                ties are kept and the witness key is the least
                                (weight, g, j, rank) over the units enumerated (visited
                                set by set, levels ascending).  d is the same as with 0
                                (the paper's Alg. 1, every set at every level).  Level
                                check only (MDIST_EINVAL with check_per_matrix);
                                single-code handles only (MDIST_EINVAL in batch and
                                server handles); mdist_run's max_units is rounded up to
                                whole levels. */
    int overlap_sets;        /* M > 0: M overlapping full information sets instead of the
                                disjoint ones (the non-disjoint case of §2, whose bound
                                the paper cites without printing).  Set j is found by
                                Gauss-Jordan on the original G scanning the columns held by
                                the fewest earlier sets first (ties by index) until rank k,
                                so every Gamma_j is systematic on k positions.  After
                                set j has all messages of weight <= h_j done, a codeword not
                                yet seen has >= h_j + 1 ones inside S_j; L is the larger of
                                sum_j max(0, h_j + 1 - (k - rho_j)), rho_j the relative rank
                                (pivots of S_j no earlier set holds), and the least w whose
                                w largest cover counts (sets holding a position) add up to
                                sum_j (h_j + 1).  Reported ranks are the relative ranks.
                                Pays off when n < 2k.  Single-code handles only; not with
                                skip_idle_sets (MDIST_EINVAL). */
    int route_work_log10;    /* batched engine and server: a code whose estimated work (every
                                set up to the predicted termination level: the hint, else
                                the Gilbert-Varshamov estimate) reaches 10^route_work_log10
                                codewords runs on the single-code tensor-core path; 0 = 9
                                (10^9), else 1..18 (MDIST_EINVAL otherwise). */
} mdist_options;

/* Witness key: the least (weight, g, j, rank) over the enumerated units (a total
 * order, so the witness is unique).  weight = INT32_MAX means "none". */
typedef struct {
    int32_t weight;
    int32_t g;
    int32_t j;
    int32_t reserved;
    uint64_t rank;
} mdist_key;

typedef struct {
    int32_t g_final, j_final; /* last unit enumerated */
    int32_t m;                /* number of information sets */
    int32_t L_final, U_final;
    int32_t launches;         /* kernel launches (enumerators and the tensor-core enumerator's tables) */
    int32_t ranks[MDIST_MAX_SETS];
    uint64_t combos[MDIST_MAX_K + 1][MDIST_MAX_SETS]; /* combinations enumerated per (g, j) */
    uint64_t total_combos;
    double seconds;           /* host wall time inside mdist_run / mdist_min_distance */
    double kernel_ms;         /* summed CUDA-event time of the enumerator launches */
    uint64_t h2d_bytes;       /* host-to-device bytes copied by mdist_prepare and the run */
    uint64_t d2h_bytes;       /* device-to-host bytes copied by the run */
    double tc_ms;             /* summed CUDA-event time of the tensor-core enumerator launches */
    int32_t tc_launches;      /* tensor-core enumerator launches */
    int32_t reserved;
    uint64_t tc_combos;       /* combinations those launches enumerated */
    uint64_t tc_candidates;   /* pairs of those launches whose accumulator reached the candidate
                                 bound (n_bits - 2 (U - base)) and were re-weighed exactly */
} mdist_stats;

typedef struct mdist_code mdist_code; /* opaque */

/* Split G (k rows of words_per_row uint64, host memory) into disjoint information
 * sets (§2): for j = 1, 2, ... Gauss-Jordan on the ORIGINAL G over the columns not
 * used by earlier sets, in ascending column order; a column is a pivot iff it is
 * independent of the set's earlier pivots; the pivot row is the lowest row at or
 * below the current pivot position with a 1 there.  Gamma_j row i < r_j carries the
 * i-th pivot; rows r_j..k-1 are the remaining rows.  Sets are formed while unused
 * columns of nonzero rank remain.  The packed Gamma_j are copied to the device.
 * `opts` may be NULL; it is copied.  `cuda_stream` is a cudaStream_t or NULL.
 * On success *out owns the handle. */
int mdist_prepare(const uint64_t *G, int n, int k, int words_per_row, const mdist_options *opts,
                  void *cuda_stream, mdist_code **out);

/* Information sets of a prepared code (§2): *m, ranks[m], pivcols[m*k] (-1 past
 * r_j), gammas[m*k*words_per_row] (Gamma_j = T_j * G) and transforms[m*k] (row r of
 * T_j as a k-bit mask of G rows).  Any output pointer except m may be NULL. */
int mdist_info_sets(const mdist_code *code, int *m, int *ranks, int32_t *pivcols, uint64_t *gammas,
                    uint64_t *transforms);

/* Enumerate unit(s) (g, j) of Alg. 1 on the GPU: every c with wt(c) = g, codeword
 * c * Gamma_j, weight (§2; §3: all combinations of g rows).  j = -1 runs every set,
 * one unit after the other.  Candidates are codewords of weight <= *U_inout; on
 * return *U_inout = min(*U_inout, least candidate weight) and *key_inout is the
 * least of itself and the candidates' keys (weight, g, j, rank).  combos_out (may be
 * NULL) receives the number of combinations enumerated, one entry per unit run
 * ([m] for j = -1, else [1]).  Does not change the state used by mdist_run. */
int mdist_enumerate_level(mdist_code *code, int g, int j, int *U_inout, mdist_key *key_inout,
                          uint64_t *combos_out);

/* Tensor-core counters of the last mdist_enumerate_level call on this handle, summed
 * over its units: *tc_combos = combinations the tensor-core enumerator covered,
 * *tc_candidates = those whose accumulator reached the candidate bound and were
 * re-weighed exactly from the packed rows (the filter's pass count: at a threshold
 * near the least weight it is a tiny fraction of *tc_combos).  Either pointer may be
 * NULL. */
int mdist_level_counters(const mdist_code *code, uint64_t *tc_combos, uint64_t *tc_candidates);

/* Debug / parity form of one unit: the full weight histogram hist[0..n] of the
 * C(k, g) codewords c * Gamma_j (weights over all n columns) and their count. */
int mdist_unit_histogram(mdist_code *code, int g, int j, uint64_t *hist, uint64_t *combos_out);

/* One slice of unit(s) (g, j), for a unit split over several ranks: the unit's work —
 * the tensor-core enumerator's work units and the ALU enumerator's tiles, each in its
 * own order — is cut into nparts near-equal contiguous slices and slice `part` is
 * enumerated, otherwise as mdist_enumerate_level (candidates weight <= *U_inout, key
 * min, combos_out the slice's combinations).  The slices of a unit partition its
 * combinations: their counts add up to C(k, g) and the least of their keys is the
 * unit's.  part in [0, nparts), else MDIST_EINVAL. */
int mdist_enumerate_level_part(mdist_code *code, int g, int j, int part, int nparts, int *U_inout,
                               mdist_key *key_inout, uint64_t *combos_out);

/* Exchange of one unit's results among the ranks of a sharded run: on entry *key (the
 * device key weight << 54 | lexicographic rank of this rank's least candidate, or
 * UINT64_MAX for none) and *count (this rank's combinations); on return the least key
 * and the summed count over all ranks.  Returns 0, or nonzero when the exchange failed
 * (a rank left). */
typedef int (*mdist_exchange_fn)(uint64_t *key, uint64_t *count, void *ctx);

/* Alg. 1 with every unit split over nparts ranks (one GPU each, or several handles of
 * one GPU): this rank enumerates slice `part` of each unit (mdist_enumerate_level_part),
 * `exchange` combines the unit's slices over the ranks, and the combined unit is folded
 * exactly as mdist_run folds it (U, key, counters, L after each level or, with
 * check_per_matrix, after each unit), so every rank stops at the same unit and
 * mdist_result then gives every rank mdist_min_distance's result.  Every rank calls this
 * with the same G, options and nparts; the exchange is on the host (no kernel waits for
 * another rank).  MDIST_ECANCELLED if an exchange fails (the run stops before folding
 * that unit).  Not with skip_idle_sets (MDIST_EINVAL).  In the stats, the combination
 * counters are the whole units' (the exchanged sums); the tensor-core counters
 * (tc_combos, tc_ms, ...) are this rank's, tc_combos as its proportional share. */
int mdist_run_sharded(mdist_code *code, int part, int nparts, mdist_exchange_fn exchange, void *ctx,
                      int *finished);

/* Advance Alg. 1 by at most max_units (g, j) units (max_units <= 0: until the end).
 * *finished = 1 once L >= U or every level is done. */
int mdist_run(mdist_code *code, int max_units, int *finished);

/* Restart Alg. 1 from its first unit (L := 1, U := n - k + 1, counters cleared); the
 * information sets and device rows are kept. */
int mdist_reset(mdist_code *code);

/* Result of a finished run: d, witness[words_per_row] (a codeword of weight d, in
 * the original column order), message[1] (the k-bit message with message*G =
 * witness), key and stats.  Any output except d may be NULL.  MDIST_EAGAIN if the
 * run has not finished. */
int mdist_result(const mdist_code *code, int *d, uint64_t *witness, uint64_t *message, mdist_key *key,
                 mdist_stats *stats);

/* mdist_run to the end, then mdist_result. */
int mdist_min_distance(mdist_code *code, int *d, uint64_t *witness, uint64_t *message, mdist_key *key,
                       mdist_stats *stats);

/* Checkpoint / resume of the Alg. 1 state after the last completed unit (next unit,
 * U, L, key, counters).  save: if buf is NULL or *len is too small, *len is set to
 * the size needed and MDIST_EINVAL is returned.  load: MDIST_ESTATE if the blob was
 * made for another code or options. */
int mdist_state_save(const mdist_code *code, void *buf, size_t *len);
int mdist_state_load(mdist_code *code, const void *buf, size_t len);

/* Change the stream later calls on this handle use. */
int mdist_set_stream(mdist_code *code, void *cuda_stream);

void mdist_free(mdist_code *code);
const char *mdist_strerror(int err);

/* SM count and the maximum SM clock (kHz) of the current device, for roofline
 * arithmetic. */
int mdist_device_info(int *sm_count, int *max_sm_clock_khz, int *cc_major, int *cc_minor);

/* ---- batched engine ------------------------------------------------------------ */

/* Many codes of different n, k through Alg. 1 together on one GPU.  Per round every
 * active code enumerates its next level (all its units); the rounds run as one CUDA
 * graph (persistent enumerator grids per row width, per-code state machines on the
 * device), relaunched only while codes remain active.  Large codes — at least 10^9
 * codewords up to the predicted termination level (the code's hint, else the
 * Gilbert-Varshamov estimate) — run instead after the graph, one after the other, on
 * the single-code path with the tensor-core enumerator (opts->tensor_cores: 0 as
 * described, 1 never, 2 every code); their device memory comes from the caller's
 * allocator, else from chunks kept for reuse during the run.  Each code's result equals
 * mdist_min_distance's for that code (same d, key, message, witness, counters).
 * Options as for mdist_prepare (check_per_matrix, max_sets, blocks_per_sm, allocator,
 * timeout_cycles). */
typedef struct mdist_batch mdist_batch;

int mdist_batch_create(const mdist_options *opts, void *cuda_stream, mdist_batch **out);

/* Add a code (host G, copied; information sets computed here).  wstar_hint > 1: a
 * predicted termination level; levels 1 .. wstar_hint-1 are then enumerated in the
 * first round (sizing only: results never depend on it).  *index = the code's index.
 * Codes cannot be added after mdist_batch_run. */
int mdist_batch_add(mdist_batch *b, const uint64_t *G, int n, int k, int words_per_row, int wstar_hint, int *index);

/* Run every code to completion.  rounds_per_graph <= 0: the batched codes' rounds are
 * ONE launch of a CUDA graph whose conditional WHILE node runs a round per iteration
 * until no code is active (a device-side counter caps it at MDIST_MAX_K + 2 rounds);
 * rounds_per_graph > 0: that many rounds captured back to back and the graph
 * relaunched while codes remain.  Then the large codes run on the single-code path.
 * Device buffers are allocated for the run and released before returning. */
int mdist_batch_run(mdist_batch *b, int rounds_per_graph);

/* Per-code result, as mdist_result (stats->launches = rounds the code took part in).
 * Returns the code's own error (e.g. MDIST_ERANGE) if it could not finish. */
int mdist_batch_result(const mdist_batch *b, int index, int *d, uint64_t *witness, uint64_t *message,
                       mdist_key *key, mdist_stats *stats);

/* Run totals: codes, graph launches, rounds, summed CUDA-event time of the graph
 * launches (ms), host wall time of mdist_batch_run (s), codes run on the single-code
 * path and the summed kernel time of those runs (ms).  Any output may be NULL. */
int mdist_batch_info(const mdist_batch *b, int *ncodes, int *graph_launches, int *rounds, double *gpu_ms,
                     double *seconds, int *large_codes, double *large_ms);

void mdist_batch_free(mdist_batch *b);

/* ---- serving loop ----------------------------------------------------------------- */

/* Continuous batching of code requests on one GPU.  A serving thread runs rounds of the
 * batched engine over a table of `max_slots` device slots.  Between rounds it retires
 * finished requests and admits queued ones, first come first served, while a slot is
 * free and the device rows pool (rows_pool_bytes) has room for the request's Gamma
 * rows; admitted requests join the next round next to those already in flight.  Gamma
 * rows and the per-request Alg. 1 state stay on the device until the request finishes.
 * A request forms at most 8 information sets (fewer if opts->max_sets is smaller); its
 * result equals mdist_min_distance's with the same max_sets.  Large requests — at least
 * 10^9 codewords up to the predicted termination level (the request's hint, else the
 * Gilbert-Varshamov estimate) — are run one at a time between two rounds on the
 * single-code path with the tensor-core enumerator instead (opts->tensor_cores: 0 as
 * described, 1 never, 2 every request); their device memory comes from chunks the
 * server allocates with cudaMalloc and keeps for reuse until mdist_server_free.  All
 * calls are thread-safe.  The server uses its own CUDA stream. */
typedef struct mdist_server mdist_server;

int mdist_server_create(const mdist_options *opts, int max_slots, size_t rows_pool_bytes, mdist_server **out);

/* Queue a request (G copied, information sets computed on the calling thread).
 * wstar_hint as in mdist_batch_add.  *request_id identifies it.  MDIST_ENOMEM if its
 * rows can never fit the pool. */
int mdist_server_submit(mdist_server *srv, const uint64_t *G, int n, int k, int words_per_row, int wstar_hint,
                        long long *request_id);

/* Result of a finished request (then forgotten): as mdist_result, plus the latency
 * from submission to completion in seconds.  Waits up to wait_ms; MDIST_EAGAIN if the
 * request is still queued or in flight. */
int mdist_server_poll(mdist_server *srv, long long request_id, int wait_ms, int *d, uint64_t *witness,
                      uint64_t *message, mdist_key *key, mdist_stats *stats, double *latency_s);

/* Cancel a request.  Still queued: it is dropped at once.  In a slot: it leaves the
 * batch at the next round boundary (its device slot and rows are freed).  Running on
 * the single-code path: that run finishes first.  Either way its poll then returns
 * MDIST_ECANCELLED.  Returns MDIST_OK if the request was queued or in flight,
 * MDIST_EAGAIN if it had already finished (its result stays available to poll),
 * MDIST_EINVAL for an unknown id (never submitted, or already polled). */
int mdist_server_cancel(mdist_server *srv, long long request_id);

/* Counters: requests admitted and completed, rounds run, requests queued and in
 * flight, summed CUDA-event time of the rounds (ms).  Returns the server's sticky
 * error, if any. */
int mdist_server_info(mdist_server *srv, long long *admitted, long long *completed, long long *rounds, int *queued,
                      int *in_flight, double *gpu_ms);

/* Stop the serving thread (requests still queued or in flight are dropped) and free. */
void mdist_server_free(mdist_server *srv);

/* ---- work predictor (sizing only) ----------------------------------------------- */

#define MDIST_NFEATURES 24

/* Predictor input features of a code (host only, no GPU): n, k, rate, number of sets,
 * the first four ranks r_j / k, the Gilbert-Varshamov estimate of d and of the
 * termination level, the least weights found at levels 1 and <= 2 and the level the
 * bound needs to pass the latter, and the column-weight histogram of the A_j of the
 * full-rank sets (8 bins of weight / k, mean, spread, fraction of weight <= 2).
 * f[MDIST_NFEATURES], each roughly in [0, 1]. */
int mdist_features(const uint64_t *G, int n, int k, int words_per_row, float *f);

/* Analytic fallback: d_GV = least w with sum_{i<=w} C(n, i) >= 2^(n-k); wstar_GV = least
 * g with L(g) = sum_j max(0, g + 1 - (k - r_j)) >= d_GV (ranks[m]).  Host only. */
int mdist_gv_estimate(int n, int k, int m, const int *ranks, int *d_gv, int *wstar_gv);

/* A small fp32 multilayer perceptron on the GPU (hand-written kernels): in_features ->
 * hidden (ReLU) x hidden_layers -> outputs, He-uniform weights from SplitMix64(seed),
 * zero biases; mean-squared-error loss, Adam.  Parameters are laid out layer by layer,
 * W_l (in x out, row-major) then b_l.  X, T, Y are host arrays, row-major. */
typedef struct mdist_mlp mdist_mlp;
int mdist_mlp_create(int in_features, int hidden, int hidden_layers, int outputs, uint64_t seed, void *cuda_stream,
                     mdist_mlp **out);
int mdist_mlp_num_params(const mdist_mlp *mlp, int *n);
int mdist_mlp_get_params(const mdist_mlp *mlp, float *params);
int mdist_mlp_set_params(mdist_mlp *mlp, const float *params);   /* also resets Adam's moments */
int mdist_mlp_forward(mdist_mlp *mlp, const float *X, int N, float *Y);
/* loss = mean over N x outputs of (Y - T)^2 and its gradient (grad may be NULL) */
int mdist_mlp_loss_grad(mdist_mlp *mlp, const float *X, const float *T, int N, float *loss, float *grad);
/* steps of Adam (lr, betas 0.9 / 0.999) on minibatches of `batch` rows drawn with
 * replacement by SplitMix64(seed); loss_curve[steps] (may be NULL) */
int mdist_mlp_train(mdist_mlp *mlp, const float *X, const float *T, int N, int steps, int batch, float lr,
                    uint64_t seed, float *loss_curve);
void mdist_mlp_free(mdist_mlp *mlp);


/* ---- one unit without any device allocation ---------------------------------------- */

/* Capacity of the fixed scratch array behind mdist_enumerate_unit_noalloc: histogram
 * bins (n_bits + g + 1 for a full-rank set, n_bits + 1 otherwise).  Both are at most
 * n + 1 (a full-rank set stores n_bits = n - k bits and g <= k), so every code with
 * n <= MDIST_MAX_N fits. */
#define MDIST_NOALLOC_MAX_HIST_BINS 513

/* Enumerate one (g, j) unit, as mdist_enumerate_level / mdist_unit_histogram do, for
 * callers that cannot allocate device memory: code running under a device-memory
 * pool or budget owned by someone else, or in a context where calling cudaMalloc is
 * not allowed.  The paper has no counterpart: this is a deployment variant of the
 * enumerator.
 *
 * Inputs: `rows` (device) = the set's stored rows, k rows of nwords 32-bit words (the
 * layout mdist_debug_set_rows of mdist_debug.h returns: for a full-rank set the n_bits = n - k
 * non-pivot columns, full_rank = 1; otherwise all n_bits = n columns, full_rank = 0).
 * Bits at positions >= n_bits of a row (the last word's padding and any whole words
 * after it) are ignored: the kernel clears them when it stages the rows.
 * level g; candidates are codewords of weight <= U.  Output `out` (device, caller-
 * owned, 3 + bins uint64): out[0] = min(U, least candidate weight), out[1] = least
 * key weight << 54 | lexicographic rank, or 2^64-1 if no candidate, out[2] =
 * combinations enumerated, out[3..] = the weight histogram when want_hist (bins as
 * above), untouched otherwise.  Work is queued on `cuda_stream` (NULL = legacy default
 * stream); read `out` after synchronising it.
 *
 * Memory: no cudaMalloc, cudaFree or other allocating call.  The unit's scratch state
 * (threshold, key, count, work counter, histogram) lives in one fixed 8 KiB device
 * array that every GPU loading the library keeps until the process exits.  The first
 * call in a CUDA context (the one current on the calling thread) looks up that array's
 * device address in that context and caches it under the context's unique id, so make
 * that first call before any stream capture starts; a new context (after
 * cudaDeviceReset, or a driver-API context the caller makes current) gets its own
 * lookup on its first call.  Each call clears the scratch it uses, but all calls share
 * it: calls that may overlap on the GPU (other streams, other host threads) race and
 * must be serialised by the caller.  MDIST_ERANGE if the histogram needs more than
 * MDIST_NOALLOC_MAX_HIST_BINS bins or C(k, g) >= 2^54; MDIST_EINVAL for bad sizes;
 * MDIST_ECUDA if a CUDA error is already pending when the call starts (the call then
 * launches nothing and leaves that error for the caller to collect) or if one of its
 * launches fails. */
int mdist_enumerate_unit_noalloc(const uint32_t *rows, int k, int nwords, int n_bits, int full_rank, int g, int U,
                                 int want_hist, unsigned long long *out, void *cuda_stream);


/* ---- host-only entry points (no CUDA call; usable without a GPU) ---------------- */

/* The information-set partition of mdist_prepare alone (same reading of §2, same
 * outputs as mdist_info_sets), computed on the host.  max_sets <= 0 means
 * MDIST_MAX_SETS.  MDIST_ERANK if rank(G) < k. */
int mdist_partition_host(const uint64_t *G, int n, int k, int words_per_row, int max_sets, int *m, int *ranks,
                         int32_t *pivcols, uint64_t *gammas, uint64_t *transforms);

/* The overlapping sets of mdist_options.overlap_sets = msets, computed on the host:
 * ranks[msets] (relative ranks), pivcols[msets*k] (in the order found), gammas,
 * transforms (as mdist_info_sets) and cover[n] (number of sets holding each column).
 * Any output may be NULL. */
int mdist_partition_overlap_host(const uint64_t *G, int n, int k, int words_per_row, int msets, int *ranks,
                                 int32_t *pivcols, uint64_t *gammas, uint64_t *transforms, int32_t *cover);

/* The lower bound L of that mode once set j has all messages of weight <= levels[j]
 * done (levels[msets]; 0 = none). */
int mdist_overlap_bound_host(const uint64_t *G, int n, int k, int words_per_row, int msets, const int *levels,
                             int *L);

#ifdef __cplusplus
}
#endif

#endif /* MDIST_H */
