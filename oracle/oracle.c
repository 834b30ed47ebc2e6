/*
 * oracle.c -- plain, slow CPU oracle for the minimum distance of a binary linear code.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference leg load this library.  It shares no code, header, table
 * or helper with the CUDA path (paper_1603_06757_gb300/), and the CUDA path never
 * calls it.
 *
 * What it computes, and from which passage of Hernando, Igual & Quintana-Orti,
 * "Fast Algorithms for the Computation of the Minimum Distance of a Random Linear
 * Code" (arXiv:1603.06757):
 *
 *   orc_weight_enumerator  -- the definitions of §2 (Hamming weight, d(C) = wt(C) =
 *                             least weight of a nonzero codeword): every one of the 2^k
 *                             codewords m*G, visited in Gray-code order.
 *   orc_partition          -- the information sets of §2 (disjoint sets S_j with
 *                             Gamma_j = (I | A_j), the last of rank k_m < k) under a
 *                             fixed greedy reading: for j = 1, 2, ... run Gauss-Jordan
 *                             on the ORIGINAL G over the columns not used by earlier
 *                             sets, in ascending column order.
 *   orc_enumerate_unit     -- one (g, j) step of Alg. 1: every c with wt(c) = g, the
 *                             codeword c*Gamma_j and its weight, in the lexicographic
 *                             order of §3.1, with the prefix reuse of Alg. 3 (sum of the
 *                             first g-1 rows kept, one more row added per codeword).
 *   orc_min_distance       -- Alg. 1: L := 1, U := n-k+1, levels g = 1, 2, ... over all
 *                             Gamma_j while g <= k and L < U, with the lower bound
 *                             L(g) = sum_j max(0, g+1-(k-r_j)) (Alg. 1 line 7 written
 *                             for any number of sets, each of rank r_j).
 *
 *   orc_min_distance_skip  -- the same loop with the sets whose bound term
 *                             max(0, g+1-(k-r_j)) is still 0 left out; a set first
 *                             enumerated at level g first runs the levels it skipped
 *                             (1 .. g), so that its term counts all of its combinations
 *                             of weight <= g.  The key is the least (weight, g, j, rank)
 *                             over the units run.
 *
 *   orc_partition_overlap  -- the non-disjoint information sets of §2 ("a different
 *   orc_min_distance_overlap  quantity if the information sets are not disjoint"): M sets,
 *                             each a full information set found by Gauss-Jordan on the
 *                             ORIGINAL G scanning the columns least covered by earlier sets
 *                             first (ties by index).  The paper cites the lower bound
 *                             without printing it; this oracle takes the larger of two
 *                             bounds that hold for any family of full information sets
 *                             S_1..S_M once every message of weight <= h_j has been
 *                             enumerated in Gamma_j (so a codeword not yet seen has at
 *                             least h_j + 1 ones inside S_j):
 *                               relative ranks: sum_j max(0, h_j + 1 - (k - rho_j)), rho_j =
 *                                 the pivots of S_j no earlier set holds (the ones inside
 *                                 S_j but outside the new positions number at most k - rho_j);
 *                               coverage: with cov(i) = number of sets holding position i,
 *                                 sum_{i in supp} cov(i) = sum_j |supp & S_j| >=
 *                                 sum_j (h_j + 1), so the weight is at least the least w
 *                                 whose w largest cov values reach that sum.
 *
 * Bit layout: an R x n matrix is R rows of W uint64 words, bit i of a row in word i>>6
 * at bit i&63.  Parallelism: POSIX threads over the first element of each combination
 * with a shared counter (the dynamic schedule over the first recursion level of §4.3).
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef uint64_t u64;

#define ORC_MAX_K 64
#define ORC_MAX_N 512
#define ORC_MAX_W (ORC_MAX_N / 64)
#define ORC_MAX_SETS 64

enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_ERANK = -2, ORC_ENOMEM = -3 };

/* ------------------------------------------------------------------------------ */
/* small helpers                                                                   */
/* ------------------------------------------------------------------------------ */

static int get_bit(const u64 *row, int i) { return (int)((row[i >> 6] >> (i & 63)) & 1u); }

static int weight_of(const u64 *v, int W) {
    int w = 0;
    for (int t = 0; t < W; t++) w += __builtin_popcountll(v[t]);
    return w;
}

/* Binomial coefficient C(a, b), exact, for 0 <= a <= 64 (Pascal's rule). */
static u64 binom(int a, int b) {
    static u64 tab[ORC_MAX_K + 1][ORC_MAX_K + 1];
    static int ready = 0;
    if (!ready) {
        for (int x = 0; x <= ORC_MAX_K; x++) {
            tab[x][0] = 1;
            for (int y = 1; y <= x; y++) tab[x][y] = tab[x - 1][y - 1] + (y <= x - 1 ? tab[x - 1][y] : 0);
        }
        ready = 1;
    }
    if (a < 0 || b < 0 || b > a) return 0;
    return tab[a][b];
}

u64 orc_binomial(int a, int b) { return binom(a, b); }

static int check_shape(const u64 *G, int n, int k, int W) {
    if (!G || k < 1 || k > ORC_MAX_K || n <= k || n > ORC_MAX_N || W < (n + 63) / 64 || W > ORC_MAX_W)
        return ORC_EINVAL;
    /* bits beyond column n must be zero */
    for (int r = 0; r < k; r++)
        for (int i = n; i < 64 * W; i++)
            if (get_bit(G + (size_t)r * W, i)) return ORC_EINVAL;
    return ORC_OK;
}

static int clamp_threads(int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    return nthreads;
}

/* ------------------------------------------------------------------------------ */
/* brute force: all 2^k codewords (definitions of §2)                              */
/* ------------------------------------------------------------------------------ */

typedef struct {
    const u64 *G;
    int n, k, W;
    u64 lo, hi;       /* Gray-sequence indices [lo, hi) */
    u64 A[ORC_MAX_N + 1];
} bf_task;

static void *bf_worker(void *arg) {
    bf_task *t = (bf_task *)arg;
    u64 x[ORC_MAX_W];
    memset(x, 0, sizeof x);
    /* codeword of Gray index lo: message gray(lo) = lo ^ (lo >> 1) */
    u64 gray = t->lo ^ (t->lo >> 1);
    for (int b = 0; b < t->k; b++)
        if ((gray >> b) & 1)
            for (int w = 0; w < t->W; w++) x[w] ^= t->G[(size_t)b * t->W + w];
    t->A[weight_of(x, t->W)]++;
    for (u64 idx = t->lo + 1; idx < t->hi; idx++) {
        int b = __builtin_ctzll(idx); /* Gray code: message idx differs from idx-1 in bit ctz(idx) */
        const u64 *row = t->G + (size_t)b * t->W;
        for (int w = 0; w < t->W; w++) x[w] ^= row[w];
        t->A[weight_of(x, t->W)]++;
    }
    return NULL;
}

/* A[0..n] := number of codewords m*G (m over all 2^k messages, m = 0 included) of each
 * weight.  k <= 40.  Returns ORC_OK. */
int orc_weight_enumerator(const u64 *G, int n, int k, int W, int nthreads, u64 *A) {
    if (check_shape(G, n, k, W) != ORC_OK || k > 40 || !A) return ORC_EINVAL;
    nthreads = clamp_threads(nthreads);
    u64 total = (u64)1 << k;
    if ((u64)nthreads > total) nthreads = (int)total;
    bf_task *tasks = (bf_task *)calloc((size_t)nthreads, sizeof(bf_task));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!tasks || !th) { free(tasks); free(th); return ORC_ENOMEM; }
    for (int i = 0; i < nthreads; i++) {
        tasks[i].G = G; tasks[i].n = n; tasks[i].k = k; tasks[i].W = W;
        tasks[i].lo = total / (u64)nthreads * (u64)i;
        tasks[i].hi = (i == nthreads - 1) ? total : total / (u64)nthreads * (u64)(i + 1);
        pthread_create(&th[i], NULL, bf_worker, &tasks[i]);
    }
    memset(A, 0, sizeof(u64) * (size_t)(n + 1));
    for (int i = 0; i < nthreads; i++) {
        pthread_join(th[i], NULL);
        for (int w = 0; w <= n; w++) A[w] += tasks[i].A[w];
    }
    free(tasks); free(th);
    return ORC_OK;
}

/* ------------------------------------------------------------------------------ */
/* information sets (§2), greedy reading                                           */
/* ------------------------------------------------------------------------------ */

/* Outputs, for each set j < *m:
 *   ranks[j]                 r_j
 *   pivcols[j*k + i]         i-th pivot column of S_j (i < r_j), -1 beyond
 *   gammas[(j*k + r)*W ...]  row r of Gamma_j = T_j * G; row i < r_j has its pivot at
 *                            pivcols[j*k+i] and is the only row with a 1 there; rows
 *                            r_j..k-1 are zero on every pivot column of S_j
 *   transforms[j*k + r]      row r of the k x k transform T_j (bit b = coefficient of G row b)
 * Returns ORC_ERANK if rank(G) < k. */
int orc_partition(const u64 *G, int n, int k, int W, int max_sets, int *m, int *ranks, int *pivcols,
                  u64 *gammas, u64 *transforms) {
    if (check_shape(G, n, k, W) != ORC_OK || !m || !ranks || !pivcols || !gammas || !transforms) return ORC_EINVAL;
    if (max_sets < 1 || max_sets > ORC_MAX_SETS) return ORC_EINVAL;
    unsigned char used[ORC_MAX_N];
    memset(used, 0, sizeof used);
    u64 M[ORC_MAX_K * ORC_MAX_W];
    u64 T[ORC_MAX_K];
    int sets = 0;
    for (int j = 0; j < max_sets; j++) {
        int any_unused = 0;
        for (int c = 0; c < n; c++) any_unused |= !used[c];
        if (!any_unused) break;
        memcpy(M, G, sizeof(u64) * (size_t)k * (size_t)W);
        for (int r = 0; r < k; r++) T[r] = (u64)1 << r;
        int p = 0;
        int piv[ORC_MAX_K];
        for (int c = 0; c < n && p < k; c++) {
            if (used[c]) continue;
            int i = p;
            while (i < k && !get_bit(M + (size_t)i * W, c)) i++;
            if (i == k) continue; /* column c depends on this set's earlier pivots */
            if (i != p) {
                for (int w = 0; w < W; w++) { u64 s = M[i * W + w]; M[i * W + w] = M[p * W + w]; M[p * W + w] = s; }
                u64 s = T[i]; T[i] = T[p]; T[p] = s;
            }
            for (int r = 0; r < k; r++) {
                if (r != p && get_bit(M + (size_t)r * W, c)) {
                    for (int w = 0; w < W; w++) M[r * W + w] ^= M[p * W + w];
                    T[r] ^= T[p];
                }
            }
            piv[p++] = c;
        }
        if (j == 0 && p < k) return ORC_ERANK;
        if (p == 0) break;
        ranks[j] = p;
        for (int i = 0; i < k; i++) pivcols[j * k + i] = (i < p) ? piv[i] : -1;
        memcpy(gammas + (size_t)j * k * W, M, sizeof(u64) * (size_t)k * (size_t)W);
        memcpy(transforms + (size_t)j * k, T, sizeof(u64) * (size_t)k);
        for (int i = 0; i < p; i++) used[piv[i]] = 1;
        sets++;
    }
    *m = sets;
    return ORC_OK;
}

/* ------------------------------------------------------------------------------ */
/* one (g, j) unit of Alg. 1, inner loop of Alg. 3                                 */
/* ------------------------------------------------------------------------------ */

typedef struct {
    const u64 *gamma;
    int n, k, W, g;
    int *next_first; /* shared counter over the first element */
    pthread_mutex_t *lock;
    /* per-thread results */
    int min_w;
    u64 min_rank;
    u64 count;
    u64 hist[ORC_MAX_N + 1];
    u64 xor_all[ORC_MAX_W];
} unit_task;

/* All combinations c_1 < ... < c_g with c_1 = a, in lexicographic order (§3.1).  The
 * prefix (c_1..c_{g-1}) is summed once and the last element c_g runs over
 * c_{g-1}+1 .. k-1 (Alg. 3).  `rank` is the lexicographic index of the first such
 * combination among all C(k, g). */
static void unit_first_element(unit_task *t, int a, u64 rank) {
    const int k = t->k, g = t->g, W = t->W;
    const u64 *R = t->gamma;
    int c[ORC_MAX_K];
    u64 prefix[ORC_MAX_W];
    /* middle elements c[1..g-2] form a (g-2)-combination of {a+1, ..., k-2} */
    const int mid = g - 2;
    for (int q = 0; q < mid; q++) c[1 + q] = a + 1 + q;
    c[0] = a;
    for (;;) {
        /* sum of the prefix rows c[0..g-2] */
        for (int w = 0; w < W; w++) prefix[w] = 0;
        for (int q = 0; q <= g - 2; q++)
            for (int w = 0; w < W; w++) prefix[w] ^= R[(size_t)c[q] * W + w];
        int first_last = c[g - 2] + 1;
        for (int last = first_last; last < k; last++) {
            u64 x[ORC_MAX_W];
            for (int w = 0; w < W; w++) x[w] = prefix[w] ^ R[(size_t)last * W + w];
            int wt = weight_of(x, W);
            if (wt < t->min_w) { t->min_w = wt; t->min_rank = rank; }
            t->hist[wt]++;
            for (int w = 0; w < W; w++) t->xor_all[w] ^= x[w];
            t->count++;
            rank++;
        }
        /* lexicographic successor of the middle part, values in [a+1, k-2] */
        int i = mid - 1;
        while (i >= 0 && c[1 + i] == (k - 2) - (mid - 1 - i)) i--;
        if (i < 0) break;
        c[1 + i]++;
        for (int q = i + 1; q < mid; q++) c[1 + q] = c[1 + q - 1] + 1;
    }
}

static void *unit_worker(void *arg) {
    unit_task *t = (unit_task *)arg;
    const int k = t->k, g = t->g;
    for (;;) {
        pthread_mutex_lock(t->lock);
        int a = (*t->next_first)++;
        pthread_mutex_unlock(t->lock);
        if (a > k - g) break;
        /* combinations whose first element is below a: C(k,g) - C(k-a,g) */
        u64 rank = binom(k, g) - binom(k - a, g);
        unit_first_element(t, a, rank);
    }
    return NULL;
}

/* Enumerate every c in F2^k with wt(c) = g (2 <= ... or g = 1) for one Gamma (k rows of
 * n bits), weights over all n columns.  Outputs the least weight and the lexicographic
 * rank of the first combination reaching it, the number of combinations visited, the
 * weight histogram hist[0..n] (optional) and the XOR of all visited codewords
 * xor_all[W] (optional). */
int orc_enumerate_unit(const u64 *gamma, int n, int k, int W, int g, int nthreads, int *min_w, u64 *min_rank,
                       u64 *count, u64 *hist, u64 *xor_all) {
    if (!gamma || k < 1 || k > ORC_MAX_K || n < 1 || n > ORC_MAX_N || W < (n + 63) / 64 || W > ORC_MAX_W)
        return ORC_EINVAL;
    if (g < 1 || g > k || !min_w || !min_rank || !count) return ORC_EINVAL;
    nthreads = clamp_threads(nthreads);
    *min_w = 1 << 30;
    *min_rank = ~(u64)0;
    *count = 0;
    if (hist) memset(hist, 0, sizeof(u64) * (size_t)(n + 1));
    if (xor_all) memset(xor_all, 0, sizeof(u64) * (size_t)W);
    if (g == 1) {
        for (int r = 0; r < k; r++) {
            int wt = weight_of(gamma + (size_t)r * W, W);
            if (wt < *min_w) { *min_w = wt; *min_rank = (u64)r; }
            if (hist) hist[wt]++;
            if (xor_all) for (int w = 0; w < W; w++) xor_all[w] ^= gamma[(size_t)r * W + w];
            (*count)++;
        }
        return ORC_OK;
    }
    int next_first = 0;
    pthread_mutex_t lock = PTHREAD_MUTEX_INITIALIZER;
    int nt = nthreads;
    if (nt > k - g + 1) nt = k - g + 1;
    unit_task *tasks = (unit_task *)calloc((size_t)nt, sizeof(unit_task));
    pthread_t *th = (pthread_t *)calloc((size_t)nt, sizeof(pthread_t));
    if (!tasks || !th) { free(tasks); free(th); return ORC_ENOMEM; }
    for (int i = 0; i < nt; i++) {
        tasks[i].gamma = gamma; tasks[i].n = n; tasks[i].k = k; tasks[i].W = W; tasks[i].g = g;
        tasks[i].next_first = &next_first; tasks[i].lock = &lock;
        tasks[i].min_w = 1 << 30; tasks[i].min_rank = ~(u64)0;
        pthread_create(&th[i], NULL, unit_worker, &tasks[i]);
    }
    for (int i = 0; i < nt; i++) {
        pthread_join(th[i], NULL);
        unit_task *t = &tasks[i];
        if (t->min_w < *min_w || (t->min_w == *min_w && t->min_rank < *min_rank)) {
            *min_w = t->min_w; *min_rank = t->min_rank;
        }
        *count += t->count;
        if (hist) for (int w = 0; w <= n; w++) hist[w] += t->hist[w];
        if (xor_all) for (int w = 0; w < W; w++) xor_all[w] ^= t->xor_all[w];
    }
    free(tasks); free(th);
    return ORC_OK;
}

/* The g-combination of {0..k-1} with lexicographic rank `rank` (as a bit mask),
 * found by walking the lexicographic order element by element. */
u64 orc_unrank_lex(int k, int g, u64 rank) {
    u64 mask = 0;
    int lo = 0;
    for (int i = 0; i < g; i++) {
        /* choose the smallest element e >= lo such that rank falls among the
         * combinations whose next element is e */
        for (int e = lo; e < k; e++) {
            u64 with_e = binom(k - 1 - e, g - 1 - i);
            if (rank < with_e) { mask |= (u64)1 << e; lo = e + 1; break; }
            rank -= with_e;
        }
    }
    return mask;
}

/* ------------------------------------------------------------------------------ */
/* Alg. 1                                                                          */
/* ------------------------------------------------------------------------------ */

typedef struct {
    int32_t d;
    int32_t key_w, key_g, key_j; /* witness key: (weight, g, j, rank), j 0-based */
    u64 key_rank;
    int32_t g_final, j_final;    /* last unit enumerated */
    int32_t m;
    int32_t L_final, U_final;
    int32_t ranks[ORC_MAX_SETS];
    u64 message;                 /* k-bit message with message*G = witness */
    u64 witness[ORC_MAX_W];
    u64 counts[(ORC_MAX_K + 1) * ORC_MAX_SETS]; /* counts[g*ORC_MAX_SETS + j] */
} orc_result;

/* lower-bound contribution of a set of rank r after all combinations of weight <= h
 * have been enumerated in it */
static int set_bound(int h, int k, int r) {
    int v = h + 1 - (k - r);
    return v > 0 ? v : 0;
}

/* (w, g, j, rank) < (key_w, key_g, key_j, key_rank) of out, lexicographically */
static int key_before(const orc_result *out, int w, int g, int j, u64 rank) {
    if (w != out->key_w) return w < out->key_w;
    if (g != out->key_g) return g < out->key_g;
    if (j != out->key_j) return j < out->key_j;
    return rank < out->key_rank;
}

static void witness_of_key(const u64 *G, int k, int W, const u64 *tr, orc_result *out) {
    u64 c = orc_unrank_lex(k, out->key_g, out->key_rank);
    u64 msg = 0;
    for (int r = 0; r < k; r++)
        if ((c >> r) & 1) msg ^= tr[(size_t)out->key_j * k + r];
    out->message = msg;
    for (int b = 0; b < k; b++)
        if ((msg >> b) & 1)
            for (int w = 0; w < W; w++) out->witness[w] ^= G[(size_t)b * W + w];
}

int orc_min_distance_skip(const u64 *G, int n, int k, int W, int max_sets, int nthreads, orc_result *out) {
    if (check_shape(G, n, k, W) != ORC_OK || !out) return ORC_EINVAL;
    memset(out, 0, sizeof *out);
    int m = 0;
    int *ranks = (int *)calloc(ORC_MAX_SETS, sizeof(int));
    int *piv = (int *)calloc((size_t)ORC_MAX_SETS * k, sizeof(int));
    u64 *gam = (u64 *)calloc((size_t)ORC_MAX_SETS * k * W, sizeof(u64));
    u64 *tr = (u64 *)calloc((size_t)ORC_MAX_SETS * k, sizeof(u64));
    int *done = (int *)calloc(ORC_MAX_SETS, sizeof(int));  /* levels run per set */
    if (!ranks || !piv || !gam || !tr || !done) {
        free(ranks); free(piv); free(gam); free(tr); free(done);
        return ORC_ENOMEM;
    }
    int rc = orc_partition(G, n, k, W, max_sets, &m, ranks, piv, gam, tr);
    if (rc != ORC_OK) { free(ranks); free(piv); free(gam); free(tr); free(done); return rc; }
    out->m = m;
    for (int j = 0; j < m; j++) out->ranks[j] = ranks[j];

    int L = 1, U = n - k + 1;
    int have_key = 0;
    int g = 1;
    while (g <= k && L < U) {
        for (int j = 0; j < m; j++) {
            if (set_bound(g, k, ranks[j]) == 0) continue;    /* idle at this level */
            for (int h = done[j] + 1; h <= g; h++) {        /* catch up, then level g */
                int w; u64 rank, cnt;
                orc_enumerate_unit(gam + (size_t)j * k * W, n, k, W, h, nthreads, &w, &rank, &cnt, NULL, NULL);
                out->counts[h * ORC_MAX_SETS + j] = cnt;
                out->g_final = h; out->j_final = j;
                if (!have_key || key_before(out, w, h, j, rank)) {
                    out->key_w = w; out->key_g = h; out->key_j = j; out->key_rank = rank;
                    have_key = 1;
                }
                if (w < U) U = w;
            }
            done[j] = g;
        }
        L = 0;
        for (int i = 0; i < m; i++) L += set_bound(g, k, ranks[i]);
        if (L >= U) break;
        g++;
    }
    out->d = U;
    out->L_final = L; out->U_final = U;
    witness_of_key(G, k, W, tr, out);
    free(ranks); free(piv); free(gam); free(tr); free(done);
    return ORC_OK;
}

int orc_min_distance(const u64 *G, int n, int k, int W, int check_per_matrix, int max_sets, int nthreads,
                     orc_result *out) {
    if (check_shape(G, n, k, W) != ORC_OK || !out) return ORC_EINVAL;
    memset(out, 0, sizeof *out);
    int m = 0;
    int *ranks = (int *)calloc(ORC_MAX_SETS, sizeof(int));
    int *piv = (int *)calloc((size_t)ORC_MAX_SETS * k, sizeof(int));
    u64 *gam = (u64 *)calloc((size_t)ORC_MAX_SETS * k * W, sizeof(u64));
    u64 *tr = (u64 *)calloc((size_t)ORC_MAX_SETS * k, sizeof(u64));
    if (!ranks || !piv || !gam || !tr) { free(ranks); free(piv); free(gam); free(tr); return ORC_ENOMEM; }
    int rc = orc_partition(G, n, k, W, max_sets, &m, ranks, piv, gam, tr);
    if (rc != ORC_OK) { free(ranks); free(piv); free(gam); free(tr); return rc; }
    out->m = m;
    for (int j = 0; j < m; j++) out->ranks[j] = ranks[j];

    int L = 1, U = n - k + 1;    /* Alg. 1, line 1 */
    int have_key = 0;
    int g = 1;
    while (g <= k && L < U) {    /* Alg. 1, line 3 */
        for (int j = 0; j < m; j++) {
            int w; u64 rank, cnt;
            orc_enumerate_unit(gam + (size_t)j * k * W, n, k, W, g, nthreads, &w, &rank, &cnt, NULL, NULL);
            out->counts[g * ORC_MAX_SETS + j] = cnt;
            out->g_final = g; out->j_final = j;
            /* units are visited in increasing (g, j); within a unit the rank is the
             * least among equal weights, so a strict improvement in weight decides */
            if (!have_key || w < out->key_w) {
                out->key_w = w; out->key_g = g; out->key_j = j; out->key_rank = rank;
                have_key = 1;
            }
            if (w < U) U = w;
            if (check_per_matrix) {
                int Lm = 0;
                for (int i = 0; i < m; i++) Lm += set_bound(i <= j ? g : g - 1, k, ranks[i]);
                if (Lm > L) L = Lm;
                if (L >= U) break;
            }
        }
        if (!check_per_matrix) {
            int Lg = 0;          /* Alg. 1, line 7, for sets of any ranks */
            for (int i = 0; i < m; i++) Lg += set_bound(g, k, ranks[i]);
            L = Lg;
        }
        if (L >= U) break;
        g++;
    }
    out->d = U;
    out->L_final = L; out->U_final = U;
    /* witness: c = the key's combination, message = c * T_j, witness = message * G */
    u64 c = orc_unrank_lex(k, out->key_g, out->key_rank);
    u64 msg = 0;
    for (int r = 0; r < k; r++)
        if ((c >> r) & 1) msg ^= tr[(size_t)out->key_j * k + r];
    out->message = msg;
    for (int b = 0; b < k; b++)
        if ((msg >> b) & 1)
            for (int w = 0; w < W; w++) out->witness[w] ^= G[(size_t)b * W + w];
    free(ranks); free(piv); free(gam); free(tr);
    return ORC_OK;
}

/* ------------------------------------------------------------------------------ */
/* overlapping information sets (the non-disjoint case of §2)                      */
/* ------------------------------------------------------------------------------ */

/* M full information sets.  Set j: Gauss-Jordan on a fresh copy of the original G over
 * ALL n columns, scanned in the order (cover count so far, column index) ascending; a
 * column is a pivot iff some row at or below the current pivot position has a 1 in it;
 * the lowest such row is swapped up and the column is cleared in every other row; the
 * scan stops at rank k.  Outputs per set j < M: rel_ranks[j] (pivots of S_j that no
 * earlier set holds), pivcols[j*k + i] (the i-th pivot in scan order), gammas and
 * transforms as orc_partition; cover[0..n-1] = number of sets holding each column. */
int orc_partition_overlap(const u64 *G, int n, int k, int W, int msets, int *rel_ranks, int *pivcols, u64 *gammas,
                          u64 *transforms, int *cover) {
    if (check_shape(G, n, k, W) != ORC_OK || !rel_ranks || !pivcols || !gammas || !transforms || !cover)
        return ORC_EINVAL;
    if (msets < 1 || msets > ORC_MAX_SETS) return ORC_EINVAL;
    u64 M[ORC_MAX_K * ORC_MAX_W];
    u64 T[ORC_MAX_K];
    int order[ORC_MAX_N];
    for (int c = 0; c < n; c++) cover[c] = 0;
    for (int j = 0; j < msets; j++) {
        /* scan order: by cover count, then by column */
        int len = 0;
        for (int cv = 0; cv <= j; cv++)
            for (int c = 0; c < n; c++)
                if (cover[c] == cv) order[len++] = c;
        memcpy(M, G, sizeof(u64) * (size_t)k * (size_t)W);
        for (int r = 0; r < k; r++) T[r] = (u64)1 << r;
        int p = 0;
        int piv[ORC_MAX_K];
        for (int q = 0; q < len && p < k; q++) {
            const int c = order[q];
            int i = p;
            while (i < k && !get_bit(M + (size_t)i * W, c)) i++;
            if (i == k) continue;
            if (i != p) {
                for (int w = 0; w < W; w++) { u64 t = M[i * W + w]; M[i * W + w] = M[p * W + w]; M[p * W + w] = t; }
                u64 t = T[i]; T[i] = T[p]; T[p] = t;
            }
            for (int r = 0; r < k; r++) {
                if (r != p && get_bit(M + (size_t)r * W, c)) {
                    for (int w = 0; w < W; w++) M[r * W + w] ^= M[p * W + w];
                    T[r] ^= T[p];
                }
            }
            piv[p++] = c;
        }
        if (p < k) return ORC_ERANK;
        int fresh = 0;
        for (int i = 0; i < k; i++) fresh += cover[piv[i]] == 0;
        rel_ranks[j] = fresh;
        for (int i = 0; i < k; i++) pivcols[j * k + i] = piv[i];
        memcpy(gammas + (size_t)j * k * W, M, sizeof(u64) * (size_t)k * (size_t)W);
        memcpy(transforms + (size_t)j * k, T, sizeof(u64) * (size_t)k);
        for (int i = 0; i < k; i++) cover[piv[i]]++;
    }
    return ORC_OK;
}

/* Lower bound once set j has all of its units of levels <= h[j] enumerated (h[j] = 0:
 * none), for full information sets with relative ranks rel[] and cover counts cover[]:
 * the larger of the relative-rank sum and the coverage bound (see the header). */
int orc_overlap_bound(int m, const int *h, int k, const int *rel, int n, const int *cover) {
    int Lrel = 0;
    long demand = 0;
    for (int j = 0; j < m; j++) {
        Lrel += set_bound(h[j], k, rel[j]);
        demand += h[j] + 1;
    }
    /* cover counts in decreasing order (counting sort: counts are at most m) */
    int Lcov = 0;
    long sum = 0;
    for (int cv = m; cv >= 1 && sum < demand; cv--)
        for (int c = 0; c < n && sum < demand; c++)
            if (cover[c] == cv) { sum += cv; Lcov++; }
    if (sum < demand) Lcov = n + 1; /* no support of any size carries the demand */
    return Lrel > Lcov ? Lrel : Lcov;
}

/* Alg. 1 over M overlapping full information sets: levels g = 1, 2, ... over every set
 * while g <= k and L < U, with L = orc_overlap_bound after each level (or, with
 * check_per_matrix, after each unit: sets up to j at level g, the later ones at g - 1).
 * Key, counts and witness as orc_min_distance; out->ranks holds the relative ranks. */
int orc_min_distance_overlap(const u64 *G, int n, int k, int W, int msets, int check_per_matrix, int nthreads,
                             orc_result *out) {
    if (check_shape(G, n, k, W) != ORC_OK || !out || msets < 1 || msets > ORC_MAX_SETS) return ORC_EINVAL;
    memset(out, 0, sizeof *out);
    int *rel = (int *)calloc(ORC_MAX_SETS, sizeof(int));
    int *piv = (int *)calloc((size_t)ORC_MAX_SETS * k, sizeof(int));
    u64 *gam = (u64 *)calloc((size_t)ORC_MAX_SETS * k * W, sizeof(u64));
    u64 *tr = (u64 *)calloc((size_t)ORC_MAX_SETS * k, sizeof(u64));
    int *cover = (int *)calloc((size_t)n, sizeof(int));
    int *h = (int *)calloc(ORC_MAX_SETS, sizeof(int));
    if (!rel || !piv || !gam || !tr || !cover || !h) {
        free(rel); free(piv); free(gam); free(tr); free(cover); free(h);
        return ORC_ENOMEM;
    }
    int rc = orc_partition_overlap(G, n, k, W, msets, rel, piv, gam, tr, cover);
    if (rc != ORC_OK) { free(rel); free(piv); free(gam); free(tr); free(cover); free(h); return rc; }
    const int m = msets;
    out->m = m;
    for (int j = 0; j < m; j++) out->ranks[j] = rel[j];
    int L = 1, U = n - k + 1;
    int have_key = 0;
    int g = 1;
    while (g <= k && L < U) {
        for (int j = 0; j < m; j++) {
            int w; u64 rank, cnt;
            orc_enumerate_unit(gam + (size_t)j * k * W, n, k, W, g, nthreads, &w, &rank, &cnt, NULL, NULL);
            out->counts[g * ORC_MAX_SETS + j] = cnt;
            out->g_final = g; out->j_final = j;
            if (!have_key || w < out->key_w) {
                out->key_w = w; out->key_g = g; out->key_j = j; out->key_rank = rank;
                have_key = 1;
            }
            if (w < U) U = w;
            h[j] = g;
            if (check_per_matrix) {
                const int Lm = orc_overlap_bound(m, h, k, rel, n, cover);
                if (Lm > L) L = Lm;
                if (L >= U) break;
            }
        }
        if (!check_per_matrix) L = orc_overlap_bound(m, h, k, rel, n, cover);
        if (L >= U) break;
        g++;
    }
    out->d = U;
    out->L_final = L; out->U_final = U;
    witness_of_key(G, k, W, tr, out);
    free(rel); free(piv); free(gam); free(tr); free(cover); free(h);
    return ORC_OK;
}
