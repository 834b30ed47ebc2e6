// api.cpp -- the C-ABI of libmdist.so (declared in include/mdist.h): code handles,
// the Alg. 1 driver (levels g = 1, 2, ... over all information sets while L < U,
// §2), the per-unit GPU launches, results, checkpoint / resume.
#include <algorithm>
#include <chrono>
#include <climits>
#include <cstdlib>
#include <cstring>
#include <new>
#include <map>
#include <mutex>
#include <vector>

#include "internal.h"
#include "prep.h"
#include "../../include/mdist_debug.h"

using mdist::DeviceRows;
using mdist::EnumParams;
using mdist::Partition;
using mdist::UnitSlot;

namespace {

struct RunState {
    int next_g = 1, next_j = 0;
    int U = 0, L = 1;
    int have_key = 0;
    mdist_key key{INT32_MAX, 0, 0, 0, 0};
    int finished = 0;
    int g_last = 0, j_last = -1;
    int launches = 0;
    double kernel_ms = 0.0;
    double tc_ms = 0.0;
    int tc_launches = 0;
    uint64_t tc_combos = 0;
    uint64_t tc_cand = 0;            // pairs the tensor-core filter passed to the exact recheck
    double seconds = 0.0;
    uint64_t h2d_bytes = 0, d2h_bytes = 0;
    int last_group = 0;
    int done_level[MDIST_MAX_SETS];  // skip_idle_sets: highest level enumerated per set
    uint64_t counts[MDIST_MAX_K + 1][MDIST_MAX_SETS];
};

uint64_t fnv1a(const void *data, size_t len, uint64_t h = 1469598103934665603ull) {
    const unsigned char *p = (const unsigned char *)data;
    for (size_t i = 0; i < len; ++i) { h ^= p[i]; h *= 1099511628211ull; }
    return h;
}

}  // namespace

struct mdist_code {
    int n = 0, k = 0, W = 0, m = 0;
    std::vector<uint64_t> G;
    Partition part;
    std::vector<DeviceRows> rows;
    mdist_options opt{};
    cudaStream_t stream = nullptr;
    int device = 0, sm_count = 0;
    std::vector<uint32_t *> d_rows;
    UnitSlot *d_slot = nullptr;
    UnitSlot *h_slot = nullptr;          // pinned (pinned_get)
    unsigned long long pinned_ctx = 0;   // context the pinned blocks belong to (0: unknown)
    unsigned long long *d_hist = nullptr;// n+1 bins, on demand
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::vector<cudaEvent_t> tc_ev;      // event pairs around tensor-core launches, one pair per unit of a wave
    uint64_t rows_bytes = 0;             // Gamma rows copied to the device by mdist_prepare
    int gram_mode = 0;                   // tensor-core plan mode the units use (see mdist_prepare)
    int wave_cap = 0;                    // units a wave can hold: m * (k + 1)
    UnitSlot *d_wave = nullptr;          // [wave_cap] per-unit slots + 1 threshold word after them
    UnitSlot *h_wave = nullptr;          // pinned copy
    // tables of the tensor-core enumerator (side_key: set, side components, expanded)
    std::map<uint64_t, void *> tabs;
    size_t tab_bytes = 0;
    // device memory of the tables: chunks from the allocator, handed out in order
    std::vector<void *> tab_chunks;
    size_t chunk_used = 0, chunk_size = 0;
    // tables allocated but not built yet (all of one set), built together by flush_tables
    int pend_j = -1;
    std::vector<mdist::GramSide> pend_sides;
    std::vector<uint32_t *> pend_outs;
    std::vector<const uint32_t *> pend_xpacked;
    std::vector<unsigned long long> pend_xcount;
    std::vector<uint8_t *> pend_xout;
    // tensor-core counters of the last mdist_enumerate_level call (summed over its units)
    uint64_t level_tc_combos = 0, level_tc_cand = 0;
    RunState st;
};

namespace {

// Page-locked host blocks kept after a handle is freed and handed to the next handle
// made in the same CUDA context: cudaMallocHost and cudaFreeHost cost tens of
// microseconds each and cudaFreeHost waits for the device.  A block belongs to the
// context that allocated it (its pages go with the context), so it is filed under that
// context's unique id and only reused there; at most kPinnedKeep blocks are kept.
struct PinnedBlock {
    unsigned long long ctx;
    size_t bytes;
    void *p;
};
constexpr size_t kPinnedKeep = 32;
std::mutex g_pinned_mu;
std::vector<PinnedBlock> g_pinned;

void *pinned_get(size_t bytes, unsigned long long *ctx) {
    unsigned long long id = 0;
    if (mdist::current_context_id(&id) == MDIST_OK) {
        std::lock_guard<std::mutex> lock(g_pinned_mu);
        for (size_t i = 0; i < g_pinned.size(); ++i)
            if (g_pinned[i].ctx == id && g_pinned[i].bytes == bytes) {
                void *p = g_pinned[i].p;
                g_pinned.erase(g_pinned.begin() + (long)i);
                *ctx = id;
                return p;
            }
    }
    void *p = nullptr;
    if (cudaMallocHost(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    *ctx = mdist::current_context_id(&id) == MDIST_OK ? id : 0;  // the context exists now
    return p;
}

void pinned_put(void *p, size_t bytes, unsigned long long ctx) {
    if (!p) return;
    if (ctx) {
        std::lock_guard<std::mutex> lock(g_pinned_mu);
        if (g_pinned.size() < kPinnedKeep) {
            g_pinned.push_back({ctx, bytes, p});
            return;
        }
    }
    if (cudaFreeHost(p) != cudaSuccess) cudaGetLastError();  // e.g. its context is gone
}

void *dev_alloc(mdist_code *c, size_t bytes) {
    if (c->opt.dev_alloc) return c->opt.dev_alloc(bytes, c->opt.alloc_ctx);
    void *p = nullptr;
    return cudaMalloc(&p, bytes) == cudaSuccess ? p : nullptr;
}

void dev_release(mdist_code *c, void *p) {
    if (!p) return;
    if (c->opt.dev_free) c->opt.dev_free(p, c->opt.alloc_ctx);
    else cudaFree(p);
}

int check_shape(const uint64_t *G, int n, int k, int W) {
    if (!G || k < 1 || k > MDIST_MAX_K || n <= k || n > MDIST_MAX_N || W < (n + 63) / 64 || W > 64)
        return MDIST_EINVAL;
    for (int r = 0; r < k; ++r)
        for (int i = n; i < 64 * W; ++i)
            if ((G[(size_t)r * W + (i >> 6)] >> (i & 63)) & 1ull) return MDIST_EINVAL;
    return MDIST_OK;
}

int set_bound(int h, int k, int r) {
    const int v = h + 1 - (k - r);
    return v > 0 ? v : 0;
}

void reset_state(mdist_code *c) {
    c->st = RunState{};
    std::memset(c->st.counts, 0, sizeof c->st.counts);
    c->st.U = c->n - c->k + 1;  // Alg. 1, line 1: L := 1, U := n - k + 1
    c->st.L = 1;
}

// At least `pairs` event pairs for timing tensor-core launches.
bool tc_events(mdist_code *c, int pairs) {
    while (c->tc_ev.size() < 2 * (size_t)pairs) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return false;
        c->tc_ev.push_back(e);
    }
    return true;
}

// Device bytes a code may hold in subset-sum tables; blocks whose tables would not fit
// stay on the ALU enumerator.
constexpr size_t kTableBudget = 16ull << 30;

// Product blocks with fewer codewords than this and a side under kGramMinSide entries
// stay on the ALU kernel; larger ones are split for the tensor cores.
constexpr unsigned long long kSplitMin = 1ull << 24;
// tensor_cores = 0 on a code whose estimated work (Gilbert-Varshamov level, as the
// routing estimate) reaches kSplitAllWork codewords plans its units as mode 3: every
// block with a small side goes to the tensor cores.  Measured on codes of 10^4 to
// 10^12 codewords: below ~10^6 the parts' tables and launches cost more than the ALU
// kernel's small blocks ([60,30] fresh run 0.34 -> 0.92 ms), from ~10^7 up they cost
// less ([100,40] 0.93 -> 0.69 ms, [260,30] 5.3 -> 2.4 ms, [192,64] -0.7 ms a run).
constexpr double kSplitAllWork = 1e7;

mdist::GramSide make_side(int off0, int kc0, int t0, int off1 = 0, int kc1 = 0, int t1 = -1) {
    mdist::GramSide S{};
    S.nc = t1 >= 0 ? 2 : 1;
    S.off[0] = (uint8_t)off0;
    S.kc[0] = (uint8_t)kc0;
    S.t[0] = (uint8_t)t0;
    S.cnt0 = (uint32_t)mdist::binom_host(kc0, t0);
    S.n = S.cnt0;
    if (t1 >= 0) {
        S.off[1] = (uint8_t)off1;
        S.kc[1] = (uint8_t)kc1;
        S.t[1] = (uint8_t)t1;
        S.n *= mdist::binom_host(kc1, t1);
    }
    return S;
}

uint64_t side_key(int j, const mdist::GramSide &S, bool expanded) {
    uint64_t key = ((uint64_t)j << 1) | (expanded ? 1u : 0u);
    key = (key << 1) | (S.nc == 2 ? 1u : 0u);
    for (int i = 0; i < 2; ++i) {
        const bool on = i < S.nc;
        key = (key << 6) | (on ? S.off[i] : 0u);
        key = (key << 6) | (on ? S.kc[i] : 0u);
        key = (key << 6) | (on ? S.t[i] : 0u);
    }
    return key;
}

// Device memory for a table: 256-byte aligned pieces of chunks that start at 64 MiB and
// double with every chunk up to 1 GiB, so that a run's hundreds of tables (several GB
// on the large codes) cost a handful of allocator calls while a small code holds one
// small chunk.  The first piece starts at the chunk's first 256-byte boundary, whatever
// the allocator's alignment (bulk copies and vector stores need 16-byte aligned tables).
void *table_alloc(mdist_code *c, size_t bytes) {
    constexpr size_t kChunk = 64ull << 20, kChunkMax = 1ull << 30, kAlign = 256;
    bytes = (bytes + kAlign - 1) / kAlign * kAlign;
    if (c->tab_chunks.empty() || c->chunk_used + bytes > c->chunk_size) {
        const size_t grown = c->tab_chunks.size() < 5 ? kChunk << c->tab_chunks.size() : kChunkMax;
        const size_t size = (bytes > grown ? bytes : grown) + kAlign;
        void *p = dev_alloc(c, size);
        if (!p) return nullptr;
        c->tab_chunks.push_back(p);
        c->chunk_size = size;
        c->chunk_used = (kAlign - (size_t)((uintptr_t)p % kAlign)) % kAlign;
    }
    void *p = (char *)c->tab_chunks.back() + c->chunk_used;
    c->chunk_used += bytes;
    return p;
}

int side_table(mdist_code *c, int j, const mdist::GramSide &S, bool expanded, const void **out);

// Low tables: the packed table of the one-component side (off0, kc0, u) of set j, built
// by an earlier flush, with the largest u in [3, t0) whose table fits in kLowTableBytes
// (it stays in the L2 while the new table streams past); 0 when there is none.
constexpr size_t kLowTableBytes = 32ull << 20;

int low_table(const mdist_code *c, int j, const mdist::GramSide &S, int nwords, const uint32_t **out) {
    *out = nullptr;
    for (int u = (int)S.t[0] - 1; u >= 3; --u) {
        if ((size_t)mdist::binom_host(S.kc[0], u) * (size_t)nwords * sizeof(uint32_t) > kLowTableBytes) continue;
        auto it = c->tabs.find(side_key(j, make_side(S.off[0], S.kc[0], u), false));
        if (it == c->tabs.end()) continue;
        if (std::find(c->pend_outs.begin(), c->pend_outs.end(), (uint32_t *)it->second) != c->pend_outs.end())
            continue;  // not written yet
        *out = (const uint32_t *)it->second;
        return u;
    }
    return 0;
}

// Build the pending tables of set c->pend_j.  First launch: the sides of t0 <= 3 (their
// low-subset sums built in shared memory) and those with a low table from an earlier
// flush; second launch: the other sides, reading the table of the 3-subsets of their
// component-0 rows written by the first (allocated here when no block needs it).  Then
// one launch for the expansions, all on the same stream.
int flush_tables(mdist_code *c) {
    if (c->pend_j < 0) return MDIST_OK;
    const int j = c->pend_j;
    const DeviceRows &dr = c->rows[(size_t)j];
    const size_t np = c->pend_sides.size();
    std::vector<const uint32_t *> lows(np);
    std::vector<int> low_t(np), wave(np);
    for (size_t i = 0; i < np; ++i) {
        const mdist::GramSide S = c->pend_sides[i];
        low_t[i] = low_table(c, j, S, dr.nwords, &lows[i]);
        if (low_t[i] || S.t[0] <= 3) continue;
        const void *t3 = nullptr;  // may append a pending table of t0 = 3 (built first)
        const int rc = side_table(c, j, make_side(S.off[0], S.kc[0], 3), false, &t3);
        if (rc != MDIST_OK) return rc;
        if (t3) {
            lows[i] = (const uint32_t *)t3;
            low_t[i] = 3;
            wave[i] = 1;
        }
    }
    lows.resize(c->pend_sides.size());
    low_t.resize(c->pend_sides.size());
    wave.resize(c->pend_sides.size());
    cudaError_t e = cudaSuccess;
    for (int w = 0; w < 2 && e == cudaSuccess; ++w) {
        std::vector<mdist::GramSide> sides;
        std::vector<uint32_t *> outs;
        std::vector<const uint32_t *> lw;
        std::vector<int> lt;
        for (size_t i = 0; i < c->pend_sides.size(); ++i) {
            if (wave[i] != w) continue;
            sides.push_back(c->pend_sides[i]);
            outs.push_back(c->pend_outs[i]);
            lw.push_back(lows[i]);
            lt.push_back(low_t[i]);
        }
        for (size_t i = 0; i < sides.size() && e == cudaSuccess; i += mdist::kMaxTableJobs) {
            const int n = (int)std::min<size_t>(mdist::kMaxTableJobs, sides.size() - i);
            e = mdist::launch_side_tables(c->d_rows[(size_t)j], c->k, dr.nwords, &sides[i], &outs[i], &lw[i], &lt[i],
                                          n, c->sm_count, c->stream);
            c->st.launches += 1;
        }
    }
    for (size_t i = 0; i < c->pend_xout.size() && e == cudaSuccess; i += mdist::kMaxTableJobs) {
        const int n = (int)std::min<size_t>(mdist::kMaxTableJobs, c->pend_xout.size() - i);
        e = mdist::launch_expand_tables(dr.nwords, dr.n_bits, &c->pend_xpacked[i], &c->pend_xcount[i],
                                        &c->pend_xout[i], n, c->sm_count, c->stream);
        c->st.launches += 1;
    }
    c->pend_j = -1;
    c->pend_sides.clear();
    c->pend_outs.clear();
    c->pend_xpacked.clear();
    c->pend_xcount.clear();
    c->pend_xout.clear();
    return e == cudaSuccess ? MDIST_OK : MDIST_ECUDA;
}

// Table of the sums of a side's entries of set j and, with `expanded`, its expansion to
// tensor-core operand tiles; allocated on first use (built by the next flush_tables)
// and kept for later levels and runs; null when over budget.
int side_table(mdist_code *c, int j, const mdist::GramSide &S, bool expanded, const void **out) {
    *out = nullptr;
    const uint64_t key = side_key(j, S, expanded);
    auto it = c->tabs.find(key);
    if (it != c->tabs.end()) {
        *out = it->second;
        return MDIST_OK;
    }
    if (c->pend_j >= 0 && c->pend_j != j) {
        const int rc = flush_tables(c);
        if (rc != MDIST_OK) return rc;
    }
    const DeviceRows &dr = c->rows[(size_t)j];
    const void *packed = nullptr;
    if (expanded) {
        const int rc = side_table(c, j, S, false, &packed);
        if (rc != MDIST_OK || !packed) return rc;
    }
    const size_t bytes = expanded ? mdist::gram_expanded_bytes(dr.nwords, S.n)
                                  : (size_t)S.n * (size_t)dr.nwords * sizeof(uint32_t);
    if (c->tab_bytes + bytes > kTableBudget) return MDIST_OK;
    void *d = table_alloc(c, bytes);
    if (!d) return MDIST_OK;
    c->pend_j = j;
    if (expanded) {
        c->pend_xpacked.push_back((const uint32_t *)packed);
        c->pend_xcount.push_back(S.n);
        c->pend_xout.push_back((uint8_t *)d);
    } else {
        c->pend_sides.push_back(S);
        c->pend_outs.push_back((uint32_t *)d);
    }
    c->tabs[key] = d;
    c->tab_bytes += bytes;
    *out = d;
    return MDIST_OK;
}

// One tensor-core block with its tables (false when a table is over budget).
int add_gram_block(mdist_code *c, int j, mdist::GramSide A, mdist::GramSide B,
                   std::vector<mdist::GramBlockSpec> &out, bool *ok) {
    *ok = false;
    if (B.n > A.n) std::swap(A, B);  // the streamed (B) side is the smaller one
    const void *a = nullptr, *b = nullptr, *bx = nullptr;
    int rc = side_table(c, j, A, false, &a);
    if (rc == MDIST_OK && a) rc = side_table(c, j, B, false, &b);
    if (rc == MDIST_OK && b) rc = side_table(c, j, B, true, &bx);
    if (rc != MDIST_OK || !a || !b || !bx) return rc;
    mdist::GramBlockSpec g;
    g.a = A;
    g.b = B;
    g.a_tab = (const uint32_t *)a;
    g.b_tab = (const uint32_t *)b;
    g.b_exp = (const uint8_t *)bx;
    out.push_back(g);
    *ok = true;
    return MDIST_OK;
}

// The tensor-core parts of product block B of a level with halves of k1 and k2 rows,
// written to A[], Bs[] (at most `cap`); returns their count, 0 when the block stays on
// the ALU kernel.  tensor_cores 0: a block whose sides both hold >= kGramMinSide
// entries is one part as it is; one with a smaller side and at least kSplitMin
// codewords is split over the two quarters of its large side's half:
// S x L_t = union over i of (S + Qa_i) x Qb_(t-i) (Vandermonde), every part with two
// large sides.  tensor_cores 3: as 0, splitting every block with a small side whatever
// its size; 2: every block as it is; 1: none.  No tables, no device calls.
int gram_block_parts(int mode, int k1, int k2, const mdist::ProductBlock &B, int cap, mdist::GramSide *A,
                     mdist::GramSide *Bs) {
    if (mode == 1) return 0;
    const int loff = B.lane_half ? k1 : 0, lkc = B.lane_half ? k2 : k1;
    const int woff = B.lane_half ? 0 : k1, wkc = B.lane_half ? k1 : k2;
    const unsigned long long small = B.lane_n < B.walk_n ? B.lane_n : B.walk_n;
    if (mode == 2 || small >= (unsigned long long)mdist::kGramMinSide) {
        if (cap < 1) return 0;
        A[0] = make_side(loff, lkc, (int)B.lane_t);
        Bs[0] = make_side(woff, wkc, (int)B.walk_t);
        return 1;
    }
    if (mode != 3 && B.lane_n * B.walk_n < kSplitMin) return 0;
    // large side L (t_L-subsets of kc_L rows at off_L), small side S
    const bool lane_large = B.lane_n >= B.walk_n;
    const int Loff = lane_large ? loff : woff, Lkc = lane_large ? lkc : wkc;
    const int Lt = (int)(lane_large ? B.lane_t : B.walk_t);
    const int Soff = lane_large ? woff : loff, Skc = lane_large ? wkc : lkc;
    const int St = (int)(lane_large ? B.walk_t : B.lane_t);
    const int qa = Lkc / 2, qb = Lkc - qa;
    const int i0 = Lt - qb > 0 ? Lt - qb : 0, i1 = Lt < qa ? Lt : qa;
    if (Lt < 1 || i1 - i0 + 1 > cap) return 0;
    for (int i = i0; i <= i1; ++i) {
        A[i - i0] = St > 0 ? make_side(Soff, Skc, St, Loff, qa, i) : make_side(Loff, qa, i);
        Bs[i - i0] = make_side(Loff + qa, qb, Lt - i);
    }
    return i1 - i0 + 1;
}

// Tables of the levels after g (set j), requested with level g's own while their sum
// stays within kPrefetchBytes, so that the small early levels share one flush (one pair
// of table launches) instead of a flush each.  Requests only: a table over budget is
// left out here as it is at its own level.
constexpr size_t kPrefetchBytes = 64ull << 20;

int prefetch_tables(mdist_code *c, int j, int g) {
    const DeviceRows &dr = c->rows[(size_t)j];
    size_t total = 0;
    for (int g2 = g + 1; g2 <= c->k; ++g2) {
        EnumParams q{};
        if (!mdist::plan_level(c->k, g2, dr.nwords, q)) return MDIST_OK;
        std::vector<std::pair<mdist::GramSide, mdist::GramSide>> parts;
        size_t bytes = 0;
        mdist::GramSide A[mdist::kMaxGramBlocks], Bs[mdist::kMaxGramBlocks];
        for (int b = 0; b < q.nblocks; ++b) {
            const int np = gram_block_parts(c->gram_mode, q.k1, q.k2, q.blocks[b],
                                            mdist::kMaxGramBlocks - (int)parts.size(), A, Bs);
            for (int i = 0; i < np; ++i) {
                mdist::GramSide a = A[i], bs = Bs[i];
                if (bs.n > a.n) std::swap(a, bs);  // as add_gram_block: B is the smaller side
                bytes += (size_t)(a.n + bs.n) * (size_t)dr.nwords * sizeof(uint32_t) +
                         mdist::gram_expanded_bytes(dr.nwords, bs.n);
                parts.push_back({a, bs});
            }
        }
        if (total + bytes > kPrefetchBytes) return MDIST_OK;
        total += bytes;
        for (const auto &pr : parts) {
            const void *t = nullptr;
            int rc = side_table(c, j, pr.first, false, &t);
            if (rc == MDIST_OK) rc = side_table(c, j, pr.second, false, &t);
            if (rc == MDIST_OK && t) rc = side_table(c, j, pr.second, true, &t);
            if (rc != MDIST_OK) return rc;
        }
    }
    return MDIST_OK;
}

// The tensor-core part of unit p (set j): gram_block_parts of every product block,
// with its tables; a block any of whose tables is over budget stays on the ALU kernel
// as a whole.  covered[b] marks the blocks handled there.
int gram_plan(mdist_code *c, int j, const EnumParams &p, std::vector<mdist::GramBlockSpec> &out, bool *covered) {
    out.clear();
    for (int b = 0; b < mdist::kMaxBlocks; ++b) covered[b] = false;
    if (!mdist::gram_eligible(p.nwords)) return MDIST_OK;
    mdist::GramSide A[mdist::kMaxGramBlocks], Bs[mdist::kMaxGramBlocks];
    for (int b = 0; b < p.nblocks; ++b) {
        const int np = gram_block_parts(c->gram_mode, p.k1, p.k2, p.blocks[b],
                                        mdist::kMaxGramBlocks - (int)out.size(), A, Bs);
        const size_t mark = out.size();
        bool all = np > 0;
        for (int i = 0; i < np && all; ++i) {
            const int rc = add_gram_block(c, j, A[i], Bs[i], out, &all);
            if (rc != MDIST_OK) return rc;
        }
        if (all) covered[b] = true;
        else out.resize(mark);  // a table over budget: the whole block stays on the ALU kernel
    }
    if (c->pend_j == j) {  // tables are built for this level: add the next levels' small ones
        const int rc = prefetch_tables(c, j, p.g);
        if (rc != MDIST_OK) return rc;
    }
    return flush_tables(c);
}

// One (g, j) unit on the GPU.  Candidates: codewords of weight <= U_thr.
// part / nparts: only that slice of the unit's work (a unit split over ranks).
int run_unit(mdist_code *c, int g, int j, int U_thr, bool hist_mode, bool *found, int *w_out, uint64_t *rank_out,
             uint64_t *count_out, int part = 0, int nparts = 1) {
    const DeviceRows &dr = c->rows[(size_t)j];
    EnumParams p{};
    if (!mdist::plan_level(c->k, g, dr.nwords, p)) return MDIST_ERANGE;
    p.rows = c->d_rows[(size_t)j];
    p.U = &c->d_slot->U;
    p.slot = c->d_slot;
    p.hist = c->d_hist;
    p.nwords = dr.nwords;
    p.n_bits = dr.n_bits;
    p.base = dr.full_rank ? g : 0;
    p.wait_polls = c->opt.timeout_cycles;
    c->h_slot->U = (unsigned)(U_thr < 0 ? 0 : U_thr);
    c->h_slot->status = 0;
    c->h_slot->key = mdist::kNoKey;
    c->h_slot->count = 0;
    c->h_slot->tile_next = 0;
    c->h_slot->tc_cand = 0;
    if (cudaMemcpyAsync(c->d_slot, c->h_slot, sizeof(UnitSlot), cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
        return MDIST_ECUDA;
    c->st.h2d_bytes += sizeof(UnitSlot);
    if (cudaEventRecord(c->ev0, c->stream) != cudaSuccess) return MDIST_ECUDA;
    int group = 0;
    if (!hist_mode) {
        const int fg = c->opt.filter_group;
        group = fg == 0 ? mdist::choose_filter_group(dr.nwords, dr.n_bits, (U_thr < 0 ? 0 : U_thr) - p.base)
                        : (fg == 1 ? 0 : fg);
        if (!mdist::filter_group_valid(group, dr.nwords)) group = 0;
    }
    c->st.last_group = group;
    std::vector<mdist::GramBlockSpec> gspecs;
    bool covered[mdist::kMaxBlocks] = {};
    if (!hist_mode) {
        const int rc = gram_plan(c, j, p, gspecs, covered);
        if (rc != MDIST_OK) return rc;
    }
    if (!tc_events(c, 1)) return MDIST_ECUDA;
    unsigned long long tc_combos = 0;
    int kernels = 0;
    if (mdist::launch_unit_split(p, dr.nwords, group, hist_mode, c->sm_count, c->opt.blocks_per_sm,
                                 gspecs.data(), (int)gspecs.size(), covered, c->stream, c->tc_ev[0], c->tc_ev[1],
                                 &tc_combos, &kernels, part, nparts) != cudaSuccess)
        return MDIST_ECUDA;
    if (cudaEventRecord(c->ev1, c->stream) != cudaSuccess) return MDIST_ECUDA;
    if (cudaMemcpyAsync(c->h_slot, c->d_slot, sizeof(UnitSlot), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
        return MDIST_ECUDA;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return MDIST_ECUDA;
    c->st.d2h_bytes += sizeof(UnitSlot);
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->ev0, c->ev1) == cudaSuccess) c->st.kernel_ms += ms;
    c->st.launches += kernels;
    if (tc_combos && cudaEventElapsedTime(&ms, c->tc_ev[0], c->tc_ev[1]) == cudaSuccess) {
        c->st.tc_ms += ms;
        c->st.tc_launches += 1;
        c->st.tc_combos += tc_combos;
    }
    c->st.tc_cand += c->h_slot->tc_cand;
    c->level_tc_combos += tc_combos;
    c->level_tc_cand += c->h_slot->tc_cand;
    if (c->h_slot->status) return MDIST_ETIMEOUT;
    const unsigned long long key = c->h_slot->key;
    *found = key != mdist::kNoKey;
    *w_out = *found ? (int)(key >> mdist::kKeyRankBits) : INT_MAX;
    *rank_out = *found ? (key & ((1ull << mdist::kKeyRankBits) - 1)) : 0;
    *count_out = c->h_slot->count;
    return MDIST_OK;
}

bool key_less(const mdist_key &a, const mdist_key &b) {
    if (a.weight != b.weight) return a.weight < b.weight;
    if (a.g != b.g) return a.g < b.g;
    if (a.j != b.j) return a.j < b.j;
    return a.rank < b.rank;
}

// g-subset of {0..k-1} with lexicographic rank `rank`, as a mask.  With
// d_i = k-1-c_i the rank satisfies C(k,g)-1-rank = sum_i C(d_i, g-i+1), the
// combinatorial number system, so the d_i are read off greedily from the top.
uint64_t unrank_lex_host(int k, int g, uint64_t rank) {
    uint64_t r = mdist::binom_host(k, g) - 1 - rank;
    uint64_t mask = 0;
    int d = k - 1;
    for (int t = g; t >= 1; --t) {
        while (mdist::binom_host(d, t) > r) --d;
        r -= mdist::binom_host(d, t);
        mask |= 1ull << (k - 1 - d);
        --d;
    }
    return mask;
}

}  // namespace

extern "C" {

const char *mdist_strerror(int err) {
    switch (err) {
        case MDIST_OK: return "ok";
        case MDIST_EINVAL: return "invalid argument";
        case MDIST_ERANK: return "generator matrix has rank < k";
        case MDIST_ENOMEM: return "out of memory";
        case MDIST_ECUDA: return "CUDA error";
        case MDIST_ETIMEOUT: return "device wait timed out";
        case MDIST_ECANCELLED: return "cancelled";
        case MDIST_ERANGE: return "level beyond the device key range (C(k,g) >= 2^54)";
        case MDIST_ESTATE: return "state blob does not match this code";
        case MDIST_EAGAIN: return "not ready / busy";
        default: return "unknown error";
    }
}

void mdist_free(mdist_code *c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    for (uint32_t *p : c->d_rows) dev_release(c, p);
    for (void *p : c->tab_chunks) dev_release(c, p);
    dev_release(c, c->d_slot);
    dev_release(c, c->d_hist);
    dev_release(c, c->d_wave);
    pinned_put(c->h_wave, sizeof(UnitSlot) * ((size_t)c->wave_cap + 1), c->pinned_ctx);
    pinned_put(c->h_slot, sizeof(UnitSlot), c->pinned_ctx);
    for (cudaEvent_t e : c->tc_ev) cudaEventDestroy(e);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    delete c;
}

int mdist_prepare(const uint64_t *G, int n, int k, int words_per_row, const mdist_options *opts, void *cuda_stream,
                  mdist_code **out) {
    if (!out) return MDIST_EINVAL;
    *out = nullptr;
    int rc = check_shape(G, n, k, words_per_row);
    if (rc != MDIST_OK) return rc;
    mdist_code *c = new (std::nothrow) mdist_code();
    if (!c) return MDIST_ENOMEM;
    if (opts) c->opt = *opts;
    if (c->opt.filter_group < 0 || c->opt.filter_group > 5 || c->opt.tensor_cores < 0 || c->opt.tensor_cores > 3 ||
        c->opt.skip_idle_sets < 0 || c->opt.skip_idle_sets > 1 || (c->opt.skip_idle_sets && c->opt.check_per_matrix) ||
        c->opt.timeout_cycles < 0 || c->opt.overlap_sets < 0 || c->opt.overlap_sets > MDIST_MAX_SETS ||
        (c->opt.overlap_sets && c->opt.skip_idle_sets)) {
        delete c;
        return MDIST_EINVAL;
    }
    if (c->opt.max_sets <= 0 || c->opt.max_sets > MDIST_MAX_SETS) c->opt.max_sets = MDIST_MAX_SETS;
    c->n = n;
    c->k = k;
    c->W = words_per_row;
    c->G.assign(G, G + (size_t)k * words_per_row);
    c->stream = (cudaStream_t)cuda_stream;
    rc = c->opt.overlap_sets > 0
             ? mdist::partition_overlapping_sets(G, n, k, words_per_row, c->opt.overlap_sets, c->part)
             : mdist::partition_info_sets(G, n, k, words_per_row, c->opt.max_sets, c->part);
    if (rc != MDIST_OK) { delete c; return rc; }
    c->m = (int)c->part.sets.size();
    c->gram_mode = c->opt.tensor_cores == 0 &&
                           mdist::estimated_work(n, k, c->part, c->opt.wstar_hint) >= kSplitAllWork
                       ? 3
                       : c->opt.tensor_cores;
    c->rows.resize((size_t)c->m);
    for (int j = 0; j < c->m; ++j) mdist::build_rows(c->part, j, c->rows[(size_t)j]);
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return MDIST_ECUDA;
    }
    if (cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess ||
        !(c->h_slot = (UnitSlot *)pinned_get(sizeof(UnitSlot), &c->pinned_ctx))) {
        mdist_free(c);
        return MDIST_ECUDA;
    }
    c->d_slot = (UnitSlot *)dev_alloc(c, sizeof(UnitSlot));
    if (!c->d_slot) { mdist_free(c); return MDIST_ENOMEM; }
    c->wave_cap = c->m * (k + 1);
    c->d_wave = (UnitSlot *)dev_alloc(c, sizeof(UnitSlot) * ((size_t)c->wave_cap + 1));
    if (!c->d_wave) { mdist_free(c); return MDIST_ENOMEM; }
    unsigned long long wave_ctx = 0;
    c->h_wave = (UnitSlot *)pinned_get(sizeof(UnitSlot) * ((size_t)c->wave_cap + 1), &wave_ctx);
    if (!c->h_wave) {
        mdist_free(c);
        return MDIST_ECUDA;
    }
    if (wave_ctx != c->pinned_ctx) c->pinned_ctx = 0;  // both blocks must belong to one context
    c->d_rows.assign((size_t)c->m, nullptr);
    for (int j = 0; j < c->m; ++j) {
        const DeviceRows &dr = c->rows[(size_t)j];
        const size_t bytes = dr.words.size() * sizeof(uint32_t);
        c->rows_bytes += bytes;
        c->d_rows[(size_t)j] = (uint32_t *)dev_alloc(c, bytes);
        if (!c->d_rows[(size_t)j]) { mdist_free(c); return MDIST_ENOMEM; }
        if (cudaMemcpyAsync(c->d_rows[(size_t)j], dr.words.data(), bytes, cudaMemcpyHostToDevice, c->stream) !=
            cudaSuccess) {
            mdist_free(c);
            return MDIST_ECUDA;
        }
    }
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) { mdist_free(c); return MDIST_ECUDA; }
    reset_state(c);
    *out = c;
    return MDIST_OK;
}

int mdist_set_stream(mdist_code *c, void *cuda_stream) {
    if (!c) return MDIST_EINVAL;
    c->stream = (cudaStream_t)cuda_stream;
    return MDIST_OK;
}

int mdist_info_sets(const mdist_code *c, int *m, int *ranks, int32_t *pivcols, uint64_t *gammas,
                    uint64_t *transforms) {
    if (!c || !m) return MDIST_EINVAL;
    *m = c->m;
    for (int j = 0; j < c->m; ++j) {
        const mdist::InfoSet &s = c->part.sets[(size_t)j];
        if (ranks) ranks[j] = s.bound_rank;
        if (pivcols)
            for (int i = 0; i < c->k; ++i) pivcols[(size_t)j * c->k + i] = i < s.rank ? s.pivcols[(size_t)i] : -1;
        if (gammas) std::memcpy(gammas + (size_t)j * c->k * c->W, s.gamma.data(), sizeof(uint64_t) * s.gamma.size());
        if (transforms) std::memcpy(transforms + (size_t)j * c->k, s.transform.data(), sizeof(uint64_t) * c->k);
    }
    return MDIST_OK;
}

int mdist_enumerate_level(mdist_code *c, int g, int j, int *U_inout, mdist_key *key_inout, uint64_t *combos_out) {
    if (!c || !U_inout || !key_inout || g < 1 || g > c->k || j < -1 || j >= c->m) return MDIST_EINVAL;
    const int j0 = j < 0 ? 0 : j;
    const int j1 = j < 0 ? c->m : j + 1;
    c->level_tc_combos = c->level_tc_cand = 0;
    for (int jj = j0; jj < j1; ++jj) {
        bool found;
        int w;
        uint64_t rank, cnt;
        const int rc = run_unit(c, g, jj, *U_inout, false, &found, &w, &rank, &cnt);
        if (rc != MDIST_OK) return rc;
        if (combos_out) combos_out[jj - j0] = cnt;
        if (found) {
            const mdist_key cand{w, g, jj, 0, rank};
            if (key_less(cand, *key_inout)) *key_inout = cand;
            if (w < *U_inout) *U_inout = w;
        }
    }
    return MDIST_OK;
}

int mdist_level_counters(const mdist_code *c, uint64_t *tc_combos, uint64_t *tc_candidates) {
    if (!c) return MDIST_EINVAL;
    if (tc_combos) *tc_combos = c->level_tc_combos;
    if (tc_candidates) *tc_candidates = c->level_tc_cand;
    return MDIST_OK;
}

int mdist_unit_histogram(mdist_code *c, int g, int j, uint64_t *hist, uint64_t *combos_out) {
    if (!c || !hist || g < 1 || g > c->k || j < 0 || j >= c->m) return MDIST_EINVAL;
    const size_t bins = (size_t)c->n + 1;
    if (!c->d_hist) {
        c->d_hist = (unsigned long long *)dev_alloc(c, bins * sizeof(unsigned long long));
        if (!c->d_hist) return MDIST_ENOMEM;
    }
    if (cudaMemsetAsync(c->d_hist, 0, bins * sizeof(unsigned long long), c->stream) != cudaSuccess) return MDIST_ECUDA;
    bool found;
    int w;
    uint64_t rank, cnt;
    const int rc = run_unit(c, g, j, 0, true, &found, &w, &rank, &cnt);
    if (rc != MDIST_OK) return rc;
    if (cudaMemcpyAsync(hist, c->d_hist, bins * sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
        return MDIST_ECUDA;
    if (combos_out) *combos_out = cnt;
    return MDIST_OK;
}

struct UnitRef {
    int g, j;
};

// Launch the units of `list` back to back, each with its own slot, sharing one
// candidate threshold that starts at U_thr (candidates: weight <= threshold); one host
// synchronisation; the results are left in c->h_wave[0 .. list.size()).  The list is
// cut at the first unit beyond the device key range (MDIST_ERANGE when that is the
// first one).
static int launch_units(mdist_code *c, std::vector<UnitRef> &list, int U_thr) {
    RunState &s = c->st;
    EnumParams p{};
    for (size_t u = 0; u < list.size(); ++u) {  // every level must be within the device key range
        if (!mdist::plan_level(c->k, list[u].g, c->rows[(size_t)list[u].j].nwords, p)) {
            if (u == 0) return MDIST_ERANGE;
            list.resize(u);
            break;
        }
    }
    const int n_units = (int)list.size();
    for (int u = 0; u < n_units; ++u) {
        c->h_wave[u].U = 0;
        c->h_wave[u].status = 0;
        c->h_wave[u].key = mdist::kNoKey;
        c->h_wave[u].count = 0;
        c->h_wave[u].tile_next = 0;
        c->h_wave[u].tc_cand = 0;
    }
    UnitSlot &thr_word = c->h_wave[c->wave_cap];
    thr_word.U = (unsigned)(U_thr < 0 ? 0 : U_thr);
    thr_word.status = 0;
    thr_word.key = thr_word.count = thr_word.tile_next = thr_word.tc_cand = 0;
    unsigned int *d_U = &c->d_wave[c->wave_cap].U;
    if (cudaMemcpyAsync(c->d_wave, c->h_wave, sizeof(UnitSlot) * (size_t)n_units, cudaMemcpyHostToDevice, c->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(&c->d_wave[c->wave_cap], &thr_word, sizeof(UnitSlot), cudaMemcpyHostToDevice, c->stream) !=
            cudaSuccess)
        return MDIST_ECUDA;
    s.h2d_bytes += sizeof(UnitSlot) * ((size_t)n_units + 1);
    if (!tc_events(c, n_units)) return MDIST_ECUDA;
    std::vector<unsigned long long> tc_combos((size_t)n_units, 0);
    std::vector<mdist::GramBlockSpec> gspecs;
    int launched = 0, kernels = 0;
    if (cudaEventRecord(c->ev0, c->stream) != cudaSuccess) return MDIST_ECUDA;
    for (int u = 0; u < n_units; ++u) {
        const int g = list[(size_t)u].g, j = list[(size_t)u].j;
        const DeviceRows &dr = c->rows[(size_t)j];
        EnumParams q{};
        mdist::plan_level(c->k, g, dr.nwords, q);
        q.rows = c->d_rows[(size_t)j];
        q.U = d_U;
        q.slot = &c->d_wave[u];
        q.hist = nullptr;
        q.nwords = dr.nwords;
        q.n_bits = dr.n_bits;
        q.base = dr.full_rank ? g : 0;
        q.wait_polls = c->opt.timeout_cycles;
        const int fg = c->opt.filter_group;
        int group = fg == 0 ? mdist::choose_filter_group(dr.nwords, dr.n_bits, U_thr - q.base) : (fg == 1 ? 0 : fg);
        if (!mdist::filter_group_valid(group, dr.nwords)) group = 0;
        bool covered[mdist::kMaxBlocks] = {};
        const int rc = gram_plan(c, j, q, gspecs, covered);
        if (rc != MDIST_OK) return rc;
        if (mdist::launch_unit_split(q, dr.nwords, group, false, c->sm_count, c->opt.blocks_per_sm, gspecs.data(),
                                     (int)gspecs.size(), covered, c->stream, c->tc_ev[2 * (size_t)u],
                                     c->tc_ev[2 * (size_t)u + 1],
                                     &tc_combos[(size_t)u], &kernels) != cudaSuccess)
            return MDIST_ECUDA;
        launched += kernels;
    }
    if (cudaEventRecord(c->ev1, c->stream) != cudaSuccess) return MDIST_ECUDA;
    if (cudaMemcpyAsync(c->h_wave, c->d_wave, sizeof(UnitSlot) * (size_t)n_units, cudaMemcpyDeviceToHost, c->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
        return MDIST_ECUDA;
    s.d2h_bytes += sizeof(UnitSlot) * (size_t)n_units;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->ev0, c->ev1) == cudaSuccess) s.kernel_ms += ms;
    s.launches += launched;
    for (int u = 0; u < n_units; ++u)
        if (tc_combos[(size_t)u] &&
            cudaEventElapsedTime(&ms, c->tc_ev[2 * (size_t)u], c->tc_ev[2 * (size_t)u + 1]) == cudaSuccess) {
            s.tc_ms += ms;
            s.tc_launches += 1;
            s.tc_combos += tc_combos[(size_t)u];
        }
    for (int u = 0; u < n_units; ++u) s.tc_cand += c->h_wave[u].tc_cand;
    for (int u = 0; u < n_units; ++u)
        if (c->h_wave[u].status) return MDIST_ETIMEOUT;
    return MDIST_OK;
}

// Fold the result of unit (g, j) — the least device key (weight << 54 | rank) among its
// candidates, or kNoKey, and its combination count — into the Alg. 1 state, then check
// the bound after the unit (per-matrix mode) or after its level (Alg. 1, line 7, or the
// overlapping sets' bound) and advance to the next unit.
static void fold_unit(mdist_code *c, int g, int j, unsigned long long key, unsigned long long count,
                      int *units_done) {
    RunState &s = c->st;
    s.counts[g][j] = count;
    s.g_last = g;
    s.j_last = j;
    ++*units_done;
    if (key != mdist::kNoKey) {
        const int w = (int)(key >> mdist::kKeyRankBits);
        if (!s.have_key || w < s.key.weight) {
            s.key = mdist_key{w, g, j, 0, key & ((1ull << mdist::kKeyRankBits) - 1)};
            s.have_key = 1;
        }
        if (w < s.U) s.U = w;
    }
    if (c->opt.check_per_matrix) {
        int h[MDIST_MAX_SETS];
        for (int i = 0; i < c->m; ++i) h[i] = i <= j ? g : g - 1;
        const int Lm = mdist::lower_bound(c->part, h);
        if (Lm > s.L) s.L = Lm;
        if (s.L >= s.U) s.finished = 1;
    }
    s.next_j = j + 1;
    if (s.next_j == c->m) {
        s.next_j = 0;
        if (!c->opt.check_per_matrix) {  // Alg. 1, line 7 (or the overlapping sets' bound)
            int h[MDIST_MAX_SETS];
            for (int i = 0; i < c->m; ++i) h[i] = g;
            s.L = mdist::lower_bound(c->part, h);
            if (s.L >= s.U) s.finished = 1;
        }
        s.next_g = g + 1;
        if (s.next_g > c->k) s.finished = 1;
    }
}

// One wave: the units from (next_g, next_j) through the end of level g_hi (at most
// max_units of them) are launched back to back, each with its own slot, sharing one
// candidate threshold (the current best weight, ties kept); one host synchronisation;
// then their results are folded in (g, j) order with the bounds checked after every
// unit (per-matrix mode) or level, exactly as if the units had run one at a time: a
// codeword first met past the termination level weighs at least L >= U, so the shared
// threshold never prunes the unit holding the final U, and folding stops at the
// termination unit.
static int run_wave(mdist_code *c, int g_hi, int max_units, int *units_done) {
    RunState &s = c->st;
    std::vector<UnitRef> list;
    for (int g = s.next_g; g <= g_hi && g <= c->k; ++g)
        for (int j = (g == s.next_g ? s.next_j : 0); j < c->m; ++j) {
            if (max_units > 0 && (int)list.size() >= max_units) break;
            list.push_back({g, j});
        }
    if (list.empty()) return MDIST_OK;
    // every unit of the wave follows the key's unit in (g, j) order, so only lighter
    // codewords can replace the key; weights found inside the wave keep their ties
    const int U_thr = s.have_key ? s.key.weight - 1 : s.U;
    const int rc = launch_units(c, list, U_thr);
    if (rc != MDIST_OK) return rc;
    const int n_units = (int)list.size();
    // fold in (g, j) order
    for (int u = 0; u < n_units && !s.finished; ++u)
        fold_unit(c, list[(size_t)u].g, list[(size_t)u].j, c->h_wave[u].key, c->h_wave[u].count, units_done);
    return MDIST_OK;
}

// skip_idle_sets: level g = next_g.  A set whose bound term t_j(g) = max(0, g+1-(k-r_j))
// is still 0 is left out; a set enumerated for the first time at level g first runs the
// levels it skipped (done_level[j]+1 .. g), so that its term rests on all of its
// combinations of weight <= g.  All units of the level are one wave; ties are
// candidates and the key is the least (weight, g, j, rank) over the enumerated units,
// visited set by set with levels ascending.
static int run_skip_level(mdist_code *c, int *units_done) {
    RunState &s = c->st;
    const int g = s.next_g;
    std::vector<UnitRef> list;
    for (int j = 0; j < c->m; ++j)
        if (set_bound(g, c->k, c->part.sets[(size_t)j].rank) > 0)
            for (int h = s.done_level[j] + 1; h <= g; ++h) list.push_back({h, j});
    if (!list.empty()) {
        const size_t want = list.size();
        const int rc = launch_units(c, list, s.U);
        if (rc != MDIST_OK) return rc;
        if (list.size() != want) return MDIST_ERANGE;
        for (size_t u = 0; u < list.size(); ++u) {
            const int h = list[u].g, j = list[u].j;
            const UnitSlot &r = c->h_wave[u];
            s.counts[h][j] = r.count;
            s.g_last = h;
            s.j_last = j;
            s.done_level[j] = h;
            ++*units_done;
            if (r.key != mdist::kNoKey) {
                const int w = (int)(r.key >> mdist::kKeyRankBits);
                const mdist_key cand{w, h, j, 0, r.key & ((1ull << mdist::kKeyRankBits) - 1)};
                if (!s.have_key || key_less(cand, s.key)) {
                    s.key = cand;
                    s.have_key = 1;
                }
                if (w < s.U) s.U = w;
            }
        }
    }
    int Lg = 0;  // Alg. 1, line 7: the idle sets' terms are 0
    for (int i = 0; i < c->m; ++i) Lg += set_bound(g, c->k, c->part.sets[(size_t)i].rank);
    s.L = Lg;
    if (s.L >= s.U) s.finished = 1;
    s.next_g = g + 1;
    s.next_j = 0;
    if (s.next_g > c->k) s.finished = 1;
    return MDIST_OK;
}

int mdist_reset(mdist_code *c) {
    if (!c) return MDIST_EINVAL;
    reset_state(c);
    return MDIST_OK;
}

int mdist_run(mdist_code *c, int max_units, int *finished) {
    if (!c) return MDIST_EINVAL;
    RunState &s = c->st;
    const auto t0 = std::chrono::steady_clock::now();
    int units = 0;
    int rc = MDIST_OK;
    while (!s.finished && (max_units <= 0 || units < max_units)) {
        if (c->opt.skip_idle_sets) {
            rc = run_skip_level(c, &units);
            if (rc != MDIST_OK) break;
            continue;
        }
        // first wave: every level below the predicted termination level at once
        int g_hi = s.next_g;
        if (c->opt.wstar_hint > 1 && s.next_g == 1 && s.next_j == 0) g_hi = std::min(c->k, c->opt.wstar_hint - 1);
        if (g_hi < s.next_g) g_hi = s.next_g;
        rc = run_wave(c, g_hi, max_units > 0 ? max_units - units : 0, &units);
        if (rc != MDIST_OK) break;
    }
    s.seconds += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (finished) *finished = s.finished;
    return rc;
}

int mdist_enumerate_level_part(mdist_code *c, int g, int j, int part, int nparts, int *U_inout, mdist_key *key_inout,
                               uint64_t *combos_out) {
    if (!c || !U_inout || !key_inout || g < 1 || g > c->k || j < -1 || j >= c->m || nparts < 1 || part < 0 ||
        part >= nparts)
        return MDIST_EINVAL;
    const int j0 = j < 0 ? 0 : j;
    const int j1 = j < 0 ? c->m : j + 1;
    c->level_tc_combos = c->level_tc_cand = 0;
    for (int jj = j0; jj < j1; ++jj) {
        bool found;
        int w;
        uint64_t rank, cnt;
        const int rc = run_unit(c, g, jj, *U_inout, false, &found, &w, &rank, &cnt, part, nparts);
        if (rc != MDIST_OK) return rc;
        if (combos_out) combos_out[jj - j0] = cnt;
        if (found) {
            const mdist_key cand{w, g, jj, 0, rank};
            if (key_less(cand, *key_inout)) *key_inout = cand;
            if (w < *U_inout) *U_inout = w;
        }
    }
    return MDIST_OK;
}

int mdist_run_sharded(mdist_code *c, int part, int nparts, mdist_exchange_fn exchange, void *ctx, int *finished) {
    if (!c || !exchange || nparts < 1 || part < 0 || part >= nparts || c->opt.skip_idle_sets) return MDIST_EINVAL;
    RunState &s = c->st;
    const auto t0 = std::chrono::steady_clock::now();
    int rc = MDIST_OK, units = 0;
    while (!s.finished) {
        const int g = s.next_g, j = s.next_j;
        // every unit after the key's only counts strictly lighter codewords; before a key
        // exists ties with U = n - k + 1 count (the same thresholds on every rank)
        const int thr = s.have_key ? s.key.weight - 1 : s.U;
        bool found;
        int w;
        uint64_t rank, cnt;
        rc = run_unit(c, g, j, thr, false, &found, &w, &rank, &cnt, part, nparts);
        if (rc != MDIST_OK) break;
        uint64_t key = found ? (((uint64_t)w << mdist::kKeyRankBits) | rank) : mdist::kNoKey;
        uint64_t count = cnt;
        if (exchange(&key, &count, ctx) != 0) {  // the ranks did not all deliver: stop here
            rc = MDIST_ECANCELLED;
            break;
        }
        fold_unit(c, g, j, key, count, &units);
    }
    s.seconds += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (finished) *finished = s.finished;
    return rc;
}

int mdist_result(const mdist_code *c, int *d, uint64_t *witness, uint64_t *message, mdist_key *key,
                 mdist_stats *stats) {
    if (!c || !d) return MDIST_EINVAL;
    const RunState &s = c->st;
    if (!s.finished || !s.have_key) return MDIST_EAGAIN;
    *d = s.U;
    const uint64_t comb = unrank_lex_host(c->k, s.key.g, s.key.rank);
    const mdist::InfoSet &set = c->part.sets[(size_t)s.key.j];
    uint64_t msg = 0;
    for (int r = 0; r < c->k; ++r)
        if ((comb >> r) & 1ull) msg ^= set.transform[(size_t)r];
    if (message) *message = msg;
    if (witness) {
        for (int w = 0; w < c->W; ++w) witness[w] = 0;
        for (int b = 0; b < c->k; ++b)
            if ((msg >> b) & 1ull)
                for (int w = 0; w < c->W; ++w) witness[w] ^= c->G[(size_t)b * c->W + w];
    }
    if (key) *key = s.key;
    if (stats) {
        std::memset(stats, 0, sizeof *stats);
        stats->g_final = s.g_last;
        stats->j_final = s.j_last;
        stats->m = c->m;
        stats->L_final = s.L;
        stats->U_final = s.U;
        stats->launches = s.launches;
        for (int j = 0; j < c->m; ++j) stats->ranks[j] = c->part.sets[(size_t)j].bound_rank;
        uint64_t tot = 0;
        for (int g = 0; g <= MDIST_MAX_K; ++g)
            for (int j = 0; j < MDIST_MAX_SETS; ++j) {
                stats->combos[g][j] = s.counts[g][j];
                tot += s.counts[g][j];
            }
        stats->total_combos = tot;
        stats->seconds = s.seconds;
        stats->kernel_ms = s.kernel_ms;
        stats->tc_ms = s.tc_ms;
        stats->tc_launches = s.tc_launches;
        stats->tc_combos = s.tc_combos;
        stats->tc_candidates = s.tc_cand;
        stats->h2d_bytes = s.h2d_bytes + c->rows_bytes;
        stats->d2h_bytes = s.d2h_bytes;
    }
    return MDIST_OK;
}

int mdist_min_distance(mdist_code *c, int *d, uint64_t *witness, uint64_t *message, mdist_key *key,
                       mdist_stats *stats) {
    if (!c || !d) return MDIST_EINVAL;
    int fin = 0;
    const int rc = mdist_run(c, 0, &fin);
    if (rc != MDIST_OK) return rc;
    return mdist_result(c, d, witness, message, key, stats);
}

// ---- checkpoint / resume --------------------------------------------------------

namespace {
struct StateBlob {
    uint64_t magic;
    uint32_t version, n, k, m;
    uint64_t code_hash;
    int32_t per_matrix;
    int32_t overlap_sets;
    RunState st;
};
constexpr uint64_t kMagic = 0x6d64697374737431ull;  // "mdistst1"

uint64_t code_hash(const mdist_code *c) {
    uint64_t h = fnv1a(c->G.data(), c->G.size() * sizeof(uint64_t));
    const int dims[3] = {c->n, c->k, c->W};
    return fnv1a(dims, sizeof dims, h);
}
}  // namespace

int mdist_state_save(const mdist_code *c, void *buf, size_t *len) {
    if (!c || !len) return MDIST_EINVAL;
    if (!buf || *len < sizeof(StateBlob)) {
        *len = sizeof(StateBlob);
        return MDIST_EINVAL;
    }
    StateBlob b;
    std::memset(static_cast<void *>(&b), 0, sizeof b);  // padding too: the blob's bytes are deterministic
    b.magic = kMagic;
    b.version = 2;
    b.n = (uint32_t)c->n;
    b.k = (uint32_t)c->k;
    b.m = (uint32_t)c->m;
    b.code_hash = code_hash(c);
    b.per_matrix = c->opt.check_per_matrix;
    b.overlap_sets = c->opt.overlap_sets;
    b.st = c->st;
    std::memcpy(buf, &b, sizeof b);
    *len = sizeof b;
    return MDIST_OK;
}

int mdist_state_load(mdist_code *c, const void *buf, size_t len) {
    if (!c || !buf) return MDIST_EINVAL;
    if (len != sizeof(StateBlob)) return MDIST_ESTATE;
    StateBlob b;
    std::memcpy(&b, buf, sizeof b);
    if (b.magic != kMagic || b.version != 2 || (int)b.n != c->n || (int)b.k != c->k || (int)b.m != c->m ||
        b.code_hash != code_hash(c) || b.per_matrix != c->opt.check_per_matrix ||
        b.overlap_sets != c->opt.overlap_sets)
        return MDIST_ESTATE;
    if (b.st.next_g < 1 || b.st.next_g > c->k + 1 || b.st.next_j < 0 || b.st.next_j >= c->m) return MDIST_ESTATE;
    c->st = b.st;
    return MDIST_OK;
}

int mdist_device_info(int *sm_count, int *max_sm_clock_khz, int *cc_major, int *cc_minor) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return MDIST_ECUDA; }
    int v = 0;
    if (sm_count) {
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return MDIST_ECUDA;
        *sm_count = v;
    }
    if (max_sm_clock_khz) {
        if (cudaDeviceGetAttribute(&v, cudaDevAttrClockRate, dev) != cudaSuccess) return MDIST_ECUDA;
        *max_sm_clock_khz = v;
    }
    if (cc_major) {
        if (cudaDeviceGetAttribute(&v, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess) return MDIST_ECUDA;
        *cc_major = v;
    }
    if (cc_minor) {
        if (cudaDeviceGetAttribute(&v, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess) return MDIST_ECUDA;
        *cc_minor = v;
    }
    return MDIST_OK;
}

int mdist_debug_gram_plan(int k, int g, int nwords, int tensor_cores, int *nparts, int *parts /* 128 * 15 */,
                          uint64_t *sizes /* 128 * 2 */, int *covered /* 34 */) {
    if (!nparts || !parts || !sizes || !covered || nwords < 1 || nwords > 16 || tensor_cores < 0 ||
        tensor_cores > 3)
        return MDIST_EINVAL;
    mdist::EnumParams p{};
    if (!mdist::plan_level(k, g, nwords, p)) return MDIST_ERANGE;
    mdist::GramSide A[mdist::kMaxGramBlocks], Bs[mdist::kMaxGramBlocks];
    int n = 0;
    for (int b = 0; b < mdist::kMaxBlocks; ++b) covered[b] = 0;
    for (int b = 0; b < p.nblocks && mdist::gram_eligible(nwords); ++b) {
        const int np = gram_block_parts(tensor_cores, p.k1, p.k2, p.blocks[b], mdist::kMaxGramBlocks - n, A, Bs);
        covered[b] = np > 0;
        for (int i = 0; i < np; ++i, ++n) {
            int *o = parts + 15 * n;
            o[0] = b;
            const mdist::GramSide *S[2] = {&A[i], &Bs[i]};
            for (int s = 0; s < 2; ++s) {
                for (int q = 0; q < 2; ++q) {
                    const bool on = q < S[s]->nc;
                    o[1 + 7 * s + 3 * q] = on ? S[s]->off[q] : -1;
                    o[2 + 7 * s + 3 * q] = on ? S[s]->kc[q] : -1;
                    o[3 + 7 * s + 3 * q] = on ? S[s]->t[q] : -1;
                }
                o[7 + 7 * s] = S[s]->nc;
            }
            sizes[2 * n] = A[i].n;
            sizes[2 * n + 1] = Bs[i].n;
        }
    }
    *nparts = n;
    return MDIST_OK;
}

int mdist_debug_side_tables(const uint32_t *rows, int k, int nwords, int n, const int *sides, uint32_t *const *outs,
                            const uint32_t *const *lows, const int *low_t, void *stream) {
    if (!rows || !sides || !outs || n < 1 || n > mdist::kMaxTableJobs || nwords < 1 ||
        nwords > mdist::kGramMaxWords || k < 1 || k > 64 || (uintptr_t)rows % 4 != 0)
        return MDIST_EINVAL;
    std::vector<mdist::GramSide> S((size_t)n);
    auto bad = [&](int off, int kc, int t) { return off < 0 || kc < 1 || kc > 32 || t < 0 || t > kc || off + kc > k; };
    for (int i = 0; i < n; ++i) {
        const int *q = sides + 6 * i;
        if (!outs[i] || (uintptr_t)outs[i] % 16 != 0 || bad(q[0], q[1], q[2]) || (q[5] >= 0 && bad(q[3], q[4], q[5])))
            return MDIST_EINVAL;
        if (q[5] >= 0 && q[0] < q[3] + q[4] && q[3] < q[0] + q[1]) return MDIST_EINVAL;  // shared rows
        if (lows && lows[i] && (!low_t || low_t[i] < 1 || low_t[i] >= q[2] || (uintptr_t)lows[i] % 16 != 0))
            return MDIST_EINVAL;
        S[(size_t)i] = make_side(q[0], q[1], q[2], q[3], q[4], q[5]);
    }
    int dev = 0, sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return MDIST_ECUDA;
    const cudaError_t e =
        mdist::launch_side_tables(rows, k, nwords, S.data(), outs, lows, low_t, n, sm, (cudaStream_t)stream);
    return e == cudaSuccess ? MDIST_OK : MDIST_ECUDA;
}

}  // extern "C"
