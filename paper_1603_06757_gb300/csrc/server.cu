// server.cu -- continuous-batching serving loop (mdist_server_* in include/mdist.h).
//
// Requests (generator matrices) are queued by any host thread.  A serving thread runs
// rounds of the batched engine (batch_launch_round) over a fixed table of device
// slots; between rounds it retires finished codes (their slot and rows memory become
// free) and admits queued requests first-come first-served while a slot is free and
// the rows pool has room for the request's Gamma rows.  Gamma_j rows, the per-code
// Alg. 1 state (U, L, key, counters) and the round's work items all stay on the
// device; a request's work overlaps with whatever else is in flight.  Each result is
// that of mdist_min_distance on the same code.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <set>
#include <thread>
#include <utility>
#include <vector>

#include "batch_kernels.cuh"
#include "chunk_cache.h"
#include "prep.h"

using namespace mdist;

namespace {

constexpr int kServeMaxSets = 8;   // information sets per request
constexpr int kServeMaxSpec = 16;  // levels a request may take in its first round

using Clock = std::chrono::steady_clock;

struct Request {
    long long id = 0;
    int n = 0, k = 0, W = 0, wstar = 0;
    bool large = false;               // routed to the single-code tensor-core path
    std::vector<uint64_t> G;
    Partition part;
    std::vector<DeviceRows> rows;
    size_t rows_words = 0;
    Clock::time_point t_submit, t_start, t_done;
    int slot = -1;
    size_t rows_off = 0;
};

struct Done {
    int status = MDIST_OK;
    int d = 0;
    mdist_key key{};
    uint64_t message = 0;
    std::vector<uint64_t> witness;
    mdist_stats stats{};
    double latency = 0, queue_wait = 0;
};

// first-fit free list over [0, capacity) words
struct Pool {
    std::map<size_t, size_t> free_;  // offset -> length
    explicit Pool(size_t cap = 0) { if (cap) free_[0] = cap; }
    bool alloc(size_t len, size_t *off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= len) {
                *off = it->first;
                const size_t rest = it->second - len, noff = it->first + len;
                free_.erase(it);
                if (rest) free_[noff] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t len) {
        auto it = free_.emplace(off, len).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) { it->second += nx->second; free_.erase(nx); }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) { pv->second += it->second; free_.erase(it); }
        }
    }
};

}  // namespace

struct mdist_server {
    mdist_options opt{};
    int device = 0, sm_count = 0;
    cudaStream_t stream = nullptr;
    int slots = 0;
    size_t pool_words = 0, gs_cap = 0, gs_used = 0;
    int item_cap = 0;
    BatchDev D{};
    std::vector<void *> allocs;
    int grid[kBatchBuckets] = {};
    // host state (guarded by mu)
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> queue;
    std::deque<Request *> large_queue;  // requests for the single-code tensor-core path
    std::map<long long, Done> done;
    std::set<long long> live;        // submitted and not finished
    std::set<long long> cancel_req;  // cancellation asked while in flight
    long long next_id = 1;
    bool stopping = false;
    // serving-thread state
    std::thread th;
    std::vector<Request *> occupant;   // per slot
    std::vector<int> free_slots;
    Pool pool;
    std::map<std::pair<int, int>, unsigned int> gs_off;
    std::vector<BatchCode> h_codes;
    std::atomic<long long> rounds{0}, completed{0}, admitted{0};
    std::atomic<int> error{MDIST_OK};
    double gpu_ms = 0;
    // device memory of the single-code handles, kept for reuse
    ChunkCache chunks;
};

namespace {

void *salloc(mdist_server *s, size_t bytes) {
    void *p = nullptr;
    if (s->opt.dev_alloc) p = s->opt.dev_alloc(bytes ? bytes : 1, s->opt.alloc_ctx);
    else if (cudaMalloc(&p, bytes ? bytes : 1) != cudaSuccess) p = nullptr;
    if (p) s->allocs.push_back(p);
    return p;
}

void sfree_all(mdist_server *s) {
    for (void *p : s->allocs) {
        if (s->opt.dev_free) s->opt.dev_free(p, s->opt.alloc_ctx);
        else cudaFree(p);
    }
    s->allocs.clear();
}

unsigned long long unrank_lex(int k, int g, unsigned long long rank) {
    unsigned long long r = binom_host(k, g) - 1 - rank, mask = 0;
    int d = k - 1;
    for (int t = g; t >= 1; --t) {
        while (binom_host(d, t) > r) --d;
        r -= binom_host(d, t);
        mask |= 1ull << (k - 1 - d);
        --d;
    }
    return mask;
}


// A large request on the single-code path (tensor-core enumerator), on the server's
// stream; the result goes to the done table like a retired slot's.
void run_large(mdist_server *s, Request *rq) {
    rq->t_start = Clock::now();
    Done out;
    mdist_options o{};
    o.check_per_matrix = s->opt.check_per_matrix;
    o.max_sets = s->opt.max_sets > 0 && s->opt.max_sets < kServeMaxSets ? s->opt.max_sets : kServeMaxSets;
    o.wstar_hint = rq->wstar;
    o.timeout_cycles = s->opt.timeout_cycles;
    o.dev_alloc = ChunkCache::alloc;
    o.dev_free = ChunkCache::release;
    o.alloc_ctx = &s->chunks;
    mdist_code *h = nullptr;
    out.status = mdist_prepare(rq->G.data(), rq->n, rq->k, rq->W, &o, s->stream, &h);
    if (out.status == MDIST_OK) {
        out.witness.assign((size_t)rq->W, 0);
        out.status = mdist_min_distance(h, &out.d, out.witness.data(), &out.message, &out.key, &out.stats);
    }
    if (h) mdist_free(h);
    s->gpu_ms += out.stats.kernel_ms;
    rq->t_done = Clock::now();
    out.latency = std::chrono::duration<double>(rq->t_done - rq->t_submit).count();
    out.queue_wait = std::chrono::duration<double>(rq->t_start - rq->t_submit).count();
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->cancel_req.erase(rq->id)) out = Done{MDIST_ECANCELLED};
        s->done[rq->id] = std::move(out);
        s->live.erase(rq->id);
    }
    s->admitted++;
    s->completed++;
    delete rq;
}

// Admit one request into slot `slot` (rows already placed at rq->rows_off).
int admit(mdist_server *s, Request *rq) {
    const int m = (int)rq->part.sets.size();
    std::vector<uint32_t> rows;
    rows.reserve(rq->rows_words);
    std::vector<BatchUnit> units((size_t)m);
    std::vector<unsigned char> gs_new;
    size_t gs_base = s->gs_used;
    for (int j = 0; j < m; ++j) {
        const DeviceRows &dr = rq->rows[(size_t)j];
        BatchUnit &u = units[(size_t)j];
        u.rows_off = (unsigned int)(rq->rows_off + rows.size());
        u.k = rq->k;
        u.k1 = (rq->k + 1) / 2;
        u.k2 = rq->k - u.k1;
        u.nwords = dr.nwords;
        u.n_bits = dr.n_bits;
        u.full_rank = dr.full_rank ? 1 : 0;
        u.rank = rq->part.sets[(size_t)j].rank;
        u.code = rq->slot;
        auto key = std::make_pair(dr.nwords, dr.n_bits);
        auto it = s->gs_off.find(key);
        if (it == s->gs_off.end()) {
            const size_t need = (size_t)dr.n_bits + 2;
            if (gs_base + gs_new.size() + need > s->gs_cap) return MDIST_ENOMEM;
            const unsigned int off = (unsigned int)(gs_base + gs_new.size());
            for (int thr = -1; thr <= dr.n_bits; ++thr)
                gs_new.push_back((unsigned char)choose_filter_group(dr.nwords, dr.n_bits, thr));
            it = s->gs_off.emplace(key, off).first;
        }
        u.gs_off = it->second;
        rows.insert(rows.end(), dr.words.begin(), dr.words.end());
    }
    BatchCode C;
    std::memset(&C, 0, sizeof C);
    C.n = rq->n;
    C.k = rq->k;
    C.m = m;
    C.unit0 = rq->slot * kServeMaxSets;
    C.active = 1;
    C.status = MDIST_OK;
    C.g_next = 1;
    C.spec = rq->wstar > 1 ? std::min(std::min(rq->wstar - 1, rq->k), kServeMaxSpec) : 1;
    C.U = rq->n - rq->k + 1;
    C.L = 1;
    C.j_final = -1;
    C.per_matrix = s->opt.check_per_matrix ? 1 : 0;
    C.counts_off = (unsigned long long)rq->slot * (MDIST_MAX_K + 1) * kServeMaxSets;
    cudaStream_t st = s->stream;
    bool ok = true;
    if (!gs_new.empty()) {
        ok &= cudaMemcpyAsync((unsigned char *)s->D.gs_table + gs_base, gs_new.data(), gs_new.size(),
                              cudaMemcpyHostToDevice, st) == cudaSuccess;
        s->gs_used = gs_base + gs_new.size();
    }
    ok &= cudaMemcpyAsync((uint32_t *)s->D.rows + rq->rows_off, rows.data(), rows.size() * sizeof(uint32_t),
                          cudaMemcpyHostToDevice, st) == cudaSuccess;
    ok &= cudaMemcpyAsync((BatchUnit *)s->D.units + C.unit0, units.data(), units.size() * sizeof(BatchUnit),
                          cudaMemcpyHostToDevice, st) == cudaSuccess;
    ok &= cudaMemsetAsync(s->D.counts + C.counts_off, 0, sizeof(unsigned long long) * (MDIST_MAX_K + 1) * kServeMaxSets,
                          st) == cudaSuccess;
    ok &= cudaMemcpyAsync(s->D.codes + rq->slot, &C, sizeof C, cudaMemcpyHostToDevice, st) == cudaSuccess;
    // the pageable sources above are copied before cudaMemcpyAsync returns
    return ok ? MDIST_OK : MDIST_ECUDA;
}

void retire(mdist_server *s, int slot, const BatchCode &S) {
    Request *rq = s->occupant[(size_t)slot];
    Done out;
    out.status = S.status;
    std::vector<unsigned long long> counts((size_t)(MDIST_MAX_K + 1) * kServeMaxSets);
    cudaMemcpy(counts.data(), s->D.counts + S.counts_off, counts.size() * sizeof(unsigned long long),
               cudaMemcpyDeviceToHost);
    if (S.status == MDIST_OK && S.have_key) {
        out.d = S.U;
        out.key = mdist_key{S.key_w, S.key_g, S.key_j, 0, S.key_rank};
        const unsigned long long comb = unrank_lex(rq->k, S.key_g, S.key_rank);
        const InfoSet &set = rq->part.sets[(size_t)S.key_j];
        uint64_t msg = 0;
        for (int r = 0; r < rq->k; ++r)
            if ((comb >> r) & 1ull) msg ^= set.transform[(size_t)r];
        out.message = msg;
        out.witness.assign((size_t)rq->W, 0);
        for (int b = 0; b < rq->k; ++b)
            if ((msg >> b) & 1ull)
                for (int w = 0; w < rq->W; ++w) out.witness[(size_t)w] ^= rq->G[(size_t)b * rq->W + w];
        mdist_stats &st = out.stats;
        std::memset(&st, 0, sizeof st);
        st.g_final = S.g_final;
        st.j_final = S.j_final;
        st.m = S.m;
        st.L_final = S.L;
        st.U_final = S.U;
        st.launches = S.rounds;
        for (int j = 0; j < S.m; ++j) st.ranks[j] = rq->part.sets[(size_t)j].rank;
        for (int g = 0; g <= rq->k; ++g)
            for (int j = 0; j < S.m; ++j) st.combos[g][j] = counts[(size_t)g * S.m + j];
        st.total_combos = S.combos;
    } else if (out.status == MDIST_OK) {
        out.status = MDIST_EAGAIN;
    }
    rq->t_done = Clock::now();
    out.latency = std::chrono::duration<double>(rq->t_done - rq->t_submit).count();
    out.queue_wait = std::chrono::duration<double>(rq->t_start - rq->t_submit).count();
    s->pool.release(rq->rows_off, rq->rows_words);
    s->occupant[(size_t)slot] = nullptr;
    s->free_slots.push_back(slot);
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->done[rq->id] = std::move(out);
        s->live.erase(rq->id);
    }
    s->completed++;
    delete rq;
}

// Requests cancelled while in a slot leave it between two rounds: the device code is
// made inactive (the next round plans nothing for it), its slot and rows are freed,
// and its result is MDIST_ECANCELLED.
void drop_cancelled(mdist_server *s) {
    std::set<long long> cx;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->cancel_req.empty()) return;
        cx = s->cancel_req;
    }
    for (int slot = 0; slot < s->slots; ++slot) {
        Request *rq = s->occupant[(size_t)slot];
        if (!rq || !cx.count(rq->id)) continue;
        if (cudaMemsetAsync(&s->D.codes[slot].active, 0, sizeof(int), s->stream) != cudaSuccess) {
            s->error = MDIST_ECUDA;
            continue;
        }
        s->pool.release(rq->rows_off, rq->rows_words);
        s->occupant[(size_t)slot] = nullptr;
        s->free_slots.push_back(slot);
        {
            std::lock_guard<std::mutex> lock(s->mu);
            s->cancel_req.erase(rq->id);
            s->done[rq->id] = Done{MDIST_ECANCELLED};
            s->live.erase(rq->id);
        }
        s->completed++;
        delete rq;
    }
    std::lock_guard<std::mutex> lock(s->mu);
    for (long long id : cx)  // finished meanwhile: nothing left to cancel
        if (!s->live.count(id)) s->cancel_req.erase(id);
}

void serve_loop(mdist_server *s) {
    cudaSetDevice(s->device);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (;;) {
        // admit first come, first served while a slot and rows memory are free
        std::vector<Request *> newly;
        Request *large = nullptr;
        {
            std::unique_lock<std::mutex> lock(s->mu);
            if (s->stopping) break;
            bool any_active = false;
            for (Request *r : s->occupant) any_active |= r != nullptr;
            if (!any_active && s->queue.empty() && s->large_queue.empty()) {
                s->cv_work.wait_for(lock, std::chrono::milliseconds(50));
                continue;
            }
            if (!s->large_queue.empty()) {
                large = s->large_queue.front();
                s->large_queue.pop_front();
            }
            while (!s->queue.empty() && !s->free_slots.empty()) {
                Request *rq = s->queue.front();
                size_t off = 0;
                if (!s->pool.alloc(rq->rows_words, &off)) break;
                s->queue.pop_front();
                rq->rows_off = off;
                rq->slot = s->free_slots.back();
                s->free_slots.pop_back();
                newly.push_back(rq);
            }
        }
        for (Request *rq : newly) {
            rq->t_start = Clock::now();
            s->occupant[(size_t)rq->slot] = rq;
            const int rc = admit(s, rq);
            if (rc != MDIST_OK) s->error = rc;
            s->admitted++;
        }
        if (large) {  // one large request between two rounds of the others
            run_large(s, large);
            s->cv_done.notify_all();
        }
        // one round over every occupied slot
        bool present[kBatchBuckets] = {};
        bool any = false;
        for (Request *r : s->occupant)
            if (r) {
                any = true;
                for (const DeviceRows &dr : r->rows) present[dr.nwords - 1] = true;
            }
        if (!any) continue;
        cudaEventRecord(e0, s->stream);
        batch_launch_round(s->D, present, s->grid, s->stream);
        cudaEventRecord(e1, s->stream);
        if (cudaMemcpyAsync(s->h_codes.data(), s->D.codes, sizeof(BatchCode) * (size_t)s->slots,
                            cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
            cudaStreamSynchronize(s->stream) != cudaSuccess) {
            s->error = MDIST_ECUDA;
            std::lock_guard<std::mutex> lock(s->mu);
            s->stopping = true;
            s->cv_done.notify_all();
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        s->gpu_ms += ms;
        s->rounds++;
        for (int slot = 0; slot < s->slots; ++slot)
            if (s->occupant[(size_t)slot] && !s->h_codes[(size_t)slot].active) retire(s, slot, s->h_codes[(size_t)slot]);
        drop_cancelled(s);
        s->cv_done.notify_all();
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
}

}  // namespace

extern "C" {

int mdist_server_create(const mdist_options *opts, int max_slots, size_t rows_pool_bytes, mdist_server **out) {
    if (!out || max_slots < 1 || max_slots > (1 << 16) || rows_pool_bytes < 4096 ||
        (opts && (opts->skip_idle_sets || opts->overlap_sets || opts->route_work_log10 < 0 ||
                  opts->route_work_log10 > 18)))
        return MDIST_EINVAL;
    *out = nullptr;
    mdist_server *s = new (std::nothrow) mdist_server();
    if (!s) return MDIST_ENOMEM;
    if (opts) s->opt = *opts;
    if (cudaGetDevice(&s->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return MDIST_ECUDA;
    }
    s->slots = max_slots;
    s->pool_words = rows_pool_bytes / sizeof(uint32_t);
    s->pool = Pool(s->pool_words);
    s->gs_cap = 1 << 20;
    s->item_cap = max_slots * kServeMaxSets * kServeMaxSpec;
    const size_t cap = (size_t)s->item_cap;
    BatchDev &D = s->D;
    D.rows = (const uint32_t *)salloc(s, s->pool_words * sizeof(uint32_t));
    D.units = (const BatchUnit *)salloc(s, (size_t)max_slots * kServeMaxSets * sizeof(BatchUnit));
    D.gs_table = (const unsigned char *)salloc(s, s->gs_cap);
    D.codes = (BatchCode *)salloc(s, (size_t)max_slots * sizeof(BatchCode));
    D.counts = (unsigned long long *)salloc(s, (size_t)max_slots * (MDIST_MAX_K + 1) * kServeMaxSets * 8);
    D.items = (BatchItem *)salloc(s, cap * sizeof(BatchItem));
    D.slots = (ItemSlot *)salloc(s, cap * sizeof(ItemSlot));
    D.plans = (unsigned long long *)salloc(s, cap * kBatchMaxPlan * sizeof(unsigned long long));
    D.bucket_items = (BucketEntry *)salloc(s, (size_t)kBatchBuckets * cap * sizeof(BucketEntry));
    unsigned long long *packed = (unsigned long long *)salloc(s, 2 * kBatchBuckets * sizeof(unsigned long long));
    D.codeU = (unsigned int *)salloc(s, (size_t)max_slots * sizeof(unsigned int));
    int *ctr = (int *)salloc(s, 2 * sizeof(int));
    if (!D.rows || !D.units || !D.gs_table || !D.codes || !D.counts || !D.items || !D.slots || !D.plans ||
        !D.bucket_items || !packed || !D.codeU || !ctr) {
        sfree_all(s);
        cudaStreamDestroy(s->stream);
        delete s;
        return MDIST_ENOMEM;
    }
    D.bucket_packed = packed;
    D.tile_ctr = packed + kBatchBuckets;
    D.item_ctr = ctr;
    D.active_ctr = ctr + 1;
    D.ncodes = max_slots;
    D.item_cap = s->item_cap;
    bool all[kBatchBuckets];
    for (bool &b : all) b = true;
    if (cudaMemsetAsync(D.codes, 0, (size_t)max_slots * sizeof(BatchCode), s->stream) != cudaSuccess ||
        batch_bucket_grids(all, s->sm_count, s->opt.blocks_per_sm, s->grid) != cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess) {
        sfree_all(s);
        cudaStreamDestroy(s->stream);
        delete s;
        return MDIST_ECUDA;
    }
    s->occupant.assign((size_t)max_slots, nullptr);
    for (int i = max_slots - 1; i >= 0; --i) s->free_slots.push_back(i);
    s->h_codes.resize((size_t)max_slots);
    s->th = std::thread(serve_loop, s);
    *out = s;
    return MDIST_OK;
}

int mdist_server_submit(mdist_server *s, const uint64_t *G, int n, int k, int words_per_row, int wstar_hint,
                        long long *request_id) {
    if (!s || !G || !request_id) return MDIST_EINVAL;
    if (k < 1 || k > MDIST_MAX_K || n <= k || n > MDIST_MAX_N || words_per_row < (n + 63) / 64) return MDIST_EINVAL;
    for (int r = 0; r < k; ++r)
        for (int i = n; i < 64 * words_per_row; ++i)
            if ((G[(size_t)r * words_per_row + (i >> 6)] >> (i & 63)) & 1ull) return MDIST_EINVAL;
    Request *rq = new (std::nothrow) Request();
    if (!rq) return MDIST_ENOMEM;
    rq->t_submit = Clock::now();
    rq->n = n;
    rq->k = k;
    rq->W = words_per_row;
    rq->wstar = wstar_hint;
    rq->G.assign(G, G + (size_t)k * words_per_row);
    const int max_sets = s->opt.max_sets > 0 && s->opt.max_sets < kServeMaxSets ? s->opt.max_sets : kServeMaxSets;
    int rc = partition_info_sets(G, n, k, words_per_row, max_sets, rq->part);
    if (rc != MDIST_OK) { delete rq; return rc; }
    rq->rows.resize(rq->part.sets.size());
    for (size_t j = 0; j < rq->part.sets.size(); ++j) {
        build_rows(rq->part, (int)j, rq->rows[j]);
        rq->rows_words += rq->rows[j].words.size();
    }
    if (rq->rows_words > s->pool_words) { delete rq; return MDIST_ENOMEM; }
    const int tc = s->opt.tensor_cores;
    rq->large = tc == 2 || (tc == 0 && estimated_work(rq->n, rq->k, rq->part, rq->wstar) >=
                                           tensor_path_work(s->opt.route_work_log10));
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->stopping) { delete rq; return MDIST_ECANCELLED; }
    rq->id = s->next_id++;
    *request_id = rq->id;
    s->live.insert(rq->id);
    if (rq->large) s->large_queue.push_back(rq);
    else s->queue.push_back(rq);
    s->cv_work.notify_one();
    return MDIST_OK;
}

int mdist_server_poll(mdist_server *s, long long request_id, int wait_ms, int *d, uint64_t *witness,
                      uint64_t *message, mdist_key *key, mdist_stats *stats, double *latency_s) {
    if (!s || !d) return MDIST_EINVAL;
    std::unique_lock<std::mutex> lock(s->mu);
    auto deadline = Clock::now() + std::chrono::milliseconds(wait_ms > 0 ? wait_ms : 0);
    for (;;) {
        auto it = s->done.find(request_id);
        if (it != s->done.end()) {
            const Done &r = it->second;
            if (r.status != MDIST_OK) {
                const int st = r.status;
                s->done.erase(it);
                return st;
            }
            *d = r.d;
            if (witness) std::copy(r.witness.begin(), r.witness.end(), witness);
            if (message) *message = r.message;
            if (key) *key = r.key;
            if (stats) *stats = r.stats;
            if (latency_s) *latency_s = r.latency;
            s->done.erase(it);
            return MDIST_OK;
        }
        if (s->error != MDIST_OK) return s->error;
        if (wait_ms <= 0 || Clock::now() >= deadline) return MDIST_EAGAIN;
        s->cv_done.wait_until(lock, deadline);
    }
}

int mdist_server_cancel(mdist_server *s, long long request_id) {
    if (!s) return MDIST_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    for (std::deque<Request *> *q : {&s->queue, &s->large_queue})
        for (auto it = q->begin(); it != q->end(); ++it)
            if ((*it)->id == request_id) {
                delete *it;
                q->erase(it);
                s->done[request_id] = Done{MDIST_ECANCELLED};
                s->live.erase(request_id);
                s->cv_done.notify_all();
                return MDIST_OK;
            }
    if (s->live.count(request_id)) {
        s->cancel_req.insert(request_id);
        s->cv_work.notify_one();
        return MDIST_OK;
    }
    return s->done.count(request_id) ? MDIST_EAGAIN : MDIST_EINVAL;
}

int mdist_server_info(mdist_server *s, long long *admitted, long long *completed, long long *rounds, int *queued,
                      int *in_flight, double *gpu_ms) {
    if (!s) return MDIST_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    if (admitted) *admitted = s->admitted;
    if (completed) *completed = s->completed;
    if (rounds) *rounds = s->rounds;
    if (queued) *queued = (int)(s->queue.size() + s->large_queue.size());
    if (in_flight) *in_flight = (int)(s->admitted - s->completed);
    if (gpu_ms) *gpu_ms = s->gpu_ms;
    return s->error;
}

void mdist_server_free(mdist_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stopping = true;
        for (Request *rq : s->queue) delete rq;
        for (Request *rq : s->large_queue) delete rq;
        s->queue.clear();
        s->large_queue.clear();
        s->cv_work.notify_all();
    }
    if (s->th.joinable()) s->th.join();
    for (Request *rq : s->occupant) delete rq;
    cudaStreamSynchronize(s->stream);
    sfree_all(s);
    s->chunks.clear();
    cudaStreamDestroy(s->stream);
    delete s;
}

}  // extern "C"
