// batch.cu -- the batched engine: kernels (layout in batch_kernels.cuh) and the C-ABI
// mdist_batch_* (include/mdist.h).  The rounds of a run are captured once into a CUDA
// graph and launched as one graph; the graph is relaunched only while some code is
// still active after all of its rounds.
#include <algorithm>
#include <chrono>
#include <climits>
#include <cstring>
#include <map>
#include <new>
#include <utility>
#include <vector>

#include "batch_kernels.cuh"
#include "chunk_cache.h"
#include "prep.h"

namespace mdist {

static __constant__ BinomTable64 c_binom_b = make_binom_table64();

__device__ __forceinline__ unsigned long long binom_dev(int a, int b) {
    return (a < 0 || b < 0 || b > a) ? 0ull : c_binom_b.v[a][b];
}

struct DevBinomB {
    __device__ __forceinline__ unsigned long long operator()(int a, int b) const { return c_binom_b.v[a][b]; }
};

__device__ __forceinline__ int set_bound_dev(int h, int k, int r) {
    const int v = h + 1 - (k - r);
    return v > 0 ? v : 0;
}

// Tiles of unit (k, g) with row width nwords, block by block (the plan of plan_level):
// plan[b] = first tile of block b.  Returns the total.
__device__ unsigned long long plan_unit_dev(int k, int g, int nwords, unsigned long long *plan, int *nblocks) {
    const int k1 = (k + 1) / 2, k2 = k - k1;
    const unsigned long long lane_chunk = 32ull * (unsigned long long)lane_entries_per_thread(nwords);
    const unsigned long long walk_chunk = (unsigned long long)walk_len_for(nwords);
    const int ilo = g - k2 > 0 ? g - k2 : 0;
    const int ihi = g < k1 ? g : k1;
    unsigned long long tiles = 0;
    int nb = 0;
    for (int i = ilo; i <= ihi; ++i) {
        const unsigned long long n1 = binom_dev(k1, i), n2 = binom_dev(k2, g - i);
        const unsigned long long ln = n1 >= n2 ? n1 : n2, wn = n1 >= n2 ? n2 : n1;
        plan[nb++] = tiles;
        tiles += ((ln + lane_chunk - 1) / lane_chunk) * ((wn + walk_chunk - 1) / walk_chunk);
    }
    *nblocks = nb;
    return tiles;
}

__global__ void batch_round_begin(BatchDev D) {
    const int t = threadIdx.x;
    if (t < kBatchBuckets) {
        D.bucket_packed[t] = 0;
        D.tile_ctr[t] = 0;
    }
    if (t == 0) {
        *D.item_ctr = 0;
        *D.active_ctr = 0;
    }
}

// One thread per code: this round's levels and one item per unit.
__global__ void batch_prep(BatchDev D) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= D.ncodes) return;
    BatchCode &C = D.codes[c];
    C.nitems = 0;
    if (!C.active) return;
    const int g0 = C.g_next;
    int g1 = g0 + (C.spec > 0 ? C.spec : 1);
    if (g1 > C.k + 1) g1 = C.k + 1;
    int gl = g0;  // levels past the device key range are not started
    while (gl < g1 && binom_dev(C.k, gl) < (1ull << kKeyRankBits)) ++gl;
    if (gl == g0) {
        C.status = MDIST_ERANGE;
        C.active = 0;
        return;
    }
    g1 = gl;
    const int n_items = (g1 - g0) * C.m;
    const int item0 = atomicAdd(D.item_ctr, n_items);
    if (item0 + n_items > D.item_cap) {  // the host sizes item_cap for every round
        C.status = MDIST_ENOMEM;
        C.active = 0;
        return;
    }
    C.item0 = item0;
    C.nitems = n_items;
    // units of this round all follow the key's unit: only lighter codewords can replace it
    D.codeU[c] = (unsigned int)(C.have_key ? C.key_w - 1 : C.U);
    int it = item0;
    for (int g = g0; g < g1; ++g) {
        for (int j = 0; j < C.m; ++j, ++it) {
            const BatchUnit &u = D.units[C.unit0 + j];
            BatchItem &I = D.items[it];
            I.unit = C.unit0 + j;
            I.code = c;
            I.g = g;
            I.tiles = plan_unit_dev(C.k, g, u.nwords, D.plans + (size_t)it * kBatchMaxPlan, &I.nblocks);
            D.slots[it].key = kNoKey;
            D.slots[it].count = 0;
            const int b = u.nwords - 1;
            const unsigned long long old =
                atomicAdd(&D.bucket_packed[b], (1ull << kTileBits) | I.tiles);
            BucketEntry &E = D.bucket_items[(size_t)b * D.item_cap + (size_t)(old >> kTileBits)];
            E.tile_begin = old & ((1ull << kTileBits) - 1);
            E.item = it;
            E.pad = 0;
        }
    }
}

// One thread per code: fold this round's units in (g, j) order, as mdist_run does.
__global__ void batch_update(BatchDev D) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= D.ncodes) return;
    BatchCode &C = D.codes[c];
    if (!C.active || C.nitems == 0) return;
    C.rounds += 1;
    const int g0 = D.items[C.item0].g;
    const int nlev = C.nitems / C.m;
    int fin = 0;
    for (int l = 0; l < nlev && !fin; ++l) {
        const int g = g0 + l;
        for (int j = 0; j < C.m && !fin; ++j) {
            const ItemSlot s = D.slots[C.item0 + l * C.m + j];
            D.counts[C.counts_off + (unsigned long long)g * C.m + j] = s.count;
            C.combos += s.count;
            C.g_final = g;
            C.j_final = j;
            if (s.key != kNoKey) {
                const int w = (int)(s.key >> kKeyRankBits);
                if (!C.have_key || w < C.key_w) {
                    C.have_key = 1;
                    C.key_w = w;
                    C.key_g = g;
                    C.key_j = j;
                    C.key_rank = s.key & ((1ull << kKeyRankBits) - 1);
                }
                if (w < C.U) C.U = w;
            }
            if (C.per_matrix) {
                int Lm = 0;
                for (int i = 0; i < C.m; ++i) Lm += set_bound_dev(i <= j ? g : g - 1, C.k, D.units[C.unit0 + i].rank);
                if (Lm > C.L) C.L = Lm;
                if (C.L >= C.U) fin = 1;
            }
        }
        if (fin) break;
        if (!C.per_matrix) {  // Alg. 1, line 7, for sets of any rank
            int Lg = 0;
            for (int i = 0; i < C.m; ++i) Lg += set_bound_dev(g, C.k, D.units[C.unit0 + i].rank);
            C.L = Lg;
            if (C.L >= C.U) fin = 1;
        }
        if (g >= C.k) fin = 1;
    }
    if (fin) {
        C.active = 0;
    } else {
        C.g_next = g0 + nlev;
        C.spec = 1;
        atomicAdd(D.active_ctr, 1);
    }
}

// Persistent enumerator of one bucket (row width NW) for one round.
template <int NW>
__global__ void __launch_bounds__(kCtaThreads, MDIST_ENUM_MIN_BLOCKS) batch_enum(const __grid_constant__ BatchDev D, int bucket) {
    constexpr int XP = lane_entries_per_thread(NW);
    constexpr int YL = walk_len_for(NW);
    constexpr int PER = YL / 32;
    constexpr int SW = walk_stride(NW);
    extern __shared__ __align__(16) uint32_t smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *wbuf = smem + warp * YL * SW;                                // this warp's walk buffer
    uint32_t *wrows = smem + kWarpsPerCta * YL * SW + warp * kMaxK * NW;    // and rows
    uint32_t *s_bn = smem + kWarpsPerCta * (YL * SW + kMaxK * NW);          // 33 x 33
    for (int i = threadIdx.x; i < kBn * kBn; i += blockDim.x) s_bn[i] = (uint32_t)c_binom_b.v[i / kBn][i % kBn];
    __syncthreads();
    const unsigned long long packed = D.bucket_packed[bucket];
    const unsigned long long total = packed & ((1ull << kTileBits) - 1);
    const int nentries = (int)(packed >> kTileBits);
    const BucketEntry *entries = D.bucket_items + (size_t)bucket * D.item_cap;
    int staged = -1;
    for (;;) {
        unsigned long long tile = 0;
        if (lane == 0) tile = atomicAdd(&D.tile_ctr[bucket], 1ull);
        tile = __shfl_sync(0xffffffffu, tile, 0);
        if (tile >= total) break;
        int lo = 0, hi = nentries - 1;  // last entry whose first tile is <= tile
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (entries[mid].tile_begin <= tile) lo = mid;
            else hi = mid - 1;
        }
        const BucketEntry E = entries[lo];
        const int it = E.item;
        const BatchItem I = D.items[it];
        const BatchUnit u = D.units[I.unit];
        if (I.unit != staged) {
            __syncwarp();
            for (int w = lane; w < u.k * NW; w += 32) wrows[w] = D.rows[u.rows_off + w];
            __syncwarp();
            staged = I.unit;
        }
        // product block of this tile within the unit
        const unsigned long long tl = tile - E.tile_begin;
        const unsigned long long *plan = D.plans + (size_t)it * kBatchMaxPlan;
        int b = 0;
        while (b + 1 < I.nblocks && plan[b + 1] <= tl) ++b;
        const int k1 = u.k1, k2 = u.k2, g = I.g;
        const int i = (g - k2 > 0 ? g - k2 : 0) + b;
        const unsigned long long n1 = binom_dev(k1, i), n2 = binom_dev(k2, g - i);
        const int lane_half = n1 >= n2 ? 0 : 1;
        const int lane_t = lane_half ? g - i : i, walk_t = lane_half ? i : g - i;
        const unsigned long long lane_n = lane_half ? n2 : n1, walk_n = lane_half ? n1 : n2;
        const unsigned long long walk_chunks = (walk_n + YL - 1) / YL;
        const unsigned long long t = tl - plan[b];
        const unsigned long long lane_chunk = t / walk_chunks;
        const unsigned long long walk_chunk = t - lane_chunk * walk_chunks;
        const int lane_kh = lane_half ? k2 : k1, walk_kh = lane_half ? k1 : k2;
        const uint32_t *lane_rows = wrows + (lane_half ? k1 : 0) * NW;
        const uint32_t *walk_rows = wrows + (lane_half ? 0 : k1) * NW;
        const int base = u.full_rank ? g : 0;
        int thr = (int)(*(volatile unsigned int *)&D.codeU[I.code]) - base;
        const int tc = thr < -1 ? -1 : (thr > u.n_bits ? u.n_bits : thr);
        const int gs = D.gs_table[u.gs_off + tc + 1];

        const unsigned long long chunk_first = lane_chunk * (unsigned long long)(32 * XP);
        const unsigned long long e_first = chunk_first + (unsigned long long)lane * XP;
        const long long left = (long long)lane_n - (long long)e_first;
        const int nvalid = left <= 0 ? 0 : (left >= XP ? XP : (int)left);
        const uint32_t e0 = (uint32_t)(e_first < lane_n ? e_first : lane_n - 1);
        uint32_t x[XP][NW];
        build_lane_entries<NW, XP>(x, s_bn, lane_rows, lane_kh, lane_t, e0, nvalid);
        const unsigned long long w_first = walk_chunk * (unsigned long long)YL;
        const unsigned long long wleft = walk_n - w_first;
        const int walk_len = wleft >= (unsigned long long)YL ? YL : (int)wleft;
        stage_walk<NW>(wbuf, s_bn, walk_rows, walk_kh, walk_t, w_first, walk_len, PER, lane);
        __syncwarp();

        auto cand = [&](int p, int s, int acc) {
            const uint32_t lm = unrank_colex(s_bn, lane_kh, lane_t, e0 + (uint32_t)p);
            const uint32_t wm = unrank_colex(s_bn, walk_kh, walk_t, (uint32_t)(w_first + s));
            const unsigned long long h1 = lane_half ? wm : lm, h2 = lane_half ? lm : wm;
            const unsigned long long rank = lexrank64(h1 | (h2 << k1), u.k, g, DevBinomB{});
            const int wt = acc + base;
            atomicMin(&D.slots[it].key, ((unsigned long long)wt << kKeyRankBits) | rank);
            atomicMin(&D.codeU[I.code], (unsigned int)wt);
            thr = acc;
        };
        switch (gs) {
            case 2: walk_tile<NW, XP, 2, false>(x, wbuf, walk_len, nvalid, thr, nullptr, base, cand); break;
            case 3: walk_tile<NW, XP, 3, false>(x, wbuf, walk_len, nvalid, thr, nullptr, base, cand); break;
            case 4: walk_tile<NW, XP, 4, false>(x, wbuf, walk_len, nvalid, thr, nullptr, base, cand); break;
            case 5: walk_tile<NW, XP, 5, false>(x, wbuf, walk_len, nvalid, thr, nullptr, base, cand); break;
            default: walk_tile<NW, XP, 0, false>(x, wbuf, walk_len, nvalid, thr, nullptr, base, cand); break;
        }
        if (lane == 0) {
            const unsigned long long in_chunk = lane_n - chunk_first;
            const unsigned long long valid = in_chunk < (unsigned long long)(32 * XP) ? in_chunk : 32 * XP;
            atomicAdd(&D.slots[it].count, valid * (unsigned long long)walk_len);
        }
        __syncwarp();
    }
}

template <int NW>
size_t batch_smem_bytes() {
    return sizeof(uint32_t) *
           ((size_t)kBn * kBn + (size_t)kWarpsPerCta * (kMaxK * NW + walk_len_for(NW) * walk_stride(NW)));
}

template <int NW>
cudaError_t batch_enum_prepare(int *grid_per_sm) {
    const size_t smem = batch_smem_bytes<NW>();
    cudaError_t e = allow_dynamic_smem((const void *)batch_enum<NW>, smem);
    if (e != cudaSuccess) return e;
    return blocks_per_sm((const void *)batch_enum<NW>, kCtaThreads, smem, grid_per_sm);
}

template <int NW>
void batch_enum_launch(const BatchDev &D, int bucket, int grid, cudaStream_t st) {
    batch_enum<NW><<<grid, kCtaThreads, batch_smem_bytes<NW>(), st>>>(D, bucket);
}

#define MDIST_NW_CASES(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16)

static cudaError_t batch_prepare_nw(int nw, int *occ) {
    switch (nw) {
#define C(N) case N: return batch_enum_prepare<N>(occ);
        MDIST_NW_CASES(C)
#undef C
        default: return cudaErrorInvalidValue;
    }
}

static void batch_launch_nw(int nw, const BatchDev &D, int grid, cudaStream_t st) {
    switch (nw) {
#define C(N) case N: batch_enum_launch<N>(D, N - 1, grid, st); break;
        MDIST_NW_CASES(C)
#undef C
        default: break;
    }
}

// Host helpers shared with the serving loop (server.cu).
cudaError_t batch_bucket_grids(const bool present[kBatchBuckets], int sm_count, int blocks_per_sm,
                               int grid[kBatchBuckets]) {
    for (int nb = 0; nb < kBatchBuckets; ++nb) {
        grid[nb] = 0;
        if (!present[nb]) continue;
        int occ = 0;
        const cudaError_t e = batch_prepare_nw(nb + 1, &occ);
        if (e != cudaSuccess) return e;
        if (occ < 1) return cudaErrorInvalidConfiguration;
        const int per_sm = blocks_per_sm > 0 && blocks_per_sm < occ ? blocks_per_sm : occ;
        grid[nb] = sm_count * per_sm;
    }
    return cudaSuccess;
}

// One thread, after a round's fold: the run's graph loops (a conditional WHILE node
// around one round) while codes remain active, for at most max_rounds rounds; the
// device-side round counter bounds the loop whatever the codes do.
__global__ void batch_continue(const int *active_ctr, int *rounds_done, int max_rounds, cudaGraphConditionalHandle h) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const int r = ++*rounds_done;
        cudaGraphSetConditional(h, (*active_ctr > 0 && r < max_rounds) ? 1u : 0u);
    }
}

void batch_launch_round(const BatchDev &D, const bool present[kBatchBuckets], const int grid[kBatchBuckets],
                        cudaStream_t st) {
    const int tb = 128, cb = (D.ncodes + tb - 1) / tb;
    batch_round_begin<<<1, 32, 0, st>>>(D);
    batch_prep<<<cb, tb, 0, st>>>(D);
    for (int nb = 0; nb < kBatchBuckets; ++nb)
        if (present[nb]) batch_launch_nw(nb + 1, D, grid[nb], st);
    batch_update<<<cb, tb, 0, st>>>(D);
}

}  // namespace mdist

// ----------------------------------------------------------------------------------
// host side
// ----------------------------------------------------------------------------------

using namespace mdist;

namespace {

struct HostCode {
    int n = 0, k = 0, W = 0, wstar = 0;
    bool large = false;          // run on the single-code path (tensor-core enumerator)
    int slot = -1;               // index among the batched codes, or among the large ones
    std::vector<uint64_t> G;
    Partition part;
    std::vector<DeviceRows> rows;
};

// Result of a code run on the single-code path.
struct LargeResult {
    int status = MDIST_EAGAIN;
    int d = 0;
    uint64_t message = 0;
    mdist_key key{};
    std::vector<uint64_t> witness;
    mdist_stats stats{};
};

unsigned long long host_unrank_lex(int k, int g, unsigned long long rank) {
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

}  // namespace

struct mdist_batch {
    mdist_options opt{};
    cudaStream_t stream = nullptr;
    int device = 0, sm_count = 0;
    std::vector<HostCode> codes;
    std::vector<void *> allocs;
    std::vector<BatchCode> res;              // per batched code, after the run
    std::vector<unsigned long long> counts;  // all batched codes
    std::vector<unsigned long long> counts_off;
    std::vector<LargeResult> large_res;      // per large code
    int n_large = 0;
    double large_ms = 0;                     // summed kernel time of the large codes' runs
    bool ran = false;
    int rounds_per_graph = 0, graph_launches = 0, rounds = 0;
    double seconds = 0, gpu_ms = 0;
    int grid_override = 0;
};

namespace {

void *balloc(mdist_batch *b, size_t bytes) {
    void *p = nullptr;
    if (b->opt.dev_alloc) p = b->opt.dev_alloc(bytes ? bytes : 1, b->opt.alloc_ctx);
    else if (cudaMalloc(&p, bytes ? bytes : 1) != cudaSuccess) p = nullptr;
    if (p) b->allocs.push_back(p);
    return p;
}

void bfree_all(mdist_batch *b) {
    for (void *p : b->allocs) {
        if (b->opt.dev_free) b->opt.dev_free(p, b->opt.alloc_ctx);
        else cudaFree(p);
    }
    b->allocs.clear();
}

int batch_run_graph(mdist_batch *b, const std::vector<int> &light, int rounds_per_graph);
int batch_run_large(mdist_batch *b);

// The loop graph of a run: a conditional WHILE node (launch value 1) whose body is one
// round followed by batch_continue.  False if the toolkit or driver cannot build it.
bool build_loop_graph(const BatchDev &D, const bool present[kBatchBuckets], const int grid[kBatchBuckets],
                      cudaStream_t st, int *d_rounds, int max_rounds, cudaGraph_t *out) {
    *out = nullptr;
    cudaGraph_t g = nullptr;
    if (cudaGraphCreate(&g, 0) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaGraphConditionalHandle h;
    cudaGraphNodeParams np{};
    cudaGraphNode_t node;
    bool ok = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) == cudaSuccess;
    if (ok) {
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        ok = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np) == cudaSuccess;
    }
    if (ok) ok = cudaStreamBeginCaptureToGraph(st, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                               cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        batch_launch_round(D, present, grid, st);
        batch_continue<<<1, 32, 0, st>>>(D.active_ctr, d_rounds, max_rounds, h);
        cudaGraph_t body = nullptr;
        ok = cudaStreamEndCapture(st, &body) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        cudaGraphDestroy(g);
        return false;
    }
    *out = g;
    return true;
}

}  // namespace

extern "C" {

int mdist_batch_create(const mdist_options *opts, void *cuda_stream, mdist_batch **out) {
    if (!out || (opts && (opts->skip_idle_sets || opts->overlap_sets || opts->tensor_cores < 0 ||
                          opts->tensor_cores > 3 || opts->route_work_log10 < 0 || opts->route_work_log10 > 18)))
        return MDIST_EINVAL;
    *out = nullptr;
    mdist_batch *b = new (std::nothrow) mdist_batch();
    if (!b) return MDIST_ENOMEM;
    if (opts) b->opt = *opts;
    if (b->opt.max_sets <= 0 || b->opt.max_sets > MDIST_MAX_SETS) b->opt.max_sets = MDIST_MAX_SETS;
    b->stream = (cudaStream_t)cuda_stream;
    if (cudaGetDevice(&b->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return MDIST_ECUDA;
    }
    *out = b;
    return MDIST_OK;
}

int mdist_batch_add(mdist_batch *b, const uint64_t *G, int n, int k, int words_per_row, int wstar_hint, int *index) {
    if (!b || !G || b->ran) return MDIST_EINVAL;
    if (k < 1 || k > MDIST_MAX_K || n <= k || n > MDIST_MAX_N || words_per_row < (n + 63) / 64) return MDIST_EINVAL;
    for (int r = 0; r < k; ++r)
        for (int i = n; i < 64 * words_per_row; ++i)
            if ((G[(size_t)r * words_per_row + (i >> 6)] >> (i & 63)) & 1ull) return MDIST_EINVAL;
    HostCode hc;
    hc.n = n;
    hc.k = k;
    hc.W = words_per_row;
    hc.wstar = wstar_hint < 0 ? 0 : wstar_hint;
    hc.G.assign(G, G + (size_t)k * words_per_row);
    const int rc = partition_info_sets(G, n, k, words_per_row, b->opt.max_sets, hc.part);
    if (rc != MDIST_OK) return rc;
    hc.rows.resize(hc.part.sets.size());
    for (size_t j = 0; j < hc.part.sets.size(); ++j) build_rows(hc.part, (int)j, hc.rows[j]);
    const int tc = b->opt.tensor_cores;
    hc.large = tc == 2 ||
               (tc == 0 && estimated_work(n, k, hc.part, hc.wstar) >= tensor_path_work(b->opt.route_work_log10));
    if (index) *index = (int)b->codes.size();
    b->codes.push_back(std::move(hc));
    return MDIST_OK;
}

int mdist_batch_run(mdist_batch *b, int rounds_per_graph) {
    if (!b || b->ran) return MDIST_EINVAL;
    const auto t0 = std::chrono::steady_clock::now();
    b->ran = true;
    std::vector<int> light;  // the codes of the graph; the others run on the single-code path
    for (int c = 0; c < (int)b->codes.size(); ++c) {
        HostCode &h = b->codes[(size_t)c];
        if (h.large) {
            h.slot = b->n_large++;
        } else {
            h.slot = (int)light.size();
            light.push_back(c);
        }
    }
    b->large_res.assign((size_t)b->n_large, LargeResult{});
    int rc = batch_run_graph(b, light, rounds_per_graph);
    if (rc == MDIST_OK) rc = batch_run_large(b);
    b->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return rc;
}

}  // extern "C"

namespace {

// The large codes one after the other through the single-code path (mdist_prepare +
// mdist_min_distance, tensor-core enumerator on), on the batch's stream, their device
// memory from the caller's allocator or else from chunks kept for reuse.
int batch_run_large(mdist_batch *b) {
    if (b->n_large == 0) return MDIST_OK;
    ChunkCache cache;
    mdist_options o{};
    o.check_per_matrix = b->opt.check_per_matrix;
    o.max_sets = b->opt.max_sets;
    o.blocks_per_sm = b->opt.blocks_per_sm;
    o.timeout_cycles = b->opt.timeout_cycles;
    if (b->opt.dev_alloc) {
        o.dev_alloc = b->opt.dev_alloc;
        o.dev_free = b->opt.dev_free;
        o.alloc_ctx = b->opt.alloc_ctx;
    } else {
        o.dev_alloc = ChunkCache::alloc;
        o.dev_free = ChunkCache::release;
        o.alloc_ctx = &cache;
    }
    int rc = MDIST_OK;
    for (const HostCode &h : b->codes) {
        if (!h.large) continue;
        LargeResult &r = b->large_res[(size_t)h.slot];
        o.wstar_hint = h.wstar;
        mdist_code *code = nullptr;
        r.status = mdist_prepare(h.G.data(), h.n, h.k, h.W, &o, b->stream, &code);
        if (r.status == MDIST_OK) {
            r.witness.assign((size_t)h.W, 0);
            r.status = mdist_min_distance(code, &r.d, r.witness.data(), &r.message, &r.key, &r.stats);
            b->large_ms += r.stats.kernel_ms;
        }
        if (code) mdist_free(code);
        if (r.status == MDIST_ECUDA) {  // the device is in trouble: stop here
            rc = MDIST_ECUDA;
            break;
        }
    }
    cache.clear();
    return rc;
}

// The batched codes `light` through the rounds of one captured graph.
int batch_run_graph(mdist_batch *b, const std::vector<int> &light, int rounds_per_graph) {
    const int C = (int)light.size();
    if (C == 0) return MDIST_OK;
    // ---- host tables ----
    std::vector<BatchUnit> units;
    std::vector<uint32_t> rows;
    std::vector<unsigned char> gs_table;
    std::map<std::pair<int, int>, unsigned int> gs_off;
    std::vector<BatchCode> codes((size_t)C);
    b->counts_off.assign((size_t)C, 0);
    unsigned long long ncounts = 0;
    long long item_cap = 0;
    bool present[kBatchBuckets] = {};
    int max_spec = 1;
    for (int c = 0; c < C; ++c) {
        const HostCode &h = b->codes[(size_t)light[(size_t)c]];
        BatchCode &S = codes[(size_t)c];
        std::memset(&S, 0, sizeof S);
        S.n = h.n;
        S.k = h.k;
        S.m = (int)h.part.sets.size();
        S.unit0 = (int)units.size();
        S.active = 1;
        S.status = MDIST_OK;
        S.g_next = 1;
        // predicted termination level: take the levels below it in the first round
        S.spec = h.wstar > 1 ? std::min(h.wstar - 1, h.k) : 1;
        max_spec = std::max(max_spec, S.spec);
        S.U = h.n - h.k + 1;  // Alg. 1, line 1
        S.L = 1;
        S.j_final = -1;
        S.per_matrix = b->opt.check_per_matrix ? 1 : 0;
        S.counts_off = ncounts;
        b->counts_off[(size_t)c] = ncounts;
        ncounts += (unsigned long long)(h.k + 1) * S.m;
        item_cap += (long long)S.m * S.spec;
        for (int j = 0; j < S.m; ++j) {
            const DeviceRows &dr = h.rows[(size_t)j];
            BatchUnit u{};
            u.rows_off = (unsigned int)rows.size();
            u.k = h.k;
            u.k1 = (h.k + 1) / 2;
            u.k2 = h.k - u.k1;
            u.nwords = dr.nwords;
            u.n_bits = dr.n_bits;
            u.full_rank = dr.full_rank ? 1 : 0;
            u.rank = h.part.sets[(size_t)j].rank;
            u.code = c;
            auto key = std::make_pair(dr.nwords, dr.n_bits);
            auto it = gs_off.find(key);
            if (it == gs_off.end()) {
                const unsigned int off = (unsigned int)gs_table.size();
                for (int thr = -1; thr <= dr.n_bits; ++thr)
                    gs_table.push_back((unsigned char)choose_filter_group(dr.nwords, dr.n_bits, thr));
                it = gs_off.emplace(key, off).first;
            }
            u.gs_off = it->second;
            rows.insert(rows.end(), dr.words.begin(), dr.words.end());
            units.push_back(u);
            present[dr.nwords - 1] = true;
        }
    }
    // ---- device buffers ----
    BatchDev D{};
    const size_t cap = (size_t)item_cap;
    uint32_t *d_rows = (uint32_t *)balloc(b, rows.size() * sizeof(uint32_t));
    BatchUnit *d_units = (BatchUnit *)balloc(b, units.size() * sizeof(BatchUnit));
    unsigned char *d_gs = (unsigned char *)balloc(b, gs_table.size());
    BatchCode *d_codes = (BatchCode *)balloc(b, codes.size() * sizeof(BatchCode));
    unsigned long long *d_counts = (unsigned long long *)balloc(b, ncounts * sizeof(unsigned long long));
    BatchItem *d_items = (BatchItem *)balloc(b, cap * sizeof(BatchItem));
    ItemSlot *d_slots = (ItemSlot *)balloc(b, cap * sizeof(ItemSlot));
    unsigned long long *d_plans = (unsigned long long *)balloc(b, cap * kBatchMaxPlan * sizeof(unsigned long long));
    BucketEntry *d_bucket = (BucketEntry *)balloc(b, (size_t)kBatchBuckets * cap * sizeof(BucketEntry));
    unsigned long long *d_packed = (unsigned long long *)balloc(b, 2 * kBatchBuckets * sizeof(unsigned long long));
    unsigned int *d_codeU = (unsigned int *)balloc(b, (size_t)C * sizeof(unsigned int));
    int *d_ctr = (int *)balloc(b, 4 * sizeof(int));  // items, active codes, rounds run
    if (!d_rows || !d_units || !d_gs || !d_codes || !d_counts || !d_items || !d_slots || !d_plans || !d_bucket ||
        !d_packed || !d_codeU || !d_ctr) {
        bfree_all(b);
        return MDIST_ENOMEM;
    }
    // graph capture is not allowed on the legacy default stream: use a private stream
    // then, after the caller's earlier work on it has finished
    cudaStream_t st = b->stream;
    cudaStream_t own = nullptr;
    if (!st) {
        if (cudaStreamSynchronize(nullptr) != cudaSuccess ||
            cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking) != cudaSuccess) {
            bfree_all(b);
            return MDIST_ECUDA;
        }
        st = own;
    }
    bool ok = cudaMemcpyAsync(d_rows, rows.data(), rows.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, st) ==
                  cudaSuccess &&
              cudaMemcpyAsync(d_units, units.data(), units.size() * sizeof(BatchUnit), cudaMemcpyHostToDevice, st) ==
                  cudaSuccess &&
              cudaMemcpyAsync(d_gs, gs_table.data(), gs_table.size(), cudaMemcpyHostToDevice, st) == cudaSuccess &&
              cudaMemcpyAsync(d_codes, codes.data(), codes.size() * sizeof(BatchCode), cudaMemcpyHostToDevice, st) ==
                  cudaSuccess &&
              cudaMemsetAsync(d_counts, 0, ncounts * sizeof(unsigned long long), st) == cudaSuccess;
    if (!ok) {
        if (own) cudaStreamDestroy(own);
        bfree_all(b);
        return MDIST_ECUDA;
    }
    D.rows = d_rows;
    D.units = d_units;
    D.gs_table = d_gs;
    D.codes = d_codes;
    D.counts = d_counts;
    D.items = d_items;
    D.slots = d_slots;
    D.plans = d_plans;
    D.bucket_items = d_bucket;
    D.bucket_packed = d_packed;
    D.tile_ctr = d_packed + kBatchBuckets;
    D.codeU = d_codeU;
    D.item_ctr = d_ctr;
    D.active_ctr = d_ctr + 1;
    D.ncodes = C;
    D.item_cap = (int)cap;
    // ---- grids per bucket ----
    int grid[kBatchBuckets] = {};
    if (batch_bucket_grids(present, b->sm_count, b->opt.blocks_per_sm, grid) != cudaSuccess) {
        if (own) cudaStreamDestroy(own);
        bfree_all(b);
        return MDIST_ECUDA;
    }
    // ---- the rounds as one graph ----
    // Default: ONE launch of a graph whose conditional WHILE node runs a round per
    // iteration until no code is active (batch_continue; at most kMaxRounds rounds).
    // rounds_per_graph > 0: that many rounds captured back to back, the graph relaunched
    // while codes remain.  Where the loop graph cannot be built, rounds of 4.
    constexpr int kMaxRounds = MDIST_MAX_K + 2;  // a code ends within k + 1 levels
    int *d_rounds = d_ctr + 2;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool looped = rounds_per_graph <= 0 && build_loop_graph(D, present, grid, st, d_rounds, kMaxRounds, &graph);
    const int R = looped ? 0 : (rounds_per_graph > 0 ? rounds_per_graph : 4);
    b->rounds_per_graph = R;
    if (!looped) {
        if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            if (own) cudaStreamDestroy(own);
            bfree_all(b);
            return MDIST_ECUDA;
        }
        for (int r = 0; r < R; ++r) batch_launch_round(D, present, grid, st);
        if (cudaStreamEndCapture(st, &graph) != cudaSuccess) graph = nullptr;
    }
    if (!graph || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        if (own) cudaStreamDestroy(own);
        bfree_all(b);
        return MDIST_ECUDA;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int rc = MDIST_OK;
    int *h_active = nullptr;
    cudaMallocHost((void **)&h_active, 2 * sizeof(int));
    const int max_launches = looped ? 1 : kMaxRounds / R + 2;
    if (cudaMemsetAsync(d_rounds, 0, sizeof(int), st) != cudaSuccess) rc = MDIST_ECUDA;
    for (int launch = 0; launch < max_launches && rc == MDIST_OK; ++launch) {
        cudaEventRecord(e0, st);
        if (cudaGraphLaunch(exec, st) != cudaSuccess) { rc = MDIST_ECUDA; break; }
        cudaEventRecord(e1, st);
        cudaMemcpyAsync(h_active, D.active_ctr, 2 * sizeof(int), cudaMemcpyDeviceToHost, st);  // active, rounds
        if (cudaStreamSynchronize(st) != cudaSuccess) { rc = MDIST_ECUDA; break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        b->gpu_ms += ms;
        b->graph_launches += 1;
        b->rounds = looped ? h_active[1] : b->rounds + R;
        if (h_active[0] == 0) break;
    }
    // codes still active here ran into the round cap, which no code reaches (their
    // results stay MDIST_EAGAIN)
    if (rc == MDIST_OK) {
        b->res.resize((size_t)C);
        b->counts.resize(ncounts);
        if (cudaMemcpy(b->res.data(), d_codes, (size_t)C * sizeof(BatchCode), cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(b->counts.data(), d_counts, ncounts * sizeof(unsigned long long), cudaMemcpyDeviceToHost) !=
                cudaSuccess)
            rc = MDIST_ECUDA;
    }
    if (h_active) cudaFreeHost(h_active);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    if (own) {
        cudaStreamSynchronize(own);
        cudaStreamDestroy(own);
    }
    bfree_all(b);
    return rc;
}

}  // namespace

extern "C" {

int mdist_batch_info(const mdist_batch *b, int *ncodes, int *graph_launches, int *rounds, double *gpu_ms,
                     double *seconds, int *large_codes, double *large_ms) {
    if (!b) return MDIST_EINVAL;
    if (large_codes) {
        int n = 0;
        for (const HostCode &h : b->codes) n += h.large ? 1 : 0;
        *large_codes = n;
    }
    if (large_ms) *large_ms = b->large_ms;
    if (ncodes) *ncodes = (int)b->codes.size();
    if (graph_launches) *graph_launches = b->graph_launches;
    if (rounds) *rounds = b->rounds;
    if (gpu_ms) *gpu_ms = b->gpu_ms;
    if (seconds) *seconds = b->seconds;
    return MDIST_OK;
}

int mdist_batch_result(const mdist_batch *b, int index, int *d, uint64_t *witness, uint64_t *message, mdist_key *key,
                       mdist_stats *stats) {
    if (!b || !d || index < 0 || index >= (int)b->codes.size()) return MDIST_EINVAL;
    if (!b->ran) return MDIST_EAGAIN;
    const HostCode &h = b->codes[(size_t)index];
    if (h.large) {
        const LargeResult &r = b->large_res[(size_t)h.slot];
        if (r.status != MDIST_OK) return r.status;
        *d = r.d;
        if (witness) std::copy(r.witness.begin(), r.witness.end(), witness);
        if (message) *message = r.message;
        if (key) *key = r.key;
        if (stats) *stats = r.stats;
        return MDIST_OK;
    }
    if (b->res.empty()) return MDIST_EAGAIN;
    const BatchCode &S = b->res[(size_t)h.slot];
    if (S.status != MDIST_OK) return S.status;
    if (S.active || !S.have_key) return MDIST_EAGAIN;
    *d = S.U;
    const unsigned long long comb = host_unrank_lex(h.k, S.key_g, S.key_rank);
    const InfoSet &set = h.part.sets[(size_t)S.key_j];
    uint64_t msg = 0;
    for (int r = 0; r < h.k; ++r)
        if ((comb >> r) & 1ull) msg ^= set.transform[(size_t)r];
    if (message) *message = msg;
    if (witness) {
        for (int w = 0; w < h.W; ++w) witness[w] = 0;
        for (int bit = 0; bit < h.k; ++bit)
            if ((msg >> bit) & 1ull)
                for (int w = 0; w < h.W; ++w) witness[w] ^= h.G[(size_t)bit * h.W + w];
    }
    if (key) *key = mdist_key{S.key_w, S.key_g, S.key_j, 0, S.key_rank};
    if (stats) {
        std::memset(stats, 0, sizeof *stats);
        stats->g_final = S.g_final;
        stats->j_final = S.j_final;
        stats->m = S.m;
        stats->L_final = S.L;
        stats->U_final = S.U;
        stats->launches = S.rounds;
        for (int j = 0; j < S.m && j < MDIST_MAX_SETS; ++j) stats->ranks[j] = h.part.sets[(size_t)j].rank;
        const unsigned long long off = b->counts_off[(size_t)h.slot];
        for (int g = 0; g <= h.k; ++g)
            for (int j = 0; j < S.m && j < MDIST_MAX_SETS; ++j) stats->combos[g][j] = b->counts[off + (size_t)g * S.m + j];
        stats->total_combos = S.combos;
    }
    return MDIST_OK;
}

void mdist_batch_free(mdist_batch *b) {
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    bfree_all(b);
    delete b;
}

}  // extern "C"
