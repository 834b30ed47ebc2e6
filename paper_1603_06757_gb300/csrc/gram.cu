// gram.cu -- the level enumerator on the tensor cores (tcgen05) for the large product
// blocks of a unit.
//
// Within a product block every codeword is x ^ y with x from one side (an i-subset sum
// of one half of the rows) and y from the other.  With the signs e(b) = 1 - 2b of the
// bits,
//     sum over the n_bits columns of e(x_c) e(y_c) = n_bits - 2 wt(x ^ y),
// so the weights of a whole 128 x 256 tile of codewords follow from a Gram matrix: a
// dense contraction over the n_bits columns.  Operand rows are the signs as E4M3 bytes
// (+1.0 / -1.0; the B side has zero bytes past n_bits), one kind::f8f6f4 MMA chain
// with f32 accumulation gives every acc = n_bits - 2 wt(x ^ y) exactly (integers of
// magnitude <= n_bits <= 256), and a codeword is a candidate iff
// acc >= n_bits - 2 thr (thr = largest reduced weight still a candidate).  The
// epilogue reads the accumulators from TMEM with loads that also return their maximum
// (tcgen05.ld.red .max); only a maximum at or above that bound sends a lane to the
// side path, which recomputes
// the weight from the bit-packed rows before touching the key.  A bound read late is
// only lower, never higher, than the current one: more candidates, all rechecked
// exactly.
//
// Neither operand depends on the threshold: the B side of a block is expanded once,
// tile by tile in the shared-memory layout, into a device table, and a tile reaches
// shared memory as one bulk copy; A tiles are expanded per work unit from the
// bit-packed subset sums.
//
// Persistent grid, one CTA per SM, 352 threads in four roles:
//   warps 0-7  epilogue   (warp w: TMEM lanes 32 (w % 4) .. + 31 = rows of the
//              accumulator tile, columns 128 (w / 4) .. + 127; four reducing loads of
//              32 f32 columns per wait),
//   warp  8    A builder  (four A rows per lane and A tile: load the packed sum, expand),
//   warp  9    B producer (one lane: a bulk copy of a whole B tile per stage),
//   warp  10   MMA issue  (one lane) and TMEM allocation.
// A work unit is (block, group of MA 128-row A tiles, up to 64 or 128 256-row B tiles:
// 128 when the launch still has at least 8 work units per SM, fewer A rebuilds); MA is
// two for rows of up to four words (one above, where two A stages of two tiles would
// leave fewer than four B stages).  Each B tile meets the MA A tiles in turn, one
// accumulator each, so a B tile copied from L2 serves 128 MA rows.  Within a block the A
// group runs fastest, so the CTAs running at the same time read the same B tiles from
// L2.  Every role walks the same static sequence of work units (CTA c takes c, c + grid,
// ...).  Stages: A two (of MA tiles), B up to four, accumulators two TMEM buffers of 256
// columns, used in turn by the MA accumulators of every B tile.  Hand-offs are
// mbarriers: A and accumulator-full by tcgen05.commit, B full by the copies'
// transaction bytes, B stages and accumulators freed by the epilogue (its thread 0
// frees a B stage once the accumulator-full commit of the tile's last accumulator has
// arrived).  Every wait is bounded; a timeout sets the status word, and the kernel
// ends after its copies and MMAs have drained.
//
#include <cstdint>

#include "combinatorics.cuh"
#include "enum_core.cuh"
#include "internal.h"
#include "tc_common.cuh"

namespace mdist {

static __constant__ BinomTable64 c_binom_g = make_binom_table64();

struct DevBinomG {
    __device__ __forceinline__ unsigned long long operator()(int a, int b) const { return c_binom_g.v[a][b]; }
};

namespace {

constexpr int kGM = 128;               // accumulator rows (A tile)
constexpr int kGN = 256;               // accumulator columns (B tile)
constexpr int kTilesPerUnit = 64;      // B tiles per work unit (doubled for large launches)
constexpr int kUnitsPerSmForLong = 8;  // work units per SM needed to use the doubled unit
constexpr int kGramThreads = 352;      // 8 epilogue warps, builder warp, producer warp, MMA warp
constexpr int kSmemOperandBudget = 200 << 10;
// Polls of a bounded wait: the default for the pipeline's hand-offs, and the floor of
// the final drains (a role's own copies and MMAs complete without any other thread, so
// those waits get at least this many polls whatever the caller's bound).
constexpr long long kDefaultWaitPolls = 200000000ll;

__host__ __device__ constexpr int gram_ka(int nw) { return 32 * nw; }  // bytes per operand row

// A tiles per work unit: every B tile meets both in turn (two accumulators per B tile),
// which halves the B bytes each multiply-add needs from L2; one where two would leave
// fewer than four B stages
__host__ __device__ constexpr int gram_ma(int nw) { return nw <= 4 ? 2 : 1; }

// B stages that fit beside the two A stages
__host__ __device__ constexpr int gram_b_stages(int nw) {
    return (kSmemOperandBudget - 2 * gram_ma(nw) * kGM * gram_ka(nw)) / (kGN * gram_ka(nw)) < 4
               ? (kSmemOperandBudget - 2 * gram_ma(nw) * kGM * gram_ka(nw)) / (kGN * gram_ka(nw))
               : 4;
}

struct GramBlock {
    GramSide a, b;               // the two sides (A: 128-row tiles, B: 256-row tiles)
    unsigned long long a_tiles;  // groups of gram_ma 128-row A tiles
    unsigned long long b_units, b_tiles;
    unsigned long long wu_begin;
    const uint32_t *a_tab;       // a.n x nwords: sums of the A side's entries
    const uint32_t *b_tab;       // b.n x nwords
    const uint8_t *b_exp;        // b_tiles x (kGN x KA) bytes: expanded B tiles (layout of write_row)
};

struct GramParams {
    unsigned int *U;
    UnitSlot *slot;
    int *status;
    int k, g, nwords, n_bits, base;
    int nblocks;
    unsigned int tiles_per_unit;  // B tiles per work unit
    unsigned long long wu_lo;     // this launch's work units: [wu_lo, total_wu)
    unsigned long long total_wu;
    long long max_wait;          // polls per hand-off wait
    long long drain_wait;        // polls per final drain wait (>= kDefaultWaitPolls)
    GramBlock blocks[kMaxGramBlocks];
};

// work unit -> (block, A tile group, B tile range); within a block the A group runs fastest
__device__ __forceinline__ void decode_wu(const GramParams &P, unsigned long long wu, int &b,
                                          unsigned long long &a_tile, unsigned long long &bt0,
                                          unsigned long long &bt1) {
    int lo = 0, hi = P.nblocks - 1;  // last block with wu_begin <= wu
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (P.blocks[mid].wu_begin <= wu) lo = mid;
        else hi = mid - 1;
    }
    b = lo;
    const GramBlock &B = P.blocks[b];
    const unsigned long long w = wu - B.wu_begin;
    const unsigned long long bu = w / B.a_tiles;
    a_tile = w - bu * B.a_tiles;
    bt0 = bu * P.tiles_per_unit;
    bt1 = bt0 + P.tiles_per_unit < B.b_tiles ? bt0 + P.tiles_per_unit : B.b_tiles;
}

// rows (as a k-bit mask) of the subset behind side entry e
__device__ __forceinline__ unsigned long long side_mask(const uint32_t *bn, const GramSide &S, unsigned long long e) {
    const unsigned long long e0 = S.nc == 2 ? e % S.cnt0 : e;
    unsigned long long m = (unsigned long long)unrank_colex(bn, S.kc[0], S.t[0], (uint32_t)e0) << S.off[0];
    if (S.nc == 2) m |= (unsigned long long)unrank_colex(bn, S.kc[1], S.t[1], (uint32_t)(e / S.cnt0)) << S.off[1];
    return m;
}

// Operand row r of a tile (K-major, no-swizzle layout): per bit of the NW words one
// E4M3 byte, +1.0 (0x38) for a clear bit and -1.0 (0xB8) for a set bit; the bits past
// `nbits` give zero bytes.
template <int NW>
__device__ __forceinline__ void write_row(uint8_t *tile, int r, const uint32_t (&x)[NW], int nbits) {
    constexpr int KA = gram_ka(NW);
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        const int vb = nbits - 32 * w;
        const uint32_t valid = vb >= 32 ? 0xFFFFFFFFu : (vb <= 0 ? 0u : (1u << vb) - 1u);
#pragma unroll
        for (int h = 0; h < 2; ++h) {  // 16 bits -> 16 bytes
            uint32_t q[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int sh = 16 * h + 4 * j;
                const uint32_t set = (((x[w] >> sh) & 0xFu) * 0x00204081u) & 0x01010101u;
                const uint32_t val = ((((valid >> sh) & 0xFu) * 0x00204081u) & 0x01010101u) * 0xFFu;
                q[j] = (0x38383838u | (set << 7)) & val;
            }
            *reinterpret_cast<uint4 *>(tile + kmajor_offset((uint32_t)r, (uint32_t)(32 * w + 16 * h), KA)) =
                make_uint4(q[0], q[1], q[2], q[3]);
        }
    }
}

template <int NW>
__global__ void __launch_bounds__(kGramThreads, 1) gram_kernel(const __grid_constant__ GramParams P) {
    constexpr int KA = gram_ka(NW);
    constexpr int KSTEPS = KA / 32;
    constexpr int S = gram_b_stages(NW);
    constexpr int MA = gram_ma(NW);  // A tiles per stage (rows 128 h .. of the group)
    constexpr int A_BYTES = kGM * KA, B_BYTES = kGN * KA;
    static_assert(S >= 2, "two B stages at least");
    extern __shared__ __align__(1024) uint8_t sm[];
    uint8_t *sA0 = sm;  // stage st, tile h at sA0 + (st * MA + h) * A_BYTES
    uint8_t *sB0 = sm + 2 * MA * A_BYTES;
    // barriers: 0-1 a_full, 2-3 a_empty, 4-5 acc_full, 6-7 acc_empty, 8 drain,
    //           9 .. 9+S-1 b_full, 9+S .. 9+2S-1 b_empty
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + 2 * MA * A_BYTES + S * B_BYTES);
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(bars + 20);
    volatile int *s_abort = reinterpret_cast<volatile int *>(s_tmem + 1);
    uint32_t *s_bn = reinterpret_cast<uint32_t *>(bars + 24);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    auto bar = [&](int i) { return smem_addr(bars + i); };
    constexpr int A_FULL = 0, A_EMPTY = 2, ACC_FULL = 4, ACC_EMPTY = 6, DRAIN = 8, B_FULL = 9, B_EMPTY = 9 + S;

    for (int i = tid; i < kBn * kBn; i += blockDim.x) s_bn[i] = (uint32_t)c_binom_g.v[i / kBn][i % kBn];
    if (warp == 10) tmem_alloc(smem_addr(s_tmem), 512);
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(bar(A_FULL + i), 32);
            mbar_init(bar(A_EMPTY + i), 1);
            mbar_init(bar(ACC_FULL + i), 1);
            mbar_init(bar(ACC_EMPTY + i), 256);
        }
        mbar_init(bar(DRAIN), 1);
        for (int i = 0; i < S; ++i) {
            mbar_init(bar(B_FULL + i), 1);
            mbar_init(bar(B_EMPTY + i), 1);
        }
        *s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *s_tmem;
    auto fail = [&]() {
        *s_abort = 1;
        atomicExch(P.status, 1);
    };

    if (warp == 8) {
        // ---------------- A builder ----------------
        unsigned long long u = 0;
        for (unsigned long long wu = P.wu_lo + blockIdx.x; wu < P.total_wu && !*s_abort; wu += gridDim.x, ++u) {
            int b;
            unsigned long long a_tile, bt0, bt1;
            decode_wu(P, wu, b, a_tile, bt0, bt1);
            const GramBlock &B = P.blocks[b];
            const int st = (int)(u & 1);
            uint32_t x[MA * kGM / 32][NW];
#pragma unroll
            for (int h = 0; h < MA * kGM / 32; ++h) {
                const unsigned long long e = a_tile * (MA * kGM) + (unsigned long long)(lane + 32 * h);
#pragma unroll
                for (int w = 0; w < NW; ++w) x[h][w] = e < B.a.n ? B.a_tab[e * NW + w] : 0u;
            }
            if (!mbar_wait(bar(A_EMPTY + st), (uint32_t)(((u >> 1) & 1) ^ 1), P.max_wait)) { fail(); break; }
#pragma unroll
            for (int h = 0; h < MA * kGM / 32; ++h)  // group row lane + 32 h: tile h / 4, row lane + 32 (h % 4)
                write_row<NW>(sA0 + (st * MA + h / (kGM / 32)) * A_BYTES, lane + 32 * (h % (kGM / 32)), x[h], 32 * NW);
            fence_async_smem();
            mbar_arrive(bar(A_FULL + st));
        }
    } else if (warp == 9) {
        // ---------------- B producer ----------------
        if (lane == 0) {
            unsigned long long t = 0;
            for (unsigned long long wu = P.wu_lo + blockIdx.x; wu < P.total_wu && !*s_abort; wu += gridDim.x) {
                int b;
                unsigned long long a_tile, bt0, bt1;
                decode_wu(P, wu, b, a_tile, bt0, bt1);
                const GramBlock &B = P.blocks[b];
                bool ok = true;
                for (unsigned long long bt = bt0; bt < bt1; ++bt, ++t) {
                    const int s = (int)(t % S);
                    if (!mbar_wait(bar(B_EMPTY + s), (uint32_t)(((t / S) & 1) ^ 1), P.max_wait)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(bar(B_FULL + s), (uint32_t)B_BYTES);
                    bulk_copy_g2s(smem_addr(sB0 + s * B_BYTES), B.b_exp + bt * (unsigned long long)B_BYTES,
                                  (uint32_t)B_BYTES, bar(B_FULL + s));
                }
                if (!ok) { fail(); break; }
            }
            // no copy may still be writing shared memory when the CTA ends: wait for the
            // last copy of every stage
            const unsigned long long first = t > (unsigned long long)S ? t - S : 0;
            for (unsigned long long i = first; i < t; ++i)
                if (!mbar_wait(bar(B_FULL + (int)(i % S)), (uint32_t)((i / S) & 1), P.drain_wait)) fail();
        }
    } else if (warp == 10) {
        // ---------------- MMA issue ----------------
        if (lane == 0) {
            const uint32_t idesc = idesc_f8f6f4_e4m3_f32(kGM, kGN);
            const uint32_t sbo = (uint32_t)(KA / 16) * 128u;
            unsigned long long t = 0, u = 0, q = 0;  // B tiles, work units, accumulators
            for (unsigned long long wu = P.wu_lo + blockIdx.x; wu < P.total_wu && !*s_abort; wu += gridDim.x, ++u) {
                int b;
                unsigned long long a_tile, bt0, bt1;
                decode_wu(P, wu, b, a_tile, bt0, bt1);
                const int st = (int)(u & 1);
                if (!mbar_wait(bar(A_FULL + st), (uint32_t)((u >> 1) & 1), P.max_wait)) { fail(); break; }
                bool ok = true;
                for (unsigned long long bt = bt0; bt < bt1 && ok; ++bt, ++t) {
                    const int s = (int)(t % S);
                    if (!mbar_wait(bar(B_FULL + s), (uint32_t)((t / S) & 1), P.max_wait)) {
                        ok = false;
                        break;
                    }
                    const uint32_t b0 = smem_addr(sB0 + s * B_BYTES);
#pragma unroll
                    for (int h = 0; h < MA; ++h, ++q) {
                        const int ab = (int)(q & 1);
                        if (!mbar_wait(bar(ACC_EMPTY + ab), (uint32_t)(((q >> 1) & 1) ^ 1), P.max_wait)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t a0 = smem_addr(sA0 + (st * MA + h) * A_BYTES);
                        const uint32_t d = tmem + (uint32_t)(ab * kGN);
#pragma unroll
                        for (int ks = 0; ks < KSTEPS; ++ks)
                            mma_f8f6f4(d, smem_desc(a0 + ks * 256, 128, sbo), smem_desc(b0 + ks * 256, 128, sbo),
                                       idesc, ks > 0 ? 1u : 0u);
                        mma_commit(bar(ACC_FULL + ab));  // accumulator ready; after tile MA-1: B stage s read
                    }
                }
                mma_commit(bar(A_EMPTY + st));  // A tile free again
                if (!ok) { fail(); break; }
            }
            mma_commit(bar(DRAIN));
            if (!mbar_wait(bar(DRAIN), 0, P.drain_wait)) fail();  // every MMA has completed
        }
    } else {
        // ---------------- epilogue (warps 0-7) ----------------
        const int row = 32 * (warp & 3) + lane;  // TMEM lane = A row
        const int col0 = 128 * (warp >> 2);      // first accumulator column of this warp
        unsigned long long t = 0, q = 0, cnt = 0;  // B tiles, accumulators, codewords counted
        unsigned int cand = 0;                     // pairs this thread re-weighed exactly (< 2^32 per launch)
        unsigned int u_next = *(volatile unsigned int *)P.U;
        bool ok = true;
        // the TMEM loads below are warp-collective (.sync.aligned), so every decision to
        // stop is taken for the whole warp: the abort flag and each wait's outcome
        for (unsigned long long wu = P.wu_lo + blockIdx.x; wu < P.total_wu && ok && !__any_sync(0xffffffffu, *s_abort != 0);
             wu += gridDim.x) {
            int b;
            unsigned long long a_tile, bt0, bt1;
            decode_wu(P, wu, b, a_tile, bt0, bt1);
            const GramBlock &B = P.blocks[b];
            // candidates: acc >= n_bits - 2 thr, with a threshold read one unit ahead
            const float bound = (float)(P.n_bits - 2 * ((int)u_next - P.base));
            u_next = *(volatile unsigned int *)P.U;
            for (unsigned long long bt = bt0; bt < bt1 && ok; ++bt, ++t) {
#pragma unroll 1
                for (int h = 0; h < MA; ++h, ++q) {
                    const int ab = (int)(q & 1);
                    if (!mbar_wait_warp(bar(ACC_FULL + ab), (uint32_t)((q >> 1) & 1), P.max_wait)) {
                        fail();
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    // the last MMA on B tile t has completed: its B stage is free (released
                    // here rather than by a commit, so that no thread but the epilogue waits
                    // on commit-driven barriers)
                    if (tid == 0 && h == MA - 1) mbar_arrive(bar(B_EMPTY + (int)(t % S)));
                    const unsigned long long a_lo = (a_tile * MA + (unsigned long long)h) * kGM;
                    const unsigned long long a_e = a_lo + (unsigned long long)row;
                    const bool a_valid = a_e < B.a.n;
                    const uint32_t base = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(ab * kGN + col0);
                    uint32_t v[4][32];  // 128 f32 accumulators
                    float m0, m1, m2, m3;
                    tmem_ldred32_max_issue(base, v[0], m0);
                    tmem_ldred32_max_issue(base + 32u, v[1], m1);
                    tmem_ldred32_max_issue(base + 64u, v[2], m2);
                    tmem_ldred32_max_issue(base + 96u, v[3], m3);
                    tmem_wait_ld(v[0]);
                    tmem_regs_ready(v[1]);
                    tmem_regs_ready(v[2]);
                    tmem_regs_ready(v[3]);
                    float_ready(m0);
                    float_ready(m1);
                    float_ready(m2);
                    float_ready(m3);
                    const float m = fmaxf(fmaxf(m0, m1), fmaxf(m2, m3));
                    if (m >= bound && a_valid) {
                        // side path: which columns reach the bound, then the exact weight
                        // from the bit-packed rows, then the key
                        uint32_t x[NW];
#pragma unroll
                        for (int w = 0; w < NW; ++w) x[w] = B.a_tab[a_e * NW + w];
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            uint32_t neg = 0;
#pragma unroll
                            for (int i = 0; i < 32; ++i) neg |= (__uint_as_float(v[c][i]) >= bound ? 1u : 0u) << i;
                            while (neg) {
                                const int i = __ffs(neg) - 1;
                                neg &= neg - 1;
                                const unsigned long long b_e = bt * kGN + (unsigned long long)(col0 + 32 * c + i);
                                if (b_e >= B.b.n) continue;
                                ++cand;
                                int w = 0;
#pragma unroll
                                for (int z = 0; z < NW; ++z) w += __popc(x[z] ^ B.b_tab[b_e * NW + z]);
                                const int weight = w + P.base;
                                if (weight > (int)(*(volatile unsigned int *)P.U)) continue;
                                const unsigned long long mask =
                                    side_mask(s_bn, B.a, a_e) | side_mask(s_bn, B.b, b_e);
                                const unsigned long long rank = lexrank64(mask, P.k, P.g, DevBinomG{});
                                atomicMin(P.U, (unsigned int)weight);
                                atomicMin(&P.slot->key, ((unsigned long long)weight << kKeyRankBits) | rank);
                            }
                        }
                    }
                    tc_fence_before();
                    mbar_arrive(bar(ACC_EMPTY + ab));
                    if (tid == 0 && a_lo < B.a.n) {
                        const unsigned long long a_rows = B.a.n - a_lo < (unsigned long long)kGM
                                                              ? B.a.n - a_lo
                                                              : (unsigned long long)kGM;
                        const unsigned long long b_left = B.b.n - bt * kGN;
                        cnt += a_rows * (b_left < (unsigned long long)kGN ? b_left : (unsigned long long)kGN);
                    }
                }
            }
        }
        if (tid == 0 && cnt) atomicAdd(&P.slot->count, cnt);
        if (cand) atomicAdd(&P.slot->tc_cand, (unsigned long long)cand);  // rare except at loose thresholds
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 10) tmem_dealloc(tmem, 512);
}

// at least 120 KB so that two CTAs never share an SM (each allocates all 512 TMEM columns)
template <int NW>
size_t gram_smem_bytes() {
    constexpr int KA = gram_ka(NW);
    const size_t need = 2 * (size_t)gram_ma(NW) * kGM * KA + (size_t)gram_b_stages(NW) * kGN * KA +
                        24 * sizeof(uint64_t) +
                        sizeof(uint32_t) * (size_t)(kBn * kBn);
    return need < (size_t)(120 << 10) ? (size_t)(120 << 10) : need;
}

template <int NW>
cudaError_t gram_launch_nw(const GramParams &p, int sm_count, cudaStream_t stream) {
    const size_t smem = gram_smem_bytes<NW>();
    cudaError_t e = cudaFuncSetAttribute(gram_kernel<NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    unsigned long long grid = (unsigned long long)sm_count;
    if (p.total_wu - p.wu_lo < grid) grid = p.total_wu - p.wu_lo;
    if (grid < 1) return cudaSuccess;
    gram_kernel<NW><<<(unsigned int)grid, kGramThreads, smem, stream>>>(p);
    return cudaGetLastError();
}

// Several tables in one launch: job i covers the global entries [begin[i], begin[i+1]).
constexpr int kTableChunk = 16;  // consecutive entries a thread builds

struct SideJobs {
    int njobs;
    unsigned long long begin[kMaxTableJobs + 1];  // chunks of kTableChunk entries
    GramSide side[kMaxTableJobs];
    uint32_t *out[kMaxTableJobs];
};

struct ExpandJobs {
    int njobs, n_bits;
    unsigned long long begin[kMaxTableJobs + 1];  // padded rows (multiples of kGN)
    unsigned long long count[kMaxTableJobs];
    const uint32_t *packed[kMaxTableJobs];
    uint8_t *out[kMaxTableJobs];
};

template <int N>
__device__ __forceinline__ int job_of(const unsigned long long (&begin)[N], int njobs, unsigned long long e) {
    int lo = 0, hi = njobs - 1;  // last job with begin <= e
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (begin[mid] <= e) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// out_i[e * NW ..] = the sum of the rows of entry e of side i (rows: the k rows of the set).
// A thread takes kTableChunk consecutive entries: it unranks the first, then steps to
// the next subset of each component in colex order (Gosper's rule; component 1 steps
// when component 0 wraps) and XORs only the rows that changed.  J.begin counts chunks.
// The 32 chunks of a warp are 512 consecutive entries of one table (when they lie in
// one table and are all full): the lanes stage their sums in shared memory (lane
// regions padded to an odd word stride, so the stores do not collide on banks) and the
// warp writes the 2 KB x NW block with coalesced 4-byte stores.  Other warps (a table
// boundary, the last partial chunk) store entry by entry.
__host__ __device__ constexpr int kStageStride(int nw) { return kTableChunk * nw + 1; }

template <int NW>
__global__ void side_tables_kernel(const uint32_t *rows, int k, const __grid_constant__ SideJobs J) {
    __shared__ uint32_t s_bn[kBn * kBn];
    __shared__ __align__(16) uint32_t s_rows[64 * NW];
    extern __shared__ uint32_t s_stage[];  // warps x 32 lanes x kStageStride(NW) words
    for (int i = threadIdx.x; i < kBn * kBn; i += blockDim.x) s_bn[i] = (uint32_t)c_binom_g.v[i / kBn][i % kBn];
    for (int i = threadIdx.x; i < k * NW; i += blockDim.x) s_rows[i] = rows[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *stage = s_stage + (size_t)warp * 32 * kStageStride(NW);
    auto add_rows = [&](uint32_t (&x)[NW], unsigned long long m) {
        while (m) {
            const int r = __ffsll((long long)m) - 1;
            m &= m - 1;
            if constexpr (NW % 4 == 0) {  // 16-byte loads of the row
#pragma unroll
                for (int v = 0; v < NW / 4; ++v) {
                    const uint4 t = reinterpret_cast<const uint4 *>(s_rows + r * NW)[v];
                    x[4 * v] ^= t.x;
                    x[4 * v + 1] ^= t.y;
                    x[4 * v + 2] ^= t.z;
                    x[4 * v + 3] ^= t.w;
                }
            } else {
#pragma unroll
                for (int w = 0; w < NW; ++w) x[w] ^= s_rows[r * NW + w];
            }
        }
    };
    const unsigned long long total = J.begin[J.njobs];
    const unsigned long long step = (unsigned long long)gridDim.x * blockDim.x;
    // every lane of a warp runs the same trips (the warp-wide votes below need them all)
    for (unsigned long long cw = blockIdx.x * (unsigned long long)blockDim.x + 32ull * warp; cw < total; cw += step) {
        const unsigned long long c = cw + lane;
        const bool active = c < total;
        const int i = active ? job_of(J.begin, J.njobs, c) : J.njobs - 1;
        const GramSide &S = J.side[i];
        unsigned long long e = active ? (c - J.begin[i]) * kTableChunk : 0;
        const unsigned long long e_end = active ? (e + kTableChunk < S.n ? e + kTableChunk : S.n) : 0;
        const int i0 = __shfl_sync(0xffffffffu, i, 0);
        const bool staged = __all_sync(0xffffffffu, active && i == i0 && e_end - e == kTableChunk);
        uint32_t *out = J.out[i];
        const unsigned long long e_first = e;
        if (active) {
            unsigned long long e0 = S.nc == 2 ? e % S.cnt0 : e;
            uint32_t m0 = unrank_colex(s_bn, S.kc[0], S.t[0], (uint32_t)e0);
            uint32_t m1 = S.nc == 2 ? unrank_colex(s_bn, S.kc[1], S.t[1], (uint32_t)(e / S.cnt0)) : 0u;
            uint32_t x[NW];
#pragma unroll
            for (int w = 0; w < NW; ++w) x[w] = 0;
            add_rows(x, ((unsigned long long)m0 << S.off[0]) | ((unsigned long long)m1 << S.off[1]));
            for (int q = 0;; ++q) {
                if (staged) {
#pragma unroll
                    for (int w = 0; w < NW; ++w) stage[lane * kStageStride(NW) + q * NW + w] = x[w];
                } else {
#pragma unroll
                    for (int w = 0; w < NW; ++w) out[e * NW + w] = x[w];
                }
                if (++e >= e_end) break;
                unsigned long long diff;
                if (e0 + 1 < S.cnt0) {
                    const uint32_t n0 = next_colex(m0);
                    diff = (unsigned long long)(m0 ^ n0) << S.off[0];
                    m0 = n0;
                    ++e0;
                } else {  // component 0 wraps to its first subset, component 1 steps
                    const uint32_t n0 = S.t[0] >= 32 ? 0xFFFFFFFFu : (1u << S.t[0]) - 1u;
                    const uint32_t n1 = next_colex(m1);
                    diff = ((unsigned long long)(m0 ^ n0) << S.off[0]) | ((unsigned long long)(m1 ^ n1) << S.off[1]);
                    m0 = n0;
                    m1 = n1;
                    e0 = 0;
                }
                add_rows(x, diff);
            }
        }
        if (staged) {
            __syncwarp();
            // lane r's 16 entries are words r * 16 NW .. of the warp's block, and they sit
            // contiguously in its staging region: copy run after run, 32 words at a time
            uint32_t *dst = out + __shfl_sync(0xffffffffu, e_first, 0) * NW;
#pragma unroll 4
            for (int r = 0; r < 32; ++r)
#pragma unroll
                for (int i = lane; i < kTableChunk * NW; i += 32)
                    dst[r * kTableChunk * NW + i] = stage[r * kStageStride(NW) + i];
            __syncwarp();
        }
    }
}

// B tiles of packed tables: row e of tile e / kGN of job i is the sign row of entry e
// (write_row with the code's n_bits); rows past the job's count are padding (zeros).
template <int NW>
__global__ void expand_tables_kernel(const __grid_constant__ ExpandJobs J) {
    constexpr int KA = gram_ka(NW);
    const unsigned long long total = J.begin[J.njobs];
    for (unsigned long long g = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; g < total;
         g += (unsigned long long)gridDim.x * blockDim.x) {
        const int i = job_of(J.begin, J.njobs, g);
        const unsigned long long e = g - J.begin[i], count = J.count[i];
        const uint32_t *packed = J.packed[i];
        uint32_t y[NW];
#pragma unroll
        for (int w = 0; w < NW; ++w) y[w] = e < count ? packed[e * NW + w] : 0u;
        write_row<NW>(J.out[i] + (e / kGN) * (unsigned long long)(kGN * KA), (int)(e % kGN), y,
                      e < count ? J.n_bits : 0);
    }
}

unsigned int table_grid(unsigned long long work, int sm_count) {
    unsigned long long grid = (work + 255) / 256;
    const unsigned long long cap = (unsigned long long)sm_count * 8;
    if (grid > cap) grid = cap;
    return (unsigned int)(grid < 1 ? 1 : grid);
}

template <int NW>
cudaError_t side_tables_nw(const uint32_t *rows, int k, const SideJobs &J, int sm_count, cudaStream_t stream) {
    const size_t smem = (size_t)(256 / 32) * 32 * kStageStride(NW) * sizeof(uint32_t);
    cudaError_t e = cudaFuncSetAttribute(side_tables_kernel<NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    side_tables_kernel<NW><<<table_grid(J.begin[J.njobs], sm_count), 256, smem, stream>>>(rows, k, J);
    return cudaGetLastError();
}

template <int NW>
cudaError_t expand_tables_nw(const ExpandJobs &J, int sm_count, cudaStream_t stream) {
    expand_tables_kernel<NW><<<table_grid(J.begin[J.njobs], sm_count), 256, 0, stream>>>(J);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_side_tables(const uint32_t *rows, int k, int nwords, const GramSide *sides, uint32_t *const *outs,
                               int n, int sm_count, cudaStream_t stream) {
    if (k < 1 || k > 64 || n < 0 || n > kMaxTableJobs) return cudaErrorInvalidValue;
    if (n == 0) return cudaSuccess;
    SideJobs J{};
    J.njobs = n;
    for (int i = 0; i < n; ++i) {
        J.side[i] = sides[i];
        J.out[i] = outs[i];
        J.begin[i + 1] = J.begin[i] + (sides[i].n + kTableChunk - 1) / kTableChunk;
    }
    switch (nwords) {
        case 1: return side_tables_nw<1>(rows, k, J, sm_count, stream);
        case 2: return side_tables_nw<2>(rows, k, J, sm_count, stream);
        case 3: return side_tables_nw<3>(rows, k, J, sm_count, stream);
        case 4: return side_tables_nw<4>(rows, k, J, sm_count, stream);
        case 5: return side_tables_nw<5>(rows, k, J, sm_count, stream);
        case 6: return side_tables_nw<6>(rows, k, J, sm_count, stream);
        case 7: return side_tables_nw<7>(rows, k, J, sm_count, stream);
        case 8: return side_tables_nw<8>(rows, k, J, sm_count, stream);
        default: return cudaErrorInvalidValue;
    }
}

size_t gram_expanded_bytes(int nwords, unsigned long long count) {
    return (size_t)((count + kGN - 1) / kGN) * (size_t)kGN * (size_t)gram_ka(nwords);
}

cudaError_t launch_expand_tables(int nwords, int n_bits, const uint32_t *const *packed,
                                 const unsigned long long *counts, uint8_t *const *outs, int n, int sm_count,
                                 cudaStream_t stream) {
    if (n < 0 || n > kMaxTableJobs) return cudaErrorInvalidValue;
    if (n == 0) return cudaSuccess;
    ExpandJobs J{};
    J.njobs = n;
    J.n_bits = n_bits;
    for (int i = 0; i < n; ++i) {
        J.packed[i] = packed[i];
        J.count[i] = counts[i];
        J.out[i] = outs[i];
        J.begin[i + 1] = J.begin[i] + (counts[i] + kGN - 1) / kGN * kGN;
    }
    switch (nwords) {
        case 1: return expand_tables_nw<1>(J, sm_count, stream);
        case 2: return expand_tables_nw<2>(J, sm_count, stream);
        case 3: return expand_tables_nw<3>(J, sm_count, stream);
        case 4: return expand_tables_nw<4>(J, sm_count, stream);
        case 5: return expand_tables_nw<5>(J, sm_count, stream);
        case 6: return expand_tables_nw<6>(J, sm_count, stream);
        case 7: return expand_tables_nw<7>(J, sm_count, stream);
        case 8: return expand_tables_nw<8>(J, sm_count, stream);
        default: return cudaErrorInvalidValue;
    }
}

bool gram_eligible(int nwords) { return nwords >= 1 && nwords <= kGramMaxWords; }

cudaError_t launch_gram_unit(const EnumParams &ep, const GramBlockSpec *blocks, int nblocks, unsigned int *U,
                             UnitSlot *slot, int *status, int sm_count, cudaStream_t stream, int part, int nparts) {
    if (nblocks > kMaxGramBlocks) return cudaErrorInvalidValue;
    GramParams p{};
    p.U = U;
    p.slot = slot;
    p.status = status;
    p.k = ep.k;
    p.g = ep.g;
    p.nwords = ep.nwords;
    p.n_bits = ep.n_bits;
    p.base = ep.base;
    p.max_wait = ep.wait_polls > 0 ? ep.wait_polls : kDefaultWaitPolls;
    p.drain_wait = p.max_wait > kDefaultWaitPolls ? p.max_wait : kDefaultWaitPolls;
    int nb = 0;
    unsigned long long wu = 0;
    for (int pass = 0; pass < 2; ++pass) {
        // first with the doubled unit; keep it if the launch still has enough units
        p.tiles_per_unit = pass == 0 ? 2 * kTilesPerUnit : kTilesPerUnit;
        nb = 0;
        wu = 0;
        for (int i = 0; i < nblocks; ++i) {
            const GramBlockSpec &S = blocks[i];
            if (!S.a_tab || !S.b_tab || !S.b_exp || S.a.n == 0 || S.b.n == 0) return cudaErrorInvalidValue;
            GramBlock &G = p.blocks[nb++];
            G.a = S.a;
            G.b = S.b;
            G.a_tab = S.a_tab;
            G.b_tab = S.b_tab;
            G.b_exp = S.b_exp;
            const unsigned long long rows = (unsigned long long)gram_ma(ep.nwords) * kGM;
            G.a_tiles = (S.a.n + rows - 1) / rows;
            G.b_tiles = (S.b.n + kGN - 1) / kGN;
            G.b_units = (G.b_tiles + p.tiles_per_unit - 1) / p.tiles_per_unit;
            G.wu_begin = wu;
            wu += G.a_tiles * G.b_units;
        }
        if (wu >= (unsigned long long)kUnitsPerSmForLong * (unsigned long long)sm_count) break;
    }
    p.nblocks = nb;
    if (nparts < 1 || part < 0 || part >= nparts) return cudaErrorInvalidValue;
    p.wu_lo = wu * (unsigned long long)part / (unsigned long long)nparts;
    p.total_wu = wu * (unsigned long long)(part + 1) / (unsigned long long)nparts;
    if (nb == 0 || p.total_wu <= p.wu_lo) return cudaSuccess;
    switch (ep.nwords) {
        case 1: return gram_launch_nw<1>(p, sm_count, stream);
        case 2: return gram_launch_nw<2>(p, sm_count, stream);
        case 3: return gram_launch_nw<3>(p, sm_count, stream);
        case 4: return gram_launch_nw<4>(p, sm_count, stream);
        case 5: return gram_launch_nw<5>(p, sm_count, stream);
        case 6: return gram_launch_nw<6>(p, sm_count, stream);
        case 7: return gram_launch_nw<7>(p, sm_count, stream);
        case 8: return gram_launch_nw<8>(p, sm_count, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace mdist
