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
#include <algorithm>
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
// which halves the B bytes each multiply-add needs from L2
__host__ __device__ constexpr int gram_ma(int) { return 2; }

// B stages that fit beside `as` A stages (at most four)
__host__ __device__ constexpr int gram_b_fit(int nw, int as) {
    return (kSmemOperandBudget - as * gram_ma(nw) * kGM * gram_ka(nw)) / (kGN * gram_ka(nw)) < 4
               ? (kSmemOperandBudget - as * gram_ma(nw) * kGM * gram_ka(nw)) / (kGN * gram_ka(nw))
               : 4;
}

// A stages: two (the builder fills the next unit's A tiles while the MMAs read these)
// where that leaves three B stages, else one (wide rows: the builder refills the A
// tiles after the unit's last MMA, a few thousand clocks per unit of 10^5)
__host__ __device__ constexpr int gram_a_stages(int nw) { return gram_b_fit(nw, 2) >= 3 ? 2 : 1; }

// B stages that fit beside the A stages
__host__ __device__ constexpr int gram_b_stages(int nw) { return gram_b_fit(nw, gram_a_stages(nw)); }

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
    constexpr int AS = gram_a_stages(NW);
    constexpr int A_BYTES = kGM * KA, B_BYTES = kGN * KA;
    static_assert(S >= 2, "two B stages at least");
    extern __shared__ __align__(1024) uint8_t sm[];
    uint8_t *sA0 = sm;  // stage st, tile h at sA0 + (st * MA + h) * A_BYTES
    uint8_t *sB0 = sm + AS * MA * A_BYTES;
    // barriers: 0-1 a_full, 2-3 a_empty, 4-5 acc_full, 6-7 acc_empty, 8 drain,
    //           9 .. 9+S-1 b_full, 9+S .. 9+2S-1 b_empty
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + AS * MA * A_BYTES + S * B_BYTES);
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
            const int st = (int)(u % AS);
            uint32_t x[MA * kGM / 32][NW];
#pragma unroll
            for (int h = 0; h < MA * kGM / 32; ++h) {
                const unsigned long long e = a_tile * (MA * kGM) + (unsigned long long)(lane + 32 * h);
#pragma unroll
                for (int w = 0; w < NW; ++w) x[h][w] = e < B.a.n ? B.a_tab[e * NW + w] : 0u;
            }
            if (!mbar_wait(bar(A_EMPTY + st), (uint32_t)(((u / AS) & 1) ^ 1), P.max_wait)) { fail(); break; }
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
                const int st = (int)(u % AS);
                if (!mbar_wait(bar(A_FULL + st), (uint32_t)((u / AS) & 1), P.max_wait)) { fail(); break; }
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
    const size_t need = (size_t)gram_a_stages(NW) * gram_ma(NW) * kGM * KA + (size_t)gram_b_stages(NW) * kGN * KA +
                        24 * sizeof(uint64_t) +
                        sizeof(uint32_t) * (size_t)(kBn * kBn);
    return need < (size_t)(120 << 10) ? (size_t)(120 << 10) : need;
}

template <int NW>
cudaError_t gram_launch_nw(const GramParams &p, int sm_count, cudaStream_t stream) {
    const size_t smem = gram_smem_bytes<NW>();
    cudaError_t e = allow_dynamic_smem((const void *)gram_kernel<NW>, smem);
    if (e != cudaSuccess) return e;
    unsigned long long grid = (unsigned long long)sm_count;
    if (p.total_wu - p.wu_lo < grid) grid = p.total_wu - p.wu_lo;
    if (grid < 1) return cudaSuccess;
    gram_kernel<NW><<<(unsigned int)grid, kGramThreads, smem, stream>>>(p);
    return cudaGetLastError();
}

// Several tables in one launch.  Entry e of a side is the sum of the rows of a subset;
// the colex rank of a t0-subset c_0 < ... < c_(t0-1) is the sum of C(c_i, i + 1), so
// the entries whose component-0 subsets share every element but the lowest u (the
// "top", least element c_u) and share the component-1 subset form one contiguous run
// of C(c_u, u) entries (all C(kc0, u) when the top is empty), and entry j of a run is
// the run's top sum XOR T[j], T the sums of the u-subsets of the component's rows in
// colex order.  T is a table built by an earlier launch (the one-component side of
// t = u on the same rows, read through the L2) or, with u = min(t0, 1), the
// component's rows themselves (the 1-subsets; for t0 = 0 a zero entry), staged in
// shared memory.  A warp task is a piece of `piece` consecutive entries: the warp
// unranks the first, then walks the runs (tops stepped by Gosper's rule, component 1
// stepping when the top wraps), writing each run's span with coalesced vector stores
// of T[j] ^ top.
constexpr int kTableThreads = 512;
constexpr int kTableWarps = kTableThreads / 32;

struct SideJob {
    GramSide side;
    uint32_t *out;
    const uint32_t *low;       // T in global memory, or null: the rows (u <= 1)
    int u;                     // elements of an entry's subset taken from T
    uint32_t first_mod;        // the job's first task in the launch-wide numbering, mod warps
    unsigned long long piece;  // entries per task
    unsigned long long ntasks;
};

struct SideJobs {
    int njobs;
    uint32_t warps;  // warps of the launch
    SideJob job[kMaxTableJobs];
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

// C(a, b) for a, b <= 32 in global memory (the table kernels stage it with coalesced
// loads; a constant-memory copy would serialise the lanes' different addresses)
struct Binom32 {
    uint32_t v[kBn * kBn];
};
constexpr Binom32 make_binom32() {
    Binom32 t{};
    for (int a = 0; a < kBn; ++a) {
        t.v[a * kBn] = 1;
        for (int b = 1; b <= a; ++b) t.v[a * kBn + b] = t.v[(a - 1) * kBn + b - 1] + (b <= a - 1 ? t.v[(a - 1) * kBn + b] : 0u);
    }
    return t;
}
static __device__ Binom32 g_binom32 = make_binom32();

// x ^= the rows of mask m (rows of NW words in shared memory)
template <int NW>
__device__ __forceinline__ void xor_rows(uint32_t (&x)[NW], const uint32_t *s_rows, unsigned long long m) {
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
}

// y = the entry at src (NW words; G: read-only global memory, else shared memory)
template <int NW, bool G>
__device__ __forceinline__ void load_entry(uint32_t (&y)[NW], const uint32_t *src) {
    if constexpr (NW % 4 == 0) {
#pragma unroll
        for (int v = 0; v < NW / 4; ++v) {
            const uint4 t = G ? __ldg(reinterpret_cast<const uint4 *>(src) + v) : reinterpret_cast<const uint4 *>(src)[v];
            y[4 * v] = t.x;
            y[4 * v + 1] = t.y;
            y[4 * v + 2] = t.z;
            y[4 * v + 3] = t.w;
        }
    } else if constexpr (NW % 2 == 0) {
#pragma unroll
        for (int v = 0; v < NW / 2; ++v) {
            const uint2 t = G ? __ldg(reinterpret_cast<const uint2 *>(src) + v) : reinterpret_cast<const uint2 *>(src)[v];
            y[2 * v] = t.x;
            y[2 * v + 1] = t.y;
        }
    } else {
#pragma unroll
        for (int w = 0; w < NW; ++w) y[w] = G ? __ldg(src + w) : src[w];
    }
}

// dst = y ^ x (one entry of NW words, vector stores where the width allows)
template <int NW>
__device__ __forceinline__ void store_entry(uint32_t *dst, const uint32_t (&y)[NW], const uint32_t (&x)[NW]) {
    if constexpr (NW % 4 == 0) {
#pragma unroll
        for (int v = 0; v < NW / 4; ++v)
            reinterpret_cast<uint4 *>(dst)[v] =
                make_uint4(y[4 * v] ^ x[4 * v], y[4 * v + 1] ^ x[4 * v + 1], y[4 * v + 2] ^ x[4 * v + 2],
                           y[4 * v + 3] ^ x[4 * v + 3]);
    } else if constexpr (NW % 2 == 0) {
#pragma unroll
        for (int v = 0; v < NW / 2; ++v)
            reinterpret_cast<uint2 *>(dst)[v] = make_uint2(y[2 * v] ^ x[2 * v], y[2 * v + 1] ^ x[2 * v + 1]);
    } else {
#pragma unroll
        for (int w = 0; w < NW; ++w) dst[w] = y[w] ^ x[w];
    }
}

// dst[i] = src[i] ^ x for i < cnt (entries of NW words), lane-strided, four entries per
// lane in flight while they last
template <int NW, bool G>
__device__ __forceinline__ void put_span(uint32_t *dst, const uint32_t *src, const uint32_t (&x)[NW], uint32_t cnt,
                                         int lane) {
    uint32_t i = lane;
    for (; i + 96 < cnt; i += 128) {
        uint32_t y0[NW], y1[NW], y2[NW], y3[NW];
        load_entry<NW, G>(y0, src + (size_t)i * NW);
        load_entry<NW, G>(y1, src + (size_t)(i + 32) * NW);
        load_entry<NW, G>(y2, src + (size_t)(i + 64) * NW);
        load_entry<NW, G>(y3, src + (size_t)(i + 96) * NW);
        store_entry<NW>(dst + (size_t)i * NW, y0, x);
        store_entry<NW>(dst + (size_t)(i + 32) * NW, y1, x);
        store_entry<NW>(dst + (size_t)(i + 64) * NW, y2, x);
        store_entry<NW>(dst + (size_t)(i + 96) * NW, y3, x);
    }
    for (; i < cnt; i += 32) {
        uint32_t y[NW];
        load_entry<NW, G>(y, src + (size_t)i * NW);
        store_entry<NW>(dst + (size_t)i * NW, y, x);
    }
}

// Task `task` of job R: entries [task * piece, min((task + 1) * piece, n)).  T: the u-subset
// sums (global memory when G).  Every T index stays below C(c_u, u) <= C(kc0, u), the
// entries of T.
template <int NW, bool G>
__device__ __forceinline__ void walk_task(const SideJob &R, unsigned long long task, const uint32_t *s_bn,
                                          const uint32_t *s_rows, const uint32_t *T, int lane) {
    const GramSide &S = R.side;
    const int u = R.u, t0 = S.t[0], kc0 = S.kc[0], off0 = S.off[0], off1 = S.off[1];
    const int tt = t0 - u;  // elements of a top, at positions 0 .. kc0 - u - 1 (element - u)
    const uint32_t first_top = (1u << tt) - 1u;                // tt <= 31 (u >= 1 once t0 > 3)
    const uint32_t last_top = first_top << (kc0 - u - tt);     // the colex-last top
    const uint32_t whole = s_bn[kc0 * kBn + u];                // run length with an empty top
    unsigned long long e = task * R.piece;
    const unsigned long long e_end = e + R.piece < S.n ? e + R.piece : S.n;
    unsigned long long e1 = S.nc == 2 ? e / S.cnt0 : 0ull;
    // the t0-subset of entry e: its lowest u elements have rank j in T, the rest is the top
    const uint32_t M = unrank_colex(s_bn, kc0, t0, (uint32_t)(e - e1 * S.cnt0));
    uint32_t j = 0, lowm = 0;
    {
        uint32_t m = M;
        for (int i = 0; i < u; ++i) {
            const int c = __ffs((int)m) - 1;
            j += s_bn[c * kBn + i + 1];
            lowm |= 1u << c;
            m &= m - 1;
        }
    }
    uint32_t top = (M ^ lowm) >> u;
    uint32_t m1 = S.nc == 2 ? unrank_colex(s_bn, S.kc[1], S.t[1], (uint32_t)e1) : 0u;
    uint32_t x[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) x[w] = 0;
    xor_rows<NW>(x, s_rows, ((unsigned long long)top << (u + off0)) | ((unsigned long long)m1 << off1));
    uint32_t len = tt > 0 ? s_bn[(__ffs((int)top) - 1 + u) * kBn + u] : whole;
    for (;;) {
        const unsigned long long left = e_end - e;
        const uint32_t cnt = (unsigned long long)(len - j) < left ? len - j : (uint32_t)left;
        put_span<NW, G>(R.out + e * NW, T + (size_t)j * NW, x, cnt, lane);
        e += cnt;
        if (e >= e_end) break;
        j = 0;
        unsigned long long diff;
        if (top != last_top) {  // the next top (tt > 0: the only top of tt = 0 is the last)
            const uint32_t nt = next_colex(top);
            diff = (unsigned long long)(top ^ nt) << (u + off0);
            top = nt;
        } else {  // the top returns to its first subset and component 1 steps
            const uint32_t n1 = next_colex(m1);
            diff = ((unsigned long long)(top ^ first_top) << (u + off0)) | ((unsigned long long)(m1 ^ n1) << off1);
            top = first_top;
            m1 = n1;
        }
        xor_rows<NW>(x, s_rows, diff);
        len = tt > 0 ? s_bn[(__ffs((int)top) - 1 + u) * kBn + u] : whole;
    }
}

// out_i[e * NW ..] = the sum of the rows of entry e of side i (rows: the k rows of the set).
// Warp w of the launch (W warps) takes the tasks t of job i with t = w - first_i mod W.
template <int NW>
__global__ void __launch_bounds__(kTableThreads) side_tables_kernel(const uint32_t *rows, int k,
                                                                      const __grid_constant__ SideJobs J) {
    __shared__ uint32_t s_bn[kBn * kBn];
    __shared__ __align__(16) uint32_t s_rows[64 * NW];
    __shared__ __align__(16) uint32_t s_zero[NW];  // T of t0 = 0: the empty sum
    for (int i = threadIdx.x; i < kBn * kBn; i += blockDim.x) s_bn[i] = g_binom32.v[i];
    for (int i = threadIdx.x; i < k * NW; i += blockDim.x) s_rows[i] = rows[i];
    if (threadIdx.x < NW) s_zero[threadIdx.x] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t W = J.warps;
    const uint32_t w = blockIdx.x * kTableWarps + (uint32_t)warp;
    for (int i = 0; i < J.njobs; ++i) {
        const SideJob &R = J.job[i];
        // this warp's first task of the job: (w - first) mod W, w < W
        for (unsigned long long t = w >= R.first_mod ? w - R.first_mod : w + W - R.first_mod; t < R.ntasks; t += W) {
            if (R.low) walk_task<NW, true>(R, t, s_bn, s_rows, R.low, lane);
            else walk_task<NW, false>(R, t, s_bn, s_rows, R.u ? s_rows + R.side.off[0] * NW : s_zero, lane);
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
cudaError_t side_tables_nw(const uint32_t *rows, int k, SideJobs &J, int sm_count, cudaStream_t stream) {
    auto kern = side_tables_kernel<NW>;
    int occ = 0;
    cudaError_t e = blocks_per_sm((const void *)kern, kTableThreads, 0, &occ);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const unsigned long long most_warps = (unsigned long long)sm_count * (unsigned long long)occ * kTableWarps;
    // pieces of one size for the launch, about 4 per warp (a small launch spreads its
    // latency-bound walks over every SM; a large one amortises each piece's unranking)
    unsigned long long total = 0;
    for (int i = 0; i < J.njobs; ++i) total += J.job[i].side.n;
    const unsigned long long piece = std::min(1ull << 20, std::max(64ull, total / (4 * most_warps)));
    unsigned long long tasks = 0;
    unsigned long long first[kMaxTableJobs];
    for (int i = 0; i < J.njobs; ++i) {
        SideJob &R = J.job[i];
        R.piece = piece;
        R.ntasks = (R.side.n + R.piece - 1) / R.piece;
        first[i] = tasks;
        tasks += R.ntasks;
    }
    const unsigned long long grid =
        std::min((unsigned long long)sm_count * occ, (tasks + kTableWarps - 1) / kTableWarps);
    J.warps = (uint32_t)(grid * kTableWarps);
    for (int i = 0; i < J.njobs; ++i) J.job[i].first_mod = (uint32_t)(first[i] % J.warps);
    kern<<<(unsigned int)grid, kTableThreads, 0, stream>>>(rows, k, J);
    return cudaGetLastError();
}

template <int NW>
cudaError_t expand_tables_nw(const ExpandJobs &J, int sm_count, cudaStream_t stream) {
    expand_tables_kernel<NW><<<table_grid(J.begin[J.njobs], sm_count), 256, 0, stream>>>(J);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_side_tables(const uint32_t *rows, int k, int nwords, const GramSide *sides, uint32_t *const *outs,
                               const uint32_t *const *lows, const int *low_t, int n, int sm_count,
                               cudaStream_t stream) {
    if (k < 1 || k > 64 || n < 0 || n > kMaxTableJobs) return cudaErrorInvalidValue;
    if (n == 0) return cudaSuccess;
    auto has_low = [&](int i) { return lows && lows[i] && low_t; };
    for (int i = 0; i < n; ++i) {
        const GramSide &S = sides[i];
        const bool ok0 = S.kc[0] <= 32 && S.t[0] <= S.kc[0] && S.off[0] + S.kc[0] <= k;
        const bool ok1 = S.nc == 1 || (S.kc[1] <= 32 && S.t[1] <= S.kc[1] && S.off[1] + S.kc[1] <= k);
        const bool okl = !has_low(i) || (low_t[i] >= 1 && low_t[i] < S.t[0]);
        if ((S.nc != 1 && S.nc != 2) || !ok0 || !ok1 || !okl || !outs[i]) return cudaErrorInvalidValue;
    }
    SideJobs J{};
    J.njobs = n;
    for (int i = 0; i < n; ++i) {
        SideJob &R = J.job[i];
        R.side = sides[i];
        R.out = outs[i];
        R.low = has_low(i) ? lows[i] : nullptr;
        R.u = has_low(i) ? low_t[i] : std::min<int>(sides[i].t[0], 1);
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
