// microbench.cu -- instruction-throughput probes for the roofline of the level
// enumerator: how many 32-bit POPC, how many 3-input LOP3 / IADD3 and how many
// "codeword steps" (the enumerator's inner-loop mix: XOR, POPC per word, sum, min)
// one SM retires per clock.  Each probe runs one CTA of 1024 threads per SM on data
// held in registers (no memory traffic) and times itself with clock64().
#include <cstdint>

#include "../csrc/internal.h"
#include "../../include/mdist_probe.h"
#include "../csrc/tc_common.cuh"

namespace mdist {
namespace {

constexpr int kProbeThreads = 1024;

__global__ void __launch_bounds__(kProbeThreads) probe_popc(int iters, unsigned int *sink, unsigned long long *cycles) {
    unsigned int a[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) a[i] = threadIdx.x * 2654435761u + i * 40503u;
    __syncthreads();
    const long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 16; ++i) a[i] = __popc(a[i]) | (a[(i + 1) & 15] << 8);
    }
    __syncthreads();
    const long long t1 = clock64();
    unsigned int s = 0;
#pragma unroll
    for (int i = 0; i < 16; ++i) s += a[i];
    if (s == 0x12345678u) sink[0] = s;
    if (threadIdx.x == 0) cycles[blockIdx.x] = (unsigned long long)(t1 - t0);
}

__global__ void __launch_bounds__(kProbeThreads) probe_lop3(int iters, unsigned int *sink, unsigned long long *cycles) {
    unsigned int a[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) a[i] = threadIdx.x * 2654435761u + i * 40503u;
    const unsigned int b = sink[1], c = sink[2];
    __syncthreads();
    const long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 16; ++i) a[i] = a[i] ^ b ^ (c + it);  // one 3-input XOR each (the add is hoisted)
    }
    __syncthreads();
    const long long t1 = clock64();
    unsigned int s = 0;
#pragma unroll
    for (int i = 0; i < 16; ++i) s += a[i];
    if (s == 0x12345678u) sink[0] = s;
    if (threadIdx.x == 0) cycles[blockIdx.x] = (unsigned long long)(t1 - t0);
}

// The enumerator's inner step for NW = 4 words and XP = 16 lane entries, with y
// taken from registers that change every iteration.
__global__ void __launch_bounds__(kProbeThreads) probe_step4(int iters, unsigned int *sink, unsigned long long *cycles) {
    unsigned int x[16][4];
#pragma unroll
    for (int p = 0; p < 16; ++p)
#pragma unroll
        for (int w = 0; w < 4; ++w) x[p][w] = (threadIdx.x + 1) * 2654435761u ^ (p * 4 + w) * 40503u;
    unsigned int y0 = sink[1], y1 = sink[2], y2 = sink[3], y3 = sink[4];
    int thr = (int)sink[5];
    int hits = 0;
    __syncthreads();
    const long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
        int mn = 1 << 30;
#pragma unroll
        for (int p = 0; p < 16; ++p) {
            const int acc = __popc(x[p][0] ^ y0) + __popc(x[p][1] ^ y1) + __popc(x[p][2] ^ y2) + __popc(x[p][3] ^ y3);
            mn = acc < mn ? acc : mn;
        }
        if (mn <= thr) ++hits;
        y0 += 0x9e3779b9u; y1 ^= y0; y2 += y1; y3 ^= y2;
    }
    __syncthreads();
    const long long t1 = clock64();
    if (hits == 0x7fffffff) sink[0] = hits;
    if (threadIdx.x == 0) cycles[blockIdx.x] = (unsigned long long)(t1 - t0);
}

// The lower-bound step of the group variants for NW = 4 (GS = 4: one POPC of the OR
// of the four XORed words; GS = 2: two POPC), threshold never reached.
template <int GS>
__global__ void __launch_bounds__(kProbeThreads) probe_step4_group(int iters, unsigned int *sink,
                                                                   unsigned long long *cycles) {
    unsigned int x[16][4];
#pragma unroll
    for (int p = 0; p < 16; ++p)
#pragma unroll
        for (int w = 0; w < 4; ++w) x[p][w] = (threadIdx.x + 1) * 2654435761u ^ (p * 4 + w) * 40503u;
    unsigned int y0 = sink[1], y1 = sink[2], y2 = sink[3], y3 = sink[4];
    const int thr = (int)sink[5] - 1;  // sink[5] = 0: bound never <= thr
    int hits = 0;
    __syncthreads();
    const long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
        int mn = 1 << 30;
#pragma unroll
        for (int p = 0; p < 16; ++p) {
            int lb;
            if (GS == 4) {
                lb = __popc((x[p][0] ^ y0) | (x[p][1] ^ y1) | (x[p][2] ^ y2) | (x[p][3] ^ y3));
            } else {
                lb = __popc((x[p][0] ^ y0) | (x[p][1] ^ y1)) + __popc((x[p][2] ^ y2) | (x[p][3] ^ y3));
            }
            mn = lb < mn ? lb : mn;
        }
        if (mn <= thr) {
#pragma unroll
            for (int p = 0; p < 16; ++p)
                hits += __popc(x[p][0] ^ y0) + __popc(x[p][1] ^ y1) + __popc(x[p][2] ^ y2) + __popc(x[p][3] ^ y3);
        }
        y0 += 0x9e3779b9u; y1 ^= y0; y2 += y1; y3 ^= y2;
    }
    __syncthreads();
    const long long t1 = clock64();
    if (hits == 0x7fffffff) sink[0] = hits;
    if (threadIdx.x == 0) cycles[blockIdx.x] = (unsigned long long)(t1 - t0);
}

// tcgen05 kind::f8f6f4 (E4M3, f16 accumulator) 128 x 256 x 32 MMAs issued back to back
// by one thread, operands resident in shared memory (zeros), four K-steps of 32 bytes
// per round as in a 128-byte operand row.  SW: 0 = no swizzle (8-row x 16-byte core
// matrices, leading byte offset 128, stride (K / 16) * 128), 2 = 128-byte swizzle
// (stride 1024, K-steps 32 bytes apart inside the swizzle atom), 6 = 32-byte swizzle
// (one atom of 8 rows x 32 bytes per K-step: stride 256, K-steps rows * 32 bytes
// apart).  cycles[blockIdx.x] = clock64 from the first issue to the completion of all.
template <int SW>
__global__ void __launch_bounds__(128, 1) probe_mma(int iters, unsigned int *sink, unsigned long long *cycles) {
    extern __shared__ __align__(1024) uint8_t sm[];
    constexpr int KROW = 128, MA = 128, NB = 256;
    uint8_t *sA = sm;
    uint8_t *sB = sm + MA * KROW;
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + (MA + NB) * KROW);
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(bar + 1);
    for (int i = threadIdx.x; i < (MA + NB) * KROW / 16; i += blockDim.x)
        reinterpret_cast<uint4 *>(sm)[i] = make_uint4(0, 0, 0, 0);
    if (threadIdx.x < 32) tmem_alloc(smem_addr(s_tmem), 256);
    if (threadIdx.x == 0) {
        mbar_init(smem_addr(bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *s_tmem;
    if (threadIdx.x == 0) {
        const uint32_t idesc = idesc_f8f6f4_e4m3_f16(MA, NB);
        const uint32_t a0 = smem_addr(sA), b0 = smem_addr(sB);
        const long long t0 = clock64();
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
                uint64_t ad, bd;
                if (SW == 0) {
                    ad = smem_desc(a0 + ks * 256, 128, (KROW / 16) * 128);
                    bd = smem_desc(b0 + ks * 256, 128, (KROW / 16) * 128);
                } else if (SW == 2) {
                    ad = smem_desc(a0 + ks * 32, 16, 1024) | ((uint64_t)2 << 61);
                    bd = smem_desc(b0 + ks * 32, 16, 1024) | ((uint64_t)2 << 61);
                } else {
                    ad = smem_desc(a0 + ks * MA * 32, 16, 256) | ((uint64_t)6 << 61);
                    bd = smem_desc(b0 + ks * NB * 32, 16, 256) | ((uint64_t)6 << 61);
                }
                mma_f8f6f4(tmem, ad, bd, idesc, (it | ks) ? 1u : 0u);
            }
        }
        mma_commit(smem_addr(bar));
        const bool done = mbar_wait(smem_addr(bar), 0, 1ll << 31);
        const long long t1 = clock64();
        cycles[blockIdx.x] = (unsigned long long)(t1 - t0);
        if (!done) sink[1] = 1;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x < 32) tmem_dealloc(tmem, 256);
}

}  // namespace
}  // namespace mdist

extern "C" int mdist_microbench(int which, int iters, double *ops_per_clock_per_sm, double *seconds) {
    using namespace mdist;
    if (!ops_per_clock_per_sm || which < 0 || which > 7 || iters < 1) return MDIST_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return MDIST_ECUDA;
    }
    unsigned int *sink = nullptr;
    unsigned long long *cyc = nullptr;
    if (cudaMalloc(&sink, 64) != cudaSuccess) return MDIST_ENOMEM;
    if (cudaMalloc(&cyc, sizeof(unsigned long long) * sms) != cudaSuccess) { cudaFree(sink); return MDIST_ENOMEM; }
    cudaMemset(sink, 0, 64);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    if (which >= 5) {
        auto *fn = which == 5 ? probe_mma<0> : (which == 6 ? probe_mma<2> : probe_mma<6>);
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 120 << 10) != cudaSuccess) {
            cudaFree(sink);
            cudaFree(cyc);
            return MDIST_ECUDA;
        }
    }
    cudaEventRecord(e0);
    if (which == 5) probe_mma<0><<<sms, 128, 120 << 10>>>(iters, sink, cyc);
    else if (which == 6) probe_mma<2><<<sms, 128, 120 << 10>>>(iters, sink, cyc);
    else if (which == 7) probe_mma<6><<<sms, 128, 120 << 10>>>(iters, sink, cyc);
    else if (which == 0) probe_popc<<<sms, kProbeThreads>>>(iters, sink, cyc);
    else if (which == 1) probe_lop3<<<sms, kProbeThreads>>>(iters, sink, cyc);
    else if (which == 2) probe_step4<<<sms, kProbeThreads>>>(iters, sink, cyc);
    else if (which == 3) probe_step4_group<2><<<sms, kProbeThreads>>>(iters, sink, cyc);
    else probe_step4_group<4><<<sms, kProbeThreads>>>(iters, sink, cyc);
    cudaEventRecord(e1);
    int rc = cudaEventSynchronize(e1) == cudaSuccess && cudaGetLastError() == cudaSuccess ? MDIST_OK : MDIST_ECUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rc == MDIST_OK) {
        unsigned long long *h = new unsigned long long[sms];
        cudaMemcpy(h, cyc, sizeof(unsigned long long) * sms, cudaMemcpyDeviceToHost);
        double mean = 0;
        for (int i = 0; i < sms; ++i) mean += (double)h[i];
        mean /= sms;
        delete[] h;
        // ops per thread per iteration: 16 POPC | 16 LOP3 | 16 codeword steps; MMA
        // probes: multiply-adds (4 x 128 x 256 x 32 per iteration)
        const double ops = which >= 5 ? 4.0 * 128 * 256 * 32 * (double)iters : 16.0 * (double)iters * kProbeThreads;
        *ops_per_clock_per_sm = ops / mean;
        if (seconds) *seconds = ms * 1e-3;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    cudaFree(cyc);
    return rc;
}
