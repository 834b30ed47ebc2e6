// microbench.cu -- instruction-throughput probes for the roofline of the level
// enumerator: how many 32-bit POPC, how many 3-input LOP3 / IADD3 and how many
// "codeword steps" (the enumerator's inner-loop mix: XOR, POPC per word, sum, min)
// one SM retires per clock.  Each probe runs one CTA of 1024 threads per SM on data
// held in registers (no memory traffic) and times itself with clock64().
#include <cstdint>

#include "internal.h"

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

}  // namespace
}  // namespace mdist

extern "C" int mdist_microbench(int which, int iters, double *ops_per_clock_per_sm, double *seconds) {
    using namespace mdist;
    if (!ops_per_clock_per_sm || which < 0 || which > 4 || iters < 1) return MDIST_EINVAL;
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
    cudaEventRecord(e0);
    if (which == 0) probe_popc<<<sms, kProbeThreads>>>(iters, sink, cyc);
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
        // ops per thread per iteration: 16 POPC | 16 LOP3 | 16 codeword steps
        const double ops = 16.0 * (double)iters * kProbeThreads;
        *ops_per_clock_per_sm = ops / mean;
        if (seconds) *seconds = ms * 1e-3;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    cudaFree(cyc);
    return rc;
}
