// tc_probe.cu -- one 128 x N x K fp8 (E4M3) product on the tensor cores (tcgen05,
// f32 accumulators in TMEM), used to check the operand layout and descriptors that
// the Gram-matrix enumerator relies on against an exact host computation.
#include <cstdint>

#include "../csrc/internal.h"
#include "../../include/mdist_probe.h"
#include "../csrc/tc_common.cuh"

namespace mdist {
namespace {

constexpr int kProbeM = 128;

// A: 128 x K bytes, B: N x K bytes (row-major, E4M3), D: 128 x N f32 (row-major).
__global__ void __launch_bounds__(128, 1) tc_probe_kernel(const uint8_t *A, const uint8_t *B, float *D, int N, int K,
                                                           int *status) {
    extern __shared__ __align__(1024) uint8_t sm[];
    uint8_t *sA = sm;                              // 128 x K
    uint8_t *sB = sm + kProbeM * K;                // N x K
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sB + N * K);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int i = tid; i < kProbeM * K; i += blockDim.x) sA[kmajor_offset(i / K, i % K, K)] = A[i];
    for (int i = tid; i < N * K; i += blockDim.x) sB[kmajor_offset(i / K, i % K, K)] = B[i];
    uint32_t ncols = 32;
    while ((int)ncols < N) ncols <<= 1;
    if (warp == 0) tmem_alloc(smem_addr(tslot), ncols);
    if (tid == 0) {
        mbar_init(smem_addr(mbar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    if (tid == 0) {
        const uint32_t idesc = idesc_f8f6f4_e4m3_f32(kProbeM, N);
        const uint32_t a0 = smem_addr(sA), b0 = smem_addr(sB);
        for (int kk = 0; kk < K / 32; ++kk) {
            // 32 bytes of K = two core matrices along K, 128 bytes apart
            const uint64_t ad = smem_desc(a0 + kk * 256, 128, (uint32_t)(K / 16) * 128);
            const uint64_t bd = smem_desc(b0 + kk * 256, 128, (uint32_t)(K / 16) * 128);
            mma_f8f6f4(tmem, ad, bd, idesc, kk > 0 ? 1u : 0u);
        }
        mma_commit(smem_addr(mbar));
    }
    const bool ok = mbar_wait(smem_addr(mbar), 0, 20000000ll);
    if (!ok && lane == 0) atomicExch(status, 1);
    tc_fence_after();
    if (ok) {
        const int row = warp * 32 + lane;  // TMEM lane = row of D
        for (int c = 0; c < N; c += 32) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
#pragma unroll
            for (int i = 0; i < 32; ++i) D[(size_t)row * N + c + i] = v[i];
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, ncols);
}

}  // namespace
}  // namespace mdist

extern "C" int mdist_tc_probe(const uint8_t *A, const uint8_t *B, int N, int K, float *D) {
    using namespace mdist;
    if (!A || !B || !D || N < 32 || N > 256 || (N % 32) || K < 32 || K > 256 || (K % 32)) return MDIST_EINVAL;
    uint8_t *dA = nullptr, *dB = nullptr;
    float *dD = nullptr;
    int *dst = nullptr;
    int rc = MDIST_OK;
    const size_t smem = (size_t)(128 + N) * K + 16;
    if (cudaMalloc(&dA, 128 * (size_t)K) != cudaSuccess || cudaMalloc(&dB, (size_t)N * K) != cudaSuccess ||
        cudaMalloc(&dD, sizeof(float) * 128 * (size_t)N) != cudaSuccess || cudaMalloc(&dst, sizeof(int)) != cudaSuccess) {
        rc = MDIST_ENOMEM;
    } else {
        cudaMemcpy(dA, A, 128 * (size_t)K, cudaMemcpyHostToDevice);
        cudaMemcpy(dB, B, (size_t)N * K, cudaMemcpyHostToDevice);
        cudaMemset(dD, 0, sizeof(float) * 128 * (size_t)N);
        cudaMemset(dst, 0, sizeof(int));
        cudaFuncSetAttribute(tc_probe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        tc_probe_kernel<<<1, 128, smem>>>(dA, dB, dD, N, K, dst);
        int st = 0;
        if (cudaDeviceSynchronize() != cudaSuccess || cudaGetLastError() != cudaSuccess) rc = MDIST_ECUDA;
        else {
            cudaMemcpy(&st, dst, sizeof(int), cudaMemcpyDeviceToHost);
            cudaMemcpy(D, dD, sizeof(float) * 128 * (size_t)N, cudaMemcpyDeviceToHost);
            if (st) rc = MDIST_ETIMEOUT;
        }
    }
    cudaFree(dA);
    cudaFree(dB);
    cudaFree(dD);
    cudaFree(dst);
    return rc;
}
