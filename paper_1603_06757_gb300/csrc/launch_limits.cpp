// launch_limits.cpp -- kernel launch settings shared by every handle and host thread of
// the process, kept per CUDA context: a kernel's dynamic shared-memory limit only ever
// rises (had one thread lowered it between another thread's setting and launch, that
// launch would fail), and occupancy answers are remembered, so a launch costs neither
// call after the first.
#include <map>
#include <mutex>
#include <tuple>

#include "internal.h"

namespace mdist {
namespace {

std::mutex g_mu;
std::map<std::pair<unsigned long long, const void *>, size_t> g_smem;  // (context, kernel) -> limit
std::map<std::tuple<unsigned long long, const void *, int, size_t>, int> g_occ;

}  // namespace

cudaError_t allow_dynamic_smem(const void *func, size_t bytes) {
    unsigned long long ctx = 0;
    if (current_context_id(&ctx) != MDIST_OK)  // no id: set it, remember nothing
        return cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_smem.find({ctx, func});
    if (it != g_smem.end() && it->second >= bytes) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) g_smem[{ctx, func}] = bytes;
    return e;
}

cudaError_t blocks_per_sm(const void *func, int threads, size_t smem, int *occ) {
    unsigned long long ctx = 0;
    if (current_context_id(&ctx) != MDIST_OK)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, func, threads, smem);
    std::lock_guard<std::mutex> lock(g_mu);
    const auto key = std::make_tuple(ctx, func, threads, smem);
    auto it = g_occ.find(key);
    if (it != g_occ.end()) {
        *occ = it->second;
        return cudaSuccess;
    }
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, func, threads, smem);
    if (e == cudaSuccess) g_occ[key] = *occ;
    return e;
}

}  // namespace mdist
