// noalloc.cu -- one (g, j) unit of the level enumerator for callers that cannot
// allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is off limits -- a host process whose
// device memory is owned by another allocator or pool it must not bypass, a plugin
// called inside someone else's tight memory budget, or a step that must not touch
// the allocator while other work holds its locks.  Such a caller already holds the
// rows of Gamma_j on the device and a small output buffer; this entry point needs
// nothing else.
//
// The enumerator's scratch state (threshold U, best key, combination count, work
// counter, and the weight histogram when asked for) lives in the file-scope array
// `g_noalloc_scratch` below, a fixed 8 KiB that every GPU loading the library keeps
// until the process exits.  Host code must not use the array's name as a device
// address: its device address is looked up once per device with
// cudaGetSymbolAddress (with that device current) on the first call made on that
// device, so that first call should be made before any stream capture starts.
// Every call shares the array and it keeps the last call's contents; each call
// clears what must start at zero before the enumeration runs.  Calls whose work
// overlaps on the GPU (different streams, or different host threads on one device)
// race on the array: serialise them.
#include <mutex>

#include "internal.h"

namespace mdist {
namespace {

constexpr int kNoAllocHistBins = MDIST_NOALLOC_MAX_HIST_BINS;
constexpr size_t kNoAllocScratchBytes = 8192;

struct NoAllocScratch {
    UnitSlot slot;
    unsigned long long hist[kNoAllocHistBins];
};
static_assert(sizeof(NoAllocScratch) <= kNoAllocScratchBytes, "scratch layout");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Clear the scratch and set the threshold; device code names the array directly.
__global__ void noalloc_init(unsigned int U, int bins) {
    NoAllocScratch *s = reinterpret_cast<NoAllocScratch *>(g_noalloc_scratch);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        s->slot.U = U;
        s->slot.status = 0;
        s->slot.key = kNoKey;
        s->slot.count = 0;
        s->slot.tile_next = 0;
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < bins; i += gridDim.x * blockDim.x) s->hist[i] = 0;
}

// Copy the results to the caller's output buffer.
__global__ void noalloc_finish(unsigned long long *out, int bins) {
    const NoAllocScratch *s = reinterpret_cast<const NoAllocScratch *>(g_noalloc_scratch);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        out[0] = s->slot.U;
        out[1] = s->slot.key;
        out[2] = s->slot.count;
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < bins; i += gridDim.x * blockDim.x) out[3 + i] = s->hist[i];
}

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void *g_scratch_addr[kMaxDevices];
int g_sm_count[kMaxDevices];

// Per-device set-up: the scratch array's device address and the SM count.
int noalloc_setup(int dev, void **addr, int *sms) {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return MDIST_ECUDA;
        }
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return MDIST_ECUDA;
        }
        g_sm_count[dev] = n;
        g_scratch_addr[dev] = p;
    }
    *addr = g_scratch_addr[dev];
    *sms = g_sm_count[dev];
    return MDIST_OK;
}

}  // namespace
}  // namespace mdist

extern "C" int mdist_enumerate_unit_noalloc(const uint32_t *rows, int k, int nwords, int n_bits, int full_rank,
                                            int g, int U, int want_hist, unsigned long long *out, void *cuda_stream) {
    using namespace mdist;
    if (!rows || !out || k < 1 || k > MDIST_MAX_K || nwords < 1 || nwords > kMaxWords32 || n_bits < 1 ||
        n_bits > 32 * nwords || g < 1 || g > k || U < 0)
        return MDIST_EINVAL;
    const int base = full_rank ? g : 0;
    const int bins = want_hist ? n_bits + base + 1 : 0;
    if (bins > kNoAllocHistBins) return MDIST_ERANGE;  // histogram larger than the scratch holds
    EnumParams p{};
    if (!plan_level(k, g, nwords, p)) return MDIST_ERANGE;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return MDIST_ECUDA;
    }
    void *scratch = nullptr;
    int sms = 0;
    const int rc = noalloc_setup(dev, &scratch, &sms);
    if (rc != MDIST_OK) return rc;
    NoAllocScratch *s = reinterpret_cast<NoAllocScratch *>(scratch);
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    p.rows = rows;
    p.U = &s->slot.U;
    p.slot = &s->slot;
    p.hist = want_hist ? s->hist : nullptr;
    p.nwords = nwords;
    p.n_bits = n_bits;
    p.base = base;
    noalloc_init<<<1, 256, 0, stream>>>((unsigned int)U, bins);
    if (cudaGetLastError() != cudaSuccess) return MDIST_ECUDA;
    if (launch_enum_unit(p, nwords, 0, want_hist != 0, sms, 0, stream) != cudaSuccess) return MDIST_ECUDA;
    noalloc_finish<<<1, 256, 0, stream>>>(out, bins);
    if (cudaGetLastError() != cudaSuccess) return MDIST_ECUDA;
    return MDIST_OK;
}
