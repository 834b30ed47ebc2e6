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
// address: its device address is looked up with cudaGetSymbolAddress on the first
// call made in a CUDA context (the context current on the calling thread, with its
// device), so that first call should be made before any stream capture starts.  The
// address belongs to that context: it is cached under the context's unique id, so a
// context created later (after cudaDeviceReset, or a driver-API context the caller
// makes current) gets its own lookup.  Every call shares the array and it keeps the
// last call's contents; each call clears what must start at zero before the
// enumeration runs.  Calls whose work overlaps on the GPU (different streams, or
// different host threads on one device) race on the array: serialise them.
#include <cuda.h>  // driver types only: the two driver calls are fetched at run time

#include <mutex>

#include "internal.h"

namespace mdist {

using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);

// Unique id of the context current on the calling thread (MDIST_OK), kNoContext when
// none is current yet, MDIST_ECUDA when the driver calls are unavailable.  The two
// driver entry points are fetched once, through the runtime.
int current_context_id(unsigned long long *id) {
    static std::once_flag once;
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    std::call_once(once, [] {
        void *f0 = nullptr, *f1 = nullptr;
        cudaDriverEntryPointQueryResult q0, q1;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f0, 12000, cudaEnableDefault, &q0) == cudaSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            q0 == cudaDriverEntryPointSuccess && q1 == cudaDriverEntryPointSuccess && f0 && f1) {
            get_current = (CtxGetCurrentFn)f0;
            get_id = (CtxGetIdFn)f1;
        }
    });
    if (!get_current || !get_id) return MDIST_ECUDA;
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS) return MDIST_ECUDA;
    if (!ctx) return kNoContext;
    if (get_id(ctx, id) != CUDA_SUCCESS) return MDIST_ECUDA;
    return MDIST_OK;
}

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
        s->slot.tc_cand = 0;
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

// Per-context set-up: the scratch array's device address and the SM count, cached
// under the unique id of the CUDA context current on the calling thread.
constexpr int kMaxContexts = 64;
struct ContextEntry {
    unsigned long long ctx_id;
    void *addr;
    int sms;
};
std::mutex g_setup_mu;
ContextEntry g_ctx[kMaxContexts];
int g_nctx = 0;
int g_next_evict = 0;

int noalloc_setup(int dev, void **addr, int *sms) {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    unsigned long long id = 0;
    void *p = nullptr;
    cudaError_t e = cudaSuccess;
    int rc = current_context_id(&id);
    if (rc == kNoContext) {
        // no context yet: the symbol lookup makes the runtime's context current
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            if (e != cudaSuccess) cudaGetLastError();  // this call's own error, not the caller's
            return MDIST_ECUDA;
        }
        rc = current_context_id(&id);
    }
    if (rc != MDIST_OK) return MDIST_ECUDA;
    for (int i = 0; i < g_nctx; ++i)
        if (g_ctx[i].ctx_id == id) {
            *addr = g_ctx[i].addr;
            *sms = g_ctx[i].sms;
            return MDIST_OK;
        }
    if (!p) {
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            if (e != cudaSuccess) cudaGetLastError();
            return MDIST_ECUDA;
        }
    }
    int n = 0;
    e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return MDIST_ECUDA;
    }
    // context ids are never reused, so a full table drops its oldest entries
    const int slot = g_nctx < kMaxContexts ? g_nctx++ : (g_next_evict++ % kMaxContexts);
    g_ctx[slot] = ContextEntry{id, p, n};
    *addr = p;
    *sms = n;
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
    // an error the caller has not collected yet stays theirs: report it, clear nothing
    if (cudaPeekAtLastError() != cudaSuccess) return MDIST_ECUDA;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
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
    // nothing was pending on entry, so each error collected below is this call's own
    noalloc_init<<<1, 256, 0, stream>>>((unsigned int)U, bins);
    if (cudaGetLastError() != cudaSuccess) return MDIST_ECUDA;
    if (launch_enum_unit(p, nwords, 0, want_hist != 0, sms, 0, stream) != cudaSuccess) {
        cudaGetLastError();
        return MDIST_ECUDA;
    }
    noalloc_finish<<<1, 256, 0, stream>>>(out, bins);
    if (cudaGetLastError() != cudaSuccess) return MDIST_ECUDA;
    return MDIST_OK;
}
