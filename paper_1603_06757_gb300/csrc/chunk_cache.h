// chunk_cache.h -- device memory for the single-code handles that the batched engine
// and the serving loop run one after the other: chunks rounded up to 2 MiB (64 MiB and
// above: to a power of two) are kept after a handle frees them and handed out again, so
// a stream of handles costs a few cudaMalloc calls instead of several per handle.  Host
// code only; not thread-safe (each owner drives its handles from one thread).
#pragma once

#include <cstddef>
#include <map>

#include <cuda_runtime.h>

namespace mdist {

struct ChunkCache {
    std::multimap<size_t, void *> free_chunks;  // size -> chunk
    std::map<void *, size_t> size_of;           // every chunk ever allocated

    static size_t rounded(size_t bytes) {
        size_t size = (bytes + (2u << 20) - 1) / (2u << 20) * (2u << 20);
        if (size >= (64u << 20)) {
            size_t p2 = 64u << 20;
            while (p2 < size) p2 <<= 1;
            size = p2;
        }
        return size;
    }
    // mdist_options.dev_alloc / dev_free with ctx = the cache
    static void *alloc(size_t bytes, void *ctx) {
        ChunkCache *c = static_cast<ChunkCache *>(ctx);
        const size_t size = rounded(bytes);
        auto it = c->free_chunks.find(size);
        if (it != c->free_chunks.end()) {
            void *p = it->second;
            c->free_chunks.erase(it);
            return p;
        }
        void *p = nullptr;
        if (cudaMalloc(&p, size) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        c->size_of[p] = size;
        return p;
    }
    static void release(void *p, void *ctx) {
        ChunkCache *c = static_cast<ChunkCache *>(ctx);
        auto it = c->size_of.find(p);
        if (it != c->size_of.end()) c->free_chunks.emplace(it->second, p);
    }
    // every chunk back to the device (the handles using them must be gone)
    void clear() {
        for (auto &kv : size_of) cudaFree(kv.first);
        size_of.clear();
        free_chunks.clear();
    }
};

}  // namespace mdist
