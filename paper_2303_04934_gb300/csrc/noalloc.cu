// reach_multi_noalloc: multi-source reachability for callers that cannot
// allocate device memory during the call.
//
// Some callers may not call cudaMalloc (or any allocating routine) at the
// point where they need a result: latency-critical loops that forbid allocator
// calls, because an allocation can block or synchronise the device, and hosts
// whose device memory is owned by their own allocator, where a library's
// allocation would bypass that allocator's accounting. This entry point serves
// them: it takes a graph handle (created earlier) and device buffers for the
// sources and the result, and it takes its working memory -- the two hash-bag
// slot arrays, the hub lists and the control block of the reachability engine
// -- from one fixed, file-scope device array instead of allocating. It
// launches the same engine kernel as reach_multi.
//
// The array is kNoAllocScratchBytes (32 MiB) per device and lives as long as
// the library is loaded on that device. Every call shares it and it keeps the
// previous call's contents, so each call resets what must start empty; two
// calls whose work overlaps on the GPU (for instance on two streams) race on it.
#include <cstring>

#include "../../include/scc.h"
#include "common.cuh"
#include "engine.cuh"
#include "internal.h"

namespace scc {

constexpr size_t kNoAllocScratchBytes = 32ull << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

// Device address of the scratch array on the current device, looked up on every
// call (host code must not use the symbol's host-side name as a pointer). A
// cached address would go stale when the module is loaded again after a
// cudaDeviceReset or a new primary context; the lookup is no stream operation
// and costs microseconds.
int scratch_address(unsigned char** out) {
    void* p = nullptr;
    SCC_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    *out = static_cast<unsigned char*>(p);
    return SCC_OK;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Carve the engine buffers for vertex items out of the scratch array; returns
// the bytes needed (the layout is only written when base != nullptr).
size_t carve(unsigned char* base, int32_t n, int64_t mt, int lambda, int num_sms, EngineBuf* b, int** bad) {
    long long items = std::max<long long>(2ll * n + 1024, lambda);
    long long nslots = (std::max<long long>(4 * items, 4ll * lambda) + bag_warp_slots(num_sms) + kSeg - 1) / kSeg * kSeg;
    int hub_cap = (int)std::min<long long>(items, 8192);
    long long segmap_cap = 2 * (mt / kHubSeg) + hub_cap + 1024;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t at = off;
        off = align256(off + bytes);
        return base ? base + at : nullptr;
    };
    unsigned char* ctl = take(sizeof(EngineCtl));
    unsigned char* badp = take(sizeof(int));
    void* slots[2];
    void* hub_item[2];
    void* hub_beg[2];
    void* hub_deg[2];
    void* hub_segbase[2];
    void* segmap[2];
    for (int k = 0; k < 2; ++k) {
        slots[k] = take((size_t)nslots * 4);
        hub_item[k] = take((size_t)hub_cap * 4);
        hub_beg[k] = take((size_t)hub_cap * 4);
        hub_deg[k] = take((size_t)hub_cap * 4);
        hub_segbase[k] = take((size_t)hub_cap * 8);
        segmap[k] = take((size_t)segmap_cap * 4);
    }
    if (base) {
        *b = EngineBuf();
        b->item_bytes = 4;
        b->nslots = nslots;
        b->items = items;
        b->hub_cap = hub_cap;
        b->segmap_cap = segmap_cap;
        b->lambda = lambda;
        b->ctl = reinterpret_cast<EngineCtl*>(ctl);
        for (int k = 0; k < 2; ++k) {
            b->slots[k] = slots[k];
            b->hub_item[k] = hub_item[k];
            b->hub_beg[k] = static_cast<int32_t*>(hub_beg[k]);
            b->hub_deg[k] = static_cast<int32_t*>(hub_deg[k]);
            b->hub_segbase[k] = static_cast<long long*>(hub_segbase[k]);
            b->segmap[k] = static_cast<int32_t*>(segmap[k]);
        }
        *bad = reinterpret_cast<int*>(badp);
    }
    return off;
}

}  // namespace

int reach_multi_noalloc_impl(const int32_t* off, const int32_t* adj, int32_t n, int64_t mt, int lambda,
                             const EngineOpts& o, const int32_t* sources, int32_t k, uint64_t* out,
                             cudaStream_t s) {
    if (carve(nullptr, n, mt, lambda, o.num_sms, nullptr, nullptr) > kNoAllocScratchBytes) return SCC_ERR_INVALID_ARG;
    unsigned char* base = nullptr;
    SCC_TRY(scratch_address(&base));
    EngineBuf b;
    int* bad = nullptr;
    carve(base, n, mt, lambda, o.num_sms, &b, &bad);
    // what must start empty: the bag, the control block, the result and the flag
    for (int j = 0; j < 2; ++j) SCC_CUDA(cudaMemsetAsync(b.slots[j], 0xff, (size_t)b.nslots * 4, s));
    SCC_CUDA(cudaMemsetAsync(b.ctl, 0, sizeof(EngineCtl), s));
    SCC_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
    SCC_CUDA(cudaMemsetAsync(out, 0, (size_t)n * 8, s));
    auto* mask = reinterpret_cast<unsigned long long*>(out);
    SCC_TRY(launch_mask_init(sources, k, n, 1, mask, bad, s));
    int hbad = 0;
    SCC_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    SCC_CUDA(cudaStreamSynchronize(s));
    if (hbad) return SCC_ERR_INVALID_ARG;
    EngineRun r;
    SCC_TRY(run_mask_fixed(off, adj, n, sources, k, mask, &b, o, &r, s));
    return r.err ? r.err : SCC_OK;
}

}  // namespace scc
