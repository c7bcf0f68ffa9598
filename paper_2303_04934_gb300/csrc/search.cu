// Reachability searches: instantiation and cooperative launch of the VGC /
// hash-bag engine (engine.cuh) for single-reachability (first SCC, Sec. 4.2),
// multi-reachability (Alg. 1; Sec. 4.3) and plain multi-source masks.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "engine.cuh"
#include "internal.h"

namespace scc {

namespace {

// The initial multi-reachability items of a batch: the pair (s, s) of every
// source (Alg. 1: each source reaches itself).
__global__ void k_pairs_from_sources(const int32_t* __restrict__ src, int32_t k, uint64_t* out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) {
        uint32_t s = (uint32_t)src[i];
        out[i] = ((uint64_t)s << 32) | s;
    }
}

template <class Pol>
int coop_grid(int num_sms, int* grid) {
    static int cached = -1;
    if (cached < 0) {
        int per_sm = 0;
        SCC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, engine_kernel<Pol>, kEngineBlock, 0));
        if (per_sm < 1) return SCC_ERR_CUDA;
        cached = engine_blocks_per_sm(per_sm);
    }
    *grid = cached * num_sms;
    return SCC_OK;
}

template <class Pol>
int launch_engine(EngineParams<typename Pol::Item>& P, Pol& pol, const EngineOpts& o, EngineRun* out,
                  cudaStream_t st, DenseParams dp = DenseParams{nullptr, nullptr, {nullptr, nullptr}, 0, 0}) {
    int grid = 0;
    SCC_TRY(coop_grid<Pol>(o.num_sms, &grid));
    SCC_CUDA(cudaMemsetAsync(P.ctl, 0, sizeof(EngineCtl), st));
    void* args[] = {(void*)&P, (void*)&pol, (void*)&dp};
    cudaEvent_t e0, e1;
    SCC_CUDA(cudaEventCreate(&e0));
    SCC_CUDA(cudaEventCreate(&e1));
    cudaEventRecord(e0, st);
    cudaError_t le =
        cudaLaunchCooperativeKernel((const void*)engine_kernel<Pol>, dim3(grid), dim3(kEngineBlock), args, 0, st);
    count_launch();
    cudaEventRecord(e1, st);
    EngineCtl h;
    cudaError_t ce = cudaMemcpyAsync(&h, P.ctl, sizeof(EngineCtl), cudaMemcpyDeviceToHost, st);
    cudaError_t se = cudaStreamSynchronize(st);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    SCC_CUDA(le);
    SCC_CUDA(ce);
    SCC_CUDA(se);
    out->ms = ms;
    out->items = h.items;
    out->err = h.err;
    out->overflow = h.search[0].overflow;
    out->rounds = h.search[0].rounds;
    out->max_chunk = h.max_chunk;
    out->edges = h.edges;
    out->inserted = h.search[0].inserted[0] + h.search[0].inserted[1];
    static const bool trace = getenv("SCC_TRACE") != nullptr;
    if (trace) {  // per-round timeline of this search on stderr
        const int nr = std::min(h.search[0].rounds, kTraceRounds);
        fprintf(stderr, "[scc-trace] %s: %d rounds, %.1f us in kernel\n", Pol::kName, h.search[0].rounds,
                1000.0 * ms);
        unsigned long long t = h.t0;
        for (int r = 0; r < nr; ++r) {
            fprintf(stderr, "[scc-trace]   round %2d %s %9.1f us  items %lld\n", r, (h.t_dense[r] & 1) ? "dense " : "sparse",
                    (h.t_end[r] - t) / 1000.0, h.t_items[r]);
            t = h.t_end[r];
        }
    }
    if (h.err != 0 && h.err != SCC_ERR_CAPACITY) return h.err;
    return SCC_OK;
}

}  // namespace

template <class Item>
EngineParams<Item> make_engine_params(const int32_t* off, const int32_t* adj, int32_t n, const EngineBuf* b,
                                      const EngineOpts& o) {
    EngineParams<Item> P;
    memset(&P, 0, sizeof(P));
    P.off = off;
    P.adj = adj;
    P.n = n;
    P.tau = o.tau;
    P.hub_thr = o.tau;
    P.seeds = o.seeds;
    for (int k = 0; k < 2; ++k) {
        P.slots[k] = (Item*)b->slots[k];
        P.hub_item[k] = (Item*)b->hub_item[k];
        P.hub_beg[k] = b->hub_beg[k];
        P.hub_deg[k] = b->hub_deg[k];
        P.hub_segbase[k] = b->hub_segbase[k];
        P.segmap[k] = b->segmap[k];
    }
    P.nslots = b->nslots;
    P.lambda = b->lambda;
    P.sigma = o.sigma;
    P.hub_cap = b->hub_cap;
    P.segmap_cap = b->segmap_cap;
    P.ctl = b->ctl;
    return P;
}
template EngineParams<uint32_t> make_engine_params<uint32_t>(const int32_t*, const int32_t*, int32_t,
                                                             const EngineBuf*, const EngineOpts&);
template EngineParams<uint64_t> make_engine_params<uint64_t>(const int32_t*, const int32_t*, int32_t,
                                                             const EngineBuf*, const EngineOpts&);

namespace {

int reserve_init(EngineBuf* b, size_t bytes, cudaStream_t st) {
    if (b->init && b->init_bytes >= bytes) return SCC_OK;
    dfree(b->init, st);
    b->init = nullptr;
    size_t want = std::max<size_t>(bytes, 1 << 16);
    SCC_TRY(dalloc(&b->init, want, st));
    b->init_bytes = want;
    return SCC_OK;
}

}  // namespace

// Restore an all-empty bag after a run that stopped early (error or overflow).
int engine_reset_slots(EngineBuf* b, cudaStream_t st) {
    for (int k = 0; k < 2; ++k)
        if (b->slots[k]) SCC_CUDA(cudaMemsetAsync(b->slots[k], 0xff, (size_t)b->nslots * b->item_bytes, st));
    return SCC_OK;
}

int engine_reserve(EngineBuf* b, int item_bytes, long long items, int lambda, int64_t m, int num_sms, cudaStream_t s) {
    if (items < 1) items = 1;
    // every warp that pushes holds a partly filled 32-slot segment, so the bag
    // needs room for two segments per warp of the largest grid besides the items
    long long need_slots = std::max<long long>(4 * items, 4ll * lambda) + bag_warp_slots(num_sms);
    need_slots = (need_slots + kSeg - 1) / kSeg * kSeg;
    if (b->slots[0] && b->item_bytes == item_bytes && b->nslots >= need_slots && b->lambda == lambda &&
        b->items >= items)
        return SCC_OK;
    engine_release(b, s);
    b->item_bytes = item_bytes;
    b->lambda = lambda;
    b->nslots = need_slots;
    b->items = items;
    b->hub_cap = (int)std::min<long long>(items, 1ll << 22);
    b->segmap_cap = 2 * (m / kHubSeg) + b->hub_cap + 1024;
    for (int k = 0; k < 2; ++k) {
        SCC_TRY(dalloc(&b->slots[k], (size_t)b->nslots * item_bytes, s));
        SCC_TRY(dalloc(&b->hub_item[k], (size_t)b->hub_cap * item_bytes, s));
        SCC_TRY(dalloc_t(&b->hub_beg[k], b->hub_cap, s));
        SCC_TRY(dalloc_t(&b->hub_deg[k], b->hub_cap, s));
        SCC_TRY(dalloc_t(&b->hub_segbase[k], b->hub_cap, s));
        SCC_TRY(dalloc_t(&b->segmap[k], b->segmap_cap, s));
        SCC_CUDA(cudaMemsetAsync(b->slots[k], 0xff, (size_t)b->nslots * item_bytes, s));
    }
    SCC_TRY(dalloc(reinterpret_cast<void**>(&b->ctl), sizeof(EngineCtl), s));
    SCC_CUDA(cudaMemsetAsync(b->ctl, 0, sizeof(EngineCtl), s));
    return SCC_OK;
}

void engine_release(EngineBuf* b, cudaStream_t s) {
    for (int k = 0; k < 2; ++k) {
        dfree(b->slots[k], s);
        dfree(b->hub_item[k], s);
        dfree(b->hub_beg[k], s);
        dfree(b->hub_deg[k], s);
        dfree(b->hub_segbase[k], s);
        dfree(b->segmap[k], s);
    }
    dfree(b->ctl, s);
    dfree(b->init, s);
    *b = EngineBuf();
}

int run_single(const int32_t* off, const int32_t* adj, int32_t n, int32_t s, uint32_t* bits, const DenseOpts& dn,
               EngineBuf* b, const EngineOpts& o, EngineRun* out, cudaStream_t st) {
    auto P = make_engine_params<uint32_t>(off, adj, n, b, o);
    SCC_TRY(reserve_init(b, sizeof(uint32_t), st));
    SCC_CUDA(cudaMemcpyAsync(b->init, &s, sizeof(int32_t), cudaMemcpyHostToDevice, st));
    P.init = reinterpret_cast<const uint32_t*>(b->init);
    P.ninit = 1;
    PolSingle pol{bits};
    DenseParams dp{dn.roff, dn.radj, {dn.fbits[0], dn.fbits[1]}, dn.n_active, dn.frac_inv, dn.m_active};
    int rc = launch_engine(P, pol, o, out, st, dp);
    if (rc != SCC_OK || out->err) SCC_TRY(engine_reset_slots(b, st));
    SCC_TRY(rc);
    return out->err ? out->err : SCC_OK;
}

int run_single_both(const int32_t* off, const int32_t* adj, const int32_t* toff, const int32_t* tadj, int32_t n,
                    int32_t s, uint32_t* bits_f, uint32_t* bits_b, EngineBuf* b, const EngineOpts& o, EngineRun* out,
                    cudaStream_t st) {
    if (n >= INT32_MAX - 2) return SCC_ERR_INVALID_ARG;  // ids must stay clear of the direction bit's sentinels
    auto P = make_engine_params<uint32_t>(off, adj, n, b, o);
    P.off2 = toff;
    P.adj2 = tadj;
    SCC_TRY(reserve_init(b, 2 * sizeof(uint32_t), st));
    const uint32_t init[2] = {(uint32_t)s, (uint32_t)s | PolSingleBoth::kDir};
    SCC_CUDA(cudaMemcpyAsync(b->init, init, sizeof(init), cudaMemcpyHostToDevice, st));
    SCC_CUDA(cudaStreamSynchronize(st));  // init is a stack array
    P.init = reinterpret_cast<const uint32_t*>(b->init);
    P.ninit = 2;
    PolSingleBoth pol;
    pol.bits[0] = bits_f;
    pol.bits[1] = bits_b;
    int rc = launch_engine(P, pol, o, out, st);
    if (rc != SCC_OK || out->err) SCC_TRY(engine_reset_slots(b, st));
    SCC_TRY(rc);
    return out->err ? out->err : SCC_OK;
}

int run_ldd(const int32_t* soff, const int32_t* sadj, int32_t n, long long soff_arcs, const int32_t* order,
            const long long* bounds_d, long long first, int nbatches, int32_t* center, uint32_t* bits, uint32_t* fbits,
            int frac_inv, EngineBuf* b, const EngineOpts& o, EngineRun* out, cudaStream_t st) {
    auto P = make_engine_params<uint32_t>(soff, sadj, n, b, o);
    P.init = reinterpret_cast<const uint32_t*>(order);  // the first batch, claimed before the launch
    P.ninit = first;
    PolLdd pol;
    pol.center = center;
    pol.bits = bits;
    pol.off = soff;
    pol.order = order;
    pol.bounds = bounds_d;
    pol.nbatches = nbatches;
    // the graph is symmetric: it is its own reverse for the bottom-up rounds
    const long long nw = ((long long)n + 31) / 32;
    DenseParams dp{soff, sadj, {fbits, fbits + nw}, (long long)n, frac_inv, soff_arcs};
    int rc = launch_engine(P, pol, o, out, st, dp);
    if (rc != SCC_OK || out->err) SCC_TRY(engine_reset_slots(b, st));
    SCC_TRY(rc);
    return out->err ? out->err : SCC_OK;
}

int run_pairs(const int32_t* off, const int32_t* adj, int32_t n, const int32_t* label, const int32_t* sources,
              int32_t k, unsigned long long* table, int64_t cap, long long max_inserted, EngineBuf* b,
              const EngineOpts& o, EngineRun* out, cudaStream_t st) {
    auto P = make_engine_params<uint64_t>(off, adj, n, b, o);
    SCC_TRY(reserve_init(b, (size_t)k * sizeof(uint64_t), st));
    uint64_t* init = reinterpret_cast<uint64_t*>(b->init);
    k_pairs_from_sources<<<std::max(1, std::min(1024, (k + 255) / 256)), 256, 0, st>>>(sources, k, init);
    SCC_LAUNCH();
    P.init = init;
    P.ninit = k;
    PolPair pol;  // every item in direction 0: one table, graph (off, adj)
    pol.label = label;
    pol.keys[0] = pol.keys[1] = table;
    pol.mask[0] = pol.mask[1] = (unsigned long long)(cap - 1);
    pol.max_ins[0] = pol.max_ins[1] = max_inserted;
    pol.overflow = &b->ctl->search[0].overflow;  // a standalone launch is search 0
    pol.ins0 = pol.ins1 = 0;
    int rc = launch_engine(P, pol, o, out, st);
    if (rc != SCC_OK || out->err || out->overflow) {
        int r2 = engine_reset_slots(b, st);
        if (rc == SCC_OK) rc = r2;
    }
    SCC_TRY(rc);
    return out->err ? out->err : SCC_OK;
}

int run_mask(const int32_t* off, const int32_t* adj, int32_t n, const int32_t* sources, int32_t k,
             unsigned long long* mask, EngineBuf* b, const EngineOpts& o, EngineRun* out, cudaStream_t st) {
    auto P = make_engine_params<uint32_t>(off, adj, n, b, o);
    P.init = reinterpret_cast<const uint32_t*>(sources);
    P.ninit = k;
    PolMask pol{mask, o.high_degree};
    int rc = launch_engine(P, pol, o, out, st);
    if (rc != SCC_OK || out->err) SCC_TRY(engine_reset_slots(b, st));
    SCC_TRY(rc);
    return out->err ? out->err : SCC_OK;
}

// reach_multi with up to 128 sources (two mask words per vertex).
int run_mask2(const int32_t* off, const int32_t* adj, int32_t n, const int32_t* sources, int32_t k,
              unsigned long long* mask2, EngineBuf* b, const EngineOpts& o, EngineRun* out, cudaStream_t st) {
    auto P = make_engine_params<uint32_t>(off, adj, n, b, o);
    P.init = reinterpret_cast<const uint32_t*>(sources);
    P.ninit = k;
    PolMask2 pol{mask2, o.high_degree};
    int rc = launch_engine(P, pol, o, out, st);
    if (rc != SCC_OK || out->err) SCC_TRY(engine_reset_slots(b, st));
    SCC_TRY(rc);
    return out->err ? out->err : SCC_OK;
}

// Mask reachability on caller-provided (fixed) engine buffers: no device
// allocation and no CUDA event; the caller has emptied the bag and the control
// block. A search that needs more bag space than the buffers hold returns
// SCC_ERR_CAPACITY.
int run_mask_fixed(const int32_t* off, const int32_t* adj, int32_t n, const int32_t* sources, int32_t k,
                   unsigned long long* mask, const EngineBuf* b, const EngineOpts& o, EngineRun* out,
                   cudaStream_t st) {
    auto P = make_engine_params<uint32_t>(off, adj, n, b, o);
    P.init = reinterpret_cast<const uint32_t*>(sources);
    P.ninit = k;
    PolMask pol{mask, o.high_degree};
    DenseParams dp{nullptr, nullptr, {nullptr, nullptr}, 0, 0};
    int grid = 0;
    SCC_TRY(coop_grid<PolMask>(o.num_sms, &grid));
    void* args[] = {(void*)&P, (void*)&pol, (void*)&dp};
    SCC_CUDA(cudaLaunchCooperativeKernel((const void*)engine_kernel<PolMask>, dim3(grid), dim3(kEngineBlock), args, 0,
                                         st));
    count_launch();
    EngineCtl h;
    SCC_CUDA(cudaMemcpyAsync(&h, P.ctl, sizeof(EngineCtl), cudaMemcpyDeviceToHost, st));
    SCC_CUDA(cudaStreamSynchronize(st));
    out->err = h.err;
    out->rounds = h.search[0].rounds;
    out->edges = h.edges;
    out->items = h.items;
    return h.err ? h.err : SCC_OK;
}

// ---------------------------------------------------------- hash bag test --
namespace {

struct BagOnlyParams {
    uint32_t* slots;
    long long nslots;
    int lambda;
    int sigma;
    EngineCtl* ctl;
};

// The hash bag alone (Sec. 3.3): every warp inserts a strided share of the items
// (Insert), one grid barrier, then ExtractAll compacts the bag into `out`; a
// test hook.
__global__ void __launch_bounds__(kEngineBlock) k_bag_only(BagOnlyParams P, const int32_t* __restrict__ items, long long count,
                                                  int32_t* out) {
    const int lane = lane_id();
    const uint32_t wid = (uint32_t)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5));
    const uint32_t nwarps = (uint32_t)(gridDim.x * (blockDim.x >> 5));
    SegState st{-1, 0, wid * 2654435761u};
    const BagRef<uint32_t> bag{P.slots, P.nslots, P.lambda, P.sigma, &P.ctl->ring[0].bag, &P.ctl->err,
                               &P.ctl->max_chunk};
    // every warp pushes a strided share, a few items at a time, as spills do
    for (long long b = (long long)wid * 32; b < count; b += (long long)nwarps * 32) {
        long long i = b + lane;
        bool has = i < count;
        uint32_t it = has ? (uint32_t)items[i] : 0u;
        // split each group of 32 into two pushes to exercise partial segments
        bag_push<uint32_t>(bag, st, has && lane < 13, it, wid, 0);
        bag_push<uint32_t>(bag, st, has && lane >= 13, it, wid, 0);
    }
    if (!grid_sync(&P.ctl->bar, &P.ctl->err)) return;
    // ExtractAll: warp-aggregated compaction of the used prefix
    const int r = ld_volatile(&P.ctl->ring[0].bag.r);
    const long long end = chunk_end(P.lambda, r, P.nslots);
    for (long long b = (long long)wid * 32; b < end; b += (long long)nwarps * 32) {
        long long i = b + lane;
        uint32_t x = i < end ? P.slots[i] : Sent<uint32_t>::empty;
        bool valid = x != Sent<uint32_t>::empty && x != Sent<uint32_t>::claimed;
        if (i < end && x != Sent<uint32_t>::empty) P.slots[i] = Sent<uint32_t>::empty;
        uint32_t msk = __ballot_sync(kFull, valid);
        long long base = 0;
        if (lane == 0 && msk)
            base = (long long)atomicAdd((unsigned long long*)&P.ctl->ring[1].items, (unsigned long long)__popc(msk));
        base = __shfl_sync(kFull, base, 0);
        if (valid) out[base + __popc(msk & lanemask_lt())] = (int32_t)x;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) P.ctl->ring[1].nhub = r;
}

// The grid barrier's failure path: every block but `absent` waits at one grid
// barrier with a limit of limit_ns; block `absent` (if any) returns without
// arriving, so the others' waits run out, record SCC_ERR_TIMEOUT in *err and
// return. arrived[b] = 1 for a block whose wait ended because all arrived.
__global__ void k_barrier_probe(GridBarrier* bar, int* err, int absent, unsigned long long limit_ns, int* arrived) {
    if ((int)blockIdx.x == absent) return;
    const bool ok = grid_sync_limit(bar, err, limit_ns);
    if (threadIdx.x == 0) arrived[blockIdx.x] = ok ? 1 : 0;
}

}  // namespace

int run_barrier_probe(int absent, int64_t limit_ns, int* n_arrived, cudaStream_t st) {
    DeviceInfo di;
    SCC_TRY(device_info(&di));
    int per_sm = 0;
    SCC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_barrier_probe, 32, 0));
    const int grid = std::max(1, std::min(per_sm, 2)) * di.num_sms;
    if (absent >= grid) return SCC_ERR_INVALID_ARG;
    Scratch tmp(st);
    GridBarrier* bar = nullptr;
    int* err = nullptr;
    int* arrived = nullptr;
    SCC_TRY(tmp.alloc(&bar, 1));
    SCC_TRY(tmp.alloc(&err, 1));
    SCC_TRY(tmp.alloc(&arrived, (size_t)grid));
    SCC_CUDA(cudaMemsetAsync(bar, 0, sizeof(GridBarrier), st));
    SCC_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    SCC_CUDA(cudaMemsetAsync(arrived, 0, sizeof(int) * (size_t)grid, st));
    unsigned long long lim = (unsigned long long)limit_ns;
    void* args[] = {(void*)&bar, (void*)&err, (void*)&absent, (void*)&lim, (void*)&arrived};
    SCC_CUDA(cudaLaunchCooperativeKernel((const void*)k_barrier_probe, dim3(grid), dim3(32), args, 0, st));
    count_launch();
    std::vector<int> h((size_t)grid);
    int herr = 0;
    SCC_CUDA(cudaMemcpyAsync(h.data(), arrived, sizeof(int) * (size_t)grid, cudaMemcpyDeviceToHost, st));
    SCC_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    SCC_CUDA(cudaStreamSynchronize(st));
    int c = 0;
    for (int x : h) c += x;
    *n_arrived = c;
    return herr;
}

int run_bag_only(const int32_t* items, int64_t count, int lambda, int sigma, int32_t* out, int64_t* nout,
                 int* chunks, cudaStream_t st) {
    DeviceInfo di;
    SCC_TRY(device_info(&di));
    BagOnlyParams P;
    P.lambda = lambda;
    P.sigma = sigma;
    P.nslots = (std::max<long long>(4 * count, 4ll * lambda) + bag_warp_slots(di.num_sms) + kSeg - 1) / kSeg * kSeg;
    Scratch tmp(st);
    SCC_TRY(tmp.alloc(&P.slots, (size_t)P.nslots));
    SCC_TRY(tmp.alloc(&P.ctl, 1));
    SCC_CUDA(cudaMemsetAsync(P.slots, 0xff, (size_t)P.nslots * 4, st));
    SCC_CUDA(cudaMemsetAsync(P.ctl, 0, sizeof(EngineCtl), st));
    int per_sm = 0;
    SCC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bag_only, kEngineBlock, 0));
    int grid = std::max(1, engine_blocks_per_sm(per_sm)) * di.num_sms;
    void* args[] = {(void*)&P, (void*)&items, (void*)&count, (void*)&out};
    int rc = cuda_err(cudaLaunchCooperativeKernel((const void*)k_bag_only, dim3(grid), dim3(kEngineBlock), args, 0, st));
    count_launch();
    EngineCtl h;
    memset(&h, 0, sizeof(h));
    if (rc == SCC_OK) rc = cuda_err(cudaMemcpyAsync(&h, P.ctl, sizeof(EngineCtl), cudaMemcpyDeviceToHost, st));
    if (rc == SCC_OK) rc = cuda_err(cudaStreamSynchronize(st));
    SCC_TRY(rc);
    if (h.err) return h.err;
    *nout = h.ring[1].items;
    if (chunks) *chunks = h.ring[1].nhub + 1;
    return SCC_OK;
}

}  // namespace scc
