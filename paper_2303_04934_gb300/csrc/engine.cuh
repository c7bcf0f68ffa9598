// Reachability engine: vertical granularity control (VGC) local searches over a
// hash-bag frontier, in persistent cooperative kernels (sm_103a).
//
// Paper: Wang, Dong, Gu, Sun, SIGMOD 2023.
//  - Alg. 3 (reachability with a hash bag): rounds; every frontier item is
//    expanded and newly visited items go to the bag that forms the next
//    frontier.
//  - Sec. 3.1-3.2 (VGC): an item is expanded by a local search that keeps
//    newly visited items in a local queue and keeps expanding them until about
//    tau arcs have been examined; what is left in the queue is flushed to the
//    bag. An item with more than tau out-arcs is expanded "in parallel".
//  - Sec. 3.3 + Fig. 5 (hash bag): a preallocated slot array split into chunks
//    of lambda, 2*lambda, ... slots; inserts go to a random position of the
//    current chunk r with CAS and linear probing; sampled inserts count towards
//    sigma, at which point r advances by CAS (also after kappa failed probes);
//    ForAll visits the used prefix and skips empty slots.
//  - Sec. 4.2: single-reachability may run dense (bottom-up) rounds.
//
// GPU mapping (what differs from the 96-core design):
//  - The hash bag is claimed in 32-slot segments (one CAS per segment at a
//    random segment of the current chunk, linear probing over segments), so a
//    warp writes its spills as full 128/256-byte lines. Sampling and the chunk
//    advance are as in Fig. 5, counted per segment claim.
//  - The next round visits the bag in place (the ForAll operation): one 32-slot
//    segment is one WARP task. The warp reads the segment, resets its slots,
//    and runs a local search from the segment's items with its queue in shared
//    memory, expanding queued items cooperatively (one arc per lane: a warp
//    scan of the batch's degrees and a 5-step shuffle search map lanes to arcs,
//    so reads of each adjacency row are coalesced). tau bounds a task's arcs.
//    Two slot arrays alternate between rounds, so a round needs one grid
//    barrier and no packing pass.
//  - "Expand in parallel" = hub items: an item with more than tau out-arcs is
//    set aside when its segment is read and cut into 1024-arc segments that all
//    warps share in the next round.
//  - Rounds are separated by grid barriers inside one cooperative launch; the
//    host is not involved between rounds.
#pragma once
#include "common.cuh"

namespace scc {

constexpr int kSeg = 32;          // slots per hash-bag segment = items of one warp task
constexpr int kHubSeg = 1024;     // arcs of one hub segment
constexpr int kMaxChunks = 48;
constexpr int kBagProbe = 16;     // kappa: segment probes before a chunk advance
constexpr int kTableProbe = 256;  // pair-table probe limit (then: overflow, regrow)
constexpr int kEngineBlock = 256;         // threads of a block of a grid-wide (cooperative) engine launch
constexpr int kEngineMaxBlocksPerSm = 4;  // cooperative engine grids are clamped to this many blocks per SM
// Blocks per SM of a cooperative engine launch, given the occupancy the
// runtime reports for the kernel.
inline int engine_blocks_per_sm(int occupancy) {
    return occupancy < kEngineMaxBlocksPerSm ? occupancy : kEngineMaxBlocksPerSm;
}
// Bag slots held by partly filled segments: two 32-slot segments for each warp
// of the largest cooperative grid on num_sms SMs (engine_blocks_per_sm bounds
// its blocks per SM), reserved beside the items of every bag.
inline long long bag_warp_slots(int num_sms) {
    return 2ll * kSeg * (kEngineBlock / kWarp) * kEngineMaxBlocksPerSm * (long long)num_sms;
}

template <class Item>
struct Sent;
template <>
struct Sent<uint32_t> {
    static constexpr uint32_t empty = 0xffffffffu, claimed = 0xfffffffeu;
};
template <>
struct Sent<uint64_t> {
    static constexpr uint64_t empty = ~0ull, claimed = ~1ull;
};

struct BagCtl {
    int r;                   // current chunk
    int sample[kMaxChunks];  // sampled segment claims per chunk
    unsigned long long tail; // reservation bag (sigma = 0): next free slot
};

// Per-round state, a ring of three indexed by the global round number g: round
// g inserts into ring[g % 3] (and slot array g % 2), reads what round g - 1 left
// in ring[(g + 2) % 3] (slot array (g + 1) % 2), and block 0 clears
// ring[(g + 1) % 3] for round g + 1 -- nobody touches that entry in round g.
// The stop flags of a round live here too: a flag raised in round g is read
// only after round g's barrier, and round g + 1 raises its own, so every block
// (and every warp) takes the same decision to stop.
struct RoundCtl {
    BagCtl bag;
    long long items;   // items inserted into this round's bag
    long long hubseg;  // hub segments reserved this round
    long long work;    // next warp task of this round (dynamic assignment)
    int nhub;          // hub items set aside this round (expanded next round)
    int overflow;      // a pair table went over its load or probe limit
    int err;           // first error of the round (SCC_ERR_*: the bag is full)
    int pad;
    long long arcs;    // arcs of the items this round pushed or set aside (of those whose degree it loaded)
};

// Per-search state, a ring of three indexed by the search index: search s
// resets entry (s + 1) % 3, last used by search s - 2, whose counters every block
// read before search s - 1 began.
struct SearchCtl {
    int overflow;                    // pair table over its load or probe limit
    int rounds;                      // rounds executed
    unsigned long long inserted[2];  // newly visited pairs, per direction (pair mode)
};

constexpr int kTraceRounds = 1024;

struct EngineCtl {
    GridBarrier bar;
    int err;        // first error (SCC_ERR_*)
    int max_chunk;  // largest bag chunk used
    RoundCtl ring[3];
    SearchCtl search[3];
    unsigned long long edges;  // arcs examined
    unsigned long long items;  // items expanded (adjacency rows read)
    // trace of the first kTraceRounds rounds of a launch, indexed by the global
    // round number: end time (globaltimer ns), items of the round's bag, and
    // dense flag | search index << 1
    unsigned long long t0;
    unsigned long long t_end[kTraceRounds];
    long long t_items[kTraceRounds];
    int t_dense[kTraceRounds];
};

template <class Item>
struct EngineParams {
    const int32_t* off;
    const int32_t* adj;
    // second graph, for policies whose items carry a direction (kTwoGraphs):
    // items of direction 1 follow off2/adj2 (the transpose)
    const int32_t* off2;
    const int32_t* adj2;
    int32_t n;
    int tau;      // VGC arc budget per warp task
    int hub_thr;  // out-degree above which an item is a hub
    int seeds;    // items of a task expanded regardless of the budget (<= 32)
    // hash bag: two slot arrays, alternating between rounds
    Item* slots[2];
    long long nslots;
    int lambda;
    int sigma;
    // hub lists, alternating between rounds
    Item* hub_item[2];
    int32_t* hub_beg[2];
    int32_t* hub_deg[2];
    long long* hub_segbase[2];
    int hub_cap;
    int32_t* segmap[2];
    long long segmap_cap;
    // initial items (standalone launches)
    const Item* init;
    long long ninit;
    EngineCtl* ctl;
};

// Synchronisation scope of a search. GridScope: every block of a cooperative
// grid works on one search, rounds end at grid barriers, and the graph arrays
// (written before the launch) are read through the read-only path. CtaScope:
// one block runs the search alone (the batched kernel gives each graph to one
// block), rounds end at __syncthreads, and the graph arrays -- which the block
// may have written itself earlier in the same launch -- are read with coherent
// loads.
struct GridScope {
    __device__ __forceinline__ static int block() { return blockIdx.x; }
    __device__ __forceinline__ static int blocks() { return gridDim.x; }
    __device__ __forceinline__ static bool sync(GridBarrier* b, int* err) { return grid_sync(b, err); }
    __device__ __forceinline__ static int32_t ld(const int32_t* p) { return __ldg(p); }
};
struct CtaScope {
    __device__ __forceinline__ static int block() { return 0; }
    __device__ __forceinline__ static int blocks() { return 1; }
    __device__ __forceinline__ static bool sync(GridBarrier*, int*) {
        __syncthreads();
        return true;
    }
    __device__ __forceinline__ static int32_t ld(const int32_t* p) { return *p; }
};

// adjacency arrays of an item's graph
template <class Pol, class Item>
__device__ __forceinline__ const int32_t* item_off(const EngineParams<Item>& P, const Pol& pol, Item it) {
    if constexpr (Pol::kTwoGraphs) return pol.graph(it) ? P.off2 : P.off;
    else return P.off;
}
template <class Pol, class Item>
__device__ __forceinline__ const int32_t* item_adj(const EngineParams<Item>& P, const Pol& pol, Item it) {
    if constexpr (Pol::kTwoGraphs) return pol.graph(it) ? P.adj2 : P.adj;
    else return P.adj;
}

// ------------------------------------------------------------ chunk geometry --
__device__ __forceinline__ long long chunk_begin(int lambda, int j) {
    return (long long)lambda * ((1ll << j) - 1);
}
__device__ __forceinline__ long long chunk_end(int lambda, int j, long long nslots) {
    long long e = (long long)lambda * ((1ll << (j + 1)) - 1);
    return e < nslots ? e : nslots;
}

// ------------------------------------------------------------- bag writer --
template <class Item>
struct BagRef {
    Item* slots;
    long long nslots;
    int lambda;
    int sigma;
    BagCtl* bc;
    int* err;
    int* max_chunk;
};

// Warp-uniform state of the segment a warp is filling.
struct SegState {
    long long base;  // slot index of the segment, -1 = none
    int fill;
    uint32_t seq;    // claim counter (random positions)
};

// Claim a free segment of the current chunk (lane 0 only). Returns slot index or
// -1 (bag exhausted: error recorded). With sigma = 0 the bag is a reservation
// bag instead (the comparison point of the sampled design): one counter hands
// out segments in order, and the chunk index only records how far the slots
// were used, so that the next round's ForAll reads the same prefix.
template <class Item>
__device__ long long bag_claim(const BagRef<Item>& b, uint32_t wid, uint32_t round, uint32_t& seq) {
    if (b.sigma == 0) {
        const long long idx = (long long)atomicAdd(&b.bc->tail, (unsigned long long)kSeg);
        if (idx + kSeg > b.nslots) {
            atomicCAS(b.err, 0, SCC_ERR_CAPACITY);
            return -1;
        }
        int j = 0;
        while (j + 1 < kMaxChunks && chunk_end(b.lambda, j, b.nslots) < idx + kSeg) ++j;
        if (j > ld_volatile(&b.bc->r)) atomicMax(&b.bc->r, j);
        if (j > ld_volatile(b.max_chunk)) atomicMax(b.max_chunk, j);
        return idx;
    }
    for (int attempt = 0; attempt < 4 * kMaxChunks; ++attempt) {
        const int r = ld_volatile(&b.bc->r);
        const long long cb = chunk_begin(b.lambda, r);
        const long long ce = chunk_end(b.lambda, r, b.nslots);
        const long long nseg = (ce - cb) / kSeg;
        if (nseg <= 0) {
            atomicCAS(b.err, 0, SCC_ERR_CAPACITY);
            return -1;
        }
        const uint64_t h = mix64(((uint64_t)wid << 40) ^ ((uint64_t)round << 20) ^ (uint64_t)(seq++) ^ 0x5bd1e995ull);
        const long long pos = (long long)(h % (uint64_t)nseg);
        for (int pr = 0; pr < kBagProbe; ++pr) {
            const long long idx = cb + ((pos + pr) % nseg) * kSeg;
            using W = typename std::conditional<sizeof(Item) == 8, unsigned long long, unsigned int>::type;
            const Item prev = atomicCAS(reinterpret_cast<W*>(&b.slots[idx]), (W)Sent<Item>::empty,
                                        (W)Sent<Item>::claimed);
            if (prev == Sent<Item>::empty) {
                // sampled claim: rate sigma / (alpha * nseg), alpha = 1/2
                const uint32_t rnd = (uint32_t)(h >> 32);
                const double rate = 2.0 * b.sigma / (double)nseg;
                if (rate >= 1.0 || (double)rnd < rate * 4294967296.0) {
                    const int s = atomicAdd(&b.bc->sample[r], 1) + 1;
                    if (s >= b.sigma && ce < b.nslots) atomicCAS(&b.bc->r, r, r + 1);
                }
                if (r > ld_volatile(b.max_chunk)) atomicMax(b.max_chunk, r);
                return idx;
            }
        }
        // kappa probes failed: the chunk is (nearly) full -> try_resize
        if (ce >= b.nslots) {
            atomicCAS(b.err, 0, SCC_ERR_CAPACITY);
            return -1;
        }
        atomicCAS(&b.bc->r, r, r + 1);
    }
    atomicCAS(b.err, 0, SCC_ERR_CAPACITY);
    return -1;
}

// Warp-cooperative insert of the items of lanes with `has` (all lanes call).
// Returns the number of items inserted by the warp.
template <class Item>
__device__ __forceinline__ int bag_push(const BagRef<Item>& b, SegState& st, bool has, Item it, uint32_t wid,
                                        uint32_t round) {
    const uint32_t m = __ballot_sync(kFull, has);
    int cnt = __popc(m);
    const int total = cnt;
    if (cnt == 0) return 0;
    int rank = __popc(m & lanemask_lt());
    while (cnt > 0) {
        if (st.base < 0 || st.fill == kSeg) {
            long long base = -1;
            if (lane_id() == 0) base = bag_claim<Item>(b, wid, round, st.seq);
            base = __shfl_sync(kFull, base, 0);
            st.seq = __shfl_sync(kFull, st.seq, 0);
            if (base < 0) return total;  // error recorded
            st.base = base;
            st.fill = 0;
        }
        const int space = kSeg - st.fill;
        if (has && rank >= 0 && rank < space) b.slots[st.base + st.fill + rank] = it;
        const int used = cnt < space ? cnt : space;
        st.fill += used;
        rank -= used;
        cnt -= used;
        if (rank < 0) has = false;
    }
    return total;
}

// ------------------------------------------------------------ warp tasks --
// The local queue of a warp's search: a ring of kQueue items, each with its
// adjacency range (first arc, out-degree), loaded while the item was visited,
// and, for policies whose arc test needs a per-item value (the class label of a
// pair's vertex), that value, inherited by the items it visits.
template <class Pol>
struct EngineSmem {  // up to 8 warps per block
    typename Pol::Item qi[8 * Pol::kQueue];
    int2 qr[8 * Pol::kQueue];
    int32_t qc[Pol::kCtxInQueue ? 8 * Pol::kQueue : 1];
};
template <class Item>
struct LocalQueue {
    Item* it;
    int2* rg;
    int32_t* cx;
};
template <class Pol>
__device__ __forceinline__ LocalQueue<typename Pol::Item> warp_queue(EngineSmem<Pol>& sm) {
    const int w = threadIdx.x >> 5;
    return {sm.qi + w * Pol::kQueue, sm.qr + w * Pol::kQueue, Pol::kCtxInQueue ? sm.qc + w * Pol::kQueue : sm.qc};
}

// Per-warp accumulators (folded into the control block at the end).
struct WarpStats {
    unsigned long long edges = 0, items = 0;
};

// Expand the next batch of queued items (up to 32, or `max_take` in the seeds
// phase, which ignores the budget and the hub test).
template <class Pol, class S>
__device__ __forceinline__ void expand_batch(const EngineParams<typename Pol::Item>& P, Pol& pol,
                                             const BagRef<typename Pol::Item>& out, SegState& st, uint32_t wid,
                                             uint32_t round, const LocalQueue<typename Pol::Item>& q, uint32_t& qh, uint32_t& qt,
                                             int& t, bool seeds_phase, int max_take, int hub_thr, WarpStats& ws,
                                             unsigned long long& pushed, unsigned long long& parcs) {
    using Item = typename Pol::Item;
    constexpr uint32_t QM = Pol::kQueue - 1;
    const int lane = lane_id();
    int avail = (int)min(32u, qt - qh);
    if (seeds_phase && avail > max_take) avail = max_take;
    Item it = Sent<Item>::empty;
    int beg = 0, deg = 0;
    using Ctx = typename Pol::Ctx;
    Ctx qctx{};
    if (lane < avail) {
        const uint32_t k = (qh + lane) & QM;
        it = q.it[k];
        const int2 r = q.rg[k];
        beg = r.x;
        deg = r.y;
        if constexpr (Pol::kCtxInQueue) qctx = (uint64_t)(uint32_t)q.cx[k];
    }
    // items past the seeds with more than hub_thr arcs go back to the bag
    bool hub = !seeds_phase && lane < avail && deg > hub_thr;
    int d = (lane < avail && !hub) ? deg : 0;
    int pre = warp_incl_scan(d);
    int take = avail;
    if (!seeds_phase) {
        const int remaining = P.tau - t;
        const uint32_t m = __ballot_sync(kFull, lane < avail && (pre - d) < remaining);
        take = __popc(m);
        if (take < 1) take = 1;
        if (lane >= take) {
            d = 0;
            hub = false;
        }
        pre = warp_incl_scan(d);
    }
    qh += take;
    pushed += bag_push<Item>(out, st, hub, it, wid, round);
    Ctx ctx = qctx;
    if constexpr (!Pol::kCtxInQueue) ctx = (lane < take && !hub) ? pol.ctx(it) : Ctx{};
    const int total = __shfl_sync(kFull, pre, 31);
    const int excl = pre - d;
    // four groups of 32 arcs per step: the adjacency loads and the visit tests of
    // the groups are independent, so their memory latencies overlap
    constexpr int U = 4;
    for (int base = 0; base < total; base += 32 * U) {
        int w[U];
        Item jit[U];
        Ctx jctx[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = base + u * 32 + lane;
            // owner lane: number of lanes whose inclusive prefix is <= e
            int j = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                const int v = __shfl_sync(kFull, pre, j + step - 1);
                if (v <= e) j += step;
            }
            const int jexcl = __shfl_sync(kFull, excl, j);
            const int jbeg = __shfl_sync(kFull, beg, j);
            jit[u] = shfl_any(it, j);
            jctx[u] = shfl_any(ctx, j);
            w[u] = e < total ? S::ld(&item_adj(P, pol, jit[u])[jbeg + (e - jexcl)]) : -1;
        }
        // the adjacency range of every target is loaded together with its visit
        // test (not after it), so a newly visited item enters the queue ready to
        // expand: one dependent memory access less per step of the search
        int rb[U], re[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int32_t* O = item_off(P, pol, jit[u]);  // a child stays in its parent's graph
            rb[u] = w[u] >= 0 ? S::ld(&O[w[u]]) : 0;
            re[u] = w[u] >= 0 ? S::ld(&O[w[u] + 1]) : 0;
        }
        bool nw[U];
        Item child[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            child[u] = Sent<Item>::empty;
            nw[u] = w[u] >= 0 && pol.visit(jit[u], jctx[u], w[u], child[u]);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            // new items: local queue while it has room, the bag otherwise
            const uint32_t m = __ballot_sync(kFull, nw[u]);
            const int cnt = __popc(m);
            if (cnt) {
                const int rank = __popc(m & lanemask_lt());
                const int room = (int)(Pol::kQueue - (qt - qh));
                const bool toq = nw[u] && rank < room;
                if (toq) {
                    const uint32_t k = (qt + rank) & QM;
                    q.it[k] = child[u];
                    q.rg[k] = make_int2(rb[u], re[u] - rb[u]);
                    if constexpr (Pol::kCtxInQueue) q.cx[k] = (int32_t)(uint32_t)jctx[u];
                }
                const int nq = cnt < room ? cnt : room;
                pushed += bag_push<Item>(out, st, nw[u] && !toq, child[u], wid, round);
                if (nw[u] && !toq) parcs += (unsigned long long)(re[u] - rb[u]);
                qt += nq;
            }
        }
        __syncwarp();
    }
    t += total;
    ws.edges += (lane == 0) ? (unsigned long long)total : 0ull;
    ws.items += (lane == 0) ? (unsigned long long)take : 0ull;
}

// Dense (bottom-up) rounds of a single-reachability search (Sec. 4.2): every
// unvisited vertex of the class scans its in-arcs (the reverse CSR) and stops at
// the first one whose tail is in the current frontier. Used when the frontier
// holds at least n_active / frac_inv items, or when its items' arcs number at
// least m_active / frac_inv (a few hubs can claim much of the graph in one
// round; their arcs, not their count, set a top-down round's cost).
struct DenseParams {
    const int32_t* roff;  // reverse CSR (G^T for a forward search, G for a backward one)
    const int32_t* radj;
    uint32_t* fbits[2];   // frontier bitmaps (alternating), ceil(n/32) words each, zero between searches
    long long n_active;   // vertices of the class
    int frac_inv;         // 0 = never dense
    long long m_active;   // arcs of the graph searched (0: the arcs test is off)
};

// The initial items of a search: an explicit list (or, for pair searches,
// InitPairs below).
template <class Item>
struct InitList {
    const Item* items;
    __device__ __forceinline__ Item operator()(long long i) const { return items[i]; }
};

// Set an item with more than hub_thr arcs aside for the next round, cut into
// hub segments. Returns false (and reserves nothing usable) when the hub list or
// the segment map is full; the caller then expands the item itself.
template <class Item>
__device__ __forceinline__ bool reserve_hub(const EngineParams<Item>& P, RoundCtl& cur, int par, Item x, int b0,
                                            int dg) {
    const int h = atomicAdd(&cur.nhub, 1);
    if (h >= P.hub_cap) return false;
    const long long ns = ceil_div(dg, kHubSeg);
    const long long sb = (long long)atomicAdd((unsigned long long*)&cur.hubseg, (unsigned long long)ns);
    const long long lim = sb + ns < P.segmap_cap ? sb + ns : P.segmap_cap;
    if (sb + ns > P.segmap_cap) {
        for (long long g = sb; g < lim; ++g) P.segmap[par][g] = -1;
        P.hub_item[par][h] = x;  // listed but without segments: skipped by the next round
        P.hub_deg[par][h] = 0;
        P.hub_beg[par][h] = b0;
        P.hub_segbase[par][h] = sb;
        return false;
    }
    P.hub_item[par][h] = x;
    P.hub_beg[par][h] = b0;
    P.hub_deg[par][h] = dg;
    P.hub_segbase[par][h] = sb;
    for (long long g = sb; g < lim; ++g) P.segmap[par][g] = h;
    return true;
}

// One complete reachability search (Alg. 3 rounds) executed by every thread of a
// cooperative grid. `g` is the global round counter (identical in all blocks;
// advanced past this search's rounds), `si` the search index (selects the
// per-search control entry). Returns false if a grid barrier timed out (the
// caller must return at once). On return every block has passed the final
// barrier, so this search's control entry is final.
template <class Pol, class Init, class S = GridScope>
__device__ bool engine_search(const EngineParams<typename Pol::Item>& P, Pol& pol, Init init, long long ninit,
                              const DenseParams* dp, const LocalQueue<typename Pol::Item>& q, WarpStats& ws, uint32_t& g,
                              uint32_t si, int& why) {
    using Item = typename Pol::Item;
    constexpr uint32_t QM = Pol::kQueue - 1;
    EngineCtl* ctl = P.ctl;
    SearchCtl& sc = ctl->search[si % 3];
    const int lane = lane_id();
    const int wib = threadIdx.x >> 5;
    const uint32_t wid = (uint32_t)(S::block() * (blockDim.x >> 5) + wib);
    const uint32_t nwarps = (uint32_t)(S::blocks() * (blockDim.x >> 5));
    const long long gtid = (long long)S::block() * blockDim.x + threadIdx.x;
    const long long gstride = (long long)S::blocks() * blockDim.x;
    const uint32_t g0 = g;
    why = 0;
    if (si == 0 && S::block() == 0 && threadIdx.x == 0) ctl->t0 = globaltimer_ns();
    bool prev_dense = false;
    uint32_t i = 0;
    for (;; ++i) {
        const uint32_t gr = g0 + i;
        const int par = (int)(gr & 1), ipar = par ^ 1;
        RoundCtl& cur = ctl->ring[gr % 3];
        RoundCtl& prev = ctl->ring[(gr + 2) % 3];
        if (S::block() == 0 && threadIdx.x == 0) {
            RoundCtl& nx = ctl->ring[(gr + 1) % 3];
            nx.bag.r = 0;
            for (int j = 0; j < kMaxChunks; ++j) nx.bag.sample[j] = 0;
            nx.bag.tail = 0;
            nx.items = 0;
            nx.hubseg = 0;
            nx.work = 0;
            nx.nhub = 0;
            nx.overflow = 0;
            nx.err = 0;
            nx.arcs = 0;
            if (i == 0) {
                SearchCtl& other = ctl->search[(si + 1) % 3];
                other.overflow = 0;
                other.rounds = 0;
                other.inserted[0] = 0;
                other.inserted[1] = 0;
            }
        }
        const BagRef<Item> out{P.slots[par], P.nslots, P.lambda, P.sigma, &cur.bag, &cur.err, &ctl->max_chunk};
        if constexpr (Pol::kCountInserts) pol.overflow = &cur.overflow;
        Item* const in_slots = P.slots[ipar];
        SegState st{-1, 0, (uint32_t)(wid * 2654435761u) ^ gr};
        unsigned long long pushed = 0, parcs = 0;
        long long in_end = i == 0 ? 0 : chunk_end(P.lambda, ld_volatile(&prev.bag.r), P.nslots);
        const long long fr_items = i == 0 ? ninit : ld_volatile(&prev.items);
        const int fr_hubs = i == 0 ? 0 : min(ld_volatile(&prev.nhub), P.hub_cap);
        bool dense = false;
        if constexpr (Pol::kDense) {
            dense = i > 0 && dp != nullptr && dp->frac_inv > 0 &&
                    ((long long)(fr_items + fr_hubs) * (long long)dp->frac_inv >= dp->n_active ||
                     (dp->m_active > 0 && ld_volatile(&prev.arcs) * (long long)dp->frac_inv >= dp->m_active));
            if (prev_dense) {  // the bitmap of the previous (dense) round
                uint32_t* old = dp->fbits[ipar];
                const long long nw = ((long long)P.n + 31) / 32;
                for (long long w = gtid; w < nw; w += gstride)
                    if (old[w]) old[w] = 0;
            }
        }
        if (dense) {
            if constexpr (Pol::kDense) {
                // ---- dense round: frontier bitmap, then bottom-up over unvisited
                // vertices. After a dense round the bitmap is ready (that round
                // wrote the vertices it found into it); the input bag (read and
                // reset) adds what the last round pushed: all of its items after
                // a sparse round, the sources a policy added after a dense one;
                // after a sparse round last round's hubs are added too.
                uint32_t* fb = dp->fbits[par];
                uint32_t* nfb = dp->fbits[ipar];  // the next round's frontier (cleared above)
                for (long long j = gtid; j < in_end; j += gstride) {
                    const Item x = in_slots[j];
                    if (x == Sent<Item>::empty) continue;
                    in_slots[j] = Sent<Item>::empty;
                    if (x == Sent<Item>::claimed) continue;
                    const int v = pol.vertex(x);
                    atomicOr(&fb[v >> 5], 1u << (v & 31));
                }
                if (!prev_dense)
                    for (long long j = gtid; j < fr_hubs; j += gstride) {
                        const int v = pol.vertex(P.hub_item[ipar][j]);
                        atomicOr(&fb[v >> 5], 1u << (v & 31));
                    }
                // sources added by the policy go into this round's bag (the next
                // round's input, as in a sparse round); they are visited before
                // the bottom-up below reads the visited words, so it leaves them
                // alone and its stores of whole words keep their bits
                if constexpr (Pol::kInject) pol.inject(i, out, st, wid, nwarps, gr, pushed);
                if (!S::sync(&ctl->bar, &ctl->err)) return false;
                const long long nw = ((long long)P.n + 31) / 32;
                // each warp takes 32 consecutive words at a time (one coalesced
                // load); their unvisited vertices form the warp's work list,
                // handed to lanes one vertex at a time: a lane whose vertex is
                // done (a parent in the frontier found, or its in-arcs
                // exhausted) takes the next entry, so a few long in-lists do not
                // hold the other lanes. A lane keeps kDV vertices in flight and
                // reads two in-arcs of each per step. Found bits gather in 32
                // shared words (the warp's local queue is idle in dense rounds)
                // and are written once per word: the warp owns its words.
                constexpr int kDV = 2;
                static_assert(sizeof(Item) * Pol::kQueue >= 32 * sizeof(uint32_t), "queue holds 32 words");
                uint32_t* s_found = reinterpret_cast<uint32_t*>(q.it);
                unsigned long long scanned = 0;
                for (long long w0 = (long long)wid * 32; w0 < nw; w0 += (long long)nwarps * 32) {
                    const uint32_t mine = w0 + lane < nw ? ld_volatile(&pol.bits[w0 + lane]) : ~0u;
                    const uint32_t unv = ~mine;  // bits past n are set by the prefill
                    const int cnt = __popc(unv);
                    const int incl = warp_incl_scan(cnt);
                    const int T = __shfl_sync(kFull, incl, 31);
                    if (T == 0) continue;  // warp-uniform
                    s_found[lane] = 0;
                    __syncwarp();
                    int next = 0;  // warp-uniform cursor into the list
                    int vv[kDV], e[kDV], e1[kDV];
#pragma unroll
                    for (int k = 0; k < kDV; ++k) vv[k] = e[k] = e1[k] = -1;
                    for (;;) {
#pragma unroll
                        for (int k = 0; k < kDV; ++k) {
                            const bool idle = vv[k] < 0;
                            const uint32_t need = __ballot_sync(kFull, idle);
                            const int idx = next + __popc(need & lanemask_lt());
                            next += __popc(need);
                            // list entry idx lies in word j, the first with incl > idx
                            int j = 0;
#pragma unroll
                            for (int sh = 16; sh >= 1; sh >>= 1)
                                if (__shfl_sync(kFull, incl, j + sh - 1) <= idx) j += sh;
                            const uint32_t uj = __shfl_sync(kFull, unv, j);
                            const int bj = __shfl_sync(kFull, incl - cnt, j);
                            if (idle && idx < T) {
                                const int v = (int)((w0 + j) * 32 + (long long)__fns(uj, 0, idx - bj + 1));
                                vv[k] = v;
                                e[k] = S::ld(&dp->roff[v]);
                                e1[k] = S::ld(&dp->roff[v + 1]);
                            }
                        }
                        bool busy = false;
#pragma unroll
                        for (int k = 0; k < kDV; ++k) busy |= vv[k] >= 0;
                        if (!__any_sync(kFull, busy)) break;  // every lane idle: the list is done
                        int u[kDV][2];
#pragma unroll
                        for (int k = 0; k < kDV; ++k)
#pragma unroll
                            for (int a = 0; a < 2; ++a)
                                u[k][a] = vv[k] >= 0 && e[k] + a < e1[k] ? S::ld(&dp->radj[e[k] + a]) : -1;
                        uint32_t fw[kDV][2];
#pragma unroll
                        for (int k = 0; k < kDV; ++k)
#pragma unroll
                            for (int a = 0; a < 2; ++a) fw[k][a] = u[k][a] >= 0 ? ld_volatile(&fb[u[k][a] >> 5]) : 0u;
#pragma unroll
                        for (int k = 0; k < kDV; ++k) {
                            bool f = false;
                            int par_u = -1;
#pragma unroll
                            for (int a = 0; a < 2; ++a)
                                if (!f && u[k][a] >= 0) {
                                    ++scanned;
                                    f = (fw[k][a] >> (u[k][a] & 31)) & 1u;
                                    if (f) par_u = u[k][a];
                                }
                            e[k] += 2;
                            if (f) {
                                atomicOr(&s_found[(vv[k] >> 5) - w0], 1u << (vv[k] & 31));
                                pol.adopt(vv[k], par_u);  // the vertex takes what its frontier neighbour carries
                            }
                            if (f || e[k] >= e1[k]) vv[k] = -1;
                        }
                    }
                    __syncwarp();
                    const uint32_t fm = s_found[lane];
                    if (fm) {  // fm != 0 only for words < nw
                        pol.bits[w0 + lane] = mine | fm;
                        nfb[w0 + lane] = fm;  // the new frontier
                    }
                    int nf = __popc(fm);
                    for (int dd = 16; dd >= 1; dd >>= 1) nf += __shfl_xor_sync(kFull, nf, dd);
                    if (lane == 0) ws.items += nf;
                    pushed += (unsigned long long)nf;
                    __syncwarp();  // the next group resets s_found
                }
                for (int dd = 16; dd >= 1; dd >>= 1) scanned += __shfl_xor_sync(kFull, scanned, dd);
                if (lane == 0) ws.edges += scanned;
            }
        } else {
            if constexpr (Pol::kDense) {
                if (prev_dense) {
                    // the last (dense) round left its new vertices in a bitmap:
                    // push them into that round's bag (read and reset the words)
                    // and read the bag as usual
                    const BagRef<Item> pin{P.slots[ipar], P.nslots, P.lambda, P.sigma, &prev.bag, &cur.err,
                                           &ctl->max_chunk};
                    SegState pst{-1, 0, (uint32_t)(wid * 2654435761u) ^ (gr - 1u)};
                    uint32_t* pfb = dp->fbits[par];
                    const long long nw = ((long long)P.n + 31) / 32;
                    for (long long w0 = (long long)wid * 32; w0 < nw; w0 += (long long)nwarps * 32) {
                        const long long w = w0 + lane;
                        uint32_t x = w < nw ? pfb[w] : 0u;
                        if (x) pfb[w] = 0;
                        while (__any_sync(kFull, x != 0)) {
                            const int b = x ? __ffs(x) - 1 : 0;
                            const bool has = x != 0;
                            if (has) x &= x - 1;
                            bag_push<Item>(pin, pst, has, (Item)(w * 32 + b), wid, gr - 1u);
                        }
                    }
                    if (!S::sync(&ctl->bar, &ctl->err)) return false;
                    in_end = chunk_end(P.lambda, ld_volatile(&prev.bag.r), P.nslots);
                }
            }
            // once a table overflows the round's work is moot: stop taking work
            // (lane 0 reads the flag for the warp, so the warp stays converged)
            auto stop = [&]() {
                if constexpr (!Pol::kCountInserts) return false;
                const int f = lane == 0 ? ld_volatile(&cur.overflow) : 0;
                return __shfl_sync(kFull, f, 0) != 0;
            };
            // ---- phase A: last round's hubs, cut into segments shared by all warps
            if (i > 0) {
                const long long nseg = min(ld_volatile(&prev.hubseg), P.segmap_cap);
                for (long long gs = wid; gs < nseg && !stop(); gs += nwarps) {
                    const int h = P.segmap[ipar][gs];
                    if (h < 0) continue;
                    const Item hit = P.hub_item[ipar][h];
                    const long long j0 = (gs - P.hub_segbase[ipar][h]) * kHubSeg;
                    const int b0 = P.hub_beg[ipar][h] + (int)j0;
                    const int len = (int)min((long long)kHubSeg, (long long)P.hub_deg[ipar][h] - j0);
                    const typename Pol::Ctx hctx = pol.ctx(hit);
                    for (int e0 = 0; e0 < len; e0 += 32) {
                        bool nw = false;
                        Item child = Sent<Item>::empty;
                        if (e0 + lane < len) {
                            const int w = S::ld(&item_adj(P, pol, hit)[b0 + e0 + lane]);
                            nw = pol.visit(hit, hctx, w, child);
                        }
                        pushed += bag_push<Item>(out, st, nw, child, wid, gr);
                    }
                    ws.edges += lane == 0 ? (unsigned long long)max(len, 0) : 0ull;
                    ws.items += (lane == 0 && gs == P.hub_segbase[ipar][h]) ? 1ull : 0ull;
                }
            }
            // ---- phase B: warp tasks over the input (ForAll over the bag, or the
            // initial items in round 0). A task covers G <= 32 slots, G halved until
            // every warp gets about two tasks; with a small frontier, items with
            // more than 64 arcs are also cut into hub segments for the next round,
            // so that a few heavy items do not serialise the round on a few warps.
            const long long in_cnt = i == 0 ? ninit : in_end;
            int G = 32;
            while (G > 1 && (long long)G * nwarps * 2 > in_cnt) G >>= 1;
            const int hub_thr = fr_items < (long long)nwarps * 8 ? min(P.hub_thr, 64) : P.hub_thr;
            const long long ntasks = (in_cnt + G - 1) / G;
            for (;;) {
                long long tk = 0;
                if (lane == 0) tk = (long long)atomicAdd((unsigned long long*)&cur.work, 1ull);
                tk = __shfl_sync(kFull, tk, 0);
                if (tk >= ntasks || stop()) break;
                const long long idx = tk * G + lane;
                Item it = Sent<Item>::empty;
                bool has = false;
                if (lane >= G || idx >= in_cnt) {
                    // not part of this task
                } else if (i == 0) {
                    it = init(idx);
                    has = pol.seed(it);
                } else {
                    it = in_slots[idx];
                    if (it != Sent<Item>::empty) {
                        in_slots[idx] = Sent<Item>::empty;
                        has = it != Sent<Item>::claimed;
                    }
                }
                int b0 = 0, dg = 0;
                int32_t cx0 = 0;
                if (has) {
                    const int v = pol.vertex(it);
                    const int32_t* O = item_off(P, pol, it);
                    b0 = S::ld(&O[v]);
                    dg = S::ld(&O[v + 1]) - b0;
                    if constexpr (Pol::kCtxInQueue) cx0 = pol.load_ctx(it);
                    if (dg > hub_thr && reserve_hub(P, cur, par, it, b0, dg)) {
                        has = false;
                        parcs += (unsigned long long)dg;
                    }
                }
                const uint32_t m = __ballot_sync(kFull, has);
                if (m == 0) continue;
                if (has) {
                    const int k = __popc(m & lanemask_lt());
                    q.it[k] = it;
                    q.rg[k] = make_int2(b0, dg);
                    if constexpr (Pol::kCtxInQueue) q.cx[k] = cx0;
                }
                __syncwarp();
                uint32_t qh = 0, qt = (uint32_t)__popc(m);
                int t = 0;
                expand_batch<Pol, S>(P, pol, out, st, wid, gr, q, qh, qt, t, true, P.seeds, hub_thr, ws, pushed,
                                     parcs);
                while (qt != qh && t < P.tau)
                    expand_batch<Pol, S>(P, pol, out, st, wid, gr, q, qh, qt, t, false, 32, hub_thr, ws, pushed,
                                         parcs);
                // budget spent: flush what is left in the local queue
                while (qt != qh) {
                    const int nrem = (int)min(32u, qt - qh);
                    const Item x = lane < nrem ? q.it[(qh + lane) & QM] : Sent<Item>::empty;
                    if (lane < nrem) parcs += (unsigned long long)q.rg[(qh + lane) & QM].y;
                    qh += nrem;
                    pushed += bag_push<Item>(out, st, lane < nrem, x, wid, gr);
                }
                __syncwarp();
                if constexpr (Pol::kCountInserts) pol.flush(sc);
            }
            if constexpr (Pol::kCountInserts) pol.flush(sc);
            // policies that add sources while the search runs (the batches of
            // the low-diameter decomposition, Alg. 4) push them into this
            // round's bag: they join the next round's frontier
            if constexpr (Pol::kInject) pol.inject(i, out, st, wid, nwarps, gr, pushed);
        }
        if (lane == 0 && pushed) atomicAdd((unsigned long long*)&cur.items, pushed);
        if constexpr (Pol::kDense) {
            for (int d = 16; d >= 1; d >>= 1) parcs += __shfl_xor_sync(kFull, parcs, d);
            if (lane == 0 && parcs) atomicAdd((unsigned long long*)&cur.arcs, parcs);
        }
        if (!S::sync(&ctl->bar, &ctl->err)) return false;
        if (gr < (uint32_t)kTraceRounds && S::block() == 0 && threadIdx.x == 0) {
            ctl->t_end[gr] = globaltimer_ns();
            ctl->t_items[gr] = ld_volatile(&cur.items);
            ctl->t_dense[gr] = (int)dense | (int)(si << 1);
        }
        prev_dense = dense;
        // the decision to stop reads only this round's entries, final now
        const int rerr = ld_volatile(&cur.err);
        if (rerr != 0) {
            why = rerr;
            break;
        }
        if (Pol::kCountInserts && ld_volatile(&cur.overflow) != 0) {
            why = 1;
            break;
        }
        if (ld_volatile(&cur.items) == 0 && ld_volatile(&cur.nhub) == 0) {
            if constexpr (Pol::kInject) {
                if (pol.more(i)) continue;  // an empty frontier, but batches of sources remain
            }
            break;
        }
    }
    // for readers after the launch (the caller inside the launch uses `why`)
    if (S::block() == 0 && threadIdx.x == 0) {
        sc.rounds = (int)i + 1;
        if (why == 1) sc.overflow = 1;
        if (why < 0) atomicCAS(&ctl->err, 0, why);
    }
    g = g0 + i + 1;
    if constexpr (Pol::kDense) {
        // a search that ended on a dense round leaves its bitmap for the next
        // search's first round... which never clears it: clear it here
        if (prev_dense && dp != nullptr) {
            uint32_t* last = dp->fbits[(g0 + i) & 1];
            const long long nw = ((long long)P.n + 31) / 32;
            for (long long w = gtid; w < nw; w += gstride)
                if (last[w]) last[w] = 0;
            if (!S::sync(&ctl->bar, &ctl->err)) return false;
        }
    }
    return true;
}

template <class Pol>
__global__ void __launch_bounds__(kEngineBlock, 3) engine_kernel(EngineParams<typename Pol::Item> P, Pol pol_in, DenseParams dp) {
    Pol pol = pol_in;
    __shared__ EngineSmem<Pol> sm;
    const LocalQueue<typename Pol::Item> q = warp_queue(sm);
    WarpStats ws;
    uint32_t g = 0;
    int why = 0;  // the host reads the outcome from the control block
    const bool ok = engine_search<Pol>(P, pol, InitList<typename Pol::Item>{P.init}, P.ninit,
                                       dp.frac_inv > 0 ? &dp : nullptr, q, ws, g, 0, why);
    if (!ok) return;
    if (lane_id() == 0 && ws.edges) atomicAdd(&P.ctl->edges, ws.edges);
    if (lane_id() == 0 && ws.items) atomicAdd(&P.ctl->items, ws.items);
}

// ---------------------------------------------------------------- policies --
// Single-reachability: vertex items, visited bitmap. Vertices outside the
// source's class (and finished ones) are pre-set in the bitmap, so the arc test
// is one bit (Alg. 3 "CAS(visit[u], false, true)").
struct PolSingle {
    using Item = uint32_t;
    static constexpr int kQueue = 256;
    static constexpr bool kCountInserts = false;
    static constexpr bool kDense = true;
    static constexpr bool kCtxInQueue = false;
    using Ctx = uint64_t;  // the per-item value an arc test reads
    static constexpr bool kTwoGraphs = false;
    static constexpr bool kInject = false;
    static constexpr const char* kName = "single-reach";
    uint32_t* bits;
    __device__ __forceinline__ int vertex(Item it) const { return (int)it; }
    __device__ __forceinline__ uint64_t ctx(Item) const { return 0; }
    __device__ __forceinline__ bool seed(Item it) const {
        uint32_t b = 1u << (it & 31);
        return (atomicOr(&bits[it >> 5], b) & b) == 0;
    }
    __device__ __forceinline__ bool visit(Item, uint64_t, int w, Item& child) const {
        uint32_t b = 1u << (w & 31);
        if (ld_volatile(&bits[w >> 5]) & b) return false;
        child = (Item)w;
        return (atomicOr(&bits[w >> 5], b) & b) == 0;
    }
    __device__ __forceinline__ void adopt(int, int) const {}
};

// Forward and backward single-reachability from the same source in one search
// (they are independent, so they can share rounds): vertex items with a
// direction bit (bit 31); direction 0 follows G and marks bits[0], direction 1
// follows G^T and marks bits[1]. No dense rounds (the dense test is per
// direction). The sentinels (0xffffffff, 0xfffffffe) are never items as long
// as vertex ids stay below 2^31 - 2.
struct PolSingleBoth {
    using Item = uint32_t;
    static constexpr int kQueue = 256;
    static constexpr bool kCountInserts = false;
    static constexpr bool kDense = false;
    static constexpr bool kCtxInQueue = false;
    using Ctx = uint64_t;  // the per-item value an arc test reads
    static constexpr bool kTwoGraphs = true;
    static constexpr bool kInject = false;
    static constexpr const char* kName = "single-reach-both";
    static constexpr uint32_t kDir = 1u << 31;
    uint32_t* bits[2];
    __device__ __forceinline__ int vertex(Item it) const { return (int)(it & ~kDir); }
    __device__ __forceinline__ int graph(Item it) const { return (int)(it >> 31); }
    __device__ __forceinline__ uint64_t ctx(Item) const { return 0; }
    __device__ __forceinline__ bool seed(Item it) const {
        uint32_t* B = graph(it) ? bits[1] : bits[0];
        const int v = vertex(it);
        const uint32_t b = 1u << (v & 31);
        return (atomicOr(&B[v >> 5], b) & b) == 0;
    }
    // the atomic is the test (no read before it): these searches run on
    // low-degree graphs, where a step's dependent accesses are its cost
    __device__ __forceinline__ bool visit(Item parent, uint64_t, int w, Item& child) const {
        uint32_t* B = (parent >> 31) ? bits[1] : bits[0];
        const uint32_t b = 1u << (w & 31);
        child = (parent & kDir) | (uint32_t)w;
        return (atomicOr(&B[w >> 5], b) & b) == 0;
    }
};

// Pair table (Sec. 4.3 phase-concurrent hash table of reachability pairs):
// open addressing over uint64 keys v << 32 | s, linear probing, insert-if-absent.
struct PairTable {
    unsigned long long* keys;
    unsigned long long mask;  // capacity - 1 (capacity a power of two)
    int* overflow;
    __device__ __forceinline__ static unsigned long long hash(unsigned long long k) { return mix64(k); }
    __device__ __forceinline__ bool insert(unsigned long long key) const { return insert_into(keys, mask, overflow, key); }
    // the CAS itself is the probe (no read before it): one memory round trip per
    // slot whether the slot is empty, holds the key or another one
    __device__ __forceinline__ static bool insert_into(unsigned long long* keys, unsigned long long mask, int* overflow,
                                                       unsigned long long key) {
        unsigned long long h = hash(key) & mask;
        for (int i = 0; i < kTableProbe; ++i) {
            const unsigned long long prev = atomicCAS(&keys[h], ~0ull, key);
            if (prev == ~0ull) return true;
            if (prev == key) return false;
            h = (h + 1) & mask;
        }
        atomicExch(overflow, 1);
        return false;
    }
    __device__ __forceinline__ bool contains(unsigned long long key) const { return contains_from(hash(key) & mask, key); }
    // lookup that starts probing at slot h (for callers that read the first
    // slot themselves)
    __device__ __forceinline__ bool contains_from(unsigned long long h, unsigned long long key) const {
        for (unsigned long long i = 0; i <= mask; ++i) {
            unsigned long long cur = keys[h];
            if (cur == key) return true;
            if (cur == ~0ull) return false;
            h = (h + 1) & mask;
        }
        return false;
    }
};

// Multi-reachability: pair items (v, s) plus a direction bit (bit 63). Direction
// 0 follows G and fills T_out with the pairs s ~> v, direction 1 follows G^T
// and fills T_in with the pairs v ~> s; the two searches of a batch are
// independent, so they share the rounds of one search. An arc (u, w) is followed
// only when label[w] == label[u] (Alg. 1: MultiReach skips (u, v) with
// L(u) != L(v); finished vertices carry kDone < 0 and never match an active
// class). Table keys are v << 32 | s without the direction bit; the sentinels
// (s with bit 31 set) are never items.
struct PolPair {
    using Item = uint64_t;
    static constexpr int kQueue = 256;
    static constexpr bool kCountInserts = true;
    static constexpr bool kDense = false;
    static constexpr bool kCtxInQueue = true;
    using Ctx = uint64_t;  // the per-item value an arc test reads
    static constexpr bool kTwoGraphs = true;
    static constexpr bool kInject = false;
    static constexpr const char* kName = "multi-reach";
    static constexpr uint64_t kDir = 1ull << 63;
    const int32_t* label;
    unsigned long long* keys[2];  // T_out, T_in
    unsigned long long mask[2];   // capacities - 1 (powers of two)
    long long max_ins[2];         // load limits (0 = none): over them the search stops
    int* overflow;                // set on a load or probe-limit overflow (per round, by the engine)
    long long ins0, ins1;         // this lane's new pairs since the last flush
    __device__ __forceinline__ int vertex(Item it) const { return (int)((it >> 32) & 0x7fffffffu); }
    __device__ __forceinline__ int graph(Item it) const { return (int)(it >> 63); }
    // labels change between the batches of one launch (the labelling passes of
    // the device-side batch loop), so they are read with coherent loads, never
    // through the read-only data path
    __device__ __forceinline__ uint64_t ctx(Item it) const { return (uint64_t)(uint32_t)label[vertex(it)]; }
    __device__ __forceinline__ int32_t load_ctx(Item it) const { return label[vertex(it)]; }
    __device__ __forceinline__ bool add(Item it) {
        const int d = graph(it);
        const bool ok = PairTable::insert_into(d ? keys[1] : keys[0], d ? mask[1] : mask[0], overflow, it & ~kDir);
        ins0 += ok && !d;
        ins1 += ok && d;
        return ok;
    }
    __device__ __forceinline__ bool seed(Item it) { return add(it); }
    __device__ __forceinline__ bool visit(Item parent, uint64_t c, int w, Item& child) {
        if (label[w] != (int32_t)(uint32_t)c) return false;
        child = (parent & kDir) | ((uint64_t)(uint32_t)w << 32) | (parent & 0xffffffffull);
        return add(child);
    }
    // warp-collective: add the warp's new pairs to the search's counters and
    // flag an overflow past a load limit (in the current round's flag, which
    // the engine points `overflow` at)
    __device__ __forceinline__ void flush(SearchCtl& sc) {
        long long c0 = ins0, c1 = ins1;
        for (int d = 16; d >= 1; d >>= 1) {
            c0 += __shfl_xor_sync(kFull, c0, d);
            c1 += __shfl_xor_sync(kFull, c1, d);
        }
        ins0 = ins1 = 0;
        if (lane_id() != 0) return;
        if (c0) {
            const unsigned long long t = atomicAdd(&sc.inserted[0], (unsigned long long)c0) + c0;
            if (max_ins[0] > 0 && (long long)t > max_ins[0]) atomicExch(overflow, 1);
        }
        if (c1) {
            const unsigned long long t = atomicAdd(&sc.inserted[1], (unsigned long long)c1) + c1;
            if (max_ins[1] > 0 && (long long)t > max_ins[1]) atomicExch(overflow, 1);
        }
    }
};

// Initial items of a pair search: (s, s) for every source, in direction 0
// (items [0, k)) and, with `both`, in direction 1 as well (items [k, 2k)).
struct InitPairs {
    const int32_t* sources;
    long long k;
    __device__ __forceinline__ uint64_t operator()(long long i) const {
        const bool d = i >= k;
        const uint32_t s = (uint32_t)sources[d ? i - k : i];
        return (d ? PolPair::kDir : 0ull) | ((uint64_t)s << 32) | s;
    }
};

// Plain multi-source reachability with 64-bit source masks: a vertex is
// (re)queued whenever it gains a source bit; at the fixpoint mask[v] is the set
// of sources reaching v.
struct PolMask {
    using Item = uint32_t;
    static constexpr int kQueue = 256;
    static constexpr bool kCountInserts = false;
    static constexpr bool kDense = false;
    static constexpr bool kCtxInQueue = false;
    using Ctx = uint64_t;  // the per-item value an arc test reads
    static constexpr bool kTwoGraphs = false;
    static constexpr bool kInject = false;
    static constexpr const char* kName = "mask-reach";
    unsigned long long* mask;
    bool test_first;  // read the target's mask before the atomic (high-degree graphs)
    __device__ __forceinline__ int vertex(Item it) const { return (int)it; }
    __device__ __forceinline__ uint64_t ctx(Item it) const { return ld_volatile(&mask[it]); }
    __device__ __forceinline__ bool seed(Item) const { return true; }
    // on low-degree graphs the atomic is the test (one dependent access less
    // per step); on high-degree ones most targets already carry the sources,
    // and a plain read first saves the atomic
    __device__ __forceinline__ bool visit(Item, uint64_t mu, int w, Item& child) const {
        if (test_first && (mu & ~ld_volatile(&mask[w])) == 0) return false;
        const unsigned long long old = atomicOr(&mask[w], (unsigned long long)mu);
        child = (Item)w;
        return (mu & ~old) != 0;
    }
};

// reach_multi with up to 128 sources: two 64-bit words per vertex, mask[2 v]
// holding sources 0..63 and mask[2 v + 1] sources 64..127 (the same search as
// PolMask, with the item's two words as its context).
struct Mask128 {
    unsigned long long lo, hi;
};
__device__ __forceinline__ Mask128 shfl_any(const Mask128& v, int src) {
    return {__shfl_sync(kFull, v.lo, src), __shfl_sync(kFull, v.hi, src)};
}
struct PolMask2 {
    using Item = uint32_t;
    static constexpr int kQueue = 256;
    static constexpr bool kCountInserts = false;
    static constexpr bool kDense = false;
    static constexpr bool kCtxInQueue = false;
    using Ctx = Mask128;
    static constexpr bool kTwoGraphs = false;
    static constexpr bool kInject = false;
    static constexpr const char* kName = "mask-reach-128";
    unsigned long long* mask;
    bool test_first;  // read the target's words before the atomics (high-degree graphs)
    __device__ __forceinline__ int vertex(Item it) const { return (int)it; }
    __device__ __forceinline__ Mask128 ctx(Item it) const {
        return {ld_volatile(&mask[2 * (size_t)it]), ld_volatile(&mask[2 * (size_t)it + 1])};
    }
    __device__ __forceinline__ bool seed(Item) const { return true; }
    __device__ __forceinline__ bool visit(Item, const Mask128& mu, int w, Item& child) const {
        unsigned long long* tw = mask + 2 * (size_t)w;
        if (test_first && ((mu.lo & ~ld_volatile(&tw[0])) | (mu.hi & ~ld_volatile(&tw[1]))) == 0) return false;
        const unsigned long long o0 = mu.lo ? atomicOr(&tw[0], mu.lo) : 0ull;
        const unsigned long long o1 = mu.hi ? atomicOr(&tw[1], mu.hi) : 0ull;
        child = (Item)w;
        return ((mu.lo & ~o0) | (mu.hi & ~o1)) != 0;
    }
};

// Low-diameter decomposition (Sec. 5.1, Alg. 4 function LDD) on the symmetric
// graph: vertex items; an arc (u, w) claims an unvisited w for u's centre
// (center[w] = center[u] by CAS from -1: Alg. 4 "visit[u] <- true, L(u) <-
// L(v)"). The centre travels with an item in the local queue; an item read
// from the bag takes it from center[]. With VGC a round explores up to tau
// arcs from an item instead of one BFS level (reachability, not BFS order, is
// what the decomposition needs; Sec. 5.1). At the end of round i the unvisited
// vertices of batch i + 1 of the seeded order become centres of their own and
// join the frontier (Alg. 4, F = F' + B_i); the search ends when the frontier
// is empty and no batch is left.
struct PolLdd {
    using Item = uint32_t;
    static constexpr int kQueue = 256;
    static constexpr bool kCountInserts = false;
    static constexpr bool kDense = true;
    static constexpr bool kCtxInQueue = true;
    using Ctx = uint64_t;  // the centre of the item's cluster
    static constexpr bool kTwoGraphs = false;
    static constexpr bool kInject = true;
    static constexpr const char* kName = "ldd";
    int32_t* center;          // -1: not yet claimed
    uint32_t* bits;           // claimed vertices (bits past n set), for dense rounds
    const int32_t* off;       // the symmetric CSR's offsets
    const int32_t* order;     // seeded order of all vertices
    const long long* bounds;  // batch i = order[bounds[i] .. bounds[i + 1])
    int nbatches;
    __device__ __forceinline__ int vertex(Item it) const { return (int)it; }
    __device__ __forceinline__ uint64_t ctx(Item it) const { return (uint64_t)(uint32_t)ld_volatile(&center[it]); }
    __device__ __forceinline__ int32_t load_ctx(Item it) const { return ld_volatile(&center[it]); }
    __device__ __forceinline__ bool seed(Item) const { return true; }  // items are claimed when pushed
    // a claim is the CAS on the centre; its winner also marks the vertex visited
    __device__ __forceinline__ bool claim(int w, int32_t c) const {
        if (ld_volatile(&center[w]) >= 0 || atomicCAS(&center[w], -1, c) != -1) return false;
        atomicOr(&bits[w >> 5], 1u << (w & 31));
        return true;
    }
    __device__ __forceinline__ bool visit(Item, uint64_t c, int w, Item& child) const {
        child = (Item)w;
        return claim(w, (int32_t)(uint32_t)c);
    }
    // dense rounds (the graph is symmetric: a vertex's in-arcs are its arcs):
    // an unvisited vertex with a neighbour in the frontier joins that
    // neighbour's cluster, whose centre was settled in an earlier round
    __device__ __forceinline__ void adopt(int v, int u) const { center[v] = ld_volatile(&center[u]); }
    __device__ __forceinline__ bool more(uint32_t i) const { return (long long)i + 2 < (long long)nbatches; }
    // warp-collective: the unvisited vertices of batch i + 1 claim themselves
    // and go into this round's bag (an isolated one is a cluster of its own
    // with nothing to expand: it is claimed but not pushed)
    __device__ __forceinline__ void inject(uint32_t i, const BagRef<Item>& out, SegState& st, uint32_t wid,
                                           uint32_t nwarps, uint32_t round, unsigned long long& pushed) const {
        if ((long long)i + 1 >= (long long)nbatches) return;
        const long long p0 = bounds[i + 1], p1 = bounds[i + 2];
        const int lane = lane_id();
        for (long long p = p0 + (long long)wid * 32; p < p1; p += (long long)nwarps * 32) {
            const long long q = p + lane;
            const int v = q < p1 ? order[q] : -1;
            const bool push = v >= 0 && claim(v, v) && off[v + 1] > off[v];
            pushed += bag_push<Item>(out, st, push, (Item)(push ? v : 0), wid, round);
        }
    }
};

}  // namespace scc
