// Reachability engine: vertical granularity control (VGC) local searches over a
// hash-bag frontier, in one persistent cooperative kernel (sm_103a).
//
// Paper: Wang, Dong, Gu, Sun, SIGMOD 2023.
//  - Alg. 3 (reachability with a hash bag): rounds; every frontier item is
//    expanded, newly visited items go to the bag H, F_{i+1} = H.ExtractAll().
//  - Sec. 3.1-3.2 (VGC): an item is expanded by a local search that keeps
//    newly visited items in a local queue and keeps expanding them until about
//    tau arcs have been examined; what is left in the queue is flushed to the
//    bag. An item with more than tau out-arcs is expanded "in parallel".
//  - Sec. 3.3 + Fig. 5 (hash bag): a preallocated slot array split into chunks
//    of lambda, 2*lambda, ... slots; inserts go to a random position of the
//    current chunk r with CAS and linear probing; sampled inserts count towards
//    sigma, at which point r advances by CAS (also after kappa failed probes);
//    ExtractAll packs the used prefix.
//
// GPU mapping (what differs from the 96-core design):
//  - The unit of a local search is a WARP task, not a thread: a warp takes up to
//    `seeds` frontier items, keeps its local queue in shared memory and expands
//    the next batch of queued items cooperatively (one arc per lane: a warp scan
//    of the batch's degrees and a 5-step shuffle search map lanes to arcs, so
//    reads of each adjacency row are coalesced). tau bounds the arcs of a task.
//  - "Expand in parallel" = hub items: an item with more than tau out-arcs
//    found inside a local search is returned to the bag; at extraction it is
//    cut into 1024-arc segments that all warps share in the next round.
//  - The hash bag is claimed in 32-slot segments (one CAS per segment, at a
//    random segment of the current chunk, linear probing over segments), so a
//    warp writes its spills as full 128/256-byte lines. Sampling and the chunk
//    advance are as in Fig. 5 but counted per segment claim.
//  - Rounds are separated by a grid barrier inside one cooperative launch; the
//    host is not involved between rounds.
#pragma once
#include "common.cuh"

namespace scc {

constexpr int kSeg = 32;         // slots per hash-bag segment
constexpr int kHubSeg = 1024;    // arcs of one hub segment
constexpr int kMaxChunks = 48;
constexpr int kBagProbe = 16;    // kappa: segment probes before a chunk advance
constexpr int kTableProbe = 256; // pair-table probe limit (then: overflow, regrow)

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
    int r;                     // current chunk
    int sample[kMaxChunks];    // sampled segment claims per chunk
};

struct EngineCtl {
    GridBarrier bar;
    int err;        // first error (SCC_ERR_*)
    int overflow;   // pair table over its load limit / probe limit
    int rounds;     // extraction rounds executed
    int max_chunk;  // largest bag chunk used
    long long fsize[2];
    long long work[2];
    long long hubseg[2];
    int nhub[2];
    BagCtl bag[2];
    unsigned long long edges;     // arcs examined
    unsigned long long inserted;  // newly visited items (pairs in pair mode)
    unsigned long long items;     // items expanded (adjacency rows read)
};

template <class Item>
struct EngineParams {
    const int32_t* off;
    const int32_t* adj;
    int32_t n;
    int tau;       // VGC arc budget per warp task
    int hub_thr;   // out-degree above which an item is a hub
    int seeds;     // frontier items per warp task (<= 32)
    // hash bag
    Item* slots;
    long long nslots;
    int lambda;
    int sigma;
    // frontier and hub lists (one buffer each; counters are double-buffered)
    Item* front;
    long long front_cap;
    Item* hub_item;
    int32_t* hub_beg;
    int32_t* hub_deg;
    long long* hub_segbase;
    int hub_cap;
    int32_t* segmap;
    long long segmap_cap;
    // initial items, pushed before round 0
    const Item* init;
    long long ninit;
    long long max_inserted;  // pair-mode load limit (0 = none)
    EngineCtl* ctl;
};

// ------------------------------------------------------------ chunk geometry --
__device__ __forceinline__ long long chunk_begin(int lambda, int j) {
    return (long long)lambda * ((1ll << j) - 1);
}
__device__ __forceinline__ long long chunk_end(int lambda, int j, long long nslots) {
    long long e = (long long)lambda * ((1ll << (j + 1)) - 1);
    return e < nslots ? e : nslots;
}

// ------------------------------------------------------------- bag writer --
// Warp-uniform state of the segment a warp is filling.
struct SegState {
    long long base;  // slot index of the segment, -1 = none
    int fill;
    uint32_t seq;    // claim counter (random positions)
};

// Claim a free segment of the current chunk (lane 0 only). Returns slot index or
// -1 (bag exhausted: error recorded).
template <class Item, class P>
__device__ long long bag_claim(const P& prm, BagCtl* bc, uint32_t wid, uint32_t round, uint32_t& seq) {
    for (int attempt = 0; attempt < 4 * kMaxChunks; ++attempt) {
        int r = ld_volatile(&bc->r);
        long long cb = chunk_begin(prm.lambda, r);
        long long ce = chunk_end(prm.lambda, r, prm.nslots);
        long long nseg = (ce - cb) / kSeg;
        if (nseg <= 0) {
            atomicCAS(&prm.ctl->err, 0, SCC_ERR_CAPACITY);
            return -1;
        }
        uint64_t h = mix64(((uint64_t)wid << 40) ^ ((uint64_t)round << 20) ^ (uint64_t)(seq++) ^ 0x5bd1e995ull);
        long long pos = (long long)(h % (uint64_t)nseg);
        for (int pr = 0; pr < kBagProbe; ++pr) {
            long long idx = cb + ((pos + pr) % nseg) * kSeg;
            Item prev = atomicCAS((typename std::conditional<sizeof(Item) == 8, unsigned long long, unsigned int>::type*)&prm.slots[idx],
                                  Sent<Item>::empty, Sent<Item>::claimed);
            if (prev == Sent<Item>::empty) {
                // sampled claim: rate sigma / (alpha * nseg), alpha = 1/2
                uint32_t rnd = (uint32_t)(h >> 32);
                double rate = 2.0 * prm.sigma / (double)nseg;
                if (rate >= 1.0 || (double)rnd < rate * 4294967296.0) {
                    int s = atomicAdd(&bc->sample[r], 1) + 1;
                    if (s >= prm.sigma && ce < prm.nslots) atomicCAS(&bc->r, r, r + 1);
                }
                if (r > ld_volatile(&prm.ctl->max_chunk)) atomicMax(&prm.ctl->max_chunk, r);
                return idx;
            }
        }
        // kappa probes failed: the chunk is (nearly) full -> try_resize
        if (ce >= prm.nslots) {
            atomicCAS(&prm.ctl->err, 0, SCC_ERR_CAPACITY);
            return -1;
        }
        atomicCAS(&bc->r, r, r + 1);
    }
    atomicCAS(&prm.ctl->err, 0, SCC_ERR_CAPACITY);
    return -1;
}

// Warp-cooperative insert of the items of lanes with `has` (all lanes call).
template <class Item, class P>
__device__ __forceinline__ void bag_push(const P& prm, BagCtl* bc, SegState& st, bool has, Item it, uint32_t wid,
                                         uint32_t round) {
    uint32_t m = __ballot_sync(kFull, has);
    int cnt = __popc(m);
    if (cnt == 0) return;
    int rank = __popc(m & lanemask_lt());
    while (cnt > 0) {
        if (st.base < 0 || st.fill == kSeg) {
            long long b = -1;
            if (lane_id() == 0) b = bag_claim<Item>(prm, bc, wid, round, st.seq);
            b = __shfl_sync(kFull, b, 0);
            st.seq = __shfl_sync(kFull, st.seq, 0);
            if (b < 0) return;  // error recorded
            st.base = b;
            st.fill = 0;
        }
        int space = kSeg - st.fill;
        if (has && rank >= 0 && rank < space) prm.slots[st.base + st.fill + rank] = it;
        int used = cnt < space ? cnt : space;
        st.fill += used;
        rank -= used;
        cnt -= used;
        if (rank < 0) has = false;
    }
}

// ------------------------------------------------------------- the kernel --
template <class Pol>
struct EngineSmem {
    typename Pol::Item q[8 * Pol::kQueue];  // up to 8 warps per block share this
};

template <class Pol>
__device__ __forceinline__ void expand_batch(const EngineParams<typename Pol::Item>& P, Pol& pol, BagCtl* bc,
                                             SegState& st, uint32_t wid, uint32_t round,
                                             typename Pol::Item* q, uint32_t& qh, uint32_t& qt, int& t,
                                             bool seeds_phase, unsigned long long& edges,
                                             unsigned long long& items) {
    using Item = typename Pol::Item;
    constexpr uint32_t QM = Pol::kQueue - 1;
    const int lane = lane_id();
    int avail = (int)min(32u, qt - qh);
    Item it = Sent<Item>::empty;
    int beg = 0, deg = 0;
    if (lane < avail) {
        it = q[(qh + lane) & QM];
        int u = pol.vertex(it);
        beg = __ldg(&P.off[u]);
        deg = __ldg(&P.off[u + 1]) - beg;
    }
    // items past the seed batch with more than hub_thr arcs go back to the bag
    bool hub = !seeds_phase && lane < avail && deg > P.hub_thr;
    int d = (lane < avail && !hub) ? deg : 0;
    int pre = warp_incl_scan(d);
    int take = avail;
    if (!seeds_phase) {
        int remaining = P.tau - t;
        uint32_t m = __ballot_sync(kFull, lane < avail && (pre - d) < remaining);
        take = __popc(m);
        if (take < 1) take = 1;
        if (lane >= take) { d = 0; hub = false; }
        pre = warp_incl_scan(d);
    }
    qh += take;
    bag_push<Item>(P, bc, st, hub, it, wid, round);
    uint64_t ctx = (lane < take && !hub) ? pol.ctx(it) : 0;
    const int total = __shfl_sync(kFull, pre, 31);
    const int excl = pre - d;
    for (int base = 0; base < total; base += 32) {
        const int e = base + lane;
        // owner lane: number of lanes whose inclusive prefix is <= e
        int j = 0;
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
            int v = __shfl_sync(kFull, pre, j + step - 1);
            if (v <= e) j += step;
        }
        const int jexcl = __shfl_sync(kFull, excl, j);
        const int jbeg = __shfl_sync(kFull, beg, j);
        const Item jit = shfl_any(it, j);
        const uint64_t jctx = shfl_any(ctx, j);
        bool nw = false;
        Item child = Sent<Item>::empty;
        if (e < total) {
            int w = __ldg(&P.adj[jbeg + (e - jexcl)]);
            nw = pol.visit(jit, jctx, w, child);
        }
        // new items: local queue while it has room, the bag otherwise
        uint32_t m = __ballot_sync(kFull, nw);
        int cnt = __popc(m);
        if (cnt) {
            int rank = __popc(m & lanemask_lt());
            int room = (int)(Pol::kQueue - (qt - qh));
            bool toq = nw && rank < room;
            if (toq) q[(qt + rank) & QM] = child;
            int nq = cnt < room ? cnt : room;
            bag_push<Item>(P, bc, st, nw && !toq, child, wid, round);
            qt += nq;
        }
        __syncwarp();
    }
    t += total;
    edges += (lane == 0) ? (unsigned long long)total : 0ull;
    items += (lane == 0) ? (unsigned long long)take : 0ull;
}

// Dense (bottom-up) rounds of a single-reachability search (Sec. 4.2): every
// unvisited vertex of the class scans its in-arcs (the reverse CSR) and stops at
// the first one whose tail is in the current frontier. Used when the frontier
// holds at least n_active / frac_inv items.
struct DenseParams {
    const int32_t* roff;  // reverse CSR (G^T for a forward search, G for a backward one)
    const int32_t* radj;
    uint32_t* fbits;      // frontier bitmap scratch, ceil(n/32) words, all zero between rounds
    long long n_active;   // vertices of the class
    int frac_inv;         // 0 = never dense
};

// The initial items of a search: either an explicit list or the pairs (s, s)
// of a source list.
template <class Item>
struct InitList {
    const Item* items;
    __device__ __forceinline__ Item operator()(long long i) const { return items[i]; }
};
struct InitPairs {
    const int32_t* sources;
    __device__ __forceinline__ uint64_t operator()(long long i) const {
        uint32_t s = (uint32_t)sources[i];
        return ((uint64_t)s << 32) | s;
    }
};

// Per-warp accumulators of a search (folded into the control block at the end).
struct WarpStats {
    unsigned long long edges = 0, items = 0;
};

// One complete reachability search (Alg. 3 rounds) executed by every thread of a
// cooperative grid. Returns false if a grid barrier timed out (the caller must
// return at once). On return all blocks have passed the final barrier, so the
// control block's counters of this search are final.
template <class Pol, class Init>
__device__ bool engine_search(EngineParams<typename Pol::Item> P, Pol& pol, Init init, long long ninit,
                              const DenseParams* dp, typename Pol::Item* q, WarpStats& ws) {
    using Item = typename Pol::Item;
    constexpr uint32_t QM = Pol::kQueue - 1;
    __shared__ long long s_tile[1];
    __shared__ int s_wsum[32];
    EngineCtl* ctl = P.ctl;
    const int lane = lane_id();
    const int wib = threadIdx.x >> 5;
    const uint32_t wid = (uint32_t)(blockIdx.x * (blockDim.x >> 5) + wib);
    const uint32_t nwarps = (uint32_t)(gridDim.x * (blockDim.x >> 5));

    // ---- fresh per-search state (the bag slots are already empty)
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        for (int p = 0; p < 2; ++p) {
            ctl->fsize[p] = 0;
            ctl->work[p] = 0;
            ctl->hubseg[p] = 0;
            ctl->nhub[p] = 0;
            ctl->bag[p].r = 0;
            for (int j = 0; j < kMaxChunks; ++j) ctl->bag[p].sample[j] = 0;
        }
        ctl->overflow = 0;
        ctl->inserted = 0;
        ctl->rounds = 0;
    }
    if (!grid_sync(&ctl->bar, &ctl->err)) return false;

    // ---- round -1: the initial items (marked visited) go into bag[1]
    {
        SegState st{-1, 0, 0};
        long long ins = 0;
        for (long long b = (long long)wid * 32; b < ninit; b += (long long)nwarps * 32) {
            long long i = b + lane;
            bool has = false;
            Item it = Sent<Item>::empty;
            if (i < ninit) {
                it = init(i);
                has = pol.seed(it);
            }
            ins += __popc(__ballot_sync(kFull, has));
            bag_push<Item>(P, &ctl->bag[1], st, has, it, wid, 0xffffu);
        }
        if constexpr (Pol::kCountInserts) {
            if (lane == 0 && ins) atomicAdd(&ctl->inserted, (unsigned long long)ins);
        }
    }
    if (!grid_sync(&ctl->bar, &ctl->err)) return false;

    bool prev_dense = false;
    for (uint32_t iter = 0;; ++iter) {
        const int p = iter & 1;
        // ---- ExtractAll: pack bag[(iter+1)&1]'s used prefix into the frontier
        // (light items) and the hub list; every slot read is reset to empty.
        {
            BagCtl* rb = &ctl->bag[(iter + 1) & 1];
            const int r = ld_volatile(&rb->r);
            const long long end = chunk_end(P.lambda, r, P.nslots);
            const long long tile = (long long)blockDim.x * 4;
            for (long long tb = (long long)blockIdx.x * tile; tb < end; tb += (long long)gridDim.x * tile) {
                Item x[4];
                bool light[4];
                int nl = 0;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    long long i = tb + threadIdx.x + (long long)k * blockDim.x;
                    x[k] = Sent<Item>::empty;
                    light[k] = false;
                    if (i < end) {
                        x[k] = P.slots[i];
                        if (x[k] != Sent<Item>::empty) P.slots[i] = Sent<Item>::empty;
                    }
                    if (x[k] != Sent<Item>::empty && x[k] != Sent<Item>::claimed) {
                        int v = pol.vertex(x[k]);
                        int b0 = __ldg(&P.off[v]);
                        int dg = __ldg(&P.off[v + 1]) - b0;
                        bool ok_hub = false;
                        if (dg > P.hub_thr) {
                            int h = atomicAdd(&ctl->nhub[p], 1);
                            if (h < P.hub_cap) {
                                long long ns = ceil_div(dg, kHubSeg);
                                long long sb = atomicAdd((unsigned long long*)&ctl->hubseg[p], (unsigned long long)ns);
                                long long lim = sb + ns < P.segmap_cap ? sb + ns : P.segmap_cap;
                                if (sb + ns <= P.segmap_cap) {
                                    P.hub_item[h] = x[k];
                                    P.hub_beg[h] = b0;
                                    P.hub_deg[h] = dg;
                                    P.hub_segbase[h] = sb;
                                    for (long long g = sb; g < lim; ++g) P.segmap[g] = h;
                                    ok_hub = true;
                                } else {
                                    for (long long g = sb; g < lim; ++g) P.segmap[g] = -1;
                                }
                            }
                        }
                        light[k] = !ok_hub;
                        nl += light[k];
                    }
                }
                // block-aggregated reservation in the frontier
                int wsum = nl;
#pragma unroll
                for (int d = 16; d >= 1; d >>= 1) wsum += __shfl_xor_sync(kFull, wsum, d);
                int wpre = warp_incl_scan(nl) - nl;
                if (lane == 0) s_wsum[wib] = wsum;
                __syncthreads();
                if (threadIdx.x == 0) {
                    long long tot = 0;
                    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                        int c = s_wsum[w];
                        s_wsum[w] = (int)tot;
                        tot += c;
                    }
                    s_tile[0] = tot ? (long long)atomicAdd((unsigned long long*)&ctl->fsize[p], (unsigned long long)tot) : 0;
                }
                __syncthreads();
                long long pos = s_tile[0] + s_wsum[wib] + wpre;
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (light[k]) {
                        if (pos < P.front_cap) P.front[pos] = x[k];
                        else atomicCAS(&ctl->err, 0, SCC_ERR_CAPACITY);
                        ++pos;
                    }
                __syncthreads();
            }
            // the frontier bitmap of a previous dense round is cleared here
            if constexpr (Pol::kDense) {
                if (prev_dense) {
                    const long long nw = ((long long)P.n + 31) / 32;
                    for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < nw;
                         w += (long long)gridDim.x * blockDim.x)
                        if (dp->fbits[w]) dp->fbits[w] = 0;
                }
            }
        }
        if (!grid_sync(&ctl->bar, &ctl->err)) return false;
        if (ld_volatile(&ctl->err) != 0) break;
        const long long fsize = ld_volatile(&ctl->fsize[p]);
        const int nhub = min(ld_volatile(&ctl->nhub[p]), P.hub_cap);
        if (fsize == 0 && nhub == 0) break;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            ctl->fsize[p ^ 1] = 0;
            ctl->work[p ^ 1] = 0;
            ctl->hubseg[p ^ 1] = 0;
            ctl->nhub[p ^ 1] = 0;
            BagCtl* nb = &ctl->bag[(iter + 1) & 1];
            nb->r = 0;
            for (int j = 0; j < kMaxChunks; ++j) nb->sample[j] = 0;
            ctl->rounds = (int)iter + 1;
        }
        BagCtl* bc = &ctl->bag[iter & 1];
        SegState st{-1, 0, (uint32_t)(wid * 2654435761u)};
        const bool stop = P.max_inserted > 0 && ld_volatile(&ctl->overflow) != 0;

        bool dense = false;
        if constexpr (Pol::kDense) {
            dense = dp != nullptr && dp->frac_inv > 0 &&
                    (long long)(fsize + nhub) * (long long)dp->frac_inv >= dp->n_active;
        }
        prev_dense = dense;
        if (dense) {
            if constexpr (Pol::kDense) {
                // ---- dense round: frontier bitmap, then bottom-up over unvisited vertices
                for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < fsize + nhub;
                     i += (long long)gridDim.x * blockDim.x) {
                    const int v = pol.vertex(i < fsize ? P.front[i] : P.hub_item[i - fsize]);
                    atomicOr(&dp->fbits[v >> 5], 1u << (v & 31));
                }
                if (!grid_sync(&ctl->bar, &ctl->err)) return false;
                const long long nw = ((long long)P.n + 31) / 32;
                for (long long w = wid; w < nw; w += nwarps) {
                    const uint32_t word = pol.bits[w];
                    const long long v = w * 32 + lane;
                    bool found = false;
                    unsigned long long scanned = 0;
                    if (v < P.n && !((word >> lane) & 1u)) {
                        const int e0 = __ldg(&dp->roff[v]), e1 = __ldg(&dp->roff[v + 1]);
                        for (int e = e0; e < e1; ++e) {
                            const int u = __ldg(&dp->radj[e]);
                            ++scanned;
                            if ((ld_volatile(&dp->fbits[u >> 5]) >> (u & 31)) & 1u) {
                                found = true;
                                break;
                            }
                        }
                    }
                    const uint32_t m = __ballot_sync(kFull, found);
                    if (lane == 0 && m) pol.bits[w] = word | m;  // this warp owns word w in this round
                    for (int d = 16; d >= 1; d >>= 1) scanned += __shfl_xor_sync(kFull, scanned, d);
                    if (lane == 0) {
                        ws.edges += scanned;
                        ws.items += __popc(m);
                    }
                    bag_push<Item>(P, bc, st, found, (Item)v, wid, iter);
                }
            }
        } else {
            // ---- phase A: hub segments, shared by all warps ("in parallel")
            const long long nseg = min(ld_volatile(&ctl->hubseg[p]), P.segmap_cap);
            for (long long g = wid; g < nseg && !stop; g += nwarps) {
                const int h = P.segmap[g];
                if (h < 0) continue;
                const Item hit = P.hub_item[h];
                const long long j0 = (g - P.hub_segbase[h]) * kHubSeg;
                const int b0 = P.hub_beg[h] + (int)j0;
                const int len = (int)min((long long)kHubSeg, (long long)P.hub_deg[h] - j0);
                const uint64_t hctx = pol.ctx(hit);
                for (int e0 = 0; e0 < len; e0 += 32) {
                    bool nw = false;
                    Item child = Sent<Item>::empty;
                    if (e0 + lane < len) {
                        int w = __ldg(&P.adj[b0 + e0 + lane]);
                        nw = pol.visit(hit, hctx, w, child);
                    }
                    bag_push<Item>(P, bc, st, nw, child, wid, iter);
                }
                ws.edges += lane == 0 ? (unsigned long long)len : 0ull;
                ws.items += (lane == 0 && g == P.hub_segbase[h]) ? 1ull : 0ull;
            }

            // ---- phase B: warp tasks over the light frontier (VGC local searches)
            for (;;) {
                long long b = 0;
                if (lane == 0) b = (long long)atomicAdd((unsigned long long*)&ctl->work[p], (unsigned long long)P.seeds);
                b = __shfl_sync(kFull, b, 0);
                if (b >= fsize) break;
                if (P.max_inserted > 0 && ld_volatile(&ctl->overflow) != 0) break;
                int cnt = (int)min((long long)P.seeds, fsize - b);
                if (lane < cnt) q[lane] = P.front[b + lane];
                __syncwarp();
                uint32_t qh = 0, qt = (uint32_t)cnt;
                int t = 0;
                expand_batch<Pol>(P, pol, bc, st, wid, iter, q, qh, qt, t, true, ws.edges, ws.items);
                while (qt != qh && t < P.tau)
                    expand_batch<Pol>(P, pol, bc, st, wid, iter, q, qh, qt, t, false, ws.edges, ws.items);
                // budget spent: flush what is left in the local queue
                while (qt != qh) {
                    int nrem = (int)min(32u, qt - qh);
                    Item it = lane < nrem ? q[(qh + lane) & QM] : Sent<Item>::empty;
                    qh += nrem;
                    bag_push<Item>(P, bc, st, lane < nrem, it, wid, iter);
                }
                __syncwarp();
                if constexpr (Pol::kCountInserts) {
                    long long c = pol.take_inserted();
                    if (c && lane == 0) {
                        unsigned long long tot = atomicAdd(&ctl->inserted, (unsigned long long)c) + c;
                        if (P.max_inserted > 0 && (long long)tot > P.max_inserted) atomicExch(&ctl->overflow, 1);
                    }
                }
            }
            if constexpr (Pol::kCountInserts) {
                long long c = pol.take_inserted();
                if (c && lane == 0) {
                    unsigned long long tot = atomicAdd(&ctl->inserted, (unsigned long long)c) + c;
                    if (P.max_inserted > 0 && (long long)tot > P.max_inserted) atomicExch(&ctl->overflow, 1);
                }
            }
        }
        if (!grid_sync(&ctl->bar, &ctl->err)) return false;
        if (P.max_inserted > 0 && ld_volatile(&ctl->overflow) != 0) break;
    }
    return true;
}

template <class Pol>
__global__ void __launch_bounds__(256) engine_kernel(EngineParams<typename Pol::Item> P, Pol pol_in, DenseParams dp) {
    Pol pol = pol_in;
    __shared__ EngineSmem<Pol> sm;
    typename Pol::Item* q = sm.q + (threadIdx.x >> 5) * Pol::kQueue;
    WarpStats ws;
    const bool ok = engine_search<Pol>(P, pol, InitList<typename Pol::Item>{P.init}, P.ninit,
                                       dp.frac_inv > 0 ? &dp : nullptr, q, ws);
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
    static constexpr int kQueue = 512;
    static constexpr bool kCountInserts = false;
    static constexpr bool kDense = true;
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
    __device__ __forceinline__ long long take_inserted() { return 0; }
};

// Pair table (Sec. 4.3 phase-concurrent hash table of reachability pairs):
// open addressing over uint64 keys v << 32 | s, linear probing, insert-if-absent.
struct PairTable {
    unsigned long long* keys;
    unsigned long long mask;  // capacity - 1 (capacity a power of two)
    int* overflow;
    __device__ __forceinline__ static unsigned long long hash(unsigned long long k) { return mix64(k); }
    __device__ __forceinline__ bool insert(unsigned long long key) const {
        unsigned long long h = hash(key) & mask;
        for (int i = 0; i < kTableProbe; ++i) {
            unsigned long long cur = ld_volatile(&keys[h]);
            if (cur == key) return false;
            if (cur == ~0ull) {
                unsigned long long prev = atomicCAS(&keys[h], ~0ull, key);
                if (prev == ~0ull) return true;
                if (prev == key) return false;
            }
            h = (h + 1) & mask;
        }
        atomicExch(overflow, 1);
        return false;
    }
    __device__ __forceinline__ bool contains(unsigned long long key) const {
        unsigned long long h = hash(key) & mask;
        for (unsigned long long i = 0; i <= mask; ++i) {
            unsigned long long cur = keys[h];
            if (cur == key) return true;
            if (cur == ~0ull) return false;
            h = (h + 1) & mask;
        }
        return false;
    }
};

// Multi-reachability: pair items (v, s); an arc (u, w) is followed only when
// label[w] == label[u] (Alg. 1: MultiReach skips (u, v) with L(u) != L(v);
// finished vertices carry kDone < 0 and never match an active class).
struct PolPair {
    using Item = uint64_t;
    static constexpr int kQueue = 256;
    static constexpr bool kCountInserts = true;
    static constexpr bool kDense = false;
    const int32_t* label;
    PairTable tab;
    long long ins;
    __device__ __forceinline__ int vertex(Item it) const { return (int)(it >> 32); }
    __device__ __forceinline__ uint64_t ctx(Item it) const { return (uint64_t)(uint32_t)__ldg(&label[it >> 32]); }
    __device__ __forceinline__ bool seed(Item it) const { return tab.insert(it); }
    __device__ __forceinline__ bool visit(Item parent, uint64_t c, int w, Item& child) {
        if (__ldg(&label[w]) != (int32_t)(uint32_t)c) return false;
        child = ((uint64_t)(uint32_t)w << 32) | (parent & 0xffffffffull);
        bool ok = tab.insert(child);
        ins += ok;
        return ok;
    }
    __device__ __forceinline__ long long take_inserted() {
        long long c = ins;
        for (int d = 16; d >= 1; d >>= 1) c += __shfl_xor_sync(kFull, c, d);
        ins = 0;
        return c;
    }
};

// Plain multi-source reachability with 64-bit source masks: a vertex is
// (re)queued whenever it gains a source bit; at the fixpoint mask[v] is the set
// of sources reaching v.
struct PolMask {
    using Item = uint32_t;
    static constexpr int kQueue = 512;
    static constexpr bool kCountInserts = false;
    static constexpr bool kDense = false;
    unsigned long long* mask;
    __device__ __forceinline__ int vertex(Item it) const { return (int)it; }
    __device__ __forceinline__ uint64_t ctx(Item it) const { return ld_volatile(&mask[it]); }
    __device__ __forceinline__ bool seed(Item) const { return true; }
    __device__ __forceinline__ bool visit(Item, uint64_t mu, int w, Item& child) const {
        if ((mu & ~ld_volatile(&mask[w])) == 0) return false;
        unsigned long long old = atomicOr(&mask[w], (unsigned long long)mu);
        child = (Item)w;
        return (mu & ~old) != 0;
    }
    __device__ __forceinline__ long long take_inserted() { return 0; }
};

}  // namespace scc
