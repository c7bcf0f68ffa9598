// Least-element lists (Sec. 5.2, Alg. 5: the BGSS LE-lists algorithm) of the
// undirected graph under the arcs of G, unweighted (sm_103a).
//
// Source v_j (position j of a seeded vertex order) belongs to L(u) iff its hop
// distance to u is smaller than that of every earlier source. Alg. 5 takes the
// sources in batches of 1, 2, 4, ... and runs one multi-source BFS per batch:
//
//   * the BFS is level-synchronous (VGC does not apply: BFS order matters,
//     Sec. 5.2) in one cooperative launch over all batches, grid barriers
//     between levels;
//   * a frontier item is a (vertex, source) pair; a pair (w, s) is new when it
//     enters the batch's hash table of visited pairs (insert-if-absent with its
//     distance, the "parallel hash table" of Sec. 5.2), and it is only tried
//     when level + 1 < delta(w), the distance from w to the closest source of
//     the earlier batches (the pruning of Alg. 5);
//   * new pairs are appended to the next level's frontier, kept packed by a
//     warp-aggregated counter (what the hash bag gives the paper's CPU code: no
//     second pass over the frontier);
//   * at the end of a batch every pair of the table goes to a log of candidate
//     entries (u, s, d) and lowers delta(u) (Alg. 5 "delta(u) <- min"); the
//     table is emptied for the next batch.
//
// A pair with d(s, w) < delta_b(w) is reached at its BFS distance (every vertex
// on a shortest path from s also passes the test), and no other pair is ever
// inserted, so after all batches the candidates at u, sorted by source
// position and kept while their distance strictly decreases (Alg. 5 "sort ...
// filter out triples that violate constraints"), are exactly L(u).
//
// A table over its load limit or a full candidate log stops the launch at the
// start of the batch; the host grows the buffer and relaunches from it.
#include <algorithm>
#include <climits>
#include <vector>

#include "common.cuh"
#include "engine.cuh"
#include "internal.h"

namespace scc {
namespace {

constexpr unsigned long long kEmpty = ~0ull;
constexpr int kLeProbe = 64;  // probes of an insert before the table counts as full

struct LeCtl {
    GridBarrier bar;
    int err;
    int status;                    // 0 done, 1 grow the table, 2 grow the log
    int batch;                     // the batch to resume at
    unsigned long long fr_n[3];    // frontier counters, a ring over the levels
    int full[3];                   // table-full flags, the same ring: a level
                                   // writes only the slot of its own output, so
                                   // a block still deciding about the previous
                                   // level never sees the next level's writes
    unsigned long long ins;        // pairs inserted in the current batch
    unsigned long long log_n;      // candidates logged so far
    int levels;                    // BFS levels run (statistics)
    unsigned long long edges;      // arcs examined (statistics)
};

struct LeParams {
    const int32_t* soff;
    const int32_t* sadj;
    int32_t n;
    const int32_t* order;
    const long long* bounds;
    int nb;
    int32_t* delta;
    unsigned long long* keys;  // visited pairs of the batch: w << 32 | s
    int32_t* kdist;
    unsigned long long mask;   // table capacity - 1
    unsigned long long* fr[2];
    int32_t* log_u;
    int32_t* log_s;
    int32_t* log_d;
    unsigned long long log_cap;
    LeCtl* ctl;
};

// Insert-if-absent of key with its distance; true if the key is new. Sets
// *full past the probe limit.
__device__ __forceinline__ bool le_insert(const LeParams& P, unsigned long long key, int32_t d, int* full) {
    unsigned long long h = mix64(key) & P.mask;
    for (int i = 0; i < kLeProbe; ++i) {
        const unsigned long long prev = atomicCAS(&P.keys[h], kEmpty, key);
        if (prev == kEmpty) {
            P.kdist[h] = d;
            return true;
        }
        if (prev == key) return false;
        h = (h + 1) & P.mask;
    }
    atomicExch(full, 1);
    return false;
}

// Warp-aggregated append of the lanes with `has` to a packed array of cap
// entries (a level appends one entry per new table pair, so cap = the table's
// capacity suffices; past it the entry is dropped and *err set).
__device__ __forceinline__ void warp_append(unsigned long long* arr, unsigned long long cap, unsigned long long* cnt,
                                            bool has, unsigned long long x, int* err) {
    const uint32_t m = __ballot_sync(kFull, has);
    if (!m) return;
    unsigned long long base = 0;
    if (lane_id() == 0) base = atomicAdd(cnt, (unsigned long long)__popc(m));
    base = __shfl_sync(kFull, base, 0);
    const unsigned long long at = base + __popc(m & lanemask_lt());
    if (has) {
        if (at < cap) arr[at] = x;
        else atomicExch(err, SCC_ERR_INTERNAL);
    }
}

__global__ void __launch_bounds__(kEngineBlock) k_le_lists(LeParams P) {
    LeCtl* ctl = P.ctl;
    const int lane = lane_id();
    const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long gstride = (long long)gridDim.x * blockDim.x;
    const long long wid = gtid >> 5, nwarps = gstride >> 5;
    unsigned long long edges = 0;
    const unsigned long long load_limit = (P.mask + 1) / 4 * 3;
    for (int b = ld_volatile(&ctl->batch); b < P.nb; ++b) {
        // ---- the batch's sources at distance 0
        if (gtid == 0) {
            for (int r = 0; r < 3; ++r) {
                ctl->fr_n[r] = 0;
                ctl->full[r] = 0;
            }
            ctl->ins = 0;
        }
        if (!grid_sync(&ctl->bar, &ctl->err)) return;
        const long long p0 = P.bounds[b], p1 = P.bounds[b + 1];
        for (long long base = p0 + (gtid - lane); base < p1; base += gstride) {
            const long long p = base + lane;
            bool nw = false;
            unsigned long long key = 0;
            if (p < p1) {
                const int s = P.order[p];
                key = ((unsigned long long)(uint32_t)s << 32) | (uint32_t)s;
                nw = ld_volatile(&P.delta[s]) > 0 && le_insert(P, key, 0, &ctl->full[0]);
            }
            warp_append(P.fr[0], P.mask + 1, &ctl->fr_n[0], nw, key, &ctl->err);
            const int c = __popc(__ballot_sync(kFull, nw));
            if (lane == 0 && c && atomicAdd(&ctl->ins, (unsigned long long)c) + c > load_limit)
                atomicExch(&ctl->full[0], 1);
        }
        if (!grid_sync(&ctl->bar, &ctl->err)) return;
        // Every block takes the same decisions below: it reads only counters
        // and flags that no block writes again before the next barrier. The
        // pairs of the batch so far (every new pair enters exactly one
        // frontier) are summed per block from the settled frontier counts.
        unsigned long long ins_b = ld_volatile(&ctl->fr_n[0]);
        bool full = ld_volatile(&ctl->full[0]) != 0 || ins_b > load_limit;
        // ---- BFS levels (one warp per frontier pair, lanes over the arcs)
        for (int lev = 0; !full; ++lev) {
            const int cur = lev & 1;
            unsigned long long* in = P.fr[cur];
            unsigned long long* out = P.fr[cur ^ 1];
            const int o = (lev + 1) % 3;
            unsigned long long* out_n = &ctl->fr_n[o];
            int* out_full = &ctl->full[o];
            if (gtid == 0) {  // read last level, written next level
                ctl->fr_n[(lev + 2) % 3] = 0;
                ctl->full[(lev + 2) % 3] = 0;
            }
            const long long cnt = (long long)ld_volatile(&ctl->fr_n[lev % 3]);
            const int32_t nd = lev + 1;
            for (long long i = wid; i < cnt; i += nwarps) {
                // once the table is over a limit the batch starts over and the
                // rest of the level is moot: stop taking items
                int stop = lane == 0 ? ld_volatile(out_full) : 0;
                if (__shfl_sync(kFull, stop, 0) != 0) break;
                const unsigned long long it = in[i];
                const int u = (int)(it >> 32);
                const unsigned long long sbits = it & 0xffffffffull;
                const int a0 = P.soff[u], a1 = P.soff[u + 1];
                for (int e0 = a0; e0 < a1; e0 += 32) {
                    const int e = e0 + lane;
                    bool nw = false;
                    unsigned long long key = 0;
                    if (e < a1) {
                        const int w = P.sadj[e];
                        key = ((unsigned long long)(uint32_t)w << 32) | sbits;
                        nw = nd < ld_volatile(&P.delta[w]) && le_insert(P, key, nd, out_full);
                    }
                    warp_append(out, P.mask + 1, out_n, nw, key, &ctl->err);
                    const int c = __popc(__ballot_sync(kFull, nw));
                    if (lane == 0 && c && atomicAdd(&ctl->ins, (unsigned long long)c) + c > load_limit)
                        atomicExch(out_full, 1);
                }
                if (lane == 0) edges += (unsigned long long)(a1 - a0);
            }
            if (!grid_sync(&ctl->bar, &ctl->err)) return;
            const unsigned long long nout = ld_volatile(out_n);
            ins_b += nout;
            full = ld_volatile(out_full) != 0 || ins_b > load_limit;
            if (gtid == 0) ctl->levels += 1;
            if (nout == 0) break;  // an empty next frontier ends the batch
        }
        // a table past its probe or load limit grows and the batch starts over
        if (full && gtid == 0) atomicExch(&ctl->status, 1);
        if (!grid_sync(&ctl->bar, &ctl->err)) return;
        if (ld_volatile(&ctl->status) == 0 && ld_volatile(&ctl->log_n) + ld_volatile(&ctl->ins) > P.log_cap &&
            gtid == 0)
            atomicExch(&ctl->status, 2);
        if (!grid_sync(&ctl->bar, &ctl->err)) return;
        if (ld_volatile(&ctl->status) != 0) {  // the host grows a buffer and resumes at this batch
            if (gtid == 0) ctl->batch = b;
            break;
        }
        // ---- the batch's pairs: candidates, delta, and an empty table
        for (long long base = gtid - lane; base <= (long long)P.mask; base += gstride) {
            const long long h = base + lane;
            unsigned long long key = kEmpty;
            if (h <= (long long)P.mask) {
                key = P.keys[h];
                if (key != kEmpty) P.keys[h] = kEmpty;
            }
            const bool has = key != kEmpty;
            const uint32_t m = __ballot_sync(kFull, has);
            if (!m) continue;
            unsigned long long o = 0;
            if (lane == 0) o = atomicAdd(&ctl->log_n, (unsigned long long)__popc(m));
            o = __shfl_sync(kFull, o, 0) + __popc(m & lanemask_lt());
            if (has) {
                const int u = (int)(key >> 32);
                const int d = P.kdist[h];
                P.log_u[o] = u;
                P.log_s[o] = (int32_t)(key & 0xffffffffull);
                P.log_d[o] = d;
                atomicMin(&P.delta[u], d);
            }
        }
        if (!grid_sync(&ctl->bar, &ctl->err)) return;
        if (gtid == 0) ctl->batch = b + 1;
    }
    if (lane == 0 && edges) atomicAdd(&ctl->edges, edges);
}

// ------------------------------------------------------------ assembly --
__global__ void k_le_count(const int32_t* __restrict__ log_u, long long total, int32_t* cnt) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x)
        atomicAdd(&cnt[log_u[i]], 1);
}
__global__ void k_le_scatter(const int32_t* __restrict__ log_u, const int32_t* __restrict__ log_s,
                             const int32_t* __restrict__ log_d, long long total, int32_t* cursor, int32_t* gs,
                             int32_t* gd) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int p = atomicAdd(&cursor[log_u[i]], 1);
        gs[p] = log_s[i];
        gd[p] = log_d[i];
    }
}
// In-place heapsort of k (source, distance) entries by the source's position.
__device__ void heap_sift(int32_t* gs, int32_t* gd, int i, int k, const int32_t* __restrict__ rank) {
    for (;;) {
        int c = 2 * i + 1;
        if (c >= k) return;
        if (c + 1 < k && rank[gs[c + 1]] > rank[gs[c]]) ++c;
        if (rank[gs[c]] <= rank[gs[i]]) return;
        const int ts = gs[i], td = gd[i];
        gs[i] = gs[c];
        gd[i] = gd[c];
        gs[c] = ts;
        gd[c] = td;
        i = c;
    }
}
__device__ void heap_sort(int32_t* gs, int32_t* gd, int k, const int32_t* __restrict__ rank) {
    for (int i = k / 2 - 1; i >= 0; --i) heap_sift(gs, gd, i, k, rank);
    for (int e = k - 1; e > 0; --e) {
        const int ts = gs[0], td = gd[0];
        gs[0] = gs[e];
        gd[0] = gd[e];
        gs[e] = ts;
        gd[e] = td;
        heap_sift(gs, gd, 0, e, rank);
    }
}

// One thread per vertex: its candidates sorted by source position, kept while
// their distance strictly decreases; keep[u] = the survivors (compacted to the
// front of the vertex's range).
__global__ void k_le_filter(int32_t n, const int32_t* __restrict__ pos, const int32_t* __restrict__ rank, int32_t* gs,
                            int32_t* gd, int32_t* keep) {
    for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (long long)gridDim.x * blockDim.x) {
        const int a0 = pos[u], a1 = pos[u + 1];
        if (a1 - a0 <= 32) {
            for (int i = a0 + 1; i < a1; ++i) {  // insertion sort by the source's position
                const int s = gs[i], d = gd[i], r = rank[s];
                int j = i - 1;
                while (j >= a0 && rank[gs[j]] > r) {
                    gs[j + 1] = gs[j];
                    gd[j + 1] = gd[j];
                    --j;
                }
                gs[j + 1] = s;
                gd[j + 1] = d;
            }
        } else {
            heap_sort(gs + a0, gd + a0, a1 - a0, rank);
        }
        int k = a0, best = INT_MAX;
        for (int i = a0; i < a1; ++i)
            if (gd[i] < best) {
                best = gd[i];
                gs[k] = gs[i];
                gd[k] = gd[i];
                ++k;
            }
        keep[u] = k - a0;
    }
}
__global__ void k_le_compact(int32_t n, const int32_t* __restrict__ pos, const int32_t* __restrict__ kpos,
                             const int32_t* __restrict__ gs, const int32_t* __restrict__ gd, int64_t* le_off,
                             int32_t* le_src, int32_t* le_dist) {
    for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (long long)gridDim.x * blockDim.x) {
        const int k0 = kpos[u], k1 = kpos[u + 1], a0 = pos[u];
        le_off[u] = k0;
        if (u == n - 1) le_off[n] = k1;
        for (int i = 0; i < k1 - k0; ++i) {
            le_src[k0 + i] = gs[a0 + i];
            le_dist[k0 + i] = gd[a0 + i];
        }
    }
}
__global__ void k_le_rank(int32_t n, const int32_t* __restrict__ order, int32_t* rank, int32_t* delta) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        rank[order[i]] = (int32_t)i;
        delta[i] = INT_MAX;
    }
}

inline int grid_for(int64_t work, int per_block, int cap) {
    int64_t g = (work + per_block - 1) / per_block;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, cap));
}

}  // namespace

int le_lists_compute(const int32_t* soff, const int32_t* sadj, int32_t n, const int32_t* order, int num_sms,
                     LeResult* res, cudaStream_t s, long long init_cap, long long init_log) {
    *res = LeResult();
    if (n == 0) return SCC_OK;
    Scratch tmp(s);
    // batches of 1, 2, 4, ... sources (Alg. 5)
    std::vector<long long> bounds{0};
    for (long long sz = 1, pos = 0; pos < n; sz *= 2) {
        pos = std::min<long long>(n, pos + sz);
        bounds.push_back(pos);
    }
    const int nb = (int)bounds.size() - 1;
    long long* bounds_d = nullptr;
    int32_t *rank = nullptr, *delta = nullptr;
    LeCtl* ctl = nullptr;
    SCC_TRY(tmp.alloc(&bounds_d, bounds.size()));
    SCC_TRY(tmp.alloc(&rank, (size_t)n));
    SCC_TRY(tmp.alloc(&delta, (size_t)n));
    SCC_TRY(tmp.alloc(&ctl, 1));
    SCC_CUDA(cudaMemcpyAsync(bounds_d, bounds.data(), sizeof(long long) * bounds.size(), cudaMemcpyHostToDevice, s));
    k_le_rank<<<grid_for(n, 1024, num_sms * 16), 256, 0, s>>>(n, order, rank, delta);
    SCC_LAUNCH();
    SCC_CUDA(cudaMemsetAsync(ctl, 0, sizeof(LeCtl), s));
    // buffers: the table (and each level's frontier, whose pairs are new table
    // entries) and the candidate log, grown on demand
    unsigned long long cap = 1024;
    while (cap < (init_cap > 0 ? (unsigned long long)init_cap : 4ull * (unsigned long long)n)) cap <<= 1;
    unsigned long long log_cap = init_log > 0 ? (unsigned long long)init_log : (unsigned long long)n * 24 + 1024;
    unsigned long long* keys = nullptr;
    int32_t* kdist = nullptr;
    unsigned long long *fr0 = nullptr, *fr1 = nullptr;
    int32_t *lu = nullptr, *ls = nullptr, *ld = nullptr;
    auto alloc_table = [&]() -> int {
        tmp.release(keys);
        tmp.release(kdist);
        tmp.release(fr0);
        tmp.release(fr1);
        SCC_TRY(tmp.alloc(&keys, (size_t)cap));
        SCC_TRY(tmp.alloc(&kdist, (size_t)cap));
        SCC_TRY(tmp.alloc(&fr0, (size_t)cap));  // a level inserts at most one pair per table slot
        SCC_TRY(tmp.alloc(&fr1, (size_t)cap));
        SCC_CUDA(cudaMemsetAsync(keys, 0xff, (size_t)cap * 8, s));
        return SCC_OK;
    };
    SCC_TRY(alloc_table());
    SCC_TRY(tmp.alloc(&lu, (size_t)log_cap));
    SCC_TRY(tmp.alloc(&ls, (size_t)log_cap));
    SCC_TRY(tmp.alloc(&ld, (size_t)log_cap));
    int per_sm = 0;
    SCC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_le_lists, kEngineBlock, 0));
    const int grid = std::max(1, engine_blocks_per_sm(per_sm)) * num_sms;
    for (int attempt = 0;; ++attempt) {
        if (attempt > 64) return SCC_ERR_CAPACITY;
        LeParams P;
        P.soff = soff;
        P.sadj = sadj;
        P.n = n;
        P.order = order;
        P.bounds = bounds_d;
        P.nb = nb;
        P.delta = delta;
        P.keys = keys;
        P.kdist = kdist;
        P.mask = cap - 1;
        P.fr[0] = fr0;
        P.fr[1] = fr1;
        P.log_u = lu;
        P.log_s = ls;
        P.log_d = ld;
        P.log_cap = log_cap;
        P.ctl = ctl;
        void* args[] = {(void*)&P};
        SCC_CUDA(cudaLaunchCooperativeKernel((const void*)k_le_lists, dim3(grid), dim3(kEngineBlock), args, 0, s));
        count_launch();
        LeCtl h;
        SCC_CUDA(cudaMemcpyAsync(&h, ctl, sizeof(LeCtl), cudaMemcpyDeviceToHost, s));
        SCC_CUDA(cudaStreamSynchronize(s));
        if (h.err) return h.err;
        res->levels = h.levels;
        res->edges = h.edges;
        res->launches = attempt + 1;
        if (h.status == 0) {
            res->candidates = (long long)h.log_n;
            break;
        }
        // grow the full buffer; the batch starts over (its pairs were never logged)
        if (h.status == 1) {
            cap *= 2;
            SCC_TRY(alloc_table());
        } else {
            const unsigned long long need = std::max(2 * log_cap, h.log_n + 2 * h.ins + 1024);
            int32_t *nu = nullptr, *ns = nullptr, *nd = nullptr;
            SCC_TRY(tmp.alloc(&nu, (size_t)need));
            SCC_TRY(tmp.alloc(&ns, (size_t)need));
            SCC_TRY(tmp.alloc(&nd, (size_t)need));
            SCC_CUDA(cudaMemcpyAsync(nu, lu, 4 * h.log_n, cudaMemcpyDeviceToDevice, s));
            SCC_CUDA(cudaMemcpyAsync(ns, ls, 4 * h.log_n, cudaMemcpyDeviceToDevice, s));
            SCC_CUDA(cudaMemcpyAsync(nd, ld, 4 * h.log_n, cudaMemcpyDeviceToDevice, s));
            tmp.release(lu);
            tmp.release(ls);
            tmp.release(ld);
            lu = nu;
            ls = ns;
            ld = nd;
            log_cap = need;
            SCC_CUDA(cudaMemsetAsync(keys, 0xff, (size_t)cap * 8, s));  // the batch's partial pairs
        }
        if (h.status == 1) {
            // alloc_table cleared the new table
        }
        h.status = 0;
        h.err = 0;
        h.bar = GridBarrier{0, 0};
        SCC_CUDA(cudaMemcpyAsync(ctl, &h, sizeof(LeCtl), cudaMemcpyHostToDevice, s));
        SCC_CUDA(cudaStreamSynchronize(s));  // h is a stack variable
    }
    // ---- assembly: group the candidates by vertex, sort and filter each list
    const long long total = res->candidates;
    if (total > (long long)INT32_MAX - 1) return SCC_ERR_CAPACITY;
    int32_t *cnt = nullptr, *pos = nullptr, *cursor = nullptr, *gs = nullptr, *gd = nullptr, *keep = nullptr,
            *kpos = nullptr;
    void* stmp = nullptr;
    SCC_TRY(tmp.alloc(&cnt, (size_t)n + 1));
    SCC_TRY(tmp.alloc(&pos, (size_t)n + 1));
    SCC_TRY(tmp.alloc(&cursor, (size_t)n + 1));
    SCC_TRY(tmp.alloc(&keep, (size_t)n + 1));
    SCC_TRY(tmp.alloc(&kpos, (size_t)n + 1));
    SCC_TRY(tmp.alloc(&gs, (size_t)std::max<long long>(total, 1)));
    SCC_TRY(tmp.alloc(&gd, (size_t)std::max<long long>(total, 1)));
    SCC_TRY(tmp.alloc(reinterpret_cast<unsigned char**>(&stmp), scan_tmp_bytes(n)));
    SCC_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * ((size_t)n + 1), s));
    const int g2 = grid_for(std::max<long long>(total, n), 1024, num_sms * 16);
    k_le_count<<<g2, 256, 0, s>>>(lu, total, cnt);
    SCC_LAUNCH();
    SCC_TRY(launch_scan(cnt, pos, n, stmp, s));
    SCC_CUDA(cudaMemcpyAsync(cursor, pos, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s));
    k_le_scatter<<<g2, 256, 0, s>>>(lu, ls, ld, total, cursor, gs, gd);
    SCC_LAUNCH();
    k_le_filter<<<grid_for(n, 256, num_sms * 16), 256, 0, s>>>(n, pos, rank, gs, gd, keep);
    SCC_LAUNCH();
    SCC_TRY(launch_scan(keep, kpos, n, stmp, s));
    int32_t kept = 0;
    SCC_CUDA(cudaMemcpyAsync(&kept, kpos + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    SCC_CUDA(cudaStreamSynchronize(s));
    // the result, kept by the caller
    SCC_TRY(dalloc_t(&res->off, (size_t)n + 1, s));
    SCC_TRY(dalloc_t(&res->src, (size_t)std::max(kept, 1), s));
    SCC_TRY(dalloc_t(&res->dist, (size_t)std::max(kept, 1), s));
    res->total = kept;
    k_le_compact<<<grid_for(n, 256, num_sms * 16), 256, 0, s>>>(n, pos, kpos, gs, gd, res->off, res->src, res->dist);
    SCC_LAUNCH();
    SCC_CUDA(cudaStreamSynchronize(s));
    return SCC_OK;
}

}  // namespace scc
