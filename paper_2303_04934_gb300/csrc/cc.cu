// Connected components by LDD-UF-JTB with VGC and the hash bag (Sec. 5.1,
// Alg. 4), on the undirected graph under the arcs of G (sm_103a).
//
//   1. The symmetric CSR: row v of G followed by row v of G^T (the paper
//      symmetrises directed inputs for connectivity). Its offsets are
//      off[v] + toff[v], so only the rows are copied.
//   2. LDD (Alg. 4 function LDD): a seeded order of all vertices cut into
//      batches growing by the factor scc_config.ldd_beta (default 2; the
//      paper's choice is 1.2, fewer batches mean fewer rounds here); the first
//      batch claims itself, then one search of the VGC engine (PolLdd) runs
//      rounds in which every frontier item claims unvisited neighbours for its
//      centre, and at the end of round i the unvisited vertices of batch i + 1
//      become centres of their own and join the frontier. A round whose
//      frontier holds at least 1/20 of the vertices runs bottom-up instead
//      (the engine's dense rounds, Sec. 4.2): every unclaimed vertex with a
//      neighbour in the frontier joins that neighbour's cluster.
//   3. Union-find over the arcs whose endpoints have different centres (Alg. 4
//      "if Find(L(v)) != Find(L(u)) then Union"): a root is hooked under the
//      smaller root by CAS, finds halve their paths; every retry loop is
//      bounded and reports SCC_ERR_INTERNAL past its limit.
//   4. labels_out[v] = the smallest vertex id of the component of v (the
//      component's root is its smallest centre, not necessarily its smallest
//      vertex: one atomicMin pass per root).
#include <algorithm>
#include <climits>
#include <vector>

#include "common.cuh"
#include "engine.cuh"
#include "internal.h"

namespace scc {
namespace {

constexpr int kBlk = 256;
constexpr int kUfLimit = 1 << 20;  // steps of one find or union before it reports an error
constexpr int kSmallRow = 32;      // rows with more arcs go to the flat pass (k_uf_flat)

inline int grid_for(int64_t work, int per_block, int cap) {
    int64_t g = (work + per_block - 1) / per_block;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, cap));
}

// Row v of the symmetric CSR: G's row, then G^T's (one warp per vertex).
__global__ void k_sym_rows(const int32_t* __restrict__ off, const int32_t* __restrict__ adj,
                           const int32_t* __restrict__ toff, const int32_t* __restrict__ tadj, int32_t n,
                           int32_t* __restrict__ soff, int32_t* __restrict__ sadj) {
    const int lane = lane_id();
    const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long v = w0; v < n; v += nw) {
        const int a0 = off[v], a1 = off[v + 1], b0 = toff[v], b1 = toff[v + 1];
        const long long s0 = (long long)a0 + b0;
        if (lane == 0) soff[v] = (int32_t)s0;
        for (int e = a0 + lane; e < a1; e += 32) sadj[s0 + (e - a0)] = adj[e];
        const long long s1 = s0 + (a1 - a0);
        for (int e = b0 + lane; e < b1; e += 32) sadj[s1 + (e - b0)] = tadj[e];
    }
    if (w0 == 0 && lane == 0) soff[n] = off[n] + toff[n];
}

// center[v] = -1 for all v and no vertex visited (the bits past n set: the
// dense rounds read whole words), then the first batch's vertices centre
// themselves.
__global__ void k_ldd_init(int32_t n, int32_t* center, uint32_t* bits) {
    const long long nw = ((long long)n + 31) / 32;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x)
        center[v] = -1;
    for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += (long long)gridDim.x * blockDim.x)
        bits[w] = (w == nw - 1 && (n & 31)) ? ~((1u << (n & 31)) - 1u) : 0u;
}
__global__ void k_ldd_first(const int32_t* __restrict__ order, long long k, int32_t* center, uint32_t* bits) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += (long long)gridDim.x * blockDim.x) {
        const int32_t v = order[i];
        center[v] = v;
        atomicOr(&bits[v >> 5], 1u << (v & 31));
    }
}

// ------------------------------------------------------------- union-find --
// parent[x] <= x always (a root is hooked under a smaller one), so the
// concurrent halving writes keep every parent a vertex of the same tree.
__device__ __forceinline__ int32_t uf_find(int32_t* parent, int32_t x, int* err) {
    for (int it = 0; it < kUfLimit; ++it) {
        const int32_t p = ld_volatile(&parent[x]);
        if (p == x) return x;
        const int32_t gp = ld_volatile(&parent[p]);
        if (gp != p) parent[x] = gp;  // halving
        x = gp;
    }
    atomicExch(err, SCC_ERR_INTERNAL);
    return x;
}
__device__ __forceinline__ void uf_union(int32_t* parent, int32_t a, int32_t b, int* err) {
    for (int it = 0; it < kUfLimit; ++it) {
        const int32_t ra = uf_find(parent, a, err), rb = uf_find(parent, b, err);
        if (ra == rb) return;
        const int32_t lo = ra < rb ? ra : rb, hi = ra < rb ? rb : ra;
        if (atomicCAS(&parent[hi], hi, lo) == hi) return;
        a = lo;
        b = hi;
    }
    atomicExch(err, SCC_ERR_INTERNAL);
}

// A vertex of x's set by plain loads and no writes (a filter in front of
// uf_union): a parent pointer only ever holds a vertex of the same set, and
// sets only merge, so even a stale chain of pointers stays inside x's set. If
// the chains from two vertices meet, the two are connected already.
__device__ __forceinline__ int32_t uf_peek(const int32_t* parent, int32_t x) {
    for (int it = 0; it < 64; ++it) {
        const int32_t p = parent[x];
        if (p == x) break;
        x = p;
    }
    return x;
}

__global__ void k_uf_init(int32_t n, int32_t* parent, int32_t* mn) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
        parent[v] = (int32_t)v;
        mn[v] = INT_MAX;
    }
}

// Arcs of G whose endpoints lie in different clusters join the clusters'
// centres (every edge of the undirected graph is an arc of G). A thread takes
// one row of at most kSmallRow arcs and walks it, four arcs at a time; longer
// rows go to a list (row, degree) whose arcs k_uf_flat spreads evenly over the
// whole grid. After the decomposition most cross arcs repeat a pair that is
// already joined (a few clusters per component, many arcs between them), and
// every union on the same pair would contend for the same few parent words:
// a row skips the centre it joined last, a warp elects one lane per distinct
// pair, and a read-only peek at both sets skips pairs already joined.
__global__ void k_uf_arcs(const int32_t* __restrict__ off, const int32_t* __restrict__ adj, int32_t n,
                          const int32_t* __restrict__ center, int32_t* parent, unsigned long long* cross,
                          int32_t* big, int32_t* bdeg, unsigned long long* nbig, long long big_cap, int* err) {
    const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long gstride = (long long)gridDim.x * blockDim.x;
    unsigned long long c = 0;
    for (long long u = gtid; u < n; u += gstride) {
        const int a0 = off[u], a1 = off[u + 1];
        if (a1 == a0) continue;
        if (a1 - a0 > kSmallRow) {
            const unsigned long long k = atomicAdd(nbig, 1ull);
            if ((long long)k < big_cap) {
                big[k] = (int32_t)u;
                bdeg[k] = a1 - a0;
            } else {
                atomicExch(err, SCC_ERR_INTERNAL);  // cannot happen: big_cap >= m / (kSmallRow + 1) + 1
            }
            continue;
        }
        const int32_t cu = center[u];
        if ((uint32_t)cu >= (uint32_t)n) {  // every vertex has a centre after the decomposition
            atomicCAS(err, 0, SCC_ERR_INTERNAL);
            continue;
        }
        // four arcs at a time: their targets, then the targets' centres, as
        // independent loads
        int32_t last = cu;
        for (int e0 = a0; e0 < a1; e0 += 4) {
            int32_t w[4], cw[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) w[j] = e0 + j < a1 ? adj[e0 + j] : -1;
#pragma unroll
            for (int j = 0; j < 4; ++j) cw[j] = w[j] >= 0 ? center[w[j]] : cu;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if ((uint32_t)cw[j] >= (uint32_t)n) {
                    atomicCAS(err, 0, SCC_ERR_INTERNAL);
                    continue;
                }
                if (cw[j] != cu) {
                    ++c;
                    if (cw[j] != last) {
                        last = cw[j];
                        if (uf_peek(parent, cu) != uf_peek(parent, cw[j])) uf_union(parent, cu, cw[j], err);
                    }
                }
            }
        }
    }
    for (int d = 16; d >= 1; d >>= 1) c += __shfl_xor_sync(kFull, c, d);
    if (lane_id() == 0 && c) atomicAdd(cross, c);
}

// The arcs of the listed rows as one flat range (row k of the list covers
// [bpre[k], bpre[k + 1])) cut into 32-arc chunks; each warp takes a contiguous
// run of chunks and walks the rows forward. A chunk meets at most two rows
// (every listed row has more than 32 arcs), so a lane's row is the warp's
// current row or the next one, whose start in the flat range, arc base and
// centre the warp keeps in registers: a chunk costs a coalesced read of its
// targets and a gather of their centres.
__global__ void k_uf_flat(const int32_t* __restrict__ off, const int32_t* __restrict__ adj,
                          const int32_t* __restrict__ center, int32_t* parent, unsigned long long* cross,
                          const int32_t* __restrict__ big, const unsigned long long* nbig, long long big_cap,
                          const int32_t* __restrict__ bpre, int32_t n, int* err) {
    const int lane = lane_id();
    const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long nb = min((long long)*nbig, big_cap);
    unsigned long long c = 0;
    const long long total = nb > 0 ? (long long)bpre[nb] : 0;
    const long long nch = (total + 31) / 32;
    const long long per = (nch + nw - 1) / nw;
    const long long ch0 = wid * per, ch1 = min(ch0 + per, nch);
    if (ch0 < ch1) {  // warp-uniform
        // the row of the run's first arc: the last k with bpre[k] <= 32 ch0
        long long lo = 0, hi = nb - 1;
        while (lo < hi) {
            const long long mid = (lo + hi + 1) >> 1;
            if ((long long)bpre[mid] <= ch0 * 32) lo = mid;
            else hi = mid - 1;
        }
        long long r = lo;
        // rows r and r + 1: start in the flat range, arc base (off[u] - start), centre
        auto row = [&](long long k, long long& st, long long& base, int32_t& cu) {
            if (k < nb) {
                const int32_t u = big[k];
                st = bpre[k];
                base = (long long)off[u] - st;
                cu = center[u];
            } else {
                st = total;
                base = 0;
                cu = 0;
            }
        };
        long long s0, b0, s1, b1;
        int32_t c0, c1;
        row(r, s0, b0, c0);
        row(r + 1, s1, b1, c1);
        int32_t lcu = -1, lcw = -1;  // the pair this lane joined last
        // two chunks a step: both targets, then both centres, as independent loads
        for (long long ch = ch0; ch < ch1; ch += 2) {
            int32_t cu[2], w[2], cw[2];
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const long long f0 = (ch + t) * 32;
                while (f0 >= s1 && r + 1 < nb) {  // at most once a chunk: every listed row has more than 32 arcs
                    ++r;
                    s0 = s1;
                    b0 = b1;
                    c0 = c1;
                    row(r + 1, s1, b1, c1);
                }
                const long long f = f0 + lane;
                const bool in = ch + t < ch1 && f < total;
                const bool nx = f >= s1;
                cu[t] = nx ? c1 : c0;
                w[t] = in ? adj[f + (nx ? b1 : b0)] : -1;
            }
#pragma unroll
            for (int t = 0; t < 2; ++t) cw[t] = w[t] >= 0 ? center[w[t]] : cu[t];
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                if (w[t] >= 0 && ((uint32_t)cu[t] >= (uint32_t)n || (uint32_t)cw[t] >= (uint32_t)n)) {
                    atomicCAS(err, 0, SCC_ERR_INTERNAL);  // every vertex has a centre
                    cw[t] = cu[t];
                }
                const bool x = w[t] >= 0 && cw[t] != cu[t];
                c += x;
                const unsigned long long key =
                    x ? ((unsigned long long)(uint32_t)cu[t] << 32 | (uint32_t)cw[t]) : ~0ull;
                const uint32_t peers = __match_any_sync(kFull, key);
                if (x && __ffs(peers) - 1 == lane && !(cu[t] == lcu && cw[t] == lcw)) {
                    lcu = cu[t];
                    lcw = cw[t];
                    if (uf_peek(parent, cu[t]) != uf_peek(parent, cw[t])) uf_union(parent, cu[t], cw[t], err);
                }
            }
        }
    }
    for (int d = 16; d >= 1; d >>= 1) c += __shfl_xor_sync(kFull, c, d);
    if (lane == 0 && c) atomicAdd(cross, c);
}

// root[v] = the root of v's centre; mn[root] = min over its vertices.
__global__ void k_uf_roots(int32_t n, const int32_t* __restrict__ center, int32_t* parent, int32_t* root, int32_t* mn,
                           int* err) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
        const int32_t c = center[v];
        if ((uint32_t)c >= (uint32_t)n) {  // every vertex has a centre after the decomposition
            atomicCAS(err, 0, SCC_ERR_INTERNAL);
            root[v] = (int32_t)v;
            continue;
        }
        const int32_t r = uf_find(parent, c, err);
        root[v] = r;
        // a read first: once a component's minimum is in place (threads take
        // vertices in increasing order) its other vertices skip the atomic
        if ((int32_t)v < ld_volatile(&mn[r])) atomicMin(&mn[r], (int32_t)v);
    }
}
__global__ void k_uf_labels(int32_t n, const int32_t* __restrict__ root, const int32_t* __restrict__ mn, int32_t* out,
                            unsigned long long* comps) {
    unsigned long long c = 0;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
        const int32_t l = mn[root[v]];
        out[v] = l;
        c += l == (int32_t)v;
    }
    for (int d = 16; d >= 1; d >>= 1) c += __shfl_xor_sync(kFull, c, d);
    if (lane_id() == 0 && c) atomicAdd(comps, c);
}
__global__ void k_iota(int32_t n, int32_t* a) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x)
        a[v] = (int32_t)v;
}
// centres: vertices with center[v] == v
__global__ void k_count_centres(int32_t n, const int32_t* __restrict__ center, unsigned long long* cnt) {
    unsigned long long c = 0;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x)
        c += center[v] == (int32_t)v;
    for (int d = 16; d >= 1; d >>= 1) c += __shfl_xor_sync(kFull, c, d);
    if (lane_id() == 0 && c) atomicAdd(cnt, c);
}

}  // namespace

int launch_sym_csr(const int32_t* off, const int32_t* adj, const int32_t* toff, const int32_t* tadj, int32_t n,
                   int32_t* soff, int32_t* sadj, int num_sms, cudaStream_t s) {
    k_sym_rows<<<num_sms * 8, kBlk, 0, s>>>(off, adj, toff, tadj, n, soff, sadj);
    SCC_LAUNCH();
    return SCC_OK;
}

int launch_iota(int32_t n, int32_t* a, int num_sms, cudaStream_t s) {
    k_iota<<<grid_for(n, kBlk * 4, num_sms * 16), kBlk, 0, s>>>(n, a);
    SCC_LAUNCH();
    return SCC_OK;
}

int launch_ldd_setup(const int32_t* order, long long first, int32_t n, int32_t* center, uint32_t* bits, int num_sms,
                     cudaStream_t s) {
    k_ldd_init<<<grid_for(n, kBlk * 4, num_sms * 16), kBlk, 0, s>>>(n, center, bits);
    SCC_LAUNCH();
    k_ldd_first<<<grid_for(first, kBlk, num_sms * 16), kBlk, 0, s>>>(order, first, center, bits);
    SCC_LAUNCH();
    return SCC_OK;
}

int launch_cc_union_label(const int32_t* off, const int32_t* adj, int32_t n, const int32_t* center, int32_t* parent,
                          int32_t* root, int32_t* mn, int32_t* out, unsigned long long* counters, int32_t* big,
                          int32_t* bdeg, int32_t* bpre, void* scan_tmp, long long big_cap, int* err, int num_sms,
                          cudaStream_t s, cudaEvent_t* ev) {
    const int g = grid_for(n, kBlk * 4, num_sms * 16);
    k_uf_init<<<g, kBlk, 0, s>>>(n, parent, mn);
    SCC_LAUNCH();
    SCC_CUDA(cudaMemsetAsync(bdeg, 0, sizeof(int32_t) * (size_t)big_cap, s));
    if (ev) cudaEventRecord(ev[0], s);
    k_uf_arcs<<<grid_for(n, kBlk * 4, num_sms * 16), kBlk, 0, s>>>(off, adj, n, center, parent, &counters[0], big, bdeg,
                                                                   &counters[3], big_cap, err);
    SCC_LAUNCH();
    SCC_TRY(launch_scan(bdeg, bpre, big_cap, scan_tmp, s));  // the listed rows' places in the flat range
    k_uf_flat<<<num_sms * 8, kBlk, 0, s>>>(off, adj, center, parent, &counters[0], big, &counters[3], big_cap, bpre, n,
                                           err);
    SCC_LAUNCH();
    if (ev) cudaEventRecord(ev[1], s);
    k_uf_roots<<<g, kBlk, 0, s>>>(n, center, parent, root, mn, err);
    SCC_LAUNCH();
    k_uf_labels<<<g, kBlk, 0, s>>>(n, root, mn, out, &counters[2]);
    SCC_LAUNCH();
    k_count_centres<<<g, kBlk, 0, s>>>(n, center, &counters[1]);
    SCC_LAUNCH();
    if (ev) cudaEventRecord(ev[2], s);
    return SCC_OK;
}

}  // namespace scc
