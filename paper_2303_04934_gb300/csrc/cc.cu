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
constexpr int kBigRow = 2048;      // rows with more arcs are split over the whole grid

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
// one row and walks its arcs; rows of more than 32 arcs are walked by the
// whole warp, one after another; rows of more than kBigRow arcs go to a list
// (at most m / kBigRow of them) whose arcs k_uf_big spreads evenly over the
// whole grid, so no warp walks a hub's row alone.
// After the decomposition most such arcs repeat a pair that is already joined
// (a few clusters per component, many arcs between them), and every union on
// the same pair would contend for the same few parent words: a row skips the
// centre it joined last, a warp on a hub row elects one lane per distinct
// centre, and a read-only peek at both sets skips pairs already joined.
__device__ __forceinline__ void uf_warp_arcs(const int32_t* __restrict__ adj, const int32_t* __restrict__ center,
                                             int32_t* parent, int32_t cu, long long b0, long long b1, long long step,
                                             unsigned long long& c, int* err) {
    const int lane = lane_id();
    for (long long e0 = b0; e0 < b1; e0 += step) {  // warp-uniform
        const long long e = e0 + lane;
        int32_t cw = e < b1 ? center[adj[e]] : cu;
        if (cw < 0) {  // every vertex has a centre after the decomposition
            atomicCAS(err, 0, SCC_ERR_INTERNAL);
            cw = cu;
        }
        const bool x = cw != cu;
        c += x;
        const uint32_t peers = __match_any_sync(kFull, x ? cw : -1);
        if (x && __ffs(peers) - 1 == lane && uf_peek(parent, cu) != uf_peek(parent, cw)) uf_union(parent, cu, cw, err);
    }
}

__global__ void k_uf_arcs(const int32_t* __restrict__ off, const int32_t* __restrict__ adj, int32_t n,
                          const int32_t* __restrict__ center, int32_t* parent, unsigned long long* cross,
                          int32_t* big, unsigned long long* nbig, long long big_cap, int* err) {
    const int lane = lane_id();
    const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long gstride = (long long)gridDim.x * blockDim.x;
    unsigned long long c = 0;
    for (long long base = gtid - lane; base < n; base += gstride) {  // warp-uniform
        const long long u = base + lane;
        int a0 = 0, a1 = 0;
        int32_t cu = 0;
        if (u < n) {
            a0 = off[u];
            a1 = off[u + 1];
            if (a1 > a0) cu = center[u];
            if ((uint32_t)cu >= (uint32_t)n) {  // every vertex has a centre after the decomposition
                atomicCAS(err, 0, SCC_ERR_INTERNAL);
                a1 = a0;
                cu = 0;
            }
        }
        if (a1 - a0 > kBigRow) {
            const unsigned long long k = atomicAdd(nbig, 1ull);
            if ((long long)k < big_cap) big[k] = (int32_t)u;
            else atomicExch(err, SCC_ERR_INTERNAL);  // cannot happen: big_cap >= m / kBigRow + 1
            a1 = a0;
        }
        const bool big = a1 - a0 > 32;
        if (!big) {
            int32_t last = cu;
            for (int e = a0; e < a1; ++e) {
                const int32_t cw = center[adj[e]];
                if ((uint32_t)cw >= (uint32_t)n) {
                    atomicCAS(err, 0, SCC_ERR_INTERNAL);
                    continue;
                }
                if (cw != cu) {
                    ++c;
                    if (cw != last) {
                        last = cw;
                        if (uf_peek(parent, cu) != uf_peek(parent, cw)) uf_union(parent, cu, cw, err);
                    }
                }
            }
        }
        uint32_t m = __ballot_sync(kFull, big);
        while (m) {
            const int j = __ffs(m) - 1;
            m &= m - 1;
            const int32_t bu = __shfl_sync(kFull, cu, j);
            const int b0 = __shfl_sync(kFull, a0, j), b1 = __shfl_sync(kFull, a1, j);
            uf_warp_arcs(adj, center, parent, bu, b0, b1, 32, c, err);
        }
    }
    for (int d = 16; d >= 1; d >>= 1) c += __shfl_xor_sync(kFull, c, d);
    if (lane == 0 && c) atomicAdd(cross, c);
}

// Offsets of the rows k_uf_arcs left in one flat range: bpre[i] = arcs of
// big[0 .. i) (one block; at most m / kBigRow + 1 rows).
__global__ void __launch_bounds__(1024) k_big_scan(const int32_t* __restrict__ off, const int32_t* __restrict__ big,
                                                   const unsigned long long* nbig, long long big_cap, long long* bpre) {
    __shared__ long long s_part[32];
    const long long nb = min((long long)*nbig, big_cap);
    const long long per = (nb + blockDim.x - 1) / blockDim.x;
    const long long i0 = (long long)threadIdx.x * per, i1 = min(i0 + per, nb);
    long long sum = 0;
    for (long long i = i0; i < i1; ++i) sum += (long long)(off[big[i] + 1] - off[big[i]]);
    // exclusive scan of the threads' sums
    long long incl = sum;
    for (int d = 1; d < 32; d <<= 1) {
        const long long y = __shfl_up_sync(kFull, incl, d);
        if (lane_id() >= d) incl += y;
    }
    if (lane_id() == 31) s_part[threadIdx.x >> 5] = incl;
    __syncthreads();
    if (threadIdx.x < 32) {
        long long x = threadIdx.x < (blockDim.x >> 5) ? s_part[threadIdx.x] : 0;
        long long y = x;
        for (int d = 1; d < 32; d <<= 1) {
            const long long z = __shfl_up_sync(kFull, y, d);
            if (lane_id() >= d) y += z;
        }
        s_part[threadIdx.x] = y - x;
    }
    __syncthreads();
    long long run = s_part[threadIdx.x >> 5] + incl - sum;
    for (long long i = i0; i < i1; ++i) {
        bpre[i] = run;
        run += (long long)(off[big[i] + 1] - off[big[i]]);
    }
    if (i1 == nb && i0 <= nb) bpre[nb] = run;  // the thread holding the last row (or the first, for none)
}

// The arcs of the rows k_uf_arcs left, as one flat range cut into 32-arc
// chunks shared by all warps of the grid; each lane finds its row among the
// big rows by a binary search over bpre.
__global__ void k_uf_big(const int32_t* __restrict__ off, const int32_t* __restrict__ adj,
                         const int32_t* __restrict__ center, int32_t* parent, unsigned long long* cross,
                         const int32_t* __restrict__ big, const unsigned long long* nbig, long long big_cap,
                         const long long* __restrict__ bpre, int32_t n, int* err) {
    const int lane = lane_id();
    const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long nb = min((long long)*nbig, big_cap);
    const long long total = nb > 0 ? bpre[nb] : 0;
    unsigned long long c = 0;
    for (long long f0 = wid * 32; f0 < total; f0 += nw * 32) {  // warp-uniform
        const long long f = f0 + lane;
        int32_t cu = 0, cw = 0;
        bool x = false;
        if (f < total) {
            long long lo = 0, hi = nb - 1;  // the last row with bpre <= f
            while (lo < hi) {
                const long long mid = (lo + hi + 1) >> 1;
                if (bpre[mid] <= f) lo = mid;
                else hi = mid - 1;
            }
            const int32_t u = big[lo];
            cu = center[u];
            cw = center[adj[(long long)off[u] + (f - bpre[lo])]];
            if ((uint32_t)cu >= (uint32_t)n || (uint32_t)cw >= (uint32_t)n) {  // every vertex has a centre
                atomicCAS(err, 0, SCC_ERR_INTERNAL);
                cw = cu;
            }
            x = cw != cu;
        }
        c += x;
        const unsigned long long key = x ? ((unsigned long long)(uint32_t)cu << 32 | (uint32_t)cw) : ~0ull;
        const uint32_t peers = __match_any_sync(kFull, key);
        if (x && __ffs(peers) - 1 == lane && uf_peek(parent, cu) != uf_peek(parent, cw)) uf_union(parent, cu, cw, err);
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
                          long long* bpre, long long big_cap, int* err, int num_sms, cudaStream_t s,
                          cudaEvent_t* ev) {
    const int g = grid_for(n, kBlk * 4, num_sms * 16);
    k_uf_init<<<g, kBlk, 0, s>>>(n, parent, mn);
    SCC_LAUNCH();
    if (ev) cudaEventRecord(ev[0], s);
    k_uf_arcs<<<grid_for(n, kBlk * 4, num_sms * 16), kBlk, 0, s>>>(off, adj, n, center, parent, &counters[0], big,
                                                                   &counters[3], big_cap, err);
    SCC_LAUNCH();
    k_big_scan<<<1, 1024, 0, s>>>(off, big, &counters[3], big_cap, bpre);
    SCC_LAUNCH();
    k_uf_big<<<num_sms * 8, kBlk, 0, s>>>(off, adj, center, parent, &counters[0], big, &counters[3], big_cap, bpre, n,
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
