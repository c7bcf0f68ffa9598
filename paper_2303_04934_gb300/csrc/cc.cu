// Connected components by LDD-UF-JTB with VGC and the hash bag (Sec. 5.1,
// Alg. 4), on the undirected graph under the arcs of G (sm_103a).
//
//   1. The symmetric CSR: row v of G followed by row v of G^T (the paper
//      symmetrises directed inputs for connectivity). Its offsets are
//      off[v] + toff[v], so only the rows are copied.
//   2. LDD (Alg. 4 function LDD): a seeded order of all vertices cut into
//      batches growing by a factor beta (1.2, the paper's choice); the first
//      batch claims itself, then one search of the VGC engine (PolLdd) runs
//      rounds in which every frontier item claims unvisited neighbours for its
//      centre, and at the end of round i the unvisited vertices of batch i + 1
//      become centres of their own and join the frontier.
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

// center[v] = -1 for all v, then the first batch's vertices centre themselves.
__global__ void k_ldd_init(int32_t n, int32_t* center) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x)
        center[v] = -1;
}
__global__ void k_ldd_first(const int32_t* __restrict__ order, long long k, int32_t* center) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += (long long)gridDim.x * blockDim.x)
        center[order[i]] = order[i];
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

__global__ void k_uf_init(int32_t n, int32_t* parent, int32_t* mn) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
        parent[v] = (int32_t)v;
        mn[v] = INT_MAX;
    }
}

// One warp per row of G: arcs whose endpoints lie in different clusters join
// the clusters' centres (an arc and its reverse join the same pair).
__global__ void k_uf_arcs(const int32_t* __restrict__ off, const int32_t* __restrict__ adj, int32_t n,
                          const int32_t* __restrict__ center, int32_t* parent, unsigned long long* cross, int* err) {
    const int lane = lane_id();
    const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    unsigned long long c = 0;
    for (long long u = w0; u < n; u += nw) {
        const int a0 = off[u], a1 = off[u + 1];
        if (a1 == a0) continue;
        const int32_t cu = center[u];
        for (int e = a0 + lane; e < a1; e += 32) {
            const int32_t cw = center[adj[e]];
            if (cw != cu) {
                ++c;
                uf_union(parent, cu, cw, err);
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
        const int32_t r = uf_find(parent, center[v], err);
        root[v] = r;
        atomicMin(&mn[r], (int32_t)v);
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

int launch_ldd_setup(const int32_t* order, long long first, int32_t n, int32_t* center, int num_sms, cudaStream_t s) {
    k_ldd_init<<<grid_for(n, kBlk * 4, num_sms * 16), kBlk, 0, s>>>(n, center);
    SCC_LAUNCH();
    k_ldd_first<<<grid_for(first, kBlk, num_sms * 16), kBlk, 0, s>>>(order, first, center);
    SCC_LAUNCH();
    return SCC_OK;
}

int launch_cc_union_label(const int32_t* off, const int32_t* adj, int32_t n, const int32_t* center, int32_t* parent,
                          int32_t* root, int32_t* mn, int32_t* out, unsigned long long* counters, int* err,
                          int num_sms, cudaStream_t s, cudaEvent_t* ev) {
    const int g = grid_for(n, kBlk * 4, num_sms * 16);
    k_uf_init<<<g, kBlk, 0, s>>>(n, parent, mn);
    SCC_LAUNCH();
    if (ev) cudaEventRecord(ev[0], s);
    k_uf_arcs<<<num_sms * 8, kBlk, 0, s>>>(off, adj, n, center, parent, &counters[0], err);
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
