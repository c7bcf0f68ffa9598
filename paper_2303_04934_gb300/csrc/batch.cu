// Batched SCC (sm_103a): many independent graphs in one persistent launch.
//
// Each thread block takes the next graph from a device work queue (graphs in
// decreasing size, so the longest ones start first) and runs the whole method
// on it alone, with __syncthreads between rounds (CtaScope of engine.cuh):
//
//   1. G^T of the graph (Sec. 2: a backward search is a forward search on
//      G^T). A run through a batch handle computes it before the persistent
//      launch for groups of consecutive graphs at once (each group, up to 2^24
//      vertices, is one graph of disjoint parts for the grid-wide transpose of
//      transpose.cu), and a block only points at its graph's part; graphs
//      outside the groups (and the server's launches) build it in the block:
//      in-degree counts, a block scan, placement.
//   2. Trimming (Sec. 4.1): vertices without in- or out-arcs are singletons.
//   3. The pivot order: a seeded Feistel permutation of the active vertices.
//   4. Single-pivot steps (Sec. 4.2): the first pivot's SCC by forward and
//      backward single-reachability with visited bitmaps -- in the same rounds
//      (vertex items with a direction bit), or, on a graph of high or skewed
//      degree, one after the other with dense (bottom-up) rounds -- then the
//      labelling of Alg. 1 for its class. The next pivots take the same step
//      while a step leaves at least 1/8 of the active vertices reached one way
//      only (a pivot that missed a giant SCC), at most kBatchSingleSteps times.
//   5. Trimming inside the classes the steps leave.
//   6. Prefix-doubling batches (Alg. 1) over the rest of the pivot order:
//      forward and backward multi-reachability sharing the rounds of one
//      search (pair items with a direction bit, Sec. 4.3 pair tables), then the
//      labelling step of Alg. 1 (labels.cuh). A batch of one source takes a
//      single-pivot step; a batch of at most kBatchSingleFallback sources whose
//      pairs overflow its tables takes one step per source; a larger one is
//      rerun with larger tables, or -- at the largest size -- with half of its
//      sources.
//   7. The canonical label: the smallest vertex id of each SCC.
//
// The working memory of a block (transpose, labels, tables, hash bag, engine
// control) is a fixed slice of one device allocation, sized for the largest
// graph of the batch; nothing is allocated during a run, so the host captures
// the launch (a reset kernel and the persistent kernel) as a CUDA graph once
// and replays it.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/scc_batch.h"
#include "common.cuh"
#include "engine.cuh"
#include "internal.h"
#include "labels.cuh"

namespace scc {
namespace {

constexpr int kBatchMaxBlock = 1024;
constexpr int kBatchTrimPasses = 4;
constexpr int kBatchSingleSteps = 8;  // single-pivot steps before the batches, at most
constexpr long long kBatchSingleFallback = 16;  // an overflowing batch this small runs as single steps
constexpr int kVU = 4;  // vertices per thread per pass of a block's vertex loops
constexpr long long kBatchMinTable = 1024;
// per-graph record: start, transpose done, first SCC done, class trimming done,
// batches done, end (globaltimer ns); block; engine rounds, pair searches, pair
// searches rerun (a table or the bag was full), batches labelled
constexpr int kTimeWords = 11;

// ------------------------------------------------------------ working memory --
// Byte offsets of a block's arrays inside its slice (all 256-byte aligned).
struct WsLayout {
    size_t toff, tadj, cnt, label, rep, act, src, fmax, bmax, hit, bits_f, bits_b, fb0, fb1, tab0, tab1, slots0, slots1,
        hub_item0, hub_item1, hub_beg0, hub_beg1, hub_deg0, hub_deg1, hub_sb0, hub_sb1, segmap0, segmap1, ctl,
        tag, bytes;
};

struct BatchDims {
    long long n_max, m_max;
    long long tcap;      // pair-table capacity per direction (power of two)
    long long nslots;    // hash-bag slots per slot array (64-bit slots)
    int hub_cap;
    long long segmap_cap;
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

WsLayout make_layout(const BatchDims& d) {
    WsLayout L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = align256(o + bytes);
        return at;
    };
    const size_t n1 = (size_t)d.n_max + 1;
    const size_t words = (size_t)(d.n_max / 32 + 2);
    L.toff = take(4 * n1);
    L.tadj = take(4 * (size_t)std::max<long long>(d.m_max, 1));
    L.cnt = take(4 * n1);
    L.label = take(4 * n1);
    L.rep = take(4 * n1);
    L.act = take(4 * n1);
    L.src = take(4 * n1);
    L.fmax = take(8 * n1);
    L.bmax = take(8 * n1);
    L.hit = take(8 * n1);
    L.bits_f = take(4 * words);
    L.bits_b = take(4 * words);
    L.fb0 = take(4 * words);
    L.fb1 = take(4 * words);
    L.tab0 = take(8 * (size_t)d.tcap);
    L.tab1 = take(8 * (size_t)d.tcap);
    L.slots0 = take(8 * (size_t)d.nslots);
    L.slots1 = take(8 * (size_t)d.nslots);
    L.hub_item0 = take(8 * (size_t)d.hub_cap);
    L.hub_item1 = take(8 * (size_t)d.hub_cap);
    L.hub_beg0 = take(4 * (size_t)d.hub_cap);
    L.hub_beg1 = take(4 * (size_t)d.hub_cap);
    L.hub_deg0 = take(4 * (size_t)d.hub_cap);
    L.hub_deg1 = take(4 * (size_t)d.hub_cap);
    L.hub_sb0 = take(8 * (size_t)d.hub_cap);
    L.hub_sb1 = take(8 * (size_t)d.hub_cap);
    L.segmap0 = take(4 * (size_t)d.segmap_cap);
    L.segmap1 = take(4 * (size_t)d.segmap_cap);
    L.ctl = take(sizeof(EngineCtl));
    L.tag = take(sizeof(uint32_t));
    L.bytes = o;
    return L;
}

struct BatchArgs {
    int32_t G;
    const long long* vbase;
    const long long* ebase;
    const int32_t* offsets;
    const int32_t* targets;
    const int32_t* order;  // graphs in processing order
    int32_t norder;
    int32_t* labels;       // output, packed like the vertices
    int* next;             // work-queue head (zeroed by the reset kernel)
    int* err;              // first error (SCC_ERR_*), zeroed by the reset kernel
    unsigned long long* times;  // per graph (kTimeWords): phase ends (globaltimer ns), block
    unsigned char* ws;
    size_t ws_stride;
    WsLayout L;
    BatchDims D;
    int tau, seeds, lambda, sigma;
    double beta;
    uint64_t seed;
    // G^T computed before the launch, packed like the input (per graph n + 1
    // local offsets at vbase[g] + g, local sources at ebase[g]) for the graphs
    // with gt_ok[g] != 0; null: every block builds its graph's G^T
    const int32_t* gt_off;
    const int32_t* gt_adj;
    const unsigned char* gt_ok;
};

// Per-block pointers into its slice.
struct Ws {
    int32_t *toff, *tadj, *cnt, *label, *rep, *act, *src;
    int32_t *toff_slice, *tadj_slice;  // the slice's own G^T arrays
    unsigned long long *fmax, *bmax, *hit;
    uint32_t *bits_f, *bits_b;
    uint32_t *fb0, *fb1;  // frontier bitmaps of the dense (bottom-up) rounds
    unsigned long long *tab0, *tab1;
    uint32_t* tag;  // the block's labelling-tag counter, kept across launches
    EngineParams<uint32_t> P32;
    EngineParams<uint64_t> P64;
};

template <class T>
__device__ __forceinline__ T* at(unsigned char* base, size_t off) {
    return reinterpret_cast<T*>(base + off);
}

__device__ void bind_ws(const BatchArgs& A, Ws& W) {
    unsigned char* b = A.ws + A.ws_stride * blockIdx.x;
    const WsLayout& L = A.L;
    W.toff = W.toff_slice = at<int32_t>(b, L.toff);
    W.tadj = W.tadj_slice = at<int32_t>(b, L.tadj);
    W.cnt = at<int32_t>(b, L.cnt);
    W.label = at<int32_t>(b, L.label);
    W.rep = at<int32_t>(b, L.rep);
    W.act = at<int32_t>(b, L.act);
    W.src = at<int32_t>(b, L.src);
    W.fmax = at<unsigned long long>(b, L.fmax);
    W.bmax = at<unsigned long long>(b, L.bmax);
    W.hit = at<unsigned long long>(b, L.hit);
    W.bits_f = at<uint32_t>(b, L.bits_f);
    W.bits_b = at<uint32_t>(b, L.bits_b);
    W.fb0 = at<uint32_t>(b, L.fb0);
    W.fb1 = at<uint32_t>(b, L.fb1);
    W.tab0 = at<unsigned long long>(b, L.tab0);
    W.tab1 = at<unsigned long long>(b, L.tab1);
    W.tag = at<uint32_t>(b, L.tag);
    EngineCtl* ctl = at<EngineCtl>(b, L.ctl);
    auto fill = [&](auto& P, auto* slot0, auto* slot1, auto* hub0, auto* hub1) {
        memset(&P, 0, sizeof(P));
        P.tau = A.tau;
        P.hub_thr = A.tau;
        P.seeds = A.seeds;
        P.slots[0] = slot0;
        P.slots[1] = slot1;
        P.nslots = A.D.nslots;
        P.lambda = A.lambda;
        P.sigma = A.sigma;
        P.hub_item[0] = hub0;
        P.hub_item[1] = hub1;
        P.hub_beg[0] = at<int32_t>(b, L.hub_beg0);
        P.hub_beg[1] = at<int32_t>(b, L.hub_beg1);
        P.hub_deg[0] = at<int32_t>(b, L.hub_deg0);
        P.hub_deg[1] = at<int32_t>(b, L.hub_deg1);
        P.hub_segbase[0] = at<long long>(b, L.hub_sb0);
        P.hub_segbase[1] = at<long long>(b, L.hub_sb1);
        P.hub_cap = A.D.hub_cap;
        P.segmap[0] = at<int32_t>(b, L.segmap0);
        P.segmap[1] = at<int32_t>(b, L.segmap1);
        P.segmap_cap = A.D.segmap_cap;
        P.ctl = ctl;
    };
    // the two hash-bag slot arrays hold 64-bit pair items or, viewed as 32-bit
    // slots, vertex items (both sentinels are all-ones bytes)
    fill(W.P32, at<uint32_t>(b, L.slots0), at<uint32_t>(b, L.slots1), at<uint32_t>(b, L.hub_item0),
         at<uint32_t>(b, L.hub_item1));
    fill(W.P64, at<uint64_t>(b, L.slots0), at<uint64_t>(b, L.slots1), at<uint64_t>(b, L.hub_item0),
         at<uint64_t>(b, L.hub_item1));
}

// ------------------------------------------------------------- block helpers --
struct BlockShared {
    int graph;
    int wsum[kBatchMaxBlock / 32];
    long long carry;
    long long count;
    unsigned long long acc;
};

// Maximum over the block (every thread gets it).
__device__ unsigned long long block_max(unsigned long long x, BlockShared& sh) {
    for (int d = 16; d >= 1; d >>= 1) x = max(x, __shfl_xor_sync(kFull, x, d));
    __syncthreads();
    if (threadIdx.x == 0) sh.acc = 0;
    __syncthreads();
    if (lane_id() == 0 && x) atomicMax(&sh.acc, x);
    __syncthreads();
    const unsigned long long t = sh.acc;
    __syncthreads();
    return t;
}

// Sum over the block (every thread gets the total).
__device__ unsigned long long block_sum(unsigned long long x, BlockShared& sh) {
    for (int d = 16; d >= 1; d >>= 1) x += __shfl_xor_sync(kFull, x, d);
    __syncthreads();
    if (threadIdx.x == 0) sh.acc = 0;
    __syncthreads();
    if (lane_id() == 0 && x) atomicAdd(&sh.acc, x);
    __syncthreads();
    const unsigned long long t = sh.acc;
    __syncthreads();
    return t;
}

// Exclusive scan in place of a[0..n) (int32), a[n] = total: tiles of 4 values
// per thread, a block scan per tile, a running carry.
__device__ void block_exclusive_scan(int32_t* a, long long n, BlockShared& sh) {
    const int nw = blockDim.x >> 5;
    if (threadIdx.x == 0) sh.carry = 0;
    __syncthreads();
    for (long long base = 0; base < n; base += 4ll * blockDim.x) {
        const long long i0 = base + 4ll * threadIdx.x;
        int v[4];
        int s = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            v[j] = i0 + j < n ? a[i0 + j] : 0;
            s += v[j];
        }
        const int incl = warp_incl_scan(s);
        if (lane_id() == 31) sh.wsum[threadIdx.x >> 5] = incl;
        __syncthreads();
        if (threadIdx.x < 32) {
            const int x = threadIdx.x < nw ? sh.wsum[threadIdx.x] : 0;
            const int y = warp_incl_scan(x);
            if (threadIdx.x < nw) sh.wsum[threadIdx.x] = y - x;
        }
        __syncthreads();
        long long run = sh.carry + sh.wsum[threadIdx.x >> 5] + (incl - s);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (i0 + j < n) a[i0 + j] = (int32_t)run;
            run += v[j];
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) sh.carry = run;
        __syncthreads();
    }
    if (threadIdx.x == 0) a[n] = (int32_t)sh.carry;
    __syncthreads();
}

// Largest r in [0, n) with off[r] <= e.
__device__ __forceinline__ int row_of(const int32_t* off, int n, long long e) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((long long)off[mid] <= e) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// ------------------------------------------------------------- initial items --
// the pivot in both directions (items 0 and 1 of a PolSingleBoth search)
struct InitPivotBoth {
    uint32_t v;
    __device__ __forceinline__ uint32_t operator()(long long i) const { return i ? (v | PolSingleBoth::kDir) : v; }
};
struct InitPivot {
    uint32_t v;
    __device__ __forceinline__ uint32_t operator()(long long) const { return v; }
};

// One single-pivot step (Sec. 4.2): forward and backward single-reachability
// from pivot p inside its class, then the labelling of Alg. 1 for that class:
// reached both ways -> p's SCC; one way -> a new class (old class, p or none,
// p or none). *c = vertices finished, *r = vertices moved to a new class. Kept
// out of line: its register use stays apart from the batch loop's. Returns
// false after an error (recorded in *A.err).
__device__ __noinline__ bool single_step(const BatchArgs& A, Ws& W, BlockShared& sh, const LocalQueue<uint32_t>& q32,
                                         uint32_t& gr, uint32_t& si, const int32_t* off, const int32_t* adj, int n,
                                         long long m, int tau_g, bool hubby, int p, unsigned long long* c_out,
                                         unsigned long long* r_out) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int words = (n + 31) / 32;
    const int wid = tid >> 5, nwarps = nt >> 5, lane = tid & 31;
    const int32_t Lp = W.label[p];
    // vertices outside the pivot's class are pre-visited (one coalesced label
    // load per 32 vertices and a ballot per bitmap word; a fixed trip count,
    // so the loads of several words are in flight together)
    unsigned long long ncls = 0;
    for (int w0 = wid * 32; w0 < words; w0 += nwarps * 32) {
        uint32_t mine = 0;
#pragma unroll 8
        for (int j = 0; j < 32; ++j) {
            const int v = (w0 + j) * 32 + lane;  // v >= n past the last word
            const uint32_t msk = __ballot_sync(kFull, v >= n || W.label[v] != Lp);
            if (lane == j) mine = msk;
        }
        if (w0 + lane < words) {
            W.bits_f[w0 + lane] = mine;
            W.bits_b[w0 + lane] = mine;
            ncls += (unsigned long long)__popc(~mine);
        }
    }
    ncls = block_sum(ncls, sh);
    if (hubby) {
        // a graph of high or skewed degree (a few rounds hold most of the
        // class): forward and backward searches one after the other, each
        // with dense (bottom-up) rounds once its frontier holds 1/20 of the
        // class or of the arcs (Sec. 4.2)
        for (int w = tid; w < words; w += nt) {
            W.fb0[w] = 0;
            W.fb1[w] = 0;
        }
        __syncthreads();
        for (int d = 0; d < 2; ++d) {
            EngineParams<uint32_t> P = W.P32;
            P.tau = P.hub_thr = tau_g;
            P.off = d == 0 ? off : W.toff;
            P.adj = d == 0 ? adj : W.tadj;
            P.n = n;
            DenseParams dp{d == 0 ? W.toff : off, d == 0 ? W.tadj : adj, {W.fb0, W.fb1}, (long long)ncls, 20, m};
            PolSingle pol;
            pol.bits = d == 0 ? W.bits_f : W.bits_b;
            WarpStats ws;
            int why = 0;
            if (!engine_search<PolSingle, InitPivot, CtaScope>(P, pol, InitPivot{(uint32_t)p}, 1, &dp, q32, ws,
                                                               gr, si, why))
                return false;
            ++si;
            if (why != 0) {  // the hash bag is sized so that this never happens
                if (tid == 0) atomicCAS(A.err, 0, why < 0 ? why : SCC_ERR_INTERNAL);
                return false;
            }
        }
    } else {
        // forward (G) and backward (G^T) searches in the same rounds
        EngineParams<uint32_t> P = W.P32;
        P.tau = P.hub_thr = tau_g;
        P.off = off;
        P.adj = adj;
        P.off2 = W.toff;
        P.adj2 = W.tadj;
        P.n = n;
        PolSingleBoth pol;
        pol.bits[0] = W.bits_f;
        pol.bits[1] = W.bits_b;
        WarpStats ws;
        int why = 0;
        const InitPivotBoth init{(uint32_t)p};
        if (!engine_search<PolSingleBoth, InitPivotBoth, CtaScope>(P, pol, init, 2, nullptr, q32, ws, gr, si, why))
            return false;
        ++si;
        if (why != 0) {  // the hash bag is sized so that this never happens
            if (tid == 0) atomicCAS(A.err, 0, why < 0 ? why : SCC_ERR_INTERNAL);
            return false;
        }
    }
    // four vertices per thread per pass, their loads issued before any store
    unsigned long long c = 0, r = 0;
    constexpr int U = 4;
    for (int v0 = tid; v0 < n; v0 += U * nt) {
        int32_t L[U];
        uint32_t wf[U], wb[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int v = v0 + u * nt;
            L[u] = v < n ? W.label[v] : kDone;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int v = v0 + u * nt;
            wf[u] = L[u] == Lp ? W.bits_f[v >> 5] : 0u;
            wb[u] = L[u] == Lp ? W.bits_b[v >> 5] : 0u;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (L[u] != Lp) continue;
            const int v = v0 + u * nt;
            const bool f = (wf[u] >> (v & 31)) & 1u, b = (wb[u] >> (v & 31)) & 1u;
            if (f && b) {
                W.label[v] = kDone;
                W.rep[v] = p;
                ++c;
            } else if (f || b) {
                W.label[v] = class_hash(Lp, f ? p : -1, b ? p : -1);
                ++r;
            }
        }
    }
    *c_out = block_sum(c, sh);
    *r_out = block_sum(r, sh);
    return true;
}

// ------------------------------------------------------------ one graph --
// Returns false after an error (recorded in *A.err): the block stops.
__device__ bool scc_one_graph(const BatchArgs& A, Ws& W, int g, BlockShared& sh,
                              const LocalQueue<uint32_t>& q32, const LocalQueue<uint64_t>& q64, uint32_t& gr,
                              uint32_t& si, uint32_t& tagc, unsigned long long* tm) {
    auto mark = [&](int k) {
        if (threadIdx.x == 0) tm[k] = globaltimer_ns();
    };
    const long long vb = A.vbase[g];
    const int n = (int)(A.vbase[g + 1] - vb);
    const long long eb = A.ebase[g];
    const long long m = A.ebase[g + 1] - eb;
    const int32_t* off = A.offsets + vb + g;
    const int32_t* adj = A.targets + eb;
    int32_t* out = A.labels + vb;
    const int tid = threadIdx.x, nt = blockDim.x;
    if (n == 0) {
        for (int k = 1; k < 5; ++k) mark(k);
        return true;
    }

    // ---- 1. G^T: computed before the launch, or in-degrees, scan, placement
    if (A.gt_ok != nullptr && A.gt_ok[g]) {
        W.toff = const_cast<int32_t*>(A.gt_off + vb + g);
        W.tadj = const_cast<int32_t*>(A.gt_adj + eb);
    } else {
        W.toff = W.toff_slice;
        W.tadj = W.tadj_slice;
        for (int v = tid; v <= n; v += nt) W.cnt[v] = 0;
        __syncthreads();
        for (long long e = tid; e < m; e += nt) atomicAdd(&W.cnt[adj[e]], 1);
        __syncthreads();
        block_exclusive_scan(W.cnt, n, sh);
        for (int v = tid; v <= n; v += nt) W.toff[v] = W.cnt[v];
        __syncthreads();
        // 16 consecutive arcs per thread: one row search, then a forward walk
        constexpr int kC = 16;
        for (long long e0 = (long long)tid * kC; e0 < m; e0 += (long long)nt * kC) {
            const long long e1 = min(e0 + kC, m);
            int u = row_of(off, n, e0);
            for (long long e = e0; e < e1; ++e) {
                while ((long long)off[u + 1] <= e) ++u;
                const int w = adj[e];
                W.tadj[atomicAdd(&W.cnt[w], 1)] = u;
            }
        }
        __syncthreads();
    }

    mark(1);
    // ---- 2. trimming; 3. active list (ordered) for the pivot permutation
    // (the vertex passes of a block take kVU vertices per thread per pass, all
    // their loads issued before any store: one memory latency per pass, not
    // one per vertex)
    unsigned long long na = 0, maxdeg = 0;
    for (int v0 = tid; v0 < n; v0 += kVU * nt) {
        int32_t o0[kVU], o1[kVU], t0[kVU], t1[kVU];
#pragma unroll
        for (int u = 0; u < kVU; ++u) {
            const int v = min(v0 + u * nt, n - 1);
            o0[u] = off[v];
            o1[u] = off[v + 1];
            t0[u] = W.toff[v];
            t1[u] = W.toff[v + 1];
        }
#pragma unroll
        for (int u = 0; u < kVU; ++u) {
            const int v = v0 + u * nt;
            if (v >= n) break;
            maxdeg = max(maxdeg, (unsigned long long)(o1[u] - o0[u]));
            const bool t = o1[u] == o0[u] || t1[u] == t0[u];
            W.label[v] = t ? kDone : 0;
            W.rep[v] = v;
            W.cnt[v] = t ? 0 : 1;
            na += t ? 0 : 1;
        }
    }
    __syncthreads();
    na = block_sum(na, sh);
    // the graph's VGC budget: the configured tau, or (tau = 0) 128 for a graph
    // with 8 arcs a vertex or more or with a row of 16 times the mean degree
    // or more (hubs: a round lasts as long as its longest local search, which
    // grows fastest where degrees are high or skewed), 2048 otherwise
    maxdeg = block_max(maxdeg, sh);
    const bool hubby = m >= 8ll * n || (long long)maxdeg * n >= 16ll * max(m, 1ll);
    const int tau_g = A.tau > 0 ? A.tau : (hubby ? 128 : 2048);
    if (na > 0) {
        block_exclusive_scan(W.cnt, n, sh);
        for (int v0 = tid; v0 < n; v0 += kVU * nt) {
            int32_t L[kVU], C[kVU];
#pragma unroll
            for (int u = 0; u < kVU; ++u) {
                const int v = min(v0 + u * nt, n - 1);
                L[u] = W.label[v];
                C[u] = W.cnt[v];
            }
#pragma unroll
            for (int u = 0; u < kVU; ++u)
                if (v0 + u * nt < n && L[u] == 0) W.act[C[u]] = v0 + u * nt;
        }
    }
    __syncthreads();
    long long active = (long long)na;
    Feistel perm;
    perm.init(A.seed, (uint64_t)max(na, 1ull));

    // ---- 4. single-pivot steps (Sec. 4.2): the first pivot's SCC by a forward
    // and a backward single-reachability search inside its class. The next
    // pivots of the order take the same step while the last one left a large
    // remainder reached but not finished (at least 1/8 of the active
    // vertices), at most kBatchSingleSteps of them. Sources whose reach is
    // much of the graph are covered far more cheaply by one bitmap search
    // each than by a batch's pair tables (so a small batch that overflows its
    // tables takes the same steps, below). The batches start after the
    // positions these steps took.
    long long pos = 0;  // pivot positions taken
    for (int step = 0; step < kBatchSingleSteps && pos < (long long)na && active > 0; ++step) {
        int p = -1;  // the next unfinished pivot (every thread walks the same positions)
        while (pos < (long long)na) {
            const int v = W.act[perm.perm((uint64_t)pos, na)];
            ++pos;
            if (W.label[v] >= 0) {
                p = v;
                break;
            }
        }
        if (p < 0) break;
        unsigned long long c = 0, r = 0;
        if (!single_step(A, W, sh, q32, gr, si, off, adj, n, m, tau_g, hubby, p, &c, &r)) return false;
        const long long before = active;
        active -= (long long)c;
        if ((long long)r * 8 < before) break;
    }

    mark(2);
    // ---- 5. trimming inside the classes: a vertex with no arc from or no arc
    // to an active vertex of its own class is a singleton
    for (int pass = 0; pass < kBatchTrimPasses && active > 0; ++pass) {
        unsigned long long c = 0;
        for (int v = tid; v < n; v += nt) {
            const int32_t L = ld_volatile(&W.label[v]);
            if (L < 0) continue;
            bool out_ok = false, in_ok = false;
            for (int e = off[v]; e < off[v + 1] && !out_ok; ++e) {
                const int w = adj[e];
                out_ok = w != v && ld_volatile(&W.label[w]) == L;
            }
            if (out_ok)
                for (int e = W.toff[v]; e < W.toff[v + 1] && !in_ok; ++e) {
                    const int w = W.tadj[e];
                    in_ok = w != v && ld_volatile(&W.label[w]) == L;
                }
            if (!(out_ok && in_ok)) {
                W.label[v] = kDone;
                W.rep[v] = v;
                ++c;
            }
        }
        const unsigned long long got = block_sum(c, sh);
        active -= (long long)got;
        if ((long long)got * 32 < active) break;
    }

    mark(3);
    const uint32_t gr_batches = gr;
    unsigned long long n_search = 0, n_retry = 0, n_batch = 0;
    // ---- 6. prefix-doubling batches over the pivot order
    long long lo = pos;
    double width = A.beta;
    long long a_prev[2] = {0, 0};
    long long k_prev = 0;     // sources of the batch whose pairs a_prev holds
    long long cap_floor = 0;  // table size forced by a retried batch
    while (lo < (long long)na && active > 0) {
        long long hi = width >= (double)na ? (long long)na : min((long long)na, lo + (long long)ceil(width));
        for (;;) {
            // sources: the still-active vertices at positions [lo, hi)
            if (tid == 0) sh.count = 0;
            __syncthreads();
            for (long long p0 = lo + tid; p0 < hi; p0 += kVU * nt) {
                int vv[kVU], L[kVU];
#pragma unroll
                for (int u = 0; u < kVU; ++u) {
                    const long long p = p0 + (long long)u * nt;
                    vv[u] = p < hi ? W.act[perm.perm((uint64_t)p, na)] : -1;
                }
#pragma unroll
                for (int u = 0; u < kVU; ++u) L[u] = vv[u] >= 0 ? ld_volatile(&W.label[vv[u]]) : -1;
#pragma unroll
                for (int u = 0; u < kVU; ++u)
                    if (L[u] >= 0) W.src[atomicAdd((unsigned long long*)&sh.count, 1ull)] = vv[u];
            }
            __syncthreads();
            const long long k = sh.count;
            __syncthreads();
            if (k == 0) break;
            if (k == 1) {
                // one source: the single-pivot step is the same search, with
                // bitmaps in place of pair tables
                unsigned long long c1 = 0, r1 = 0;
                if (!single_step(A, W, sh, q32, gr, si, off, adj, n, m, tau_g, hubby, W.src[0], &c1, &r1))
                    return false;
                active -= (long long)c1;
                ++n_batch;
                break;
            }
            // table sizes (Sec. 4.5 heuristic, capped by the slice; the previous
            // batch's pairs scaled by the ratio of the sources, as batches grow)
            long long cap[2];
            const double grow_k = k_prev > 0 ? (double)k / (double)k_prev : 1.0;
            for (int d = 0; d < 2; ++d) {
                long long want = max((long long)ceil(0.3 * (double)active),
                                     (long long)ceil(1.5 * (double)a_prev[d] * grow_k));
                want = max(want, k);
                long long c2 = kBatchMinTable;
                while (c2 < 2 * want && c2 < A.D.tcap) c2 <<= 1;
                cap[d] = min(max(c2, cap_floor), A.D.tcap);
            }
            EngineParams<uint64_t> P = W.P64;
            P.tau = P.hub_thr = tau_g;
            P.off = off;
            P.adj = adj;
            P.off2 = W.toff;
            P.adj2 = W.tadj;
            P.n = n;
            SearchCtl& sc = W.P64.ctl->search[si % 3];
            PolPair pol;
            pol.label = W.label;
            pol.keys[0] = W.tab0;
            pol.keys[1] = W.tab1;
            for (int d = 0; d < 2; ++d) {
                pol.mask[d] = (unsigned long long)(cap[d] - 1);
                pol.max_ins[d] = (long long)(0.75 * (double)cap[d]);
            }
            pol.overflow = &sc.overflow;
            pol.ins0 = pol.ins1 = 0;
            WarpStats ws;
            int why = 0;  // 1: a table overflowed; < 0: error (same in every thread)
            if (!engine_search<PolPair, InitPairs, CtaScope>(P, pol, InitPairs{W.src, k}, 2 * k, nullptr, q64, ws, gr,
                                                             si, why))
                return false;
            ++si;
            ++n_search;
            const long long pairs0 = (long long)ld_volatile(&sc.inserted[0]);
            const long long pairs1 = (long long)ld_volatile(&sc.inserted[1]);
            __syncthreads();
            if (why < 0 && why != SCC_ERR_CAPACITY) {
                if (tid == 0) atomicCAS(A.err, 0, why);
                return false;
            }
            if (why == 1 || why == SCC_ERR_CAPACITY) {  // a table or the hash bag is full
                // the search stopped early: empty both tables and the used part of
                // both hash-bag slot arrays, then take a small batch's sources
                // one at a time, or grow the tables or, at full size, halve the
                // batch
                for (long long i = tid; i < cap[0]; i += nt) W.tab0[i] = ~0ull;
                for (long long i = tid; i < cap[1]; i += nt) W.tab1[i] = ~0ull;
                const long long used = chunk_end(A.lambda, ld_volatile(&W.P64.ctl->max_chunk), A.D.nslots);
                for (long long i = tid; i < used; i += nt) {
                    W.P64.slots[0][i] = ~0ull;
                    W.P64.slots[1][i] = ~0ull;
                }
                __syncthreads();
                ++n_retry;
                if (k <= kBatchSingleFallback) {
                    // a few sources whose reach fills a table: a single-pivot
                    // step each (bitmaps, not pairs), and the batch is done
                    for (long long j = 0; j < k; ++j) {
                        const int sj = W.src[j];
                        if (W.label[sj] < 0) continue;  // finished by an earlier step
                        unsigned long long c1 = 0, r1 = 0;
                        if (!single_step(A, W, sh, q32, gr, si, off, adj, n, m, tau_g, hubby, sj, &c1, &r1))
                            return false;
                        active -= (long long)c1;
                    }
                    cap_floor = 0;
                    break;
                }
                const long long c = max(cap[0], cap[1]);
                if (why == 1 && c < A.D.tcap) {
                    cap_floor = 2 * c;
                } else if (hi - lo > 1) {
                    hi = lo + (hi - lo) / 2;
                } else {
                    if (tid == 0) atomicCAS(A.err, 0, SCC_ERR_CAPACITY);
                    return false;
                }
                continue;
            }
            // labelling (Alg. 1; Sec. 4.4), which also empties both tables
            ++tagc;
            const unsigned long long tag = (unsigned long long)tagc << 32;
            const PairTable tb{W.tab1, (unsigned long long)(cap[1] - 1), nullptr};
            label_scan(tid, nt, W.tab0, cap[0], tb, tag, W.fmax, W.bmax, W.hit);
            __syncthreads();
            const unsigned long long c = label_finalize(tid, nt, W.tab0, cap[0], W.tab1, cap[1], tag, W.fmax, W.bmax,
                                                        W.hit, W.label, W.rep, true);
            active -= (long long)block_sum(c, sh);
            a_prev[0] = pairs0;
            a_prev[1] = pairs1;
            k_prev = k;
            cap_floor = 0;
            ++n_batch;
            break;
        }
        if (width < (double)na) width *= A.beta;
        lo = hi;
    }

    mark(4);
    if (threadIdx.x == 0) {
        tm[7] = gr - gr_batches;
        tm[8] = n_search;
        tm[9] = n_retry;
        tm[10] = n_batch;
    }
    // ---- 7. canonical labels: the smallest vertex of each SCC (by its rep)
    for (int v = tid; v < n; v += nt) W.cnt[v] = INT_MAX;
    __syncthreads();
    for (int v0 = tid; v0 < n; v0 += kVU * nt) {
        int32_t R[kVU];
#pragma unroll
        for (int u = 0; u < kVU; ++u) R[u] = W.rep[min(v0 + u * nt, n - 1)];
#pragma unroll
        for (int u = 0; u < kVU; ++u)
            if (v0 + u * nt < n) atomicMin(&W.cnt[R[u]], v0 + u * nt);
    }
    __syncthreads();
    for (int v0 = tid; v0 < n; v0 += kVU * nt) {
        int32_t R[kVU], M[kVU];
#pragma unroll
        for (int u = 0; u < kVU; ++u) R[u] = W.rep[min(v0 + u * nt, n - 1)];
#pragma unroll
        for (int u = 0; u < kVU; ++u) M[u] = W.cnt[R[u]];
#pragma unroll
        for (int u = 0; u < kVU; ++u)
            if (v0 + u * nt < n) out[v0 + u * nt] = M[u];
    }
    __syncthreads();
    return true;
}

// The persistent launch's work counter and error flag, reset inside the
// captured graph before every replay.
__global__ void k_batch_reset(int* next, int* err) {
    *next = 0;
    *err = 0;
}

// Dynamic shared memory: the warps' local queues, sized for the larger of the
// two item kinds (pairs: 8 B item + 8 B range + 4 B label per entry).
constexpr int kBQ = 256;  // = PolPair::kQueue = PolSingle::kQueue
static_assert(PolPair::kQueue == kBQ && PolSingle::kQueue == kBQ, "one queue size for both searches");
size_t batch_smem_bytes(int block) { return (size_t)(block / 32) * kBQ * (8 + 8 + 4); }

__device__ __forceinline__ void batch_body(const BatchArgs& A) {
    extern __shared__ unsigned char dsm[];
    __shared__ BlockShared sh;
    const int nw = blockDim.x >> 5, w = threadIdx.x >> 5;
    // queues of the two searches overlay the same bytes (never live together)
    LocalQueue<uint64_t> q64{reinterpret_cast<uint64_t*>(dsm) + w * kBQ,
                             reinterpret_cast<int2*>(dsm + (size_t)nw * kBQ * 8) + w * kBQ,
                             reinterpret_cast<int32_t*>(dsm + (size_t)nw * kBQ * 16) + w * kBQ};
    LocalQueue<uint32_t> q32{reinterpret_cast<uint32_t*>(dsm) + w * kBQ,
                             reinterpret_cast<int2*>(dsm + (size_t)nw * kBQ * 8) + w * kBQ, nullptr};
    Ws W;
    bind_ws(A, W);
    // a fresh engine control block for this launch
    {
        uint32_t* c = reinterpret_cast<uint32_t*>(W.P64.ctl);
        for (size_t i = threadIdx.x; i < sizeof(EngineCtl) / 4; i += blockDim.x) c[i] = 0;
    }
    __syncthreads();
    // labelling tags (the high word of the per-vertex maxima) must never repeat
    // while a stale maximum could carry them: the counter lives in the slice
    uint32_t gr = 0, si = 0, tagc = ld_volatile(W.tag);
    for (;;) {
        if (threadIdx.x == 0) {
            const int i = atomicAdd(A.next, 1);
            sh.graph = (i < A.norder && ld_volatile(A.err) == 0) ? A.order[i] : -1;
        }
        __syncthreads();
        const int g = sh.graph;
        __syncthreads();
        if (g < 0) break;
        unsigned long long* tm = A.times + (size_t)kTimeWords * g;
        if (threadIdx.x == 0) {
            tm[0] = globaltimer_ns();
            tm[6] = blockIdx.x;
            for (int k = 7; k < kTimeWords; ++k) tm[k] = 0;
        }
        if (!scc_one_graph(A, W, g, sh, q32, q64, gr, si, tagc, tm)) break;
        if (threadIdx.x == 0) tm[5] = globaltimer_ns();
    }
    if (threadIdx.x == 0) *W.tag = tagc;
}

// 64 registers a thread, so that one SM holds 1,024 threads: a block's
// searches wait on chains of dependent loads, and 32 warps on a graph hide
// more of that latency than 16 warps at 128 registers, in spite of the spills
// (on the mixed batch of tori and R-MAT graphs: 1.12x the graphs/s, and the
// largest graph 1.2x faster)
__global__ void __launch_bounds__(kBatchMaxBlock, 1) k_batch_scc(BatchArgs A) { batch_body(A); }

using BatchKernel = void (*)(BatchArgs);
BatchKernel batch_kernel_for(const scc_batch_config&) { return k_batch_scc; }

// Fresh slices: everything zero except the tables and the hash-bag slot
// arrays, which start empty (all-ones).
__global__ void k_batch_init_ws(unsigned char* ws, size_t stride, int blocks, WsLayout L, BatchDims d) {
    const size_t t0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x, ts = (size_t)gridDim.x * blockDim.x;
    for (int b = 0; b < blocks; ++b) {
        unsigned char* base = ws + stride * (size_t)b;
        unsigned long long* regions[4] = {reinterpret_cast<unsigned long long*>(base + L.tab0),
                                          reinterpret_cast<unsigned long long*>(base + L.tab1),
                                          reinterpret_cast<unsigned long long*>(base + L.slots0),
                                          reinterpret_cast<unsigned long long*>(base + L.slots1)};
        const size_t len[4] = {(size_t)d.tcap, (size_t)d.tcap, (size_t)d.nslots, (size_t)d.nslots};
        for (int r = 0; r < 4; ++r)
            for (size_t i = t0; i < len[r]; i += ts) regions[r][i] = ~0ull;
    }
}

}  // namespace
}  // namespace scc

// ---------------------------------------------------------------- host side --
using scc::BatchDims;
using scc::DeviceInfo;
using scc::TransposeScratch;
using scc::WsLayout;

namespace scc {
namespace {

// ------------------------------------------------------ groups of graphs --
// Graphs [g0, g1) of a packed batch as one graph: vertices [v0, v0 + ng),
// arcs [e0, e0 + mg). The vertex (or arc) -> graph map is a search for the
// first of 16 consecutive entries of a thread, then a walk.
constexpr long long kGroupVerts = 1ll << 24;  // the bucketed transpose's limit
constexpr long long kGroupArcs = 1ll << 27;   // bounds the groups' scratch

struct GroupPlan {
    int g0, g1;
    long long v0, v1, e0, e1;
};

// Groups of consecutive graphs (host only): greedily, as many consecutive
// graphs as fit in max_v vertices and max_a arcs; a graph larger than either
// limit ends the current group and belongs to none (its block builds its
// G^T). Groups without vertices are dropped. ok[g] = 1 for the grouped graphs.
void plan_groups(int G, const long long* vb, const long long* eb, long long max_v, long long max_a,
                 std::vector<GroupPlan>& groups, std::vector<unsigned char>& ok) {
    groups.clear();
    ok.assign((size_t)G + 1, 0);
    GroupPlan cur{0, 0, vb[0], vb[0], eb[0], eb[0]};
    auto flush = [&](int g) {
        if (cur.g1 > cur.g0 && cur.v1 > cur.v0) {
            groups.push_back(cur);
        } else {
            for (int k = cur.g0; k < cur.g1; ++k) ok[k] = 0;
        }
        cur = {g, g, vb[g], vb[g], eb[g], eb[g]};
    };
    for (int g = 0; g < G; ++g) {
        const long long n = vb[g + 1] - vb[g], m = eb[g + 1] - eb[g];
        if (n > max_v || m > max_a) {
            flush(g + 1);  // the current group ends before g
            continue;
        }
        if ((cur.v1 - cur.v0) + n > max_v || (cur.e1 - cur.e0) + m > max_a) flush(g);
        cur.g1 = g + 1;
        cur.v1 = vb[g + 1];
        cur.e1 = eb[g + 1];
        ok[g] = 1;
    }
    flush(G);
}

// last g in [lo, hi) with a[g] <= x (a non-decreasing, a[lo] <= x)
__device__ __forceinline__ int last_le(const long long* __restrict__ a, int lo, int hi, long long x) {
    while (hi - lo > 1) {
        const int mid = lo + ((hi - lo) >> 1);
        if (a[mid] <= x) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Elements [0, cnt) of a group (its vertices or arcs; global index base + i):
// a warp takes one contiguous run of 512-element chunks, lane l the elements
// l, l + 32, ... of a chunk (loads and stores coalesce). Per chunk, first the
// graph g of each of the lane's 16 elements (bnd = vbase or ebase: the graphs'
// first elements; one search for the run's first element, then the graph only
// walks forward, in L1-resident reads), then the 16 loads ld(i, g), all in
// flight together, then the 16 stores st(i, g, value).
template <class Ld, class St>
__device__ __forceinline__ void for_group_elems(const long long* __restrict__ bnd, int g0, int g1, long long base,
                                                long long cnt, Ld ld, St st) {
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long per = ((cnt + nwarps - 1) / nwarps + 511) / 512 * 512;
    const long long lo = warp * per, hi = min(cnt, lo + per);
    if (lo >= hi) return;  // warp-uniform
    int g = lane == 0 ? last_le(bnd, g0, g1, base + lo) : 0;
    g = __shfl_sync(kFull, g, 0);
    for (long long c0 = lo; c0 < hi; c0 += 512) {
        int gk[16];
        int32_t v[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const long long i = c0 + k * 32 + lane;
            if (i < hi)
                while (g + 1 < g1 && bnd[g + 1] <= base + i) ++g;
            gk[k] = g;
        }
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const long long i = c0 + k * 32 + lane;
            v[k] = i < hi ? ld(i, gk[k]) : 0;
        }
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const long long i = c0 + k * 32 + lane;
            if (i < hi) st(i, gk[k], v[k]);
        }
        g = (int)__reduce_max_sync(kFull, (unsigned)g);  // the graph of the chunk's last element
    }
}

// The group's CSR: offsets from its first arc, targets from its first vertex
// (graph g's local row offsets start at offsets[vbase[g] + g]).
__global__ void k_group_csr(const long long* __restrict__ vbase, const long long* __restrict__ ebase,
                            const int32_t* __restrict__ offsets, const int32_t* __restrict__ targets, int g0, int g1,
                            long long v0, long long e0, long long ng, long long mg, int32_t* __restrict__ goff,
                            int32_t* __restrict__ gadj) {
    for_group_elems(
        vbase, g0, g1, v0, ng, [&](long long i, int g) { return offsets[v0 + i + g] + (int32_t)(ebase[g] - e0); },
        [&](long long i, int, int32_t x) { goff[i] = x; });
    if (blockIdx.x == 0 && threadIdx.x == 0) goff[ng] = (int32_t)mg;
    for_group_elems(
        ebase, g0, g1, e0, mg, [&](long long j, int g) { return targets[e0 + j] + (int32_t)(vbase[g] - v0); },
        [&](long long j, int, int32_t x) { gadj[j] = x; });
}

// The group's G^T back to per-graph local form, packed like the input:
// offsets from each graph's first arc (and its closing offset), sources from
// its first vertex (in place: the group's G^T arcs are gt_adj[e0 ..)).
__global__ void k_group_localize(const long long* __restrict__ vbase, const long long* __restrict__ ebase, int g0,
                                 int g1, long long v0, long long e0, long long ng, long long mg,
                                 const int32_t* __restrict__ gtoff, int32_t* __restrict__ gt_off, int32_t* gt_adj) {
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for_group_elems(
        vbase, g0, g1, v0, ng, [&](long long i, int g) { return gtoff[i] - (int32_t)(ebase[g] - e0); },
        [&](long long i, int g, int32_t x) { gt_off[v0 + i + g] = x; });
    for (long long g = g0 + tid; g < g1; g += stride) gt_off[vbase[g + 1] + g] = (int32_t)(ebase[g + 1] - ebase[g]);
    for_group_elems(
        ebase, g0, g1, e0, mg, [&](long long j, int g) { return gt_adj[e0 + j] - (int32_t)(vbase[g] - v0); },
        [&](long long j, int, int32_t x) { gt_adj[e0 + j] = x; });
}

}  // namespace
}  // namespace scc

struct scc_batch {
    DeviceInfo di;
    int32_t G = 0;
    long long nv = 0, na = 0;
    long long n_max = 0, m_max = 0;
    long long* vbase = nullptr;
    long long* ebase = nullptr;
    int32_t* offsets = nullptr;
    int32_t* targets = nullptr;
    int32_t* order = nullptr;       // all graphs, largest first
    std::vector<int32_t> order_h;
    std::vector<long long> vb_h, eb_h;
    int* flags = nullptr;           // [0] work-queue head, [1] error
    unsigned long long* times = nullptr;  // per graph: start, end, block (3 words)
    int32_t* labels = nullptr;      // internal output (host destinations, tuning)
    // G^T computed before the persistent launch, for groups of consecutive
    // graphs (one grid-wide transpose each)
    std::vector<scc::GroupPlan> groups;
    int32_t* gt_off = nullptr;       // packed like offsets
    int32_t* gt_adj = nullptr;       // packed like targets
    unsigned char* gt_ok = nullptr;  // graph is in a group
    int32_t *grp_off = nullptr, *grp_adj = nullptr, *grp_toff = nullptr;  // one group's CSR and G^T offsets
    unsigned char* grp_scratch = nullptr;
    TransposeScratch ts{};
    scc_batch_config cfg;
    // working memory for the current configuration
    unsigned char* ws = nullptr;
    size_t ws_bytes = 0;
    size_t ws_stride = 0;
    int blocks = 0;
    WsLayout L;
    BatchDims D;
    // captured launch
    cudaGraphExec_t exec = nullptr;
    int exec_kernels = 0;  // kernel nodes of the captured graph (launches per replay)
    int32_t* exec_out = nullptr;
    const int32_t* exec_order = nullptr;
    int exec_norder = -1;
    bool exec_valid = false;
    scc_batch_stats st;
};

namespace scc {
namespace {

bool valid_config(const scc_batch_config* c) {
    if (!c) return false;
    if (c->tau < 0 || c->tau > 65536) return false;
    if (c->block != 128 && c->block != 256 && c->block != 512 && c->block != 1024) return false;
    if (c->lambda < 256 || c->lambda > 65536 || (c->lambda & (c->lambda - 1))) return false;
    if (c->sigma < 1 || c->seeds < 1 || c->seeds > 32) return false;
    if (!(c->beta > 1.0 && c->beta <= 64.0)) return false;
    if (c->blocks_per_sm < 0 || c->blocks_per_sm > 16) return false;
    return true;
}

void drop_exec(scc_batch* h) {
    if (h->exec) cudaGraphExecDestroy(h->exec);
    h->exec = nullptr;
    h->exec_valid = false;
}

// Working-memory plan for a configuration: one slice per block, sized for the
// largest graph (n_max, m_max), as many blocks as fit on the device (at most
// `gcap`, the graphs of one launch) within `budget` bytes.
int plan_workspace(const DeviceInfo& di, const scc_batch_config& cfg, long long n_max, long long m_max, long long gcap,
                   size_t budget, WsLayout* Lo, BatchDims* Do, int* blocks_out) {
    BatchDims d;
    d.n_max = std::max<long long>(n_max, 1);
    d.m_max = std::max<long long>(m_max, 1);
    long long t = kBatchMinTable;
    while (t < 2 * d.n_max) t <<= 1;  // one source never fills 3/4 of a table
    d.tcap = t;
    // the bag holds a round's new items, sized for a pair search from one
    // source (each vertex at most once per direction), four times that in
    // slots; a pair search from many sources that fills it is rerun with fewer
    // sources, like one that fills a table
    const long long items = 2 * d.n_max + 1024;
    d.nslots = ((std::max<long long>(4 * items, 4ll * cfg.lambda) + kSeg - 1) / kSeg) * kSeg;
    d.hub_cap = (int)std::min<long long>(items, 8192);
    d.segmap_cap = 2 * (d.m_max / kHubSeg) + d.hub_cap + 1024;
    WsLayout L = make_layout(d);
    int per_sm = 0;
    const size_t smem = batch_smem_bytes(cfg.block);
    const BatchKernel kern = batch_kernel_for(cfg);
    SCC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    SCC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, cfg.block, smem));
    if (per_sm < 1) return SCC_ERR_INVALID_ARG;
    if (cfg.blocks_per_sm > 0) per_sm = std::min(per_sm, cfg.blocks_per_sm);
    long long blocks = (long long)per_sm * di.num_sms;
    blocks = std::min<long long>(blocks, std::max<long long>(1, (long long)(budget / L.bytes)));
    blocks = std::min<long long>(blocks, std::max<long long>(gcap, 1));
    *Lo = L;
    *Do = d;
    *blocks_out = (int)blocks;
    return SCC_OK;
}

// Every slice starts with empty bags and tables and untagged maxima.
int init_workspace(unsigned char* ws, const WsLayout& L, const BatchDims& d, int blocks, int num_sms, cudaStream_t s) {
    SCC_CUDA(cudaMemsetAsync(ws, 0, L.bytes * (size_t)blocks, s));
    k_batch_init_ws<<<num_sms * 4, 256, 0, s>>>(ws, L.bytes, blocks, L, d);
    SCC_LAUNCH();
    return SCC_OK;
}

size_t default_budget() {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return 0;
    return std::min<size_t>(free_b / 2, (size_t)96 << 30);
}

// Working memory of a batch handle for its current configuration.
int prepare(scc_batch* h, cudaStream_t s) {
    WsLayout L;
    BatchDims d;
    int blocks = 0;
    SCC_TRY(plan_workspace(h->di, h->cfg, h->n_max, h->m_max, h->G, default_budget(), &L, &d, &blocks));
    const size_t need = L.bytes * (size_t)blocks;
    if (h->ws && (h->ws_bytes < need)) {
        dfree(h->ws, s);
        h->ws = nullptr;
        h->ws_bytes = 0;
    }
    if (!h->ws) {
        SCC_TRY(dalloc(reinterpret_cast<void**>(&h->ws), need, s));
        h->ws_bytes = need;
    }
    SCC_TRY(init_workspace(h->ws, L, d, blocks, h->di.num_sms, s));
    h->ws_stride = L.bytes;
    h->blocks = blocks;
    h->L = L;
    h->D = d;
    h->st.blocks = h->blocks;
    h->st.workspace_bytes = (int64_t)need;
    return SCC_OK;
}

BatchArgs args_for(const scc_batch_config& cfg, unsigned char* ws, const WsLayout& L, const BatchDims& D, int* flags,
                   unsigned long long* times, int32_t G, const long long* vbase, const long long* ebase,
                   const int32_t* offsets, const int32_t* targets, const int32_t* order, int norder, int32_t* out,
                   const int32_t* gt_off = nullptr, const int32_t* gt_adj = nullptr,
                   const unsigned char* gt_ok = nullptr) {
    BatchArgs A;
    memset(&A, 0, sizeof(A));
    A.gt_off = gt_off;
    A.gt_adj = gt_adj;
    A.gt_ok = gt_ok;
    A.G = G;
    A.vbase = vbase;
    A.ebase = ebase;
    A.offsets = offsets;
    A.targets = targets;
    A.order = order;
    A.norder = norder;
    A.labels = out;
    A.next = flags;
    A.err = flags + 1;
    A.times = times;
    A.ws = ws;
    A.ws_stride = L.bytes;
    A.L = L;
    A.D = D;
    A.tau = cfg.tau;
    A.seeds = cfg.seeds;
    A.lambda = cfg.lambda;
    A.sigma = cfg.sigma;
    A.beta = cfg.beta;
    A.seed = cfg.seed;
    return A;
}

BatchArgs make_args(scc_batch* h, const int32_t* order, int norder, int32_t* out) {
    return args_for(h->cfg, h->ws, h->L, h->D, h->flags, h->times, h->G, h->vbase, h->ebase, h->offsets, h->targets,
                    order, norder, out, h->gt_off, h->gt_adj, h->gt_ok);
}

// G^T of every group (after the reset kernel, before the persistent launch);
// the passes' self-check errors go to the batch's error flag.
int enqueue_groups(scc_batch* h, cudaStream_t s) {
    TransposeScratch ts = h->ts;
    ts.err = h->flags + 1;
    for (const auto& gr : h->groups) {
        const long long ng = gr.v1 - gr.v0, mg = gr.e1 - gr.e0;
        const int grid = h->di.num_sms * 4;
        k_group_csr<<<grid, 256, 0, s>>>(h->vbase, h->ebase, h->offsets, h->targets, gr.g0, gr.g1, gr.v0, gr.e0, ng,
                                         mg, h->grp_off, h->grp_adj);
        SCC_LAUNCH();
        SCC_TRY(launch_transpose_keep_self(h->grp_off, h->grp_adj, (int32_t)ng, mg, ts, h->grp_toff,
                                           h->gt_adj + gr.e0, h->di.num_sms, s));
        k_group_localize<<<grid, 256, 0, s>>>(h->vbase, h->ebase, gr.g0, gr.g1, gr.v0, gr.e0, ng, mg, h->grp_toff,
                                              h->gt_off, h->gt_adj);
        SCC_LAUNCH();
    }
    return SCC_OK;
}

int enqueue(scc_batch* h, const int32_t* order, int norder, int32_t* out, cudaStream_t s) {
    BatchArgs A = make_args(h, order, norder, out);
    k_batch_reset<<<1, 1, 0, s>>>(h->flags, h->flags + 1);
    SCC_LAUNCH();
    SCC_TRY(enqueue_groups(h, s));
    batch_kernel_for(h->cfg)<<<h->blocks, h->cfg.block, batch_smem_bytes(h->cfg.block), s>>>(A);
    SCC_LAUNCH();
    return SCC_OK;
}

// Capture the reset and the persistent kernel as one CUDA graph.
int capture(scc_batch* h, const int32_t* order, int norder, int32_t* out) {
    drop_exec(h);
    cudaStream_t cs;
    SCC_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    int rc = cuda_err(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    if (rc == SCC_OK) {
        BatchArgs A = make_args(h, order, norder, out);
        k_batch_reset<<<1, 1, 0, cs>>>(h->flags, h->flags + 1);
        rc = enqueue_groups(h, cs);
        if (rc == SCC_OK) {
            batch_kernel_for(h->cfg)<<<h->blocks, h->cfg.block, batch_smem_bytes(h->cfg.block), cs>>>(A);
            rc = cuda_err(cudaGetLastError());
        }
        const int rc2 = cuda_err(cudaStreamEndCapture(cs, &graph));
        if (rc == SCC_OK) rc = rc2;
    }
    if (rc == SCC_OK) {
        size_t nn = 0;
        rc = cuda_err(cudaGraphGetNodes(graph, nullptr, &nn));
        std::vector<cudaGraphNode_t> nodes(nn);
        if (rc == SCC_OK && nn > 0) rc = cuda_err(cudaGraphGetNodes(graph, nodes.data(), &nn));
        h->exec_kernels = 0;
        for (size_t k = 0; rc == SCC_OK && k < nn; ++k) {
            cudaGraphNodeType t;
            if (cudaGraphNodeGetType(nodes[k], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) h->exec_kernels++;
        }
    }
    if (rc == SCC_OK) rc = cuda_err(cudaGraphInstantiate(&h->exec, graph, 0));
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    SCC_TRY(rc);
    h->exec_out = out;
    h->exec_order = order;
    h->exec_norder = norder;
    h->exec_valid = true;
    h->st.captures++;
    return SCC_OK;
}

// One run over `order` into `out` (device), timed with CUDA events.
int run_order(scc_batch* h, const int32_t* order, int norder, int32_t* out, cudaStream_t s, double* ms) {
    if (!h->ws) SCC_TRY(prepare(h, s));
    cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
    SCC_CUDA(cudaStreamIsCapturing(s, &cst));
    if (cst != cudaStreamCaptureStatusNone) {
        // the caller is capturing: add the launches to the caller's graph
        return enqueue(h, order, norder, out, s);
    }
    if (!h->exec_valid || h->exec_out != out || h->exec_order != order || h->exec_norder != norder)
        SCC_TRY(capture(h, order, norder, out));
    cudaEvent_t e0, e1;
    SCC_CUDA(cudaEventCreate(&e0));
    SCC_CUDA(cudaEventCreate(&e1));
    cudaEventRecord(e0, s);
    cudaError_t le = cudaGraphLaunch(h->exec, s);
    cudaEventRecord(e1, s);
    for (int k = 0; k < h->exec_kernels; ++k) count_launch();  // the graph's kernels (reset, G^T, persistent)
    int herr = 0;
    cudaError_t ce = cudaMemcpyAsync(&herr, h->flags + 1, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaError_t se = cudaStreamSynchronize(s);
    float f = 0;
    cudaEventElapsedTime(&f, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    SCC_CUDA(le);
    SCC_CUDA(ce);
    SCC_CUDA(se);
    h->st.replays++;
    h->st.ms_last_run = f;
    if (ms) *ms = f;
    return herr ? herr : SCC_OK;
}

void batch_free(scc_batch* h, cudaStream_t s) {
    drop_exec(h);
    dfree(h->ws, s);
    dfree(h->gt_off, s);
    dfree(h->gt_adj, s);
    dfree(h->gt_ok, s);
    dfree(h->grp_off, s);
    dfree(h->grp_adj, s);
    dfree(h->grp_toff, s);
    dfree(h->grp_scratch, s);
    dfree(h->vbase, s);
    dfree(h->ebase, s);
    dfree(h->offsets, s);
    dfree(h->targets, s);
    dfree(h->order, s);
    dfree(h->flags, s);
    dfree(h->times, s);
    dfree(h->labels, s);
}

// One block per graph: its CSR is well formed (offsets start at 0, do not
// decrease and end at its arc count; targets in [0, n_g)); *bad set otherwise.
__global__ void k_batch_validate(int32_t G, const long long* vbase, const long long* ebase, const int32_t* off,
                                 const int32_t* adj, int* bad) {
    for (int g = blockIdx.x; g < G; g += gridDim.x) {
        const long long n = vbase[g + 1] - vbase[g];
        const long long m = ebase[g + 1] - ebase[g];
        const int32_t* o = off + vbase[g] + g;
        const int32_t* a = adj + ebase[g];
        if (threadIdx.x == 0 && (o[0] != 0 || (long long)o[n] != m)) atomicExch(bad, 1);
        for (long long v = threadIdx.x; v < n; v += blockDim.x)
            if (o[v] > o[v + 1]) atomicExch(bad, 1);
        for (long long e = threadIdx.x; e < m; e += blockDim.x)
            if (a[e] < 0 || (long long)a[e] >= n) atomicExch(bad, 1);
    }
}

int batch_create_impl(scc_batch* h, int32_t G, const int64_t* vbase, const int64_t* ebase, const int32_t* offsets,
                      const int32_t* targets, cudaStream_t s) {
    SCC_TRY(device_info(&h->di));
    h->G = G;
    // bases on the host (sizes, processing order) and on the device
    h->vb_h.resize((size_t)G + 1);
    h->eb_h.resize((size_t)G + 1);
    SCC_CUDA(cudaMemcpyAsync(h->vb_h.data(), vbase, sizeof(long long) * ((size_t)G + 1), cudaMemcpyDefault, s));
    SCC_CUDA(cudaMemcpyAsync(h->eb_h.data(), ebase, sizeof(long long) * ((size_t)G + 1), cudaMemcpyDefault, s));
    SCC_CUDA(cudaStreamSynchronize(s));
    if (h->vb_h[0] != 0 || h->eb_h[0] != 0) return SCC_ERR_INVALID_ARG;
    for (int32_t g = 0; g < G; ++g) {
        const long long n = h->vb_h[g + 1] - h->vb_h[g], m = h->eb_h[g + 1] - h->eb_h[g];
        if (n < 0 || m < 0 || n > (1ll << 30) || m > (long long)INT32_MAX) return SCC_ERR_INVALID_ARG;
        h->n_max = std::max(h->n_max, n);
        h->m_max = std::max(h->m_max, m);
    }
    h->nv = h->vb_h[G];
    h->na = h->eb_h[G];
    SCC_TRY(dalloc_t(&h->vbase, (size_t)G + 1, s));
    SCC_TRY(dalloc_t(&h->ebase, (size_t)G + 1, s));
    SCC_TRY(dalloc_t(&h->offsets, (size_t)(h->nv + G) + 1, s));
    SCC_TRY(dalloc_t(&h->targets, (size_t)h->na + 1, s));
    SCC_TRY(dalloc_t(&h->flags, 2, s));
    SCC_TRY(dalloc_t(&h->times, (size_t)kTimeWords * G + 1, s));
    SCC_TRY(dalloc_t(&h->labels, (size_t)h->nv + 1, s));
    SCC_CUDA(cudaMemcpyAsync(h->vbase, h->vb_h.data(), sizeof(long long) * ((size_t)G + 1), cudaMemcpyHostToDevice, s));
    SCC_CUDA(cudaMemcpyAsync(h->ebase, h->eb_h.data(), sizeof(long long) * ((size_t)G + 1), cudaMemcpyHostToDevice, s));
    if (h->nv + G > 0)
        SCC_CUDA(cudaMemcpyAsync(h->offsets, offsets, sizeof(int32_t) * (size_t)(h->nv + G), cudaMemcpyDefault, s));
    if (h->na > 0)
        SCC_CUDA(cudaMemcpyAsync(h->targets, targets, sizeof(int32_t) * (size_t)h->na, cudaMemcpyDefault, s));
    Scratch tmp(s);
    int* bad = nullptr;
    SCC_TRY(tmp.alloc(&bad, 1));
    SCC_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
    if (G > 0) {
        k_batch_validate<<<std::min<int32_t>(G, 65535), 256, 0, s>>>(G, h->vbase, h->ebase, h->offsets, h->targets,
                                                                     bad);
        SCC_LAUNCH();
    }
    int hbad = 0;
    SCC_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    SCC_CUDA(cudaStreamSynchronize(s));
    tmp.release(bad);
    if (hbad) return SCC_ERR_INVALID_ARG;
    // processing order: decreasing work (arcs + vertices), so long graphs start first
    h->order_h.resize((size_t)G);
    for (int32_t g = 0; g < G; ++g) h->order_h[g] = g;
    std::stable_sort(h->order_h.begin(), h->order_h.end(), [&](int32_t a, int32_t b) {
        const long long wa = (h->eb_h[a + 1] - h->eb_h[a]) + (h->vb_h[a + 1] - h->vb_h[a]);
        const long long wb = (h->eb_h[b + 1] - h->eb_h[b]) + (h->vb_h[b + 1] - h->vb_h[b]);
        return wa > wb;
    });
    SCC_TRY(dalloc_t(&h->order, (size_t)G + 1, s));
    if (G > 0)
        SCC_CUDA(cudaMemcpyAsync(h->order, h->order_h.data(), sizeof(int32_t) * (size_t)G, cudaMemcpyHostToDevice, s));
    // groups of consecutive graphs for the G^T computed before each launch: up
    // to kGroupVerts vertices and kGroupArcs arcs each; a larger graph is left
    // to its block
    std::vector<unsigned char> ok;
    plan_groups(G, h->vb_h.data(), h->eb_h.data(), kGroupVerts, kGroupArcs, h->groups, ok);
    long long ng_max = 0, mg_max = 0;
    for (const auto& gr : h->groups) {
        ng_max = std::max(ng_max, gr.v1 - gr.v0);
        mg_max = std::max(mg_max, gr.e1 - gr.e0);
    }
    if (!h->groups.empty()) {
        SCC_TRY(dalloc_t(&h->gt_off, (size_t)(h->nv + G) + 1, s));
        SCC_TRY(dalloc_t(&h->gt_adj, (size_t)h->na + 1, s));
        SCC_TRY(dalloc_t(&h->gt_ok, (size_t)G + 1, s));
        SCC_CUDA(cudaMemcpyAsync(h->gt_ok, ok.data(), (size_t)G, cudaMemcpyHostToDevice, s));
        SCC_TRY(dalloc_t(&h->grp_off, (size_t)ng_max + 1, s));
        SCC_TRY(dalloc_t(&h->grp_toff, (size_t)ng_max + 1, s));
        SCC_TRY(dalloc_t(&h->grp_adj, (size_t)mg_max + 8, s));
        SCC_TRY(dalloc_t(&h->grp_scratch, transpose_scratch_bytes(mg_max), s));
        transpose_scratch_carve(h->grp_scratch, mg_max, &h->ts);
        SCC_TRY(transpose_set_attributes());  // before any capture
    }
    SCC_CUDA(cudaStreamSynchronize(s));
    memset(&h->st, 0, sizeof(h->st));
    h->st.graphs = G;
    h->st.vertices = h->nv;
    h->st.arcs = h->na;
    h->st.max_vertices = (int32_t)h->n_max;
    h->st.max_arcs = h->m_max;
    return SCC_OK;
}

}  // namespace

// ------------------------------------------------------------ batch runner --
// The batched kernel on caller-owned packed device arrays, with working memory
// allocated once (for graphs of up to n_max vertices and m_max arcs, up to
// gcap graphs per launch): what a serving loop launches over and over.
struct BatchRunner {
    DeviceInfo di;
    scc_batch_config cfg;
    long long gcap = 0;
    unsigned char* ws = nullptr;
    size_t bytes = 0;
    WsLayout L;
    BatchDims D;
    int blocks = 0;
    int* flags = nullptr;
    unsigned long long* times = nullptr;
};

int batch_runner_create(const scc_batch_config* cfg, long long n_max, long long m_max, long long gcap, size_t budget,
                        cudaStream_t s, BatchRunner** out) {
    *out = nullptr;
    BatchRunner* r = new (std::nothrow) BatchRunner();
    if (!r) return SCC_ERR_OOM;
    auto fail = [&](int rc) {
        batch_runner_destroy(r, s);
        return rc;
    };
    r->gcap = std::max<long long>(gcap, 1);
    if (cfg) r->cfg = *cfg;
    else scc_batch_config_default(&r->cfg);
    if (!valid_config(&r->cfg)) return fail(SCC_ERR_INVALID_ARG);
    int rc = device_info(&r->di);
    if (rc == SCC_OK) rc = plan_workspace(r->di, r->cfg, n_max, m_max, r->gcap, budget ? budget : default_budget(),
                                          &r->L, &r->D, &r->blocks);
    if (rc == SCC_OK) rc = dalloc(reinterpret_cast<void**>(&r->ws), r->L.bytes * (size_t)r->blocks, s);
    if (rc == SCC_OK) rc = dalloc_t(&r->flags, 2, s);
    if (rc == SCC_OK) rc = dalloc_t(&r->times, (size_t)kTimeWords * r->gcap, s);
    if (rc == SCC_OK) rc = init_workspace(r->ws, r->L, r->D, r->blocks, r->di.num_sms, s);
    if (rc != SCC_OK) return fail(rc);
    r->bytes = r->L.bytes * (size_t)r->blocks + 8 * (size_t)kTimeWords * r->gcap;
    *out = r;
    return SCC_OK;
}

void batch_runner_destroy(BatchRunner* r, cudaStream_t s) {
    if (!r) return;
    dfree(r->ws, s);
    dfree(r->flags, s);
    dfree(r->times, s);
    delete r;
}

// bad[g] = 1 when graph g of a packed batch is malformed (offsets not starting
// at 0, decreasing or not ending at m_g; a target outside [0, n_g)), else 0.
__global__ void k_batch_validate_each(int32_t G, const long long* vbase, const long long* ebase, const int32_t* off,
                                      const int32_t* adj, int* bad) {
    for (int g = blockIdx.x; g < G; g += gridDim.x) {
        const long long n = vbase[g + 1] - vbase[g];
        const long long m = ebase[g + 1] - ebase[g];
        const int32_t* o = off + vbase[g] + g;
        const int32_t* a = adj + ebase[g];
        __shared__ int s_bad;
        if (threadIdx.x == 0) s_bad = (o[0] != 0 || (long long)o[n] != m);
        __syncthreads();
        bool b = false;
        for (long long v = threadIdx.x; v < n; v += blockDim.x) b |= o[v] > o[v + 1];
        for (long long e = threadIdx.x; e < m; e += blockDim.x) b |= a[e] < 0 || (long long)a[e] >= n;
        if (b) s_bad = 1;
        __syncthreads();
        if (threadIdx.x == 0) bad[g] = s_bad;
        __syncthreads();
    }
}

int batch_validate_each(int32_t G, const long long* vbase, const long long* ebase, const int32_t* offsets,
                        const int32_t* targets, int* bad, cudaStream_t s) {
    if (G <= 0) return SCC_OK;
    k_batch_validate_each<<<std::min<int32_t>(G, 65535), 256, 0, s>>>(G, vbase, ebase, offsets, targets, bad);
    SCC_LAUNCH();
    return SCC_OK;
}

bool batch_runner_fits(const BatchRunner* r, long long n, long long m) { return n <= r->D.n_max && m <= r->D.m_max; }
size_t batch_runner_bytes(const BatchRunner* r) { return r->bytes; }
const int* batch_runner_err(const BatchRunner* r) { return r->flags + 1; }

int batch_runner_enqueue(BatchRunner* r, int32_t G, const long long* vbase, const long long* ebase,
                         const int32_t* offsets, const int32_t* targets, const int32_t* order, int32_t norder,
                         int32_t* out, cudaStream_t s) {
    if (norder > r->gcap) return SCC_ERR_INVALID_ARG;
    BatchArgs A = args_for(r->cfg, r->ws, r->L, r->D, r->flags, r->times, G, vbase, ebase, offsets, targets, order,
                           norder, out);
    k_batch_reset<<<1, 1, 0, s>>>(r->flags, r->flags + 1);
    SCC_LAUNCH();
    batch_kernel_for(r->cfg)<<<r->blocks, r->cfg.block, batch_smem_bytes(r->cfg.block), s>>>(A);
    SCC_LAUNCH();
    return SCC_OK;
}

}  // namespace scc

using namespace scc;

extern "C" {

SCC_API int scc_batch_config_default(scc_batch_config* cfg) {
    if (!cfg) return SCC_ERR_INVALID_ARG;
    cfg->tau = 0;
    cfg->block = 1024;
    cfg->lambda = 256;
    cfg->sigma = 50;
    cfg->seeds = 32;
    cfg->beta = 2.0;
    cfg->blocks_per_sm = 0;
    cfg->seed = 0x5CC00;
    return SCC_OK;
}

SCC_API int scc_batch_create(int32_t G, const int64_t* vbase, const int64_t* ebase, const int32_t* offsets,
                             const int32_t* targets, void* stream_, scc_batch_handle* out) {
    cudaStream_t stream = (cudaStream_t)stream_;
    if (!out || G < 0 || !vbase || !ebase) return SCC_ERR_INVALID_ARG;
    *out = nullptr;
    scc_batch* h = new (std::nothrow) scc_batch();
    if (!h) return SCC_ERR_OOM;
    scc_batch_config_default(&h->cfg);
    int rc = batch_create_impl(h, G, vbase, ebase, offsets, targets, stream);
    if (rc == SCC_OK && ((h->nv + G > 0 && !offsets) || (h->na > 0 && !targets))) rc = SCC_ERR_INVALID_ARG;
    if (rc != SCC_OK) {
        cudaStreamSynchronize(stream);
        batch_free(h, stream);
        cudaStreamSynchronize(stream);
        delete h;
        return rc;
    }
    *out = h;
    return SCC_OK;
}

SCC_API int scc_batch_destroy(scc_batch_handle h) {
    if (!h) return SCC_OK;
    cudaDeviceSynchronize();
    batch_free(h, 0);
    cudaDeviceSynchronize();
    delete h;
    return SCC_OK;
}

SCC_API int scc_batch_set_config(scc_batch_handle h, const scc_batch_config* cfg) {
    if (!h || !valid_config(cfg)) return SCC_ERR_INVALID_ARG;
    const bool relayout = cfg->block != h->cfg.block || cfg->lambda != h->cfg.lambda ||
                          cfg->blocks_per_sm != h->cfg.blocks_per_sm;
    h->cfg = *cfg;
    drop_exec(h);
    if (relayout && h->ws) {
        cudaDeviceSynchronize();
        dfree(h->ws, 0);
        cudaDeviceSynchronize();
        h->ws = nullptr;
        h->ws_bytes = 0;
    }
    return SCC_OK;
}

SCC_API int scc_batch_get_config(scc_batch_handle h, scc_batch_config* cfg) {
    if (!h || !cfg) return SCC_ERR_INVALID_ARG;
    *cfg = h->cfg;
    return SCC_OK;
}

SCC_API int scc_batch_run(scc_batch_handle h, int32_t* labels_out, void* stream_) {
    cudaStream_t stream = (cudaStream_t)stream_;
    if (!h || (!labels_out && h->nv > 0)) return SCC_ERR_INVALID_ARG;
    if (h->G == 0 || h->nv == 0) return SCC_OK;
    const bool dev_out = is_device_ptr(labels_out);
    int32_t* dst = dev_out ? labels_out : h->labels;
    SCC_TRY(run_order(h, h->order, h->G, dst, stream, nullptr));
    if (!dev_out) {
        SCC_CUDA(cudaMemcpyAsync(labels_out, h->labels, sizeof(int32_t) * (size_t)h->nv, cudaMemcpyDeviceToHost, stream));
        SCC_CUDA(cudaStreamSynchronize(stream));
    }
    return SCC_OK;
}

SCC_API int scc_batch_autotune(scc_batch_handle h, int32_t sample, void* stream_, scc_batch_config* best,
                               double* best_ms) {
    cudaStream_t stream = (cudaStream_t)stream_;
    if (!h) return SCC_ERR_INVALID_ARG;
    const scc_batch_config base = h->cfg;
    if (h->G == 0) {
        if (best) *best = base;
        if (best_ms) *best_ms = 0;
        return SCC_OK;
    }
    // the sample: every k-th graph of the size order, so it spans the size range
    std::vector<int32_t> sub;
    const int32_t want = (sample <= 0 || sample >= h->G) ? h->G : sample;
    const double step = (double)h->G / (double)want;
    for (int32_t i = 0; i < want; ++i) sub.push_back(h->order_h[(size_t)std::min<double>(h->G - 1, i * step)]);
    Scratch tmp(stream);
    int32_t* dsub = nullptr;
    SCC_TRY(tmp.alloc(&dsub, sub.size()));
    SCC_CUDA(cudaMemcpyAsync(dsub, sub.data(), sizeof(int32_t) * sub.size(), cudaMemcpyHostToDevice, stream));
    const int taus[] = {16, 64, 256, 1024, 4096};
    const int blocks[] = {128, 256, 512, 1024};
    const int lambdas[] = {256, 1024, 4096, 16384};
    // The objective is the sample's total block time (every sampled graph
    // runs on its own block, from the kernel's per-graph clock), not the
    // launch's span: a sample smaller than the grid finishes when its largest
    // graph does, while a full batch's time is its total work spread over the
    // blocks. It is not divided by the blocks a full launch keeps resident:
    // the sample's few blocks each have an SM to themselves, so a small block
    // runs faster here than beside the others of a full batch, and that
    // division favoured 512-thread blocks that lost on the full batch (span
    // 516 against 477 ms). The configuration in the handle stays unless
    // another one cuts the objective by more than 3%.
    std::vector<unsigned long long> tms((size_t)kTimeWords * h->G);
    auto measure = [&](const scc_batch_config& c, double* work, double* span) -> int {
        SCC_TRY(scc_batch_set_config(h, &c));
        double ms = 0;
        SCC_TRY(run_order(h, dsub, (int)sub.size(), h->labels, stream, &ms));  // warm-up (and capture)
        SCC_TRY(run_order(h, dsub, (int)sub.size(), h->labels, stream, span));
        SCC_CUDA(cudaMemcpyAsync(tms.data(), h->times, sizeof(unsigned long long) * tms.size(),
                                 cudaMemcpyDeviceToHost, stream));
        SCC_CUDA(cudaStreamSynchronize(stream));
        double w = 0;
        for (int32_t g : sub) {
            const unsigned long long* t = &tms[(size_t)kTimeWords * g];
            w += t[5] > t[0] ? 1e-6 * (double)(t[5] - t[0]) : 0.0;
        }
        *work = w;
        return SCC_OK;
    };
    scc_batch_config bc = base;
    double bwork = 1e300, bms = 0, base_work = 0, base_ms = 0;
    int rc = measure(base, &base_work, &base_ms);
    for (int blk : blocks) {
        if (rc != SCC_OK) break;
        for (int lam : lambdas) {
            if (rc != SCC_OK) break;
            for (int tau : taus) {
                scc_batch_config c = base;
                c.block = blk;
                c.lambda = lam;
                c.tau = tau;
                double work = 0, ms2 = 0;
                rc = measure(c, &work, &ms2);
                if (rc != SCC_OK) break;
                if (work < bwork) {
                    bwork = work;
                    bms = ms2;
                    bc = c;
                }
            }
        }
    }
    if (rc == SCC_OK && !(bwork < 0.97 * base_work)) {
        bc = base;
        bms = base_ms;
    }
    tmp.release(dsub);
    cudaStreamSynchronize(stream);
    const int rc2 = scc_batch_set_config(h, rc == SCC_OK ? &bc : &base);
    if (rc != SCC_OK) return rc;
    if (rc2 != SCC_OK) return rc2;
    if (best) *best = bc;
    if (best_ms) *best_ms = bms;
    return SCC_OK;
}

SCC_API int scc_debug_batch_groups(int32_t G, const int64_t* vbase, const int64_t* ebase, int64_t max_vertices,
                                   int64_t max_arcs, int32_t* groups, int32_t* ngroups) {
    if (G < 0 || !ngroups || max_vertices < 1 || max_arcs < 0 || (G > 0 && (!vbase || !ebase || !groups)))
        return SCC_ERR_INVALID_ARG;
    std::vector<long long> vb((size_t)G + 1), eb((size_t)G + 1);
    for (int32_t g = 0; g <= G; ++g) {
        vb[g] = vbase[g];
        eb[g] = ebase[g];
        if (g > 0 && (vb[g] < vb[g - 1] || eb[g] < eb[g - 1])) return SCC_ERR_INVALID_ARG;
    }
    std::vector<scc::GroupPlan> plan;
    std::vector<unsigned char> ok;
    scc::plan_groups(G, vb.data(), eb.data(), max_vertices, max_arcs, plan, ok);
    for (size_t k = 0; k < plan.size(); ++k) {
        groups[2 * k] = plan[k].g0;
        groups[2 * k + 1] = plan[k].g1;
    }
    *ngroups = (int32_t)plan.size();
    return SCC_OK;
}

SCC_API int scc_debug_batch_times(scc_batch_handle h, uint64_t* out) {
    if (!h || (!out && h->G > 0)) return SCC_ERR_INVALID_ARG;
    if (h->G == 0) return SCC_OK;
    SCC_CUDA(cudaMemcpy(out, h->times, sizeof(uint64_t) * kTimeWords * (size_t)h->G, cudaMemcpyDeviceToHost));
    return SCC_OK;
}

SCC_API int scc_batch_get_stats(scc_batch_handle h, scc_batch_stats* out) {
    if (!h || !out) return SCC_ERR_INVALID_ARG;
    *out = h->st;
    return SCC_OK;
}

}  // extern "C"
