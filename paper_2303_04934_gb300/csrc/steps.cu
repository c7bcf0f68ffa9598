// SCC steps other than the reachability searches (sm_103a):
//  - CSR validation, transposed-CSR construction (histogram, scan, scatter);
//  - trimming (Sec. 4.1);
//  - pivot permutation and prefix-doubling batches (Alg. 1; Sec. 2);
//  - labelling/partition after the first SCC and after each multi-search round
//    (Alg. 1; Sec. 4.4);
//  - canonical minimum labels.
// Paper: Wang, Dong, Gu, Sun, "Parallel Strong Connectivity Based on Faster
// Reachability", SIGMOD 2023.
#include <climits>

#include "common.cuh"
#include "engine.cuh"
#include "internal.h"

namespace scc {

namespace {

constexpr int kBlk = 256;
constexpr int kEdgeTile = kBlk * 8;  // arcs per block tile in the CSR passes

inline int grid_for(int64_t work, int per_block, int cap = 152 * 32) {
    int64_t g = (work + per_block - 1) / per_block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

// Largest r in [lo, hi] with off[r] <= e (off non-decreasing, off[lo] <= e).
__device__ __forceinline__ int row_of(const int32_t* __restrict__ off, int lo, int hi, int64_t e) {
    while (lo < hi) {
        int mid = lo + ((hi - lo + 1) >> 1);
        if ((int64_t)__ldg(&off[mid]) <= e) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Row range of the arcs [e0, e1) of a tile, found once per block.
__device__ __forceinline__ void tile_rows(const int32_t* off, int32_t n, int64_t e0, int64_t e1, int* r0, int* r1) {
    __shared__ int s_r[2];
    if (threadIdx.x == 0) {
        s_r[0] = row_of(off, 0, n - 1, e0);
        s_r[1] = row_of(off, s_r[0], n - 1, e1 - 1);
    }
    __syncthreads();
    *r0 = s_r[0];
    *r1 = s_r[1];
    __syncthreads();
}

// ---------------------------------------------------------------- validate --
__global__ void k_validate_offsets(const int32_t* __restrict__ off, int32_t n, int64_t m, int* bad) {
    int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (tid == 0 && (off[0] != 0 || (int64_t)off[n] != m)) atomicExch(bad, 1);
    for (int64_t i = tid; i < n; i += stride)
        if (off[i] > off[i + 1]) atomicExch(bad, 1);
}

// Forward CSR without self-loops. Rows without self-loops are copied arc-parallel;
// rows with self-loops (rare) are copied by one thread each.
__global__ void __launch_bounds__(kBlk) k_drop_self_arcs(const int32_t* __restrict__ off,
                                                         const int32_t* __restrict__ adj, int32_t n, int64_t m,
                                                         const int32_t* __restrict__ selfrow,
                                                         const int32_t* __restrict__ off2, int32_t* adj2) {
    for (int64_t t0 = (int64_t)blockIdx.x * kEdgeTile; t0 < m; t0 += (int64_t)gridDim.x * kEdgeTile) {
        int64_t t1 = t0 + kEdgeTile < m ? t0 + kEdgeTile : m;
        int r0, r1;
        tile_rows(off, n, t0, t1, &r0, &r1);
        for (int64_t e = t0 + threadIdx.x; e < t1; e += blockDim.x) {
            int u = row_of(off, r0, r1, e);
            if (selfrow[u] == 0) adj2[off2[u] + (e - off[u])] = adj[e];
        }
    }
}
// The rows with self-loops: one thread copies a row, skipping its self-loops.
__global__ void k_drop_self_rows(const int32_t* __restrict__ off, const int32_t* __restrict__ adj, int32_t n,
                                 const int32_t* __restrict__ selfrow, const int32_t* __restrict__ off2,
                                 int32_t* adj2) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
        if (selfrow[u] == 0) continue;
        int o = off2[u];
        for (int e = off[u]; e < off[u + 1]; ++e)
            if (adj[e] != u) adj2[o++] = adj[e];
    }
}
// out[u] = arcs of row u that are not self-loops (the new CSR's row lengths).
__global__ void k_sub(const int32_t* __restrict__ off, const int32_t* __restrict__ selfrow, int32_t n, int32_t* out) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x)
        out[u] = off[u + 1] - off[u] - selfrow[u];
}

// ------------------------------------------------------------------- scan --
constexpr int kScanItems = 8;
constexpr int kScanTile = kBlk * kScanItems;

__device__ __forceinline__ long long block_excl_scan(long long x, long long* total) {
    __shared__ long long s_w[kBlk / 32];
    const int lane = lane_id(), w = threadIdx.x >> 5;
    long long incl = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        long long y = __shfl_up_sync(kFull, incl, d);
        if (lane >= d) incl += y;
    }
    if (lane == 31) s_w[w] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long s = 0;
        for (int i = 0; i < kBlk / 32; ++i) {
            long long c = s_w[i];
            s_w[i] = s;
            s += c;
        }
        *total = s;
    }
    __syncthreads();
    long long r = s_w[w] + incl - x;
    __syncthreads();
    return r;
}

// Exclusive scan of int32 counts in three passes: per-tile sums, a scan of the
// sums in one block, then each tile's scan from its offset.
__global__ void __launch_bounds__(kBlk) k_scan_reduce(const int32_t* __restrict__ in, int64_t n, long long* sums) {
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    long long s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n) s += in[base + k];
    __shared__ long long tot;
    block_excl_scan(s, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}
__global__ void __launch_bounds__(1024) k_scan_sums(long long* sums, int64_t nb, long long* total) {
    // one block: each thread owns a contiguous run of block sums
    __shared__ long long s_part[1024];
    int64_t per = (nb + 1023) / 1024;
    int64_t b0 = (int64_t)threadIdx.x * per, b1 = b0 + per < nb ? b0 + per : nb;
    long long s = 0;
    for (int64_t i = b0; i < b1; ++i) s += sums[i];
    s_part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long a = 0;
        for (int i = 0; i < 1024; ++i) {
            long long c = s_part[i];
            s_part[i] = a;
            a += c;
        }
        *total = a;
    }
    __syncthreads();
    long long a = s_part[threadIdx.x];
    for (int64_t i = b0; i < b1; ++i) {
        long long c = sums[i];
        sums[i] = a;
        a += c;
    }
}
__global__ void __launch_bounds__(kBlk) k_scan_down(const int32_t* __restrict__ in, int32_t* out, int64_t n,
                                                   const long long* __restrict__ sums, const long long* total) {
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int32_t v[kScanItems];
    long long s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = base + k < n ? in[base + k] : 0;
        s += v[k];
    }
    __shared__ long long tot;
    long long pre = block_excl_scan(s, &tot) + sums[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) out[base + k] = (int32_t)pre;
        pre += v[k];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = (int32_t)*total;
}

// ------------------------------------------------------------------- trim --
__global__ void k_trim(const int32_t* __restrict__ off, const int32_t* __restrict__ toff, int32_t n, uint8_t* flags) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        flags[v] = (off[v + 1] == off[v]) || (toff[v + 1] == toff[v]);
}

// Four consecutive vertices per thread (16-byte loads and stores; the arrays
// are 16-byte aligned), the last partial group one by one.
__global__ void k_init_labels(const int32_t* __restrict__ off, const int32_t* __restrict__ toff, int32_t n,
                              int32_t* label, int32_t* rep, unsigned long long* nact) {
    unsigned long long c = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; 4 * i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v0 = 4 * i;
        if (v0 + 4 <= n) {
            const int4 a = __ldg(reinterpret_cast<const int4*>(off + v0));
            const int4 b = __ldg(reinterpret_cast<const int4*>(toff + v0));
            const int a4 = __ldg(off + v0 + 4), b4 = __ldg(toff + v0 + 4);
            const bool t0 = a.y == a.x || b.y == b.x, t1 = a.z == a.y || b.z == b.y;
            const bool t2 = a.w == a.z || b.w == b.z, t3 = a4 == a.w || b4 == b.w;
            *reinterpret_cast<int4*>(label + v0) = make_int4(t0 ? kDone : 0, t1 ? kDone : 0, t2 ? kDone : 0,
                                                             t3 ? kDone : 0);
            const int u = (int)v0;
            *reinterpret_cast<int4*>(rep + v0) = make_int4(t0 ? u : -1, t1 ? u + 1 : -1, t2 ? u + 2 : -1,
                                                           t3 ? u + 3 : -1);
            c += (unsigned long long)(!t0 + !t1 + !t2 + !t3);
        } else {
            for (int64_t v = v0; v < n; ++v) {
                const bool tr = (off[v + 1] == off[v]) || (toff[v + 1] == toff[v]);
                label[v] = tr ? kDone : 0;
                rep[v] = tr ? (int32_t)v : -1;
                c += !tr;
            }
        }
    }
    for (int d = 16; d >= 1; d >>= 1) c += __shfl_xor_sync(kFull, c, d);
    if (lane_id() == 0 && c) atomicAdd(nact, c);
}

// ----------------------------------------------------------------- pivots --
__global__ void k_pivot_order(const int32_t* __restrict__ act, int64_t N, Feistel f, int32_t* order) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x)
        order[p] = act[f.perm((uint64_t)p, (uint64_t)N)];
}

// Remaining pivot positions p >= p0 whose vertex is still active, in order.
__global__ void k_rem_flags(const int32_t* __restrict__ act, int64_t N, Feistel f, int64_t p0,
                            const int32_t* __restrict__ label, int32_t* flags) {
    for (int64_t p = p0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x)
        flags[p - p0] = label[act[f.perm((uint64_t)p, (uint64_t)N)]] >= 0;
}
// rem_pos/rem_v of the remaining pivots, at the places the scan of the flags gives.
__global__ void k_rem_scatter(const int32_t* __restrict__ act, int64_t N, Feistel f, int64_t p0,
                              const int32_t* __restrict__ flags, const int32_t* __restrict__ pos, int32_t* rem_pos,
                              int32_t* rem_v) {
    for (int64_t p = p0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x)
        if (flags[p - p0]) {
            const int32_t j = pos[p - p0];
            rem_pos[j] = (int32_t)p;
            rem_v[j] = act[f.perm((uint64_t)p, (uint64_t)N)];
        }
}

// Active list (vertices with label >= 0, in increasing order) in two passes
// over the labels: per-tile counts, then (after the scan of the counts) a
// block scan of the flags and the scatter. Thread t of a tile owns the
// kScanItems consecutive vertices from tile + t * kScanItems.
__device__ __forceinline__ int active_bits(const int32_t* __restrict__ label, int32_t n, int64_t base) {
    int f = 0;
    if (base + kScanItems <= n && (base & 3) == 0) {
        const int4* p = reinterpret_cast<const int4*>(label + base);
#pragma unroll
        for (int q = 0; q < kScanItems / 4; ++q) {
            const int4 x = __ldg(p + q);
            f |= (x.x >= 0) << (4 * q) | (x.y >= 0) << (4 * q + 1) | (x.z >= 0) << (4 * q + 2) |
                 (x.w >= 0) << (4 * q + 3);
        }
    } else {
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) f |= (base + k < n && __ldg(&label[base + k]) >= 0) << k;
    }
    return f;
}
// act = increasing list of the active vertices: counts per tile, then a scatter.
__global__ void __launch_bounds__(kBlk) k_active_count(const int32_t* __restrict__ label, int32_t n, long long* sums) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int c = __popc(active_bits(label, n, base));
    for (int d = 16; d >= 1; d >>= 1) c += __shfl_xor_sync(kFull, c, d);
    __shared__ int s_c[kBlk / 32];
    if (lane_id() == 0) s_c[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int i = 0; i < kBlk / 32; ++i) t += s_c[i];
        sums[blockIdx.x] = t;
    }
}
__global__ void __launch_bounds__(kBlk) k_active_scatter(const int32_t* __restrict__ label, int32_t n,
                                                         const long long* __restrict__ sums, int32_t* act) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int f = active_bits(label, n, base);
    __shared__ long long tot;
    long long pos = block_excl_scan(__popc(f), &tot) + sums[blockIdx.x];
    while (f) {
        const int k = __ffs(f) - 1;
        f &= f - 1;
        act[pos++] = (int32_t)(base + k);
    }
}

// --------------------------------------------------------------- bitmaps --
// Bit v set for every vertex outside class L (and past n): lane l of a warp
// reads vertex 32 w + l, a ballot makes word w. bits2, if not null, gets the
// same words.
__global__ void k_prefill_bits(const int32_t* __restrict__ label, int32_t L, int32_t n, uint32_t* bits,
                               uint32_t* bits2) {
    const int64_t nw = ((int64_t)n + 31) / 32;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nw; w += warps) {
        const int64_t v = w * 32 + lane_id();
        const bool out = v >= n || (label != nullptr && __ldg(&label[v]) != L);
        const uint32_t b = __ballot_sync(kFull, out);
        if (lane_id() == 0) {
            bits[w] = b;
            if (bits2) bits2[w] = b;
        }
    }
}
// out[v] = 1 iff bit v is set and v is in class L (all classes when label is
// NULL): a visited bitmap as bytes, for the test hooks.
__global__ void k_bits_to_bytes(const uint32_t* __restrict__ bits, const int32_t* __restrict__ label, int32_t L,
                                int32_t n, uint8_t* out) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        bool in = label == nullptr || label[v] == L;
        out[v] = in && ((bits[v >> 5] >> (v & 31)) & 1u);
    }
}

// ---------------------------------------------------------------- labels --
// After the first SCC (one pivot s, class L = label[s]): a vertex of class L
// reached both ways is finished with representative s; otherwise its class
// becomes hash(L, s if reached from s, s if it reaches s) (Alg. 1 label step).
// Trimming inside classes: an active vertex with no out-arc or no in-arc to an
// active vertex of its own class cannot share a cycle with any other vertex, so
// it is a singleton SCC (Sec. 4.1 trimming, applied to the classes of Alg. 1).
// Arcs to finished vertices (label kDone, never equal to a class) are ignored.
// A vertex finished concurrently by another thread may or may not be seen as
// active; either way the decision is exact. Per thread one vertex of the active
// list, four arcs in flight, early exit at the first arc inside the class.
__device__ __forceinline__ bool has_class_arc(const int32_t* __restrict__ off, const int32_t* __restrict__ adj,
                                              const int32_t* label, int32_t v, int32_t L) {
    const int e1 = off[v + 1];
    for (int e = off[v]; e < e1; e += 4) {
        int w[4], lw[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) w[k] = e + k < e1 ? adj[e + k] : -1;
#pragma unroll
        for (int k = 0; k < 4; ++k) lw[k] = w[k] >= 0 ? ld_volatile(&label[w[k]]) : kDone;
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (lw[k] == L) return true;
    }
    return false;
}
__global__ void k_class_trim(const int32_t* __restrict__ act, int64_t N, const int32_t* __restrict__ off,
                             const int32_t* __restrict__ adj, const int32_t* __restrict__ toff,
                             const int32_t* __restrict__ tadj, int32_t* label, int32_t* rep,
                             unsigned long long* ndone) {
    unsigned long long c = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = act[i];
        const int32_t L = ld_volatile(&label[v]);
        if (L < 0) continue;
        if (has_class_arc(off, adj, label, v, L) && has_class_arc(toff, tadj, label, v, L)) continue;
        label[v] = kDone;
        rep[v] = v;
        ++c;
    }
    for (int d = 16; d >= 1; d >>= 1) c += __shfl_xor_sync(kFull, c, d);
    if (lane_id() == 0 && c) atomicAdd(ndone, c);
}

// Four consecutive vertices per thread (one 16-byte label load; their bits
// share a bitmap word).
__global__ void k_label_first(const uint32_t* __restrict__ bf, const uint32_t* __restrict__ bb, int32_t n, int32_t s,
                              int32_t L, int32_t* label, int32_t* rep, unsigned long long* ndone) {
    unsigned long long c = 0;
    auto one = [&](int64_t v, int lv, uint32_t wf, uint32_t wb) -> int {
        if (lv != L) return lv;
        const bool f = (wf >> (v & 31)) & 1u, b = (wb >> (v & 31)) & 1u;
        if (f && b) {
            rep[v] = s;
            ++c;
            return kDone;
        }
        return (f || b) ? class_hash(L, f ? s : -1, b ? s : -1) : lv;
    };
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; 4 * i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v0 = 4 * i;
        if (v0 + 4 <= n) {
            const int4 lab = *reinterpret_cast<const int4*>(label + v0);
            if (lab.x != L && lab.y != L && lab.z != L && lab.w != L) continue;
            const uint32_t wf = __ldg(&bf[v0 >> 5]), wb = __ldg(&bb[v0 >> 5]);
            const int4 o = make_int4(one(v0, lab.x, wf, wb), one(v0 + 1, lab.y, wf, wb), one(v0 + 2, lab.z, wf, wb),
                                     one(v0 + 3, lab.w, wf, wb));
            *reinterpret_cast<int4*>(label + v0) = o;
        } else {
            for (int64_t v = v0; v < n; ++v) label[v] = one(v, label[v], bf[v >> 5], bb[v >> 5]);
        }
    }
    for (int d = 16; d >= 1; d >>= 1) c += __shfl_xor_sync(kFull, c, d);
    if (lane_id() == 0 && c) atomicAdd(ndone, c);
}

// ---------------------------------------------------------- canonicalise --
// minid[v] = v where v is its own representative (every trimmed singleton, and
// the representative of each larger SCC), INT_MAX elsewhere: the pass below
// then needs no atomic for a vertex with rep[v] = v. Four vertices per thread.
__global__ void k_minid_init(const int32_t* __restrict__ rep, int32_t n, int32_t* minid) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; 4 * i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v0 = 4 * i;
        if (v0 + 4 <= n) {
            const int4 r = __ldg(reinterpret_cast<const int4*>(rep + v0));
            const int u = (int)v0;
            *reinterpret_cast<int4*>(minid + v0) = make_int4(r.x == u ? u : INT_MAX, r.y == u + 1 ? u + 1 : INT_MAX,
                                                             r.z == u + 2 ? u + 2 : INT_MAX,
                                                             r.w == u + 3 ? u + 3 : INT_MAX);
        } else {
            for (int64_t v = v0; v < n; ++v) minid[v] = rep[v] == (int32_t)v ? (int32_t)v : INT_MAX;
        }
    }
}
// minid[rep[v]] = min v. Lanes of a warp hold consecutive v, so among lanes with
// the same rep the lowest lane has the smallest v: one atomic per group, and
// only when it can still lower the stored minimum (an SCC of millions of
// vertices then costs a few atomics instead of one per vertex). A warp's v only
// grow, so a lane that has already offered its v for a rep skips that rep
// after: a large SCC is then read once per warp, not once per iteration (its
// minid word would otherwise take every warp's reads).
__global__ void k_min_of_rep(const int32_t* __restrict__ rep, int32_t n, int32_t* minid, int* bad) {
    int last = -1;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x; b < n; b += (int64_t)gridDim.x * blockDim.x) {
        int64_t v = b + threadIdx.x;
        int r = v < n ? rep[v] : -1;
        bool ok = r >= 0 && r < n;
        if (v < n && !ok) atomicExch(bad, 1);
        ok = ok && r != (int)v;  // minid[v] = v already (k_minid_init)
        int key = ok ? r : -1;
        // lanes whose reps are all one SCC's (the common case: a large SCC
        // among singletons) need no match: their first lane has the smallest v
        const uint32_t okm = __ballot_sync(kFull, ok);
        if (okm == 0) continue;
        const int key0 = __shfl_sync(kFull, key, __ffs(okm) - 1);
        const uint32_t peers = __ballot_sync(kFull, ok && key != key0) == 0 ? okm : __match_any_sync(kFull, key);
        if (ok && lane_id() == __ffs(peers & okm) - 1 && r != last) {
            last = r;
            if (ld_volatile(&minid[r]) > (int32_t)v) atomicMin(&minid[r], (int32_t)v);
        }
    }
}
// out[v] = minid[rep[v]], the last rep looked up kept per thread (a large SCC
// is then one read per thread). Four vertices per thread; out may be any
// device buffer, so the 16-byte stores are used only when it is aligned.
__global__ void k_write_labels(const int32_t* __restrict__ rep, int32_t n, const int32_t* __restrict__ minid,
                               int32_t* out) {
    int ck = -1, cv = -1;
    auto look = [&](int r) {
        if (r < 0 || r >= n) return -1;
        if (r != ck) {
            ck = r;
            cv = __ldg(&minid[r]);
        }
        return cv;
    };
    const bool vec = ((uintptr_t)out & 15) == 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; 4 * i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v0 = 4 * i;
        if (v0 + 4 <= n) {
            const int4 r = __ldg(reinterpret_cast<const int4*>(rep + v0));
            const int4 o = make_int4(look(r.x), look(r.y), look(r.z), look(r.w));
            if (vec) {
                *reinterpret_cast<int4*>(out + v0) = o;
            } else {
                out[v0] = o.x;
                out[v0 + 1] = o.y;
                out[v0 + 2] = o.z;
                out[v0 + 3] = o.w;
            }
        } else {
            for (int64_t v = v0; v < n; ++v) out[v] = look(rep[v]);
        }
    }
}

// ------------------------------------------------------------- pair table --
__global__ void k_table_gather(const unsigned long long* __restrict__ tab, int64_t cap, unsigned long long* out,
                               int64_t out_cap, unsigned long long* count) {
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x; b < cap; b += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = b + threadIdx.x;
        unsigned long long k = i < cap ? tab[i] : ~0ull;
        uint32_t msk = __ballot_sync(kFull, k != ~0ull);
        unsigned long long base = 0;
        if (lane_id() == 0 && msk) base = atomicAdd(count, (unsigned long long)__popc(msk));
        base = __shfl_sync(kFull, base, 0);
        unsigned long long pos = base + __popc(msk & lanemask_lt());
        if (k != ~0ull && (int64_t)pos < out_cap) out[pos] = k;
    }
}
// Insert-if-absent of every key (Sec. 4.5 pair table); *inserted += the keys
// that were new.
__global__ void k_table_insert(const unsigned long long* __restrict__ keys, int64_t count, PairTable t,
                               unsigned long long* inserted) {
    unsigned long long c = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        c += t.insert(keys[i]);
    for (int d = 16; d >= 1; d >>= 1) c += __shfl_xor_sync(kFull, c, d);
    if (lane_id() == 0 && c && inserted) atomicAdd(inserted, c);
}

}  // namespace

// ================================================================ launchers ==
int launch_validate_offsets(const int32_t* off, int32_t n, int64_t m, int* bad, cudaStream_t s) {
    k_validate_offsets<<<grid_for((int64_t)n + 1, kBlk * 4), kBlk, 0, s>>>(off, n, m, bad);
    SCC_LAUNCH();
    return SCC_OK;
}

size_t scan_tmp_bytes(int64_t n) { return (size_t)(ceil_div(n + 1, kScanTile) + 2) * sizeof(long long); }

int launch_scan(const int32_t* in, int32_t* out, int64_t n, void* tmp, cudaStream_t s) {
    int64_t nb = ceil_div(n > 0 ? n : 1, kScanTile);
    long long* sums = (long long*)tmp;
    long long* total = sums + nb;
    k_scan_reduce<<<(unsigned)nb, kBlk, 0, s>>>(in, n, sums);
    SCC_LAUNCH();
    k_scan_sums<<<1, 1024, 0, s>>>(sums, nb, total);
    SCC_LAUNCH();
    k_scan_down<<<(unsigned)nb, kBlk, 0, s>>>(in, out, n, sums, total);
    SCC_LAUNCH();
    return SCC_OK;
}

int launch_drop_self_loops(const int32_t* off, const int32_t* adj, int32_t n, int64_t m, const int32_t* selfrow,
                           const int32_t* off2, int32_t* adj2, cudaStream_t s) {
    if (m > 0) {
        k_drop_self_arcs<<<grid_for(m, kEdgeTile, 152 * 16), kBlk, 0, s>>>(off, adj, n, m, selfrow, off2, adj2);
        SCC_LAUNCH();
    }
    k_drop_self_rows<<<grid_for(n, kBlk), kBlk, 0, s>>>(off, adj, n, selfrow, off2, adj2);
    SCC_LAUNCH();
    return SCC_OK;
}

int launch_row_nonself(const int32_t* off, const int32_t* selfrow, int32_t n, int32_t* cnt, cudaStream_t s) {
    if (n == 0) return SCC_OK;
    k_sub<<<grid_for(n, kBlk), kBlk, 0, s>>>(off, selfrow, n, cnt);
    SCC_LAUNCH();
    return SCC_OK;
}

namespace {
// bit j of vertex sources[j]'s mask (words 64-bit words per vertex)
__global__ void k_mask_init(const int32_t* __restrict__ src, int32_t k, int32_t n, int words,
                            unsigned long long* mask, int* bad) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= k) return;
    int v = src[j];
    if (v < 0 || v >= n) {
        atomicExch(bad, 1);
        return;
    }
    atomicOr(&mask[(size_t)words * v + (j >> 6)], 1ull << (j & 63));
}
// The sources given to the test hook that are in [0, n) and unfinished (an
// id out of range sets *bad), compacted into out.
__global__ void k_filter_sources(const int32_t* __restrict__ in, int32_t k, int32_t n,
                                 const int32_t* __restrict__ label, int32_t* out, int* cnt, int* bad) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < k; j += gridDim.x * blockDim.x) {
        int v = in[j];
        if (v < 0 || v >= n) {
            atomicExch(bad, 1);
            continue;
        }
        if (label[v] >= 0) out[atomicAdd(cnt, 1)] = v;
    }
}
}  // namespace

int launch_mask_init(const int32_t* sources, int32_t k, int32_t n, int words, unsigned long long* mask, int* bad,
                     cudaStream_t s) {
    if (k < 1 || k > 64 * words) return SCC_ERR_INVALID_ARG;
    k_mask_init<<<1, 64 * words, 0, s>>>(sources, k, n, words, mask, bad);
    SCC_LAUNCH();
    return SCC_OK;
}

int launch_filter_sources(const int32_t* in, int32_t k, int32_t n, const int32_t* label, int32_t* out, int* cnt,
                          int* bad, cudaStream_t s) {
    k_filter_sources<<<grid_for(k, kBlk), kBlk, 0, s>>>(in, k, n, label, out, cnt, bad);
    SCC_LAUNCH();
    return SCC_OK;
}

int launch_trim(const int32_t* off, const int32_t* toff, int32_t n, uint8_t* flags, cudaStream_t s) {
    if (n == 0) return SCC_OK;
    k_trim<<<grid_for(n, kBlk), kBlk, 0, s>>>(off, toff, n, flags);
    SCC_LAUNCH();
    return SCC_OK;
}

int launch_init_labels(const int32_t* off, const int32_t* toff, int32_t n, int32_t* label, int32_t* rep,
                       unsigned long long* nact, cudaStream_t s) {
    if (n == 0) return SCC_OK;
    k_init_labels<<<grid_for(ceil_div((int64_t)n, 4), kBlk), kBlk, 0, s>>>(off, toff, n, label, rep, nact);
    SCC_LAUNCH();
    return SCC_OK;
}

int launch_compact_active(const int32_t* label, int32_t n, void* scan_tmp, int32_t* act, cudaStream_t s) {
    if (n == 0) return SCC_OK;
    const int64_t nb = ceil_div((int64_t)n, kScanTile);
    long long* sums = (long long*)scan_tmp;
    k_active_count<<<(unsigned)nb, kBlk, 0, s>>>(label, n, sums);
    SCC_LAUNCH();
    k_scan_sums<<<1, 1024, 0, s>>>(sums, nb, sums + nb);
    SCC_LAUNCH();
    k_active_scatter<<<(unsigned)nb, kBlk, 0, s>>>(label, n, sums, act);
    SCC_LAUNCH();
    return SCC_OK;
}

int64_t feistel_perm_host(int64_t p, int64_t N, uint64_t seed) {
    Feistel f;
    f.init(seed, (uint64_t)N);
    return (int64_t)f.perm((uint64_t)p, (uint64_t)N);
}

int launch_remaining(const int32_t* act, int64_t N, uint64_t seed, int64_t p0, const int32_t* label,
                     int32_t* flags_tmp, int32_t* pos_tmp, void* scan_tmp, int32_t* rem_pos, int32_t* rem_v,
                     cudaStream_t s) {
    const int64_t cnt = N - p0;
    if (cnt <= 0) return SCC_OK;
    Feistel f;
    f.init(seed, (uint64_t)N);
    k_rem_flags<<<grid_for(cnt, kBlk), kBlk, 0, s>>>(act, N, f, p0, label, flags_tmp);
    SCC_LAUNCH();
    SCC_TRY(launch_scan(flags_tmp, pos_tmp, cnt, scan_tmp, s));
    k_rem_scatter<<<grid_for(cnt, kBlk), kBlk, 0, s>>>(act, N, f, p0, flags_tmp, pos_tmp, rem_pos, rem_v);
    SCC_LAUNCH();
    return SCC_OK;
}

int launch_pivot_order(const int32_t* act, int64_t N, uint64_t seed, int32_t* order, cudaStream_t s) {
    if (N == 0) return SCC_OK;
    Feistel f;
    f.init(seed, (uint64_t)N);
    k_pivot_order<<<grid_for(N, kBlk), kBlk, 0, s>>>(act, N, f, order);
    SCC_LAUNCH();
    return SCC_OK;
}

int launch_prefill_bits(const int32_t* label, int32_t L, int32_t n, uint32_t* bits, uint32_t* bits2, cudaStream_t s) {
    int64_t nw = ((int64_t)n + 31) / 32;
    if (nw == 0) return SCC_OK;
    k_prefill_bits<<<grid_for(nw, kBlk / 32), kBlk, 0, s>>>(label, L, n, bits, bits2);
    SCC_LAUNCH();
    return SCC_OK;
}

int launch_bits_to_bytes(const uint32_t* bits, const int32_t* label, int32_t L, int32_t n, uint8_t* out,
                         cudaStream_t s) {
    if (n == 0) return SCC_OK;
    k_bits_to_bytes<<<grid_for(n, kBlk), kBlk, 0, s>>>(bits, label, L, n, out);
    SCC_LAUNCH();
    return SCC_OK;
}

int launch_class_trim(const int32_t* act, int64_t N, const int32_t* off, const int32_t* adj, const int32_t* toff,
                      const int32_t* tadj, int32_t* label, int32_t* rep, unsigned long long* ndone, cudaStream_t s) {
    if (N <= 0) return SCC_OK;
    k_class_trim<<<grid_for(N, kBlk), kBlk, 0, s>>>(act, N, off, adj, toff, tadj, label, rep, ndone);
    SCC_LAUNCH();
    return SCC_OK;
}

int launch_label_first(const uint32_t* bf, const uint32_t* bb, int32_t n, int32_t s, int32_t* label, int32_t* rep,
                       unsigned long long* ndone, cudaStream_t st) {
    if (n == 0) return SCC_OK;
    // the class of the pivot is 0 in the first round (every untrimmed vertex)
    k_label_first<<<grid_for(ceil_div((int64_t)n, 4), kBlk), kBlk, 0, st>>>(bf, bb, n, s, 0, label, rep, ndone);
    SCC_LAUNCH();
    return SCC_OK;
}

int launch_canonicalize(const int32_t* rep, int32_t n, int32_t* minid, int32_t* labels_out, int* bad,
                        cudaStream_t s) {
    if (n == 0) return SCC_OK;
    k_minid_init<<<grid_for(ceil_div((int64_t)n, 4), kBlk), kBlk, 0, s>>>(rep, n, minid);
    SCC_LAUNCH();
    k_min_of_rep<<<grid_for(n, kBlk), kBlk, 0, s>>>(rep, n, minid, bad);
    SCC_LAUNCH();
    k_write_labels<<<grid_for(ceil_div((int64_t)n, 4), kBlk), kBlk, 0, s>>>(rep, n, minid, labels_out);
    SCC_LAUNCH();
    return SCC_OK;
}

int launch_table_gather(const unsigned long long* tab, int64_t cap, unsigned long long* out, int64_t out_cap,
                        unsigned long long* count, cudaStream_t s) {
    k_table_gather<<<grid_for(cap, kBlk), kBlk, 0, s>>>(tab, cap, out, out_cap, count);
    SCC_LAUNCH();
    return SCC_OK;
}

namespace {
// Every key of the old table into the new one (the regrowth of Sec. 4.5).
__global__ void k_table_rehash(const unsigned long long* __restrict__ src, int64_t src_cap, PairTable dst) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < src_cap; i += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long k = src[i];
        if (k != ~0ull) dst.insert(k);
    }
}
}  // namespace

int launch_table_rehash(const unsigned long long* src, int64_t src_cap, unsigned long long* dst, int64_t dst_cap,
                        int* overflow, cudaStream_t s) {
    PairTable t{dst, (unsigned long long)(dst_cap - 1), overflow};
    k_table_rehash<<<grid_for(src_cap, kBlk), kBlk, 0, s>>>(src, src_cap, t);
    SCC_LAUNCH();
    return SCC_OK;
}

int launch_table_insert(const unsigned long long* keys, int64_t count, unsigned long long* tab, int64_t cap,
                        int* overflow, unsigned long long* inserted, cudaStream_t s) {
    if (count == 0) return SCC_OK;
    PairTable t{tab, (unsigned long long)(cap - 1), overflow};
    k_table_insert<<<grid_for(count, kBlk), kBlk, 0, s>>>(keys, count, t, inserted);
    SCC_LAUNCH();
    return SCC_OK;
}

}  // namespace scc
