// Transposed CSR G^T from the CSR of G (sm_103a).
//
// Every non-self arc (u, v) of G becomes the entry u of row v of G^T (Sec. 2: a
// backward reachability search is a forward search on G^T). This is a counting
// sort of the arcs by target in three levels, so that every per-arc atomic is a
// shared-memory atomic and every pass writes in runs:
//
//   A. coarse partition by bucket b = v >> shift (at most 512 buckets):
//      A1 histogram of sub-buckets (2^sb vertices, up to 32 per bucket;
//         per-block shared histogram, one global add per block and bin), fused
//         with the copy and range check of the targets: it needs no arc
//         sources, so it reads the targets once as a flat array. One scan
//         gives the start of every sub-bucket's rows in G^T; a bucket's run
//         starts where its first sub-bucket's rows start.
//      A2 partition: a block takes a tile of 8k arcs, counting-sorts it by
//         bucket in shared memory, reserves one run per non-empty bucket with a
//         global atomicAdd, and writes the sorted tile out, so consecutive lanes
//         store consecutive positions of a run.
//      Each arc is written as its source u (4 B) and its target's offset within
//      the bucket (2 B: buckets hold at most 2^15 vertices).
//   B. split: one block per bucket cuts its run into the runs of its
//      sub-buckets (tiles counting-sorted in shared memory by a warp
//      multi-split, written out through per-sub-bucket cursors the block owns).
//   C. rows: one block per sub-bucket (those with more arcs than the window
//      first): per-vertex counts in shared memory, their scan gives the rows
//      of G^T, then each arc's source is placed in a shared-memory copy of the
//      sub-bucket's rows, which is written out in order. A sub-bucket with more
//      arcs than the window places its arcs directly; its rows span only it.
//   Placing arcs straight into a bucket's rows instead (2 MB of rows per block,
//   about 300 MB in flight over the GPU, far more than L2) cost more than the
//   split pass: the scattered 4-byte stores left L2 before their sectors filled.
//
// Rows of each arc tile are found by one binary search per thread followed by a
// forward walk over the tile's row offsets staged in shared memory.
#include <algorithm>
#include <climits>
#include <numeric>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace scc {
namespace {

constexpr int kMaxBuckets = 512;
constexpr int kBucketLog = 15;          // at most 2^15 vertices per bucket (16-bit offsets within it)
constexpr int kSubLog = 5;              // at most 2^5 sub-buckets per bucket
constexpr int kMaxSubVertsLog = 10;     // at most 2^10 vertices per sub-bucket
constexpr int kMaxBins = kMaxBuckets << kSubLog;  // 16384 sub-buckets
constexpr int kMaxChunks = 8;                     // intake/partition chunks (host input)
constexpr int kBlkA = 512;
static_assert(kMaxBuckets <= kBlkA, "bucket scan uses one thread per bucket");
constexpr int kChunk = 16;              // consecutive arcs per thread per step
constexpr int kStep = kBlkA * kChunk;   // arcs per block step (8192) = partition tile
constexpr int kRowsCap = 4096;          // row offsets of one step staged in shared memory
constexpr int kBlkS = 256;                     // split pass (four blocks per SM)
constexpr int kSplitTile = kBlkS * 8;           // arcs per split tile
constexpr int kBlkR = 512;                      // rows pass
constexpr int kWinArcs = 16384;                 // rows staged in shared memory (64 KB)

// Largest r in [lo, hi] with off[r] <= e.
__device__ __forceinline__ int row_search_g(const int32_t* __restrict__ off, int lo, int hi, int64_t e) {
    while (lo < hi) {
        int mid = lo + ((hi - lo + 1) >> 1);
        if ((int64_t)__ldg(&off[mid]) <= e) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// One step of a block: arcs [s0, s1), thread t owns [s0 + 16 t, s0 + 16 t + 16).
// Calls f(q, u, v) for its q-th arc (q < 16, a compile-time index after unrolling). Row offsets of the step are staged in
// shared memory when they fit; each thread binary-searches its first arc's row
// and walks forward.
template <class F>
__device__ __forceinline__ void for_step_arcs(const int32_t* __restrict__ off, const int32_t* __restrict__ adj,
                                              int32_t n, int64_t s0, int64_t s1, const int32_t* __restrict__ trow,
                                              int32_t* s_off, F&& f) {
    // rows of the step: trow[t] holds the row of arc t * kStep, so rows
    // trow[t] .. trow[t + 1] contain every arc of [s0, s1)
    const int64_t t = s0 / kStep;
    const int r0 = __ldg(&trow[t]), r1 = __ldg(&trow[t + 1]);
    const int cnt = r1 - r0 + 2;  // offsets off[r0 .. r1 + 1]
    const bool sm = cnt <= kRowsCap;
    __syncthreads();  // the previous step's readers of s_off are done
    if (sm)
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) s_off[i] = off[r0 + i];
    __syncthreads();
    const int64_t e0 = s0 + (int64_t)threadIdx.x * kChunk;
    if (e0 < s1) {
        const int64_t e1 = min(e0 + (int64_t)kChunk, s1);
        int r;
        if (sm) {
            const int ei = (int)e0;  // offsets fit 32 bits (m <= INT32_MAX)
            int lo = 0, hi = cnt - 2;
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (s_off[mid] <= ei) lo = mid;
                else hi = mid - 1;
            }
            r = lo;  // relative row
        } else {
            r = row_search_g(off, r0, r1, e0) - r0;
        }
        int32_t a[kChunk];
        if (e1 - e0 == kChunk && ((e0 & 3) == 0)) {
            const int4* p = reinterpret_cast<const int4*>(adj + e0);
#pragma unroll
            for (int q = 0; q < kChunk / 4; ++q) {
                int4 x = __ldg(p + q);
                a[4 * q] = x.x;
                a[4 * q + 1] = x.y;
                a[4 * q + 2] = x.z;
                a[4 * q + 3] = x.w;
            }
        } else {
#pragma unroll
            for (int q = 0; q < kChunk; ++q) a[q] = (e0 + q < e1) ? __ldg(&adj[e0 + q]) : 0;
        }
        if (sm) {
            // offsets fit 32 bits (m <= INT32_MAX); the next row's start stays in
            // a register, so an arc costs one compare unless its row changes
            const int ei0 = (int)e0, ne = (int)(e1 - e0);
            int nxt = s_off[r + 1];
#pragma unroll
            for (int q = 0; q < kChunk; ++q) {
                if (q < ne) {
                    while (r + 1 < cnt - 1 && nxt <= ei0 + q) nxt = s_off[++r + 1];
                    f(q, r0 + r, a[q]);
                }
            }
        } else {
#pragma unroll
            for (int q = 0; q < kChunk; ++q) {
                const int64_t e = e0 + q;
                if (e < e1) {
                    // advance to the row containing e
                    // (bounded by the rows r0..r1, which always contain e)
                    while (r0 + r + 1 <= r1 && (int64_t)__ldg(&off[r0 + r + 1]) <= e) ++r;
                    f(q, r0 + r, a[q]);
                }
            }
        }
    }
    __syncthreads();
}

// A1 fused with graph intake: dst[e] = src[e] (unless dst == src), every target
// checked against [0, n) (*bad set otherwise, the arc skipped), and the bucket
// histogram of all arcs (self-loops included: the partition pass finds them).
// 16-byte loads and stores when both arrays are 16-byte aligned.
__global__ void __launch_bounds__(kBlkA) k_copy_check_hist(const int32_t* __restrict__ src, int32_t* __restrict__ dst,
                                                           int64_t m, int32_t n, int shift, int nb,
                                                           unsigned long long* bucket_cnt, int* bad) {
    extern __shared__ unsigned int s_hist[];  // nb bins
    for (int i = threadIdx.x; i < nb; i += blockDim.x) s_hist[i] = 0;
    __syncthreads();
    const bool copy = src != dst;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
    bool badl = false;
    auto one = [&](int32_t t) {
        if (t < 0 || t >= n) badl = true;
        else atomicAdd(&s_hist[t >> shift], 1u);
    };
    int64_t done = 0;
    if ((((uintptr_t)src | (uintptr_t)dst) & 15) == 0) {
        const int64_t m4 = m / 4;
        const int4* s4 = reinterpret_cast<const int4*>(src);
        int4* d4 = reinterpret_cast<int4*>(dst);
        for (int64_t i = tid; i < m4; i += stride) {
            const int4 x = __ldg(s4 + i);
            if (copy) d4[i] = x;
            one(x.x);
            one(x.y);
            one(x.z);
            one(x.w);
        }
        done = m4 * 4;
    }
    for (int64_t e = done + tid; e < m; e += stride) {
        const int32_t t = __ldg(src + e);
        if (copy) dst[e] = t;
        one(t);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nb; i += blockDim.x)
        if (s_hist[i]) atomicAdd(&bucket_cnt[i], (unsigned long long)s_hist[i]);
    if (badl) atomicExch(bad, 1);
}

// Row of the first arc of every step (trow[t], t < T) and of the last arc
// (trow[T]): one binary search per step instead of one per block step.
__global__ void k_tile_rows(const int32_t* __restrict__ off, int32_t n, int64_t m, int64_t T, int32_t* trow) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t <= T; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = t < T ? t * kStep : m - 1;
        trow[t] = row_search_g(off, 0, n - 1, e);
    }
}

// A1. bucket histogram of non-self arcs; self-loops counted per row.
__global__ void __launch_bounds__(kBlkA) k_bucket_hist(const int32_t* __restrict__ off, const int32_t* __restrict__ adj,
                                                       const int32_t* __restrict__ trow, int32_t n, int64_t m,
                                                       int shift, int nb,
                                                       unsigned long long* bucket_cnt, int32_t* selfrow,
                                                       unsigned long long* nself) {
    __shared__ int32_t s_off[kRowsCap];
    __shared__ unsigned int s_hist[kMaxBuckets];
    for (int i = threadIdx.x; i < nb; i += blockDim.x) s_hist[i] = 0;
    __syncthreads();
    unsigned long long my_self = 0;
    for (int64_t s0 = (int64_t)blockIdx.x * kStep; s0 < m; s0 += (int64_t)gridDim.x * kStep) {
        const int64_t s1 = min(s0 + (int64_t)kStep, m);
        for_step_arcs(off, adj, n, s0, s1, trow, s_off, [&](int, int u, int v) {
            if (u == v) {
                atomicAdd(&selfrow[u], 1);
                ++my_self;
            } else {
                atomicAdd(&s_hist[v >> shift], 1u);
            }
        });
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nb; i += blockDim.x)
        if (s_hist[i]) atomicAdd(&bucket_cnt[i], (unsigned long long)s_hist[i]);
    if (my_self) atomicAdd(nself, my_self);
}

// Block-wide exclusive scan (blockDim.x a multiple of 32, <= 1024); *total
// gets the sum. Every thread must call it.
__device__ __forceinline__ unsigned long long block_scan_u64(unsigned long long x, unsigned long long* s_w,
                                                             unsigned long long* total) {
    unsigned long long incl = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long y = __shfl_up_sync(kFull, incl, d);
        if (lane_id() >= d) incl += y;
    }
    if (lane_id() == 31) s_w[threadIdx.x >> 5] = incl;
    __syncthreads();
    if (threadIdx.x < 32) {
        const int nw = (int)(blockDim.x >> 5);
        unsigned long long w = threadIdx.x < nw ? s_w[threadIdx.x] : 0ull;
        unsigned long long wi = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned long long y = __shfl_up_sync(kFull, wi, d);
            if (lane_id() >= d) wi += y;
        }
        if (threadIdx.x < nw) s_w[threadIdx.x] = wi - w;
        if (threadIdx.x == 31) *total = wi;
    }
    __syncthreads();
    const unsigned long long r = s_w[threadIdx.x >> 5] + incl - x;
    __syncthreads();
    return r;
}

// One block of 512 threads: chunk c's partition cursors. Bucket b's arcs of
// the chunk form segment (c, b) = [seg_start, seg_start + seg_len), laid out in
// bucket order from the chunk's first arc base (the chunk's arcs keep their
// range); cursor = seg_start (advanced by the partition's reservations).
__global__ void __launch_bounds__(512) k_chunk_cursor(const unsigned long long* __restrict__ hist, int nb, int sublog,
                                                     long long base, unsigned long long* seg_start,
                                                     unsigned long long* seg_len, unsigned long long* cursor) {
    __shared__ unsigned long long s_w[32];
    __shared__ unsigned long long s_tot;
    const int b = threadIdx.x;
    unsigned long long len = 0;
    if (b < nb)
        for (int q = 0; q < (1 << sublog); ++q) len += hist[((size_t)b << sublog) + q];
    const unsigned long long pre = block_scan_u64(len, s_w, &s_tot);
    if (b < nb) {
        seg_start[b] = (unsigned long long)base + pre;
        seg_len[b] = len;
        cursor[b] = (unsigned long long)base + pre;
    }
}

// One block of 1024 threads over the sub-bucket counts (the sum of K chunk
// histograms of nf bins): start[0 .. nf] (exclusive scan) and gcur = start
// (the split pass's cursors), order = the sub-buckets with more than kWinArcs
// arcs, then the others (each group increasing), the split pass's tiles (each
// segment, from its first multiple of 8, in tiles of kSplitTile arcs:
// tile_base[g] = the first tile of segment g = c * nb + b, tile_seg[t] = the
// segment of tile t), counters[0] = 0 (work counter of the rows pass).
__global__ void __launch_bounds__(1024) k_fine_scan(const unsigned long long* __restrict__ hist, int K, int nf,
                                                   int nb, unsigned long long* start, unsigned long long* gcur,
                                                   int32_t* order, const unsigned long long* __restrict__ seg_start,
                                                   const unsigned long long* __restrict__ seg_len,
                                                   unsigned long long* tile_base, int32_t* tile_seg,
                                                   long long tile_cap, unsigned int* counters, int* err) {
    __shared__ unsigned long long s_w[32];
    __shared__ unsigned long long s_tot, s_hot;
    __shared__ unsigned long long s_wsum[32], s_whot[32];
    auto count = [&](int i) {
        unsigned long long c = 0;
        for (int k = 0; k < K; ++k) c += hist[(size_t)k * nf + i];
        return c;
    };
    // each warp scans a contiguous range of the bins, 32 consecutive bins per
    // step (coalesced loads and stores); the warps' totals are scanned first
    const int lane = lane_id(), warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int per_w = ((nf + nwarps - 1) / nwarps + 31) & ~31;
    const int w0 = min(warp * per_w, nf), w1 = min(w0 + per_w, nf);
    unsigned long long sum = 0, hot = 0;
    for (int i = w0 + lane; i < w1; i += 32) {
        const unsigned long long c = count(i);
        sum += c;
        hot += c > (unsigned long long)kWinArcs;
    }
    for (int d = 16; d >= 1; d >>= 1) {
        sum += __shfl_xor_sync(kFull, sum, d);
        hot += __shfl_xor_sync(kFull, hot, d);
    }
    if (lane == 0) {
        s_wsum[warp] = sum;
        s_whot[warp] = hot;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long a = 0, b = 0;
        for (int w = 0; w < nwarps; ++w) {
            const unsigned long long x = s_wsum[w], y = s_whot[w];
            s_wsum[w] = a;
            s_whot[w] = b;
            a += x;
            b += y;
        }
        s_tot = a;
        s_hot = b;
        start[nf] = a;
        counters[0] = 0;
    }
    __syncthreads();
    const unsigned long long nhot = s_hot;
    unsigned long long run = s_wsum[warp], hrun = s_whot[warp];
    for (int b0 = w0; b0 < w1; b0 += 32) {
        const int i = b0 + lane;
        const unsigned long long c = i < w1 ? count(i) : 0ull;
        const unsigned long long h = c > (unsigned long long)kWinArcs ? 1ull : 0ull;
        unsigned long long ci = c, hi = h;  // inclusive scans over the 32 lanes
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned long long yc = __shfl_up_sync(kFull, ci, d), yh = __shfl_up_sync(kFull, hi, d);
            if (lane >= d) {
                ci += yc;
                hi += yh;
            }
        }
        if (i < w1) {
            const unsigned long long st = run + ci - c;
            start[i] = st;
            gcur[i] = st;
            const unsigned long long hb = hrun + hi - h;  // hot bins before i
            order[h ? hb : nhot + (unsigned long long)i - hb] = i;
        }
        run += __shfl_sync(kFull, ci, 31);
        hrun += __shfl_sync(kFull, hi, 31);
    }
    // split tiles per segment (up to 8 x 512 segments: a run of them per thread)
    const int ns = K * nb;
    const int sper = (ns + (int)blockDim.x - 1) / (int)blockDim.x;
    const int s0 = min((int)threadIdx.x * sper, ns), s1 = min(s0 + sper, ns);
    auto tiles_of = [&](int g) {
        const long long r0 = (long long)seg_start[g], r1 = r0 + (long long)seg_len[g];
        return r1 > r0 ? (unsigned long long)(((r1 - (r0 & ~7ll)) + kSplitTile - 1) / kSplitTile) : 0ull;
    };
    unsigned long long nt = 0;
    for (int g = s0; g < s1; ++g) nt += tiles_of(g);
    unsigned long long tb = block_scan_u64(nt, s_w, &s_tot);
    unsigned long long ntot = s_tot;
    if (ntot > (unsigned long long)tile_cap) {  // the tile table is too small: report, split nothing past it
        if (threadIdx.x == 0) atomicExch(err, SCC_ERR_INTERNAL);
        ntot = (unsigned long long)tile_cap;
    }
    for (int g = s0; g < s1; ++g) {
        tile_base[g] = tb;
        tb += tiles_of(g);
    }
    if (threadIdx.x == 0) tile_base[ns] = ntot;
}

// The segment of every split tile: a warp per segment fills its run of
// tile_seg (tile_base written by k_fine_scan; runs past tile_cap are cut).
__global__ void k_tile_seg(const unsigned long long* __restrict__ tile_base, int ns, long long tile_cap,
                           int32_t* tile_seg) {
    const int lane = lane_id();
    const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long g = w0; g < ns; g += nw) {
        const long long t0 = (long long)tile_base[g], t1 = min((long long)tile_base[g + 1], tile_cap);
        for (long long t = t0 + lane; t < t1; t += 32) tile_seg[t] = (int32_t)g;
    }
}

// A2. partition: per 8k-arc tile, a shared-memory counting sort by bucket,
// one global reservation per non-empty bucket, then a coalesced write-out.
__global__ void __launch_bounds__(kBlkA, 2) k_bucket_part(const int32_t* __restrict__ off, const int32_t* __restrict__ adj,
                                                       const int32_t* __restrict__ trow, int32_t n, int64_t a_lo,
                                                       int64_t a_hi, int shift, int nb,
                                                       unsigned long long* cursor, int32_t* out_u, uint16_t* out_lv,
                                                       unsigned long long mt, int32_t* selfrow,
                                                       unsigned long long* nself, const int* bad, int* err) {
    if (bad != nullptr && ld_volatile(bad) != 0) return;  // a target out of range: nothing is partitioned
    __shared__ int32_t s_off[kRowsCap];
    __shared__ unsigned int s_cnt[kMaxBuckets];
    __shared__ unsigned int s_start[kMaxBuckets];
    __shared__ int s_disp[kMaxBuckets];  // staged position -> output position, per bucket
    extern __shared__ uint2 s_stage[];    // the sorted tile: (u, v)[kStep]
    __shared__ unsigned int s_wsum[kBlkA / 32];
    __shared__ unsigned int s_total;
    for (int64_t t0 = a_lo + (int64_t)blockIdx.x * kStep; t0 < a_hi; t0 += (int64_t)gridDim.x * kStep) {
        const int64_t t1 = min(t0 + (int64_t)kStep, a_hi);
        for (int i = threadIdx.x; i < nb; i += blockDim.x) s_cnt[i] = 0;
        __syncthreads();
        // ranks within (tile, bucket), kept per thread two to a word (< kStep)
        unsigned int rk[kChunk / 2];
        int uu[kChunk], vv[kChunk];
#pragma unroll
        for (int q = 0; q < kChunk; ++q) vv[q] = -1;
#pragma unroll
        for (int q = 0; q < kChunk / 2; ++q) rk[q] = 0;
        // every arc is placed (the histogram counted self-loops too); a self-loop
        // is also counted per row, and any self-loop makes the caller rebuild
        // the CSR without them and start over
        for_step_arcs(off, adj, n, t0, t1, trow, s_off, [&](int q, int u, int v) {
            uu[q] = u;
            vv[q] = v;
            rk[q >> 1] |= atomicAdd(&s_cnt[v >> shift], 1u) << (16 * (q & 1));
            if (u == v && selfrow != nullptr) {  // without selfrow, self-loops are kept
                atomicAdd(&selfrow[u], 1);
                atomicAdd(nself, 1ull);
            }
        });
        // exclusive scan of the bucket counts (nb <= 512 = blockDim)
        {
            const int i = threadIdx.x;
            const unsigned int c = i < nb ? s_cnt[i] : 0u;
            const int incl = warp_incl_scan((int)c);
            if (lane_id() == 31) s_wsum[i >> 5] = incl;
            __syncthreads();
            if (i < 32) {
                unsigned int x = i < (int)(blockDim.x >> 5) ? s_wsum[i] : 0u;
                unsigned int y = (unsigned int)warp_incl_scan((int)x);
                if (i < (int)(blockDim.x >> 5)) s_wsum[i] = y - x;
                if (i == 31) s_total = y;
            }
            __syncthreads();
            if (i < nb) s_start[i] = s_wsum[i >> 5] + incl - c;
            __syncthreads();
            // reserve the tile's run in each bucket; the atomics' latency
            // overlaps the staging below
            const unsigned long long g = (i < nb && c) ? atomicAdd(&cursor[i], (unsigned long long)c) : 0ull;
            // stage the tile sorted by bucket
#pragma unroll
            for (int q = 0; q < kChunk; ++q)
                if (vv[q] >= 0)
                    s_stage[s_start[vv[q] >> shift] + ((rk[q >> 1] >> (16 * (q & 1))) & 0xffffu)] =
                        make_uint2((uint32_t)uu[q], (uint32_t)vv[q]);
            // positions fit 32 bits (m <= INT32_MAX): one displacement per bucket
            if (i < nb) s_disp[i] = (int)((long long)g - (long long)s_start[i]);
            __syncthreads();
        }
        const int total = (int)s_total;
        const unsigned int lmask = (1u << shift) - 1u;
        for (int j = threadIdx.x; j < total; j += kBlkA) {
            const uint2 x = s_stage[j];
            const int pos = s_disp[x.y >> shift] + j;
            if ((unsigned int)pos < (unsigned int)mt) {  // mt <= INT32_MAX
                out_u[pos] = (int32_t)x.x;
                out_lv[pos] = (uint16_t)(x.y & lmask);  // the target within its bucket
            } else {
                atomicExch(err, SCC_ERR_INTERNAL);
            }
        }
        __syncthreads();
    }
}

__device__ __forceinline__ void unpack8(const uint4 r, unsigned int (&lv)[8]) {
    lv[0] = r.x & 0xffffu;
    lv[1] = r.x >> 16;
    lv[2] = r.y & 0xffffu;
    lv[3] = r.y >> 16;
    lv[4] = r.z & 0xffffu;
    lv[5] = r.z >> 16;
    lv[6] = r.w & 0xffffu;
    lv[7] = r.w >> 16;
}

// B. split over tiles: tile t of bucket b = tile_bucket[t] covers kSplitTile
// arcs of the bucket's run from its first multiple of 8 (8 per thread; the
// arrays are padded by 8 entries), blocks take tiles in a grid-stride loop and
// load the next tile while they work on this one. A tile's arcs are counted
// per sub-bucket in shared memory (the count is the arc's rank); one global
// atomicAdd per non-empty sub-bucket reserves the tile's run in it; the tile is
// staged in sub-bucket order and written out, consecutive lanes to consecutive
// positions. The target is kept as its offset within the sub-bucket.
struct SplitLoad {
    uint4 lv;
    int4 ua, ub;
    long long c, r0, r1;
    int b;  // the bucket
};
__device__ __forceinline__ SplitLoad split_load(const int32_t* __restrict__ uu, const uint16_t* __restrict__ lvv,
                                                const unsigned long long* __restrict__ seg_start,
                                                const unsigned long long* __restrict__ seg_len,
                                                const unsigned long long* __restrict__ tile_base,
                                                const int32_t* __restrict__ tile_seg, int nb, long long t) {
    SplitLoad L;
    const int g = __ldg(&tile_seg[t]);
    L.b = g % nb;
    L.r0 = (long long)__ldg(&seg_start[g]);
    L.r1 = L.r0 + (long long)__ldg(&seg_len[g]);
    L.c = (L.r0 & ~7ll) + ((long long)t - (long long)__ldg(&tile_base[g])) * kSplitTile + 8ll * threadIdx.x;
    const bool in = L.c < L.r1;
    L.lv = in ? __ldg(reinterpret_cast<const uint4*>(lvv + L.c)) : make_uint4(0, 0, 0, 0);
    L.ua = in ? __ldg(reinterpret_cast<const int4*>(uu + L.c)) : make_int4(0, 0, 0, 0);
    L.ub = in ? __ldg(reinterpret_cast<const int4*>(uu + L.c + 4)) : make_int4(0, 0, 0, 0);
    return L;
}

__global__ void __launch_bounds__(kBlkS, 4) k_bucket_split(const int32_t* __restrict__ uu,
                                                           const uint16_t* __restrict__ lvv,
                                                           const unsigned long long* __restrict__ start,
                                                           const unsigned long long* __restrict__ seg_start,
                                                           const unsigned long long* __restrict__ seg_len,
                                                           const unsigned long long* __restrict__ tile_base,
                                                           const int32_t* __restrict__ tile_seg, int nseg, int nb,
                                                           int sublog, int sb, unsigned long long* gcur, int32_t* u2,
                                                           uint16_t* lv2, int* err) {
    __shared__ unsigned int s_tcnt[1 << kSubLog];
    __shared__ unsigned int s_tstart[1 << kSubLog];
    __shared__ int s_disp[1 << kSubLog];           // staged position -> output position, per sub-bucket
    __shared__ unsigned int s_end[1 << kSubLog];   // end of each sub-bucket's range
    extern __shared__ uint2 s_st[];                // [kSplitTile] (u, local target)
    const int S = 1 << sublog;
    const unsigned int lmask = (1u << sb) - 1u;
    const long long ntiles = (long long)tile_base[nseg];
    long long t = blockIdx.x;
    if (t >= ntiles) return;
    SplitLoad cur = split_load(uu, lvv, seg_start, seg_len, tile_base, tile_seg, nb, t);
    for (; t < ntiles; t += gridDim.x) {
        const long long tn = t + gridDim.x;
        SplitLoad nxt;
        if (tn < ntiles) nxt = split_load(uu, lvv, seg_start, seg_len, tile_base, tile_seg, nb, tn);
        const size_t f0 = (size_t)cur.b << sublog;
        if (threadIdx.x < (unsigned)S) {
            s_tcnt[threadIdx.x] = 0;
            s_end[threadIdx.x] = (unsigned int)__ldg(&start[f0 + threadIdx.x + 1]);
        }
        __syncthreads();
        unsigned int lv[8];
        unpack8(cur.lv, lv);
        unsigned int rk[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const bool valid = cur.c + j >= cur.r0 && cur.c + j < cur.r1;
            const unsigned int sub = lv[j] >> sb;
            rk[j] = ~0u;
            if (valid) {
                if (sub < (unsigned)S) rk[j] = atomicAdd(&s_tcnt[sub], 1u);
                else atomicExch(err, SCC_ERR_INTERNAL);
            }
        }
        __syncthreads();
        unsigned int x = 0;
        if (threadIdx.x < 32) {  // scan of the tile's sub-bucket counts
            x = threadIdx.x < (unsigned)S ? s_tcnt[threadIdx.x] : 0u;
            const unsigned int y = (unsigned int)warp_incl_scan((int)x);
            s_tstart[threadIdx.x] = y - x;
        }
        __syncthreads();
        // reserve the tile's run in each sub-bucket; the atomics' latency
        // overlaps the staging below
        const unsigned long long g = x ? atomicAdd(&gcur[f0 + threadIdx.x], (unsigned long long)x) : 0ull;
        const int u8[8] = {cur.ua.x, cur.ua.y, cur.ua.z, cur.ua.w, cur.ub.x, cur.ub.y, cur.ub.z, cur.ub.w};
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (rk[j] != ~0u) s_st[s_tstart[lv[j] >> sb] + rk[j]] = make_uint2((uint32_t)u8[j], lv[j]);
        // positions fit 32 bits (m <= INT32_MAX): one displacement per sub-bucket
        if (x) s_disp[threadIdx.x] = (int)((long long)g - (long long)s_tstart[threadIdx.x]);
        __syncthreads();
        const int total = (int)(s_tstart[S - 1] + s_tcnt[S - 1]);
        for (int q = threadIdx.x; q < total; q += kBlkS) {
            const uint2 y = s_st[q];
            const unsigned int sub = y.y >> sb;
            const unsigned int pos = (unsigned int)(s_disp[sub] + q);
            if (pos < s_end[sub]) {
                u2[pos] = (int32_t)y.x;
                lv2[pos] = (uint16_t)(y.y & lmask);
            } else {
                atomicExch(err, SCC_ERR_INTERNAL);
            }
        }
        __syncthreads();  // the staging and the counts are reused by the next tile
        if (tn < ntiles) cur = nxt;
    }
}

// C. rows: block takes the next sub-bucket of `order` (a work counter). Counter
// i of the sub-bucket lives at i + i / 32 in shared memory: the scan gives each
// thread a run of consecutive counters, and with one padding word per 32 the
// lanes of a warp reading the j-th counter of their runs hit 32 different banks.
__device__ __forceinline__ int cpad(int i) { return i + (i >> 5); }
constexpr int kCntWords = (1 << kMaxSubVertsLog) + (1 << kMaxSubVertsLog) / 32 + 4;  // 16-byte multiple
size_t rows_smem_bytes() { return sizeof(int) * ((size_t)kCntWords + kWinArcs); }

__global__ void __launch_bounds__(kBlkR, 3) k_sub_rows(const int32_t* __restrict__ u2, const uint16_t* __restrict__ lv2,
                                                      const unsigned long long* __restrict__ start,
                                                      const int32_t* __restrict__ order, int nf, int sb, int32_t n,
                                                      int32_t* toff, int32_t* tadj, unsigned int* next, int* err) {
    extern __shared__ int s_dyn[];
    int* s_cnt = s_dyn;                // 2^sb counters, padded (cpad)
    int32_t* s_win = s_dyn + kCntWords;  // the sub-bucket's rows while they fit
    __shared__ int s_wsum[kBlkR / 32];
    __shared__ int s_oi;
    const int W = 1 << sb;
    for (;;) {
        if (threadIdx.x == 0) s_oi = (int)atomicAdd(next, 1u);
        __syncthreads();
        const int oi = s_oi;
        if (oi >= nf) break;
        const int f = order[oi];
        const long long v0 = (long long)f << sb;
        const int vw = (int)min((long long)W, (long long)n - v0);
        if (vw <= 0) {  // bins past the last vertex hold nothing; uniform
            __syncthreads();  // every thread has read s_oi before it is rewritten
            continue;
        }
        const long long a0 = (long long)start[f], a1 = (long long)start[f + 1];
        const bool win = a1 - a0 <= kWinArcs;
        for (int i = threadIdx.x; i < cpad(vw); i += blockDim.x) s_cnt[i] = 0;
        __syncthreads();
        const long long c0 = (a0 & ~7ll) + 8ll * threadIdx.x;
        const long long cstep = 8ll * blockDim.x;
        for (long long c = c0; c < a1; c += cstep) {
            unsigned int lv[8];
            unpack8(__ldg(reinterpret_cast<const uint4*>(lv2 + c)), lv);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (c + j < a0 || c + j >= a1) continue;
                if (lv[j] < (unsigned int)vw) atomicAdd(&s_cnt[cpad((int)lv[j])], 1);
                else atomicExch(err, SCC_ERR_INTERNAL);  // arc outside its sub-bucket: skip it, report
            }
        }
        __syncthreads();
        // exclusive scan of s_cnt[0..vw) in place; each thread owns a contiguous run
        const int per = (vw + blockDim.x - 1) / blockDim.x;
        const int q0 = min((int)threadIdx.x * per, vw), q1 = min(q0 + per, vw);
        int sum = 0;
        for (int i = q0; i < q1; ++i) sum += s_cnt[cpad(i)];
        int incl = warp_incl_scan(sum);
        if (lane_id() == 31) s_wsum[threadIdx.x >> 5] = incl;
        __syncthreads();
        if (threadIdx.x < 32) {
            int x = threadIdx.x < (int)(blockDim.x >> 5) ? s_wsum[threadIdx.x] : 0;
            int y = warp_incl_scan(x);
            if (threadIdx.x < (int)(blockDim.x >> 5)) s_wsum[threadIdx.x] = y - x;
        }
        __syncthreads();
        int run = s_wsum[threadIdx.x >> 5] + incl - sum;
        for (int i = q0; i < q1; ++i) {
            const int cn = s_cnt[cpad(i)];
            s_cnt[cpad(i)] = run;
            run += cn;
        }
        __syncthreads();
        // the sub-bucket's row offsets, written coalesced (before the placement
        // below advances the counters)
        for (int i = threadIdx.x; i < vw; i += blockDim.x) toff[v0 + i] = (int32_t)(a0 + s_cnt[cpad(i)]);
        __syncthreads();
        for (long long c = c0; c < a1; c += cstep) {
            unsigned int lv[8];
            unpack8(__ldg(reinterpret_cast<const uint4*>(lv2 + c)), lv);
            const int4 ua = __ldg(reinterpret_cast<const int4*>(u2 + c));
            const int4 ub = __ldg(reinterpret_cast<const int4*>(u2 + c + 4));
            const int u8[8] = {ua.x, ua.y, ua.z, ua.w, ub.x, ub.y, ub.z, ub.w};
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (c + j < a0 || c + j >= a1 || lv[j] >= (unsigned int)vw) continue;
                const int p = atomicAdd(&s_cnt[cpad((int)lv[j])], 1);
                if (p < a1 - a0) {
                    if (win) s_win[p] = u8[j];
                    else tadj[a0 + p] = u8[j];
                } else {
                    atomicExch(err, SCC_ERR_INTERNAL);
                }
            }
        }
        __syncthreads();
        if (win)
            for (int i = threadIdx.x; i < (int)(a1 - a0); i += blockDim.x) tadj[a0 + i] = s_win[i];
        __syncthreads();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) toff[n] = (int32_t)start[nf];
}

// Direct path for graphs too large for shared per-bucket counters: global
// in-degree atomics, scan, global cursor atomics.
__global__ void __launch_bounds__(kBlkA) k_direct_count(const int32_t* __restrict__ off,
                                                        const int32_t* __restrict__ adj,
                                                        const int32_t* __restrict__ trow, int32_t n, int64_t m,
                                                        int32_t* indeg) {
    __shared__ int32_t s_off[kRowsCap];
    for (int64_t s0 = (int64_t)blockIdx.x * kStep; s0 < m; s0 += (int64_t)gridDim.x * kStep)
        for_step_arcs(off, adj, n, s0, min(s0 + (int64_t)kStep, m), trow, s_off, [&](int, int u, int v) {
            if (u != v) atomicAdd(&indeg[v], 1);
        });
}
__global__ void __launch_bounds__(kBlkA) k_direct_place(const int32_t* __restrict__ off,
                                                        const int32_t* __restrict__ adj,
                                                        const int32_t* __restrict__ trow, int32_t n, int64_t m,
                                                        int32_t* cursor, int32_t* tadj) {
    __shared__ int32_t s_off[kRowsCap];
    for (int64_t s0 = (int64_t)blockIdx.x * kStep; s0 < m; s0 += (int64_t)gridDim.x * kStep)
        for_step_arcs(off, adj, n, s0, min(s0 + (int64_t)kStep, m), trow, s_off, [&](int, int u, int v) {
            if (u != v) tadj[atomicAdd(&cursor[v], 1)] = u;
        });
}

int grid_for_arcs(int64_t m, int per_block, int num_sms, int per_sm) {
    int64_t t = (m + per_block - 1) / per_block;
    return (int)std::max<int64_t>(1, std::min(t, (int64_t)num_sms * per_sm));
}

}  // namespace

// sub-buckets: 2^sb vertices, 2^sublog of them per bucket
inline int sub_vert_log(int shift) { return std::min(shift, std::max(shift - kSubLog, 5)); }
inline int sub_log(int shift) { return shift - sub_vert_log(shift); }

int transpose_set_attributes_impl();
// The kernels' shared-memory limits, set once per process (the first call is
// outside any stream capture: graph creation, or the batched setup).
int ensure_attributes() {
    static const int rc = transpose_set_attributes_impl();
    return rc;
}

int bucket_shift(int32_t n) {
    int shift = 6;
    while (((int64_t)n + (1ll << shift) - 1) >> shift > kMaxBuckets) ++shift;
    return shift;
}

size_t tile_rows_count(int64_t m) { return (size_t)((m + kStep - 1) / kStep) + 1; }

// Tiles of the split pass: one run per segment (chunk, bucket), each from its
// first multiple of 8, so at most m / T + 7 ns / T + ns tiles for ns segments.
size_t transpose_split_tiles(int64_t m, int32_t n, int shift, int K) {
    const int nb = std::max(1, (int)(((int64_t)n + (1ll << shift) - 1) >> shift));
    const size_t ns = (size_t)K * nb;
    return (size_t)(m / kSplitTile) + ns + (7 * ns) / kSplitTile + 2;
}

int transpose_bins(int32_t n, int shift) {
    const int nb = std::max(1, (int)(((int64_t)n + (1ll << shift) - 1) >> shift));
    return nb << sub_log(shift);
}

int launch_copy_check_hist(const int32_t* src, int32_t* dst, int32_t n, int64_t m, int shift,
                           unsigned long long* bucket_cnt, int* bad, int num_sms, cudaStream_t s) {
    if (m == 0) return SCC_OK;
    const int nf = transpose_bins(n, shift);  // sub-bucket bins (<= 16384)
    const size_t smem = sizeof(unsigned int) * (size_t)nf;
    SCC_TRY(ensure_attributes());
    k_copy_check_hist<<<grid_for_arcs(m, 4 * kBlkA * 4, num_sms, 2), kBlkA, smem, s>>>(src, dst, m, n,
                                                                                      sub_vert_log(shift), nf,
                                                                                      bucket_cnt, bad);
    SCC_LAUNCH();
    return SCC_OK;
}

int launch_tile_rows(const int32_t* off, int32_t n, int64_t m, int32_t* trow, cudaStream_t s) {
    if (m == 0 || n == 0) return SCC_OK;
    const int64_t T = (m + kStep - 1) / kStep;
    k_tile_rows<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((T + 256) / 256, 4096)), 256, 0, s>>>(off, n, m, T,
                                                                                                     trow);
    SCC_LAUNCH();
    return SCC_OK;
}

int launch_bucket_hist(const int32_t* off, const int32_t* adj, const int32_t* trow, int32_t n, int64_t m, int shift,
                       unsigned long long* bucket_cnt, int32_t* selfrow, unsigned long long* nself, int num_sms,
                       cudaStream_t s) {
    if (m == 0 || n == 0) return SCC_OK;
    int nb = (int)(((int64_t)n + (1ll << shift) - 1) >> shift);
    k_bucket_hist<<<grid_for_arcs(m, kStep, num_sms, 2), kBlkA, 0, s>>>(off, adj, trow, n, m, shift, nb, bucket_cnt,
                                                                          selfrow, nself);
    SCC_LAUNCH();
    return SCC_OK;
}

int launch_transpose_direct(const int32_t* off, const int32_t* adj, const int32_t* trow, int32_t n, int64_t m,
                            int32_t* indeg, void* scan_tmp, int32_t* toff, int32_t* tadj, int num_sms,
                            cudaStream_t s) {
    SCC_CUDA(cudaMemsetAsync(indeg, 0, sizeof(int32_t) * ((size_t)n + 1), s));
    if (m > 0) {
        k_direct_count<<<grid_for_arcs(m, kStep, num_sms, 2), kBlkA, 0, s>>>(off, adj, trow, n, m, indeg);
        SCC_LAUNCH();
    }
    SCC_TRY(launch_scan(indeg, toff, n, scan_tmp, s));
    if (m > 0) {
        SCC_CUDA(cudaMemcpyAsync(indeg, toff, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s));
        k_direct_place<<<grid_for_arcs(m, kStep, num_sms, 2), kBlkA, 0, s>>>(off, adj, trow, n, m, indeg, tadj);
        SCC_LAUNCH();
    }
    return SCC_OK;
}

bool transpose_bucketed(int shift) { return shift <= kBucketLog; }

int transpose_chunks(int64_t m, bool overlap) {
    if (!overlap) return 1;
    const int64_t T = (m + kStep - 1) / kStep;
    return (int)std::max<int64_t>(1, std::min<int64_t>(kMaxChunks, T / 64));
}
size_t transpose_hist_words(int32_t n, int shift, int K) { return (size_t)K * transpose_bins(n, shift) + 2; }
size_t transpose_tmp_words(int32_t n, int shift, int K) {
    const int nb = std::max(1, (int)(((int64_t)n + (1ll << shift) - 1) >> shift));
    return 2 * (size_t)transpose_bins(n, shift) + 4 * (size_t)K * nb + 4;
}

namespace {
// bucket_tmp: start [nf + 1] | gcur [nf] | tile_base [K nb + 1] | counter |
// seg_start [K nb] | seg_len [K nb] | cursor [K nb]
struct TmpLayout {
    unsigned long long *start, *gcur, *tile_base, *seg_start, *seg_len, *cursor;
    unsigned int* counters;
};
TmpLayout tmp_layout(unsigned long long* t, int nf, int nb, int K) {
    TmpLayout L;
    L.start = t;
    L.gcur = L.start + nf + 1;
    L.tile_base = L.gcur + nf;
    L.counters = reinterpret_cast<unsigned int*>(L.tile_base + (size_t)K * nb + 1);
    L.seg_start = L.tile_base + (size_t)K * nb + 2;
    L.seg_len = L.seg_start + (size_t)K * nb;
    L.cursor = L.seg_len + (size_t)K * nb;
    return L;
}
}  // namespace

int launch_intake_partition(const int32_t* src, int32_t* adj, const int32_t* off, const int32_t* trow, int32_t n,
                            int64_t m, int shift, int K, unsigned long long* hist, unsigned long long* bucket_tmp,
                            int32_t* tmp_u, uint16_t* tmp_lv, int32_t* selfrow, unsigned long long* nself, int* bad,
                            int* err, int num_sms, cudaStream_t s, cudaStream_t s2, cudaEvent_t* cev, cudaEvent_t* ev) {
    const int nb = std::max(1, (int)(((int64_t)n + (1ll << shift) - 1) >> shift));
    const int sublog = sub_log(shift);
    const int nf = nb << sublog;
    const TmpLayout T = tmp_layout(bucket_tmp, nf, nb, K);
    SCC_TRY(ensure_attributes());
    SCC_CUDA(cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * (size_t)K * nf, s));
    if (n == 0) return SCC_OK;
    const int64_t tiles = (m + kStep - 1) / kStep;
    const int64_t tpc = (tiles + K - 1) / K;  // tiles per chunk
    cudaStream_t sp = K > 1 ? s2 : s;          // the partitions' stream
    if (ev) cudaEventRecord(ev[0], s);
    for (int c = 0; c < K; ++c) {
        const int64_t e0 = std::min<int64_t>(m, (int64_t)c * tpc * kStep);
        const int64_t e1 = std::min<int64_t>(m, (int64_t)(c + 1) * tpc * kStep);
        unsigned long long* hc = hist + (size_t)c * nf;
        if (e1 > e0) {
            // chunk c's intake (a multiple of kStep arcs in: 16-byte aligned)
            k_copy_check_hist<<<grid_for_arcs(e1 - e0, 4 * kBlkA * 4, num_sms, 2), kBlkA, sizeof(unsigned int) * nf,
                                s>>>(src + e0, adj + e0, e1 - e0, n, sub_vert_log(shift), nf, hc, bad);
            SCC_LAUNCH();
        }
        if (ev && c == K - 1) cudaEventRecord(ev[1], s);  // the last intake
        if (K > 1) {
            SCC_CUDA(cudaEventRecord(cev[c], s));
            SCC_CUDA(cudaStreamWaitEvent(sp, cev[c], 0));
        }
        if (ev && c == 0) cudaEventRecord(ev[2], sp);
        k_chunk_cursor<<<1, 512, 0, sp>>>(hc, nb, sublog, (long long)e0, T.seg_start + (size_t)c * nb,
                                         T.seg_len + (size_t)c * nb, T.cursor + (size_t)c * nb);
        SCC_LAUNCH();
        if (e1 > e0) {
            const int stage = 2 * kStep * (int)sizeof(int32_t);
            k_bucket_part<<<grid_for_arcs(e1 - e0, kStep, num_sms, 2), kBlkA, stage, sp>>>(
                off, adj, trow, n, e0, e1, shift, nb, T.cursor + (size_t)c * nb, tmp_u, tmp_lv, (unsigned long long)m,
                selfrow, nself, bad, err);
            SCC_LAUNCH();
        }
    }
    if (ev) cudaEventRecord(ev[3], sp);
    if (K > 1) {  // the stream continues after the last partition
        SCC_CUDA(cudaEventRecord(cev[K], sp));
        SCC_CUDA(cudaStreamWaitEvent(s, cev[K], 0));
    }
    return SCC_OK;
}

int launch_transpose_rest(int32_t n, int64_t mt, int shift, int K, const unsigned long long* hist,
                          unsigned long long* bucket_tmp, const int32_t* tmp_u, const uint16_t* tmp_lv, int32_t* tmp2_u,
                          uint16_t* tmp2_lv, int32_t* order_tmp, int32_t* tile_tmp, int32_t* toff, int32_t* tadj,
                          const unsigned long long* nself, bool* self_found, int* err, int num_sms, cudaStream_t s,
                          cudaEvent_t* ev) {
    // nself == nullptr: self-loops are kept as arcs of G^T and nothing is read
    // back to the host (the launches can be captured in a CUDA graph)
    *self_found = false;
    const int nb = std::max(1, (int)(((int64_t)n + (1ll << shift) - 1) >> shift));
    const int sb = sub_vert_log(shift), sublog = sub_log(shift);
    const int nf = nb << sublog;
    const TmpLayout T = tmp_layout(bucket_tmp, nf, nb, K);
    if (n == 0) {
        SCC_CUDA(cudaMemsetAsync(toff, 0, sizeof(int32_t), s));
        return SCC_OK;
    }
    SCC_TRY(ensure_attributes());
    const long long tile_cap = (long long)transpose_split_tiles(mt, n, shift, K);
    k_fine_scan<<<1, 1024, 0, s>>>(hist, K, nf, nb, T.start, T.gcur, order_tmp, T.seg_start, T.seg_len, T.tile_base,
                                   tile_tmp, tile_cap, T.counters, err);
    SCC_LAUNCH();
    k_tile_seg<<<std::max(1, std::min(num_sms * 4, (K * nb + 7) / 8)), 256, 0, s>>>(T.tile_base, K * nb, tile_cap,
                                                                                    tile_tmp);
    SCC_LAUNCH();
    if (nself != nullptr) {
        unsigned long long hself = 0;
        SCC_CUDA(cudaMemcpyAsync(&hself, nself, sizeof(hself), cudaMemcpyDeviceToHost, s));
        SCC_CUDA(cudaStreamSynchronize(s));
        if (hself > 0) {  // the caller drops the self-loops and calls again
            *self_found = true;
            return SCC_OK;
        }
    }
    int per_sm = 0;
    const size_t split_smem = (size_t)kSplitTile * sizeof(uint2);
    SCC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bucket_split, kBlkS, split_smem));
    if (ev) cudaEventRecord(ev[0], s);
    if (mt > 0) {  // the tile count is read on the device; spare blocks return at once
        k_bucket_split<<<num_sms * std::max(1, per_sm), kBlkS, split_smem, s>>>(tmp_u, tmp_lv, T.start, T.seg_start,
                                                                               T.seg_len, T.tile_base, tile_tmp, K * nb,
                                                                               nb, sublog, sb, T.gcur, tmp2_u, tmp2_lv,
                                                                               err);
        SCC_LAUNCH();
    }
    if (ev) cudaEventRecord(ev[1], s);
    const size_t smem = rows_smem_bytes();
    SCC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sub_rows, kBlkR, smem));
    if (ev) cudaEventRecord(ev[2], s);
    k_sub_rows<<<std::min(nf, num_sms * std::max(1, per_sm)), kBlkR, smem, s>>>(tmp2_u, tmp2_lv, T.start, order_tmp, nf,
                                                                                 sb, n, toff, tadj, T.counters, err);
    SCC_LAUNCH();
    if (ev) cudaEventRecord(ev[3], s);
    return SCC_OK;
}

// ---------------------------------------------------- packed graph groups --
// Scratch of launch_transpose_keep_self for graphs of up to 2^24 vertices and
// m_max arcs, carved from one allocation.
size_t transpose_scratch_bytes(int64_t m_max) {
    const size_t nf = (size_t)kMaxBins, nb = (size_t)kMaxBuckets;
    auto a = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t m8 = (size_t)std::max<int64_t>(m_max, 1) + 8;
    return a(8 * (nf + 2)) + a(8 * (2 * nf + 4 * nb + 4)) + 2 * a(4 * m8) + 2 * a(2 * m8) + a(4 * nf) +
           a(4 * ((size_t)m_max / kSplitTile + nb + (7 * nb) / kSplitTile + 2)) +
           a(4 * tile_rows_count(std::max<int64_t>(m_max, 1))) +
           2 * a(sizeof(int));
}
void transpose_scratch_carve(unsigned char* base, int64_t m_max, TransposeScratch* ts) {
    const size_t nf = (size_t)kMaxBins, nb = (size_t)kMaxBuckets;
    size_t o = 0;
    auto take = [&](size_t x) {
        unsigned char* p = base + o;
        o += (x + 255) & ~(size_t)255;
        return p;
    };
    const size_t m8 = (size_t)std::max<int64_t>(m_max, 1) + 8;
    ts->bcnt = reinterpret_cast<unsigned long long*>(take(8 * (nf + 2)));
    ts->btmp = reinterpret_cast<unsigned long long*>(take(8 * (2 * nf + 4 * nb + 4)));
    ts->tmp_u = reinterpret_cast<int32_t*>(take(4 * m8));
    ts->tmp2_u = reinterpret_cast<int32_t*>(take(4 * m8));
    ts->tmp_lv = reinterpret_cast<uint16_t*>(take(2 * m8));
    ts->tmp2_lv = reinterpret_cast<uint16_t*>(take(2 * m8));
    ts->order = reinterpret_cast<int32_t*>(take(4 * nf));
    ts->tiles = reinterpret_cast<int32_t*>(take(4 * ((size_t)m_max / kSplitTile + nb + (7 * nb) / kSplitTile + 2)));
    ts->trow = reinterpret_cast<int32_t*>(take(4 * tile_rows_count(std::max<int64_t>(m_max, 1))));
    ts->bad = reinterpret_cast<int*>(take(sizeof(int)));
    ts->err = reinterpret_cast<int*>(take(sizeof(int)));
}

// G^T of a CSR whose targets were validated already, self-loops kept, with no
// host synchronisation: the launches can be captured in a CUDA graph. Needs
// n <= 2^24 (transpose_bucketed) and m within the scratch. Errors of the
// passes' self-checks go to ts.err (device).
int launch_transpose_keep_self(const int32_t* off, const int32_t* adj, int32_t n, int64_t m, const TransposeScratch& ts,
                               int32_t* toff, int32_t* tadj, int num_sms, cudaStream_t s) {
    const int shift = bucket_shift(n);
    if (!transpose_bucketed(shift)) return SCC_ERR_INVALID_ARG;
    SCC_TRY(launch_tile_rows(off, n, m, ts.trow, s));
    SCC_CUDA(cudaMemsetAsync(ts.bad, 0, sizeof(int), s));
    SCC_TRY(launch_intake_partition(adj, const_cast<int32_t*>(adj), off, ts.trow, n, m, shift, 1, ts.bcnt, ts.btmp,
                                    ts.tmp_u, ts.tmp_lv, nullptr, nullptr, ts.bad, ts.err, num_sms, s, s, nullptr,
                                    nullptr));
    bool self_found = false;
    return launch_transpose_rest(n, m, shift, 1, ts.bcnt, ts.btmp, ts.tmp_u, ts.tmp_lv, ts.tmp2_u, ts.tmp2_lv, ts.order,
                                 ts.tiles, toff, tadj, nullptr, &self_found, ts.err, num_sms, s, nullptr);
}

int transpose_set_attributes() { return ensure_attributes(); }
int transpose_set_attributes_impl() {
    SCC_CUDA(cudaFuncSetAttribute(k_copy_check_hist, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(sizeof(unsigned int) * kMaxBins)));
    SCC_CUDA(cudaFuncSetAttribute(k_bucket_part, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  2 * kStep * (int)sizeof(int32_t)));
    SCC_CUDA(cudaFuncSetAttribute(k_bucket_split, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)((size_t)kSplitTile * sizeof(uint2))));
    SCC_CUDA(cudaFuncSetAttribute(k_sub_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rows_smem_bytes()));
    return SCC_OK;
}

}  // namespace scc
