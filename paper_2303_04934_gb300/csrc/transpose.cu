// Transposed CSR G^T from the CSR of G (sm_103a).
//
// Every non-self arc (u, v) of G becomes the entry u of row v of G^T (Sec. 2: a
// backward reachability search is a forward search on G^T). This is a counting
// sort of the arcs by target, done in two levels so that every per-arc atomic is
// a shared-memory atomic:
//
//   A. coarse partition by bucket b = v >> shift (at most 512 buckets):
//      A1 histogram of buckets (per-block shared histogram, one global add per
//         block and bucket), fused with the copy and range check of the
//         targets: it needs no arc sources, so it reads the targets once as a
//         flat array;
//      A2 partition: a block takes a tile of 8k arcs, counting-sorts it by
//         bucket in shared memory, reserves one run per non-empty bucket with a
//         global atomicAdd, and writes the sorted tile out, so consecutive lanes
//         store consecutive positions of a run.
//      Each arc is written as its source u (4 B) and its target's offset within
//      the bucket (2 B: buckets hold at most 2^15 vertices).
//   B. one block per bucket (largest buckets first): per-vertex counts of the
//      bucket in shared memory, their scan gives the bucket's rows of G^T
//      (offsets written directly: the bucket's first row starts at the bucket's
//      start), then the arcs are placed with shared-memory cursors. The rows a
//      block writes span one bucket, so partial-sector writes merge in L2.
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
constexpr int kBucketLog = 15;          // at most 2^15 vertices per bucket (128 KB of shared counters)
constexpr int kBlkA = 512;
static_assert(kMaxBuckets <= kBlkA, "bucket scan uses one thread per bucket");
constexpr int kChunk = 16;              // consecutive arcs per thread per step
constexpr int kStep = kBlkA * kChunk;   // arcs per block step (8192) = partition tile
constexpr int kRowsCap = 4096;          // row offsets of one step staged in shared memory
constexpr int kBlkB = 1024;

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
            int lo = 0, hi = cnt - 2;
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if ((int64_t)s_off[mid] <= e0) lo = mid;
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
#pragma unroll
        for (int q = 0; q < kChunk; ++q) {
            const int64_t e = e0 + q;
            if (e < e1) {
                // advance to the row containing e
                // (bounded by the staged rows: r0..r1 always contain e)
                if (sm) {
                    while (r + 1 < cnt - 1 && (int64_t)s_off[r + 1] <= e) ++r;
                } else {
                    while (r0 + r + 1 <= r1 && (int64_t)__ldg(&off[r0 + r + 1]) <= e) ++r;
                }
                f(q, r0 + r, a[q]);
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
    __shared__ unsigned int s_hist[kMaxBuckets];
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

// exclusive scan of the bucket counts (one block, sequential: nb <= 2048);
// also zeroes the work counter of the rows pass
__global__ void k_bucket_scan(const unsigned long long* cnt, int nb, unsigned long long* start,
                              unsigned long long* cursor, unsigned int* rows_next) {
    if (threadIdx.x == 0) {
        unsigned long long s = 0;
        for (int i = 0; i < nb; ++i) {
            start[i] = s;
            cursor[i] = s;
            s += cnt[i];
        }
        start[nb] = s;
        *rows_next = 0;
    }
}

// A2. partition: per 8k-arc tile, a shared-memory counting sort by bucket,
// one global reservation per non-empty bucket, then a coalesced write-out.
__global__ void __launch_bounds__(kBlkA) k_bucket_part(const int32_t* __restrict__ off, const int32_t* __restrict__ adj,
                                                       const int32_t* __restrict__ trow, int32_t n, int64_t m,
                                                       int shift, int nb,
                                                       unsigned long long* cursor, int32_t* out_u, uint16_t* out_lv,
                                                       unsigned long long mt, int32_t* selfrow,
                                                       unsigned long long* nself, int* err) {
    __shared__ int32_t s_off[kRowsCap];
    __shared__ unsigned int s_cnt[kMaxBuckets];
    __shared__ unsigned int s_start[kMaxBuckets];
    __shared__ unsigned long long s_gbase[kMaxBuckets];
    extern __shared__ int32_t s_stage[];  // the sorted tile: u[kStep], v[kStep]
    int32_t* s_u = s_stage;
    int32_t* s_v = s_stage + kStep;
    __shared__ unsigned int s_wsum[kBlkA / 32];
    __shared__ unsigned int s_total;
    for (int64_t t0 = (int64_t)blockIdx.x * kStep; t0 < m; t0 += (int64_t)gridDim.x * kStep) {
        const int64_t t1 = min(t0 + (int64_t)kStep, m);
        for (int i = threadIdx.x; i < nb; i += blockDim.x) s_cnt[i] = 0;
        __syncthreads();
        // ranks within (tile, bucket), kept per thread
        unsigned int rk[kChunk];
        int uu[kChunk], vv[kChunk];
#pragma unroll
        for (int q = 0; q < kChunk; ++q) vv[q] = -1;
        // every arc is placed (the histogram counted self-loops too); a self-loop
        // is also counted per row, and any self-loop makes the caller rebuild
        // the CSR without them and start over
        for_step_arcs(off, adj, n, t0, t1, trow, s_off, [&](int q, int u, int v) {
            uu[q] = u;
            vv[q] = v;
            rk[q] = atomicAdd(&s_cnt[v >> shift], 1u);
            if (u == v) {
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
            if (i < nb) {
                s_start[i] = s_wsum[i >> 5] + incl - c;
                s_gbase[i] = c ? atomicAdd(&cursor[i], (unsigned long long)c) : 0ull;
            }
            __syncthreads();
        }
        // stage the tile sorted by bucket
#pragma unroll
        for (int q = 0; q < kChunk; ++q)
            if (vv[q] >= 0) {
                const unsigned int j = s_start[vv[q] >> shift] + rk[q];
                s_u[j] = uu[q];
                s_v[j] = vv[q];
            }
        __syncthreads();
        const unsigned int total = s_total;
        for (unsigned int j = threadIdx.x; j < total; j += blockDim.x) {
            const int v = s_v[j];
            const int b = v >> shift;
            const unsigned long long pos = s_gbase[b] + (j - s_start[b]);
            if (pos < mt) {
                out_u[pos] = s_u[j];
                out_lv[pos] = (uint16_t)(v & ((1 << shift) - 1));  // the target within its bucket
            } else {
                atomicExch(err, SCC_ERR_INTERNAL);
            }
        }
        __syncthreads();
    }
}

// B. one block per bucket: per-vertex counts in shared memory, row offsets of
// G^T for the bucket's vertices, placement with shared cursors. The grid is
// persistent (the resident blocks); each block takes the next bucket of the
// largest-first order from a global counter when it is done with one. The arcs are
// read in aligned chunks of 8 (one 16-byte load of local targets, two of
// sources), two chunks per thread per step; the arrays are padded by 8 entries
// so the last chunk may read past the last arc.
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
// Counter i of a bucket lives at i + i / 32 in shared memory: the scan below
// gives each thread a run of consecutive counters, and with one padding word
// per 32 the lanes of a warp reading the j-th counter of their runs hit 32
// different banks (without it they would all hit one).
__device__ __forceinline__ int cpad(int i) { return i + (i >> 5); }

__global__ void __launch_bounds__(kBlkB) k_bucket_rows(const int32_t* __restrict__ uu, const uint16_t* __restrict__ lvv,
                                                       const unsigned long long* __restrict__ start,
                                                       const int32_t* __restrict__ order, int nb, int shift,
                                                       int32_t n, int32_t* toff, int32_t* tadj,
                                                       unsigned int* rows_next, int* err) {
    extern __shared__ int s_cnt[];  // 2^shift counters, padded (cpad)
    __shared__ int s_wsum[kBlkB / 32];
    __shared__ int s_oi;
    const int W = 1 << shift;
    constexpr int kCh = 2;  // chunks per thread per step
    for (;;) {
        if (threadIdx.x == 0) s_oi = (int)atomicAdd(rows_next, 1u);
        __syncthreads();
        const int oi = s_oi;
        if (oi >= nb) break;
        const int b = order[oi];
        const int v0 = b << shift;
        const int vw = min(W, n - v0);
        const long long a0 = (long long)start[b], a1 = (long long)start[b + 1];
        for (int i = threadIdx.x; i < cpad(vw); i += blockDim.x) s_cnt[i] = 0;
        __syncthreads();
        const long long c0 = (a0 & ~7ll) + 8ll * threadIdx.x;
        const long long cstep = 8ll * blockDim.x;
        for (long long c = c0; c < a1; c += kCh * cstep) {
            uint4 r[kCh];
#pragma unroll
            for (int k = 0; k < kCh; ++k) {
                const long long cc = c + k * cstep;
                r[k] = cc < a1 ? __ldg(reinterpret_cast<const uint4*>(lvv + cc)) : make_uint4(0, 0, 0, 0);
            }
#pragma unroll
            for (int k = 0; k < kCh; ++k) {
                const long long cc = c + k * cstep;
                unsigned int lv[8];
                unpack8(r[k], lv);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    if (cc + j < a0 || cc + j >= a1) continue;
                    if (lv[j] < (unsigned int)vw) atomicAdd(&s_cnt[cpad((int)lv[j])], 1);
                    else atomicExch(err, SCC_ERR_INTERNAL);  // arc outside its bucket: skip it, report
                }
            }
        }
        __syncthreads();
        // exclusive scan of s_cnt[0..vw) in place; each thread owns a contiguous run
        const int per = (vw + blockDim.x - 1) / blockDim.x;
        const int q0 = threadIdx.x * per, q1 = min(q0 + per, vw);
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
        // the bucket's row offsets, written coalesced (before the placement
        // below advances the counters)
        for (int i = threadIdx.x; i < vw; i += blockDim.x) toff[v0 + i] = (int32_t)(a0 + s_cnt[cpad(i)]);
        __syncthreads();
        for (long long c = c0; c < a1; c += kCh * cstep) {
            uint4 r[kCh];
            int4 ua[kCh], ub[kCh];
#pragma unroll
            for (int k = 0; k < kCh; ++k) {
                const long long cc = c + k * cstep;
                const bool in = cc < a1;
                r[k] = in ? __ldg(reinterpret_cast<const uint4*>(lvv + cc)) : make_uint4(0, 0, 0, 0);
                ua[k] = in ? __ldg(reinterpret_cast<const int4*>(uu + cc)) : make_int4(0, 0, 0, 0);
                ub[k] = in ? __ldg(reinterpret_cast<const int4*>(uu + cc + 4)) : make_int4(0, 0, 0, 0);
            }
#pragma unroll
            for (int k = 0; k < kCh; ++k) {
                const long long cc = c + k * cstep;
                unsigned int lv[8];
                unpack8(r[k], lv);
                const int u8[8] = {ua[k].x, ua[k].y, ua[k].z, ua[k].w, ub[k].x, ub[k].y, ub[k].z, ub[k].w};
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    if (cc + j < a0 || cc + j >= a1 || lv[j] >= (unsigned int)vw) continue;
                    const int p = atomicAdd(&s_cnt[cpad((int)lv[j])], 1);
                    if (a0 + p < a1) tadj[a0 + p] = u8[j];
                    else atomicExch(err, SCC_ERR_INTERNAL);
                }
            }
        }
        __syncthreads();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) toff[n] = (int32_t)start[nb];
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

int bucket_shift(int32_t n) {
    int shift = 6;
    while (((int64_t)n + (1ll << shift) - 1) >> shift > kMaxBuckets) ++shift;
    return shift;
}

size_t tile_rows_count(int64_t m) { return (size_t)((m + kStep - 1) / kStep) + 1; }

int launch_copy_check_hist(const int32_t* src, int32_t* dst, int32_t n, int64_t m, int shift,
                           unsigned long long* bucket_cnt, int* bad, int num_sms, cudaStream_t s) {
    if (m == 0) return SCC_OK;
    const int nb = std::max(1, (int)(((int64_t)n + (1ll << shift) - 1) >> shift));
    k_copy_check_hist<<<grid_for_arcs(m, 4 * kBlkA * 4, num_sms, 2), kBlkA, 0, s>>>(src, dst, m, n, shift, nb,
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

int launch_transpose(const int32_t* off, const int32_t* adj, const int32_t* trow, int32_t n, int64_t m, int64_t mt,
                     int shift,
                     const unsigned long long* bucket_cnt, unsigned long long* bucket_tmp, int32_t* tmp_u,
                     uint16_t* tmp_lv, int32_t* order_tmp, int32_t* toff, int32_t* tadj, int32_t* selfrow,
                     unsigned long long* nself, bool* self_found, int* err, int num_sms, cudaStream_t s,
                     cudaEvent_t* ev) {
    *self_found = false;
    const int nb = std::max(1, (int)(((int64_t)n + (1ll << shift) - 1) >> shift));
    unsigned long long* start = bucket_tmp;
    unsigned long long* cursor = bucket_tmp + nb + 1;
    unsigned int* rows_next = reinterpret_cast<unsigned int*>(bucket_tmp + 2 * nb + 1);
    if (n == 0) {
        SCC_CUDA(cudaMemsetAsync(toff, 0, sizeof(int32_t), s));
        return SCC_OK;
    }
    k_bucket_scan<<<1, 32, 0, s>>>(bucket_cnt, nb, start, cursor, rows_next);
    SCC_LAUNCH();
    if (mt > 0) {
        const int stage = 2 * kStep * (int)sizeof(int32_t);
        SCC_CUDA(cudaFuncSetAttribute(k_bucket_part, cudaFuncAttributeMaxDynamicSharedMemorySize, stage));
        if (ev) cudaEventRecord(ev[0], s);
        k_bucket_part<<<grid_for_arcs(m, kStep, num_sms, 2), kBlkA, stage, s>>>(off, adj, trow, n, m, shift, nb, cursor,
                                                                                  tmp_u, tmp_lv,
                                                                                  (unsigned long long)mt, selfrow,
                                                                                  nself, err);
        SCC_LAUNCH();
        if (ev) cudaEventRecord(ev[1], s);
    }
    // buckets by decreasing size (longest first), from the host copy of the counts
    std::vector<unsigned long long> hc(nb);
    unsigned long long hself = 0;
    SCC_CUDA(cudaMemcpyAsync(hc.data(), bucket_cnt, sizeof(unsigned long long) * nb, cudaMemcpyDeviceToHost, s));
    SCC_CUDA(cudaMemcpyAsync(&hself, nself, sizeof(hself), cudaMemcpyDeviceToHost, s));
    SCC_CUDA(cudaStreamSynchronize(s));
    if (hself > 0) {  // the caller drops the self-loops and calls again
        *self_found = true;
        return SCC_OK;
    }
    std::vector<int32_t> ord(nb);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return hc[a] > hc[b]; });
    SCC_CUDA(cudaMemcpyAsync(order_tmp, ord.data(), sizeof(int32_t) * nb, cudaMemcpyHostToDevice, s));
    const size_t smem = sizeof(int) * (((size_t)1 << shift) + ((size_t)1 << shift) / 32 + 1);
    if (smem > 48 * 1024)
        SCC_CUDA(cudaFuncSetAttribute(k_bucket_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    SCC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bucket_rows, kBlkB, smem));
    if (ev) cudaEventRecord(ev[2], s);
    k_bucket_rows<<<std::min(nb, num_sms * std::max(1, per_sm)), kBlkB, smem, s>>>(tmp_u, tmp_lv, start, order_tmp,
                                                                                     nb, shift, n, toff, tadj,
                                                                                     rows_next, err);
    SCC_LAUNCH();
    if (ev) cudaEventRecord(ev[3], s);
    SCC_CUDA(cudaStreamSynchronize(s));  // ord (host) must outlive the copy
    return SCC_OK;
}

}  // namespace scc
