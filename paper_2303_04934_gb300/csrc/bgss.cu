// Device-side loop over the multi-reachability batches of Alg. 1 (sm_103a).
//
// After the first SCC, every remaining prefix-doubling batch runs inside ONE
// cooperative launch: batch sources (P_i n V'), the pair-table sizing of
// Sec. 4.5, the forward and the backward multi-reachability searches (VGC +
// hash bag, engine.cuh; the two are independent and share the rounds of one
// search) and the labelling passes (labels.cuh), separated by grid barriers. The host is involved only when a table or bag must grow: the
// kernel then stops before labelling that batch and reports it; the host
// enlarges the buffers and relaunches from that batch (nothing of the batch has
// been committed, so rerunning it is exact).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "common.cuh"
#include "engine.cuh"
#include "internal.h"
#include "labels.cuh"

namespace scc {

template <class Item>
EngineParams<Item> make_engine_params(const int32_t* off, const int32_t* adj, int32_t n, const EngineBuf* b,
                                      const EngineOpts& o);

struct BgssCtl {
    int status;                 // 0 finished, 1 grow tables/bag and resume at `batch`, 2 relaunch smaller
    int batch;
    long long need_cap;
    unsigned long long ndone;   // finished vertices so far (first SCC included)
    unsigned long long a[2];    // pairs of the previous batch, per direction
    int ka;                     // that batch's sources (0: unknown)
    int k[2];                   // sources of the batch (double-buffered)
    unsigned long long pairs;   // statistics
    int batches;
    int rounds;
    unsigned long long edges;
    unsigned long long items;
    unsigned long long active_sum;  // active vertices summed over the batches run
};

namespace {

struct BgssParams {
    const int32_t* off;
    const int32_t* adj;
    const int32_t* toff;
    const int32_t* tadj;
    int32_t n;
    int32_t* label;
    int32_t* rep;
    unsigned long long* fmax;
    unsigned long long* bmax;
    unsigned long long* hit;
    const int32_t* rem_pos;
    const int32_t* rem_v;
    long long nrem;
    long long N;
    const long long* bounds;
    int nb;
    int first;
    long long first_min_cap;  // table size for the resumed batch after an overflow
    long long shrink_below;   // stop (status 2) when fewer vertices are active: a smaller grid is cheaper
    int32_t* sources;
    unsigned long long* tab[2];
    long long tab_alloc;
    EngineParams<uint64_t> P;
    BgssCtl* bc;
};

// first j in [0, n) with a[j] >= x (n if none)
__device__ __forceinline__ long long lower_bound_d(const int32_t* a, long long n, long long x) {
    long long lo = 0, hi = n;
    while (lo < hi) {
        long long mid = (lo + hi) >> 1;
        if ((long long)a[mid] < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ long long pow2ceil_d(long long x) {
    long long p = 1;
    while (p < x) p <<= 1;
    return p;
}

// The remaining batches of Alg. 1 in one cooperative launch (the loop the file
// header describes); B.ctl tells the host why it stopped.
__global__ void __launch_bounds__(kEngineBlock, 2) bgss_kernel(BgssParams B) {
    __shared__ EngineSmem<PolPair> sm;
    const LocalQueue<uint64_t> q = warp_queue(sm);
    WarpStats ws;
    EngineCtl* ctl = B.P.ctl;
    BgssCtl* bc = B.bc;
    const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long gstride = (long long)gridDim.x * blockDim.x;
    const int lane = lane_id();
    int status = 0, stop_batch = B.nb;
    long long need = 0;
    uint32_t g = 0;   // global round counter of the engine (same in every block)
    uint32_t si = 0;  // search index
    for (int i = B.first; i < B.nb; ++i) {
        const int kb = i & 1;
        // ---- sources of batch i: the still-active vertices among its pivot
        // positions, a contiguous range of the remaining-position list
        if (gtid == 0) bc->k[kb ^ 1] = 0;
        const long long j0 = lower_bound_d(B.rem_pos, B.nrem, B.bounds[i]);
        const long long j1 = lower_bound_d(B.rem_pos, B.nrem, B.bounds[i + 1]);
        for (long long base = j0 + (gtid - lane); base < j1; base += gstride) {
            const long long j = base + lane;
            int v = -1;
            if (j < j1) {
                v = B.rem_v[j];
                if (B.label[v] < 0) v = -1;
            }
            const uint32_t m = __ballot_sync(kFull, v >= 0);
            int o = 0;
            if (lane == 0 && m) o = atomicAdd(&bc->k[kb], __popc(m));
            o = __shfl_sync(kFull, o, 0);
            if (v >= 0) B.sources[o + __popc(m & lanemask_lt())] = v;
        }
        if (!grid_sync(&ctl->bar, &ctl->err)) return;
        const int k = ld_volatile(&bc->k[kb]);
        const long long b_active = B.N - (long long)ld_volatile(&bc->ndone);
        if (b_active <= 0) break;
        if (gtid == 0) bc->active_sum += (unsigned long long)b_active;
        if (b_active < B.shrink_below) {
            status = 2;
            stop_batch = i;
            break;
        }
        if (k == 0) continue;
        // ---- pair-table sizes (Sec. 4.5): the expected pairs max(0.3 b, 1.5 a) (at
        // least k) at load factor 1/2, rounded up to a power of two; a batch
        // resumed after an overflow keeps the grown size. a is the previous
        // batch's pairs scaled by the ratio of this batch's sources to that
        // batch's: batches grow by beta, and their pairs with them
        long long cap[2];
        const int ka = ld_volatile(&bc->ka);
        const double grow_k = ka > 0 ? (double)k / (double)ka : 1.0;
        for (int d = 0; d < 2; ++d) {
            const double a = (double)ld_volatile(&bc->a[d]) * grow_k;
            long long want = max((long long)ceil(0.3 * (double)b_active), (long long)ceil(1.5 * a));
            want = max(want, (long long)k);
            cap[d] = max(1024ll, pow2ceil_d(2 * want));
            if (i == B.first) cap[d] = max(cap[d], B.first_min_cap);
        }
        if (cap[0] > B.tab_alloc || cap[1] > B.tab_alloc) {
            status = 1;
            stop_batch = i;
            need = max(cap[0], cap[1]);
            break;
        }
        // (the tables are empty: the previous batch's last pass reset every entry)
        // ---- forward (G) and backward (G^T) multi-reachability: independent
        // searches, run in the same rounds (items carry their direction)
        long long pairs[2];
        bool grow = false;
        {
            EngineParams<uint64_t> P = B.P;
            P.off = B.off;
            P.adj = B.adj;
            P.off2 = B.toff;
            P.adj2 = B.tadj;
            SearchCtl& sc = ctl->search[si % 3];
            PolPair pol;
            pol.label = B.label;
            for (int d = 0; d < 2; ++d) {
                pol.keys[d] = B.tab[d];
                pol.mask[d] = (unsigned long long)(cap[d] - 1);
                pol.max_ins[d] = (long long)(0.75 * (double)cap[d]);
            }
            pol.overflow = &sc.overflow;
            pol.ins0 = pol.ins1 = 0;
            int why = 0;  // 1: a table overflowed; < 0: error (same in every block)
            if (!engine_search<PolPair>(P, pol, InitPairs{B.sources, k}, 2 * (long long)k, nullptr, q, ws, g, si,
                                        why))
                return;
            ++si;
            pairs[0] = (long long)ld_volatile(&sc.inserted[0]);
            pairs[1] = (long long)ld_volatile(&sc.inserted[1]);
            const int rounds = ld_volatile(&sc.rounds);
            if (why < 0 && why != SCC_ERR_CAPACITY) return;
            if (why == 1 || why == SCC_ERR_CAPACITY) {
                grow = true;
                need = 2 * max(cap[0], cap[1]);
            }
            if (gtid == 0) bc->rounds += rounds;
        }
        if (grow) {
            status = 1;
            stop_batch = i;
            break;
        }
        // ---- labelling (Alg. 1; Sec. 4.4)
        const unsigned long long tag = (unsigned long long)i << 32;
        const PairTable tb{B.tab[1], (unsigned long long)(cap[1] - 1), nullptr};
        label_scan(gtid, gstride, B.tab[0], cap[0], tb, tag, B.fmax, B.bmax, B.hit);
        if (!grid_sync(&ctl->bar, &ctl->err)) return;
        unsigned long long c = label_finalize(gtid, gstride, B.tab[0], cap[0], B.tab[1], cap[1], tag, B.fmax,
                                              B.bmax, B.hit, B.label, B.rep, true);
        for (int d = 16; d >= 1; d >>= 1) c += __shfl_xor_sync(kFull, c, d);
        if (lane == 0 && c) atomicAdd(&bc->ndone, c);
        if (gtid == 0) {
            bc->a[0] = (unsigned long long)pairs[0];
            bc->a[1] = (unsigned long long)pairs[1];
            bc->ka = k;
            bc->pairs += (unsigned long long)(pairs[0] + pairs[1]);
            bc->batches += 1;
        }
        if (!grid_sync(&ctl->bar, &ctl->err)) return;
    }
    if (lane == 0 && ws.edges) atomicAdd(&bc->edges, ws.edges);
    if (lane == 0 && ws.items) atomicAdd(&bc->items, ws.items);
    if (gtid == 0) {
        bc->status = status;
        bc->batch = stop_batch;
        bc->need_cap = need;
    }
}

}  // namespace

int run_bgss_device(const BgssArgs& a, BgssResult* res, cudaStream_t st) {
    BgssParams B;
    memset(&B, 0, sizeof(B));
    B.off = a.off;
    B.adj = a.adj;
    B.toff = a.toff;
    B.tadj = a.tadj;
    B.n = a.n;
    B.label = a.label;
    B.rep = a.rep;
    B.fmax = a.fmax;
    B.bmax = a.bmax;
    B.hit = a.hit;
    B.rem_pos = a.rem_pos;
    B.rem_v = a.rem_v;
    B.nrem = a.nrem;
    B.N = a.N;
    B.bounds = a.bounds;
    B.nb = a.nb;
    B.first = a.first;
    B.first_min_cap = a.first_min_cap;
    B.shrink_below = a.shrink_below;
    B.sources = a.sources;
    B.tab[0] = a.tab[0];
    B.tab[1] = a.tab[1];
    B.tab_alloc = a.tab_alloc;
    EngineBuf* b = a.eb;
    B.P = make_engine_params<uint64_t>(a.off, a.adj, a.n, b, a.o);
    // control block for this launch
    BgssCtl* dbc = reinterpret_cast<BgssCtl*>(a.bgss_ctl);
    BgssCtl h;
    memset(&h, 0, sizeof(h));
    h.ndone = a.ndone;
    h.a[0] = a.a_prev[0];
    h.a[1] = a.a_prev[1];
    h.ka = a.ka_prev;
    B.bc = dbc;
    SCC_CUDA(cudaMemcpyAsync(dbc, &h, sizeof(h), cudaMemcpyHostToDevice, st));
    SCC_CUDA(cudaMemsetAsync(b->ctl, 0, sizeof(EngineCtl), st));
    static int per_sm = -1;
    if (per_sm < 0) {
        SCC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bgss_kernel, kEngineBlock, 0));
        if (per_sm < 1) return SCC_ERR_CUDA;
        per_sm = engine_blocks_per_sm(per_sm);
    }
    void* args[] = {(void*)&B};
    cudaEvent_t e0, e1;
    SCC_CUDA(cudaEventCreate(&e0));
    SCC_CUDA(cudaEventCreate(&e1));
    cudaEventRecord(e0, st);
    const int full = per_sm * a.o.num_sms;
    const int grid = a.grid > 0 ? std::min(a.grid, full) : full;
    cudaError_t le = cudaLaunchCooperativeKernel((const void*)bgss_kernel, dim3(grid), dim3(kEngineBlock), args, 0, st);
    count_launch();
    cudaEventRecord(e1, st);
    EngineCtl ec;
    cudaError_t c1 = cudaMemcpyAsync(&h, dbc, sizeof(h), cudaMemcpyDeviceToHost, st);
    cudaError_t c2 = cudaMemcpyAsync(&ec, b->ctl, sizeof(ec), cudaMemcpyDeviceToHost, st);
    cudaError_t se = cudaStreamSynchronize(st);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    SCC_CUDA(le);
    SCC_CUDA(c1);
    SCC_CUDA(c2);
    SCC_CUDA(se);
    res->ms = ms;
    res->status = h.status;
    res->batch = h.batch;
    res->need_cap = h.need_cap;
    res->ndone = h.ndone;
    res->a_prev[0] = h.a[0];
    res->a_prev[1] = h.a[1];
    res->ka_prev = h.ka;
    res->pairs = h.pairs;
    res->active_sum = h.active_sum;
    res->batches = h.batches;
    res->rounds = h.rounds;
    res->edges = h.edges;
    res->items = h.items;
    static const bool trace = getenv("SCC_TRACE") != nullptr;
    if (trace) {  // per-round timeline of the batches on stderr
        fprintf(stderr, "[scc-trace] multi-reach batches %d..%d: %d batches, %d rounds, %.1f us in kernel\n", a.first,
                h.batch, h.batches, h.rounds, 1000.0 * ms);
        unsigned long long t = ec.t0;
        const int nr = std::min(h.rounds, kTraceRounds);
        for (int r = 0; r < nr; ++r) {
            fprintf(stderr, "[scc-trace]   round %3d search %3d %s %9.1f us  items %lld\n", r, ec.t_dense[r] >> 1,
                    (ec.t_dense[r] & 1) ? "dense " : "sparse", (ec.t_end[r] - t) / 1000.0, ec.t_items[r]);
            t = ec.t_end[r];
        }
    }
    if (ec.err != 0 && ec.err != SCC_ERR_CAPACITY) return ec.err;
    return SCC_OK;
}

size_t bgss_ctl_bytes() { return sizeof(BgssCtl); }

int bgss_full_grid(int num_sms) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bgss_kernel, kEngineBlock, 0) != cudaSuccess) {
        cudaGetLastError();
        return num_sms;
    }
    return std::max(1, engine_blocks_per_sm(per_sm)) * num_sms;
}

}  // namespace scc
