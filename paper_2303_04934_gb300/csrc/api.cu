// C ABI (include/scc.h, include/scc_debug.h): graph handles, the SCC round
// driver (Alg. 1 with the paper's Sec. 4 engineering), multi-source
// reachability and the step-level test hooks.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <mutex>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/scc.h"
#include "../../include/scc_debug.h"
#include "common.cuh"
#include "engine.cuh"
#include "internal.h"

using namespace scc;

struct scc_graph {
    DeviceInfo di;
    int32_t n = 0;
    int64_t m_in = 0;      // arcs of the input
    int64_t mt = 0;        // arcs without self-loops (= arcs of G^T)
    int32_t* off = nullptr;
    int32_t* adj = nullptr;
    int32_t* toff = nullptr;
    int32_t* tadj = nullptr;
    scc_config cfg;
    cudaStream_t last = nullptr;
    // run state (allocated on first use, reused)
    int32_t* label = nullptr;
    int32_t* rep = nullptr;
    int32_t* act = nullptr;
    int32_t* tmp_a = nullptr;  // n+1
    int32_t* tmp_b = nullptr;  // n+1
    void* scan_tmp = nullptr;
    int32_t* sources = nullptr;
    unsigned long long* fmax = nullptr;
    unsigned long long* bmax = nullptr;
    unsigned long long* hit = nullptr;
    uint32_t* bits_f = nullptr;
    uint32_t* bits_b = nullptr;
    uint32_t* fbits = nullptr;               // dense-round frontier bitmap (kept zero)
    long long* bounds_d = nullptr;           // batch bounds on the device
    int32_t* rem_pos = nullptr;              // remaining active pivot positions / vertices
    int32_t* rem_v = nullptr;
    int bounds_cap = 0;
    void* bgss_ctl = nullptr;
    unsigned long long* counters = nullptr;  // [0] nact [1] ndone [2] scratch
    int* flags = nullptr;                    // [0] k [1] bad [2] overflow
    unsigned long long* tab[2] = {nullptr, nullptr};
    int64_t tab_alloc[2] = {0, 0};
    EngineBuf eb32, eb64;
    scc_stats stats;
    double create_ms[5] = {0, 0, 0, 0, 0};  // total, histogram, partition, rows, split
    // connectivity: the symmetric CSR (built on the first cc_run) and its stats
    int32_t* soff = nullptr;
    int32_t* sadj = nullptr;
    scc_cc_stats cc_stats;
    // least-element lists of the last le_lists_run
    int32_t* le_order = nullptr;
    int64_t* le_off = nullptr;
    int32_t* le_src = nullptr;
    int32_t* le_dist = nullptr;
    long long le_total = -1;  // -1: none computed
    scc_le_stats le_stats;
};

namespace scc {

static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(); }

// The library's stream-ordered allocations come from its own memory pool on the
// current device, whose release threshold keeps freed memory for reuse: creating
// and destroying graphs of similar size then costs no new device mappings.
static cudaMemPool_t library_pool() {
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    if (!pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        if (cudaMemPoolCreate(&p, &props) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        uint64_t thr = ~0ull;
        cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &thr);
        pools[dev] = p;
    }
    return pools[dev];
}

int dalloc(void** p, size_t bytes, cudaStream_t s) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaMemPool_t pool = library_pool();
    cudaError_t e = pool ? cudaMallocFromPoolAsync(p, bytes, pool, s) : cudaMallocAsync(p, bytes, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return e == cudaErrorMemoryAllocation ? SCC_ERR_OOM : SCC_ERR_CUDA;
    }
    return SCC_OK;
}
void dfree(void* p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}
bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// The device address of page-locked host memory (NULL for pageable memory).
const void* mapped_host_ptr(const void* p) {
    if (!p) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}
int device_info(DeviceInfo* out) {
    SCC_CUDA(cudaGetDevice(&out->dev));
    SCC_CUDA(cudaDeviceGetAttribute(&out->num_sms, cudaDevAttrMultiProcessorCount, out->dev));
    return SCC_OK;
}

}  // namespace scc

namespace {

int64_t pow2ceil(int64_t x) {
    int64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

// Copy count elements from a host-or-device pointer into device memory dst.
int to_device(void* dst, const void* src, size_t bytes, cudaStream_t s) {
    if (bytes == 0) return SCC_OK;
    cudaMemcpyKind kind = is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    SCC_CUDA(cudaMemcpyAsync(dst, src, bytes, kind, s));
    return SCC_OK;
}
int from_device(void* dst, const void* src, size_t bytes, cudaStream_t s) {
    if (bytes == 0) return SCC_OK;
    cudaMemcpyKind kind = is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    SCC_CUDA(cudaMemcpyAsync(dst, src, bytes, kind, s));
    return SCC_OK;
}

// average degree from which the first SCC's two searches run one after the
// other with dense rounds (below it they share one launch without)
constexpr double kDenseDegree = 8.0;

// automatic VGC budgets (config tau 0), by average degree
constexpr int kAutoTauHighDegree = 128;
constexpr int kAutoTauLowDegree = 2048;

EngineOpts opts_of(const scc_graph* h) {
    EngineOpts o;
    o.seeds = h->cfg.seeds;
    o.sigma = h->cfg.sigma;
    o.block = h->cfg.block;
    o.num_sms = h->di.num_sms;
    o.high_degree = (double)h->mt >= kDenseDegree * (double)std::max<int32_t>(h->n, 1);
    o.tau = h->cfg.tau ? h->cfg.tau : (o.high_degree ? kAutoTauHighDegree : kAutoTauLowDegree);
    return o;
}

int valid_config(const scc_config* c) {
    if (!c) return SCC_ERR_INVALID_ARG;
    if (c->tau < 0 || c->tau > (1 << 20)) return SCC_ERR_INVALID_ARG;
    if (!(c->beta > 1.0 && c->beta <= 64.0)) return SCC_ERR_INVALID_ARG;
    if (c->lambda < 1024 || c->lambda > (1 << 24) || (c->lambda & (c->lambda - 1))) return SCC_ERR_INVALID_ARG;
    if (c->sigma < 0 || c->sigma > (1 << 20)) return SCC_ERR_INVALID_ARG;
    if (c->block != 256) return SCC_ERR_INVALID_ARG;
    if (c->seeds < 1 || c->seeds > 32) return SCC_ERR_INVALID_ARG;
    if (c->dense < 0 || c->dense > 1024) return SCC_ERR_INVALID_ARG;
    if (!(c->ldd_beta > 1.0 && c->ldd_beta <= 64.0)) return SCC_ERR_INVALID_ARG;
    return SCC_OK;
}

int reserve_run_state(scc_graph* h, cudaStream_t s) {
    if (h->label) return SCC_OK;
    const int64_t n = h->n;
    const int64_t nw = (n + 31) / 32;
    SCC_TRY(dalloc_t(&h->label, n, s));
    SCC_TRY(dalloc_t(&h->rep, n, s));
    SCC_TRY(dalloc_t(&h->act, n, s));
    SCC_TRY(dalloc_t(&h->tmp_a, n + 1, s));
    SCC_TRY(dalloc_t(&h->tmp_b, n + 1, s));
    SCC_TRY(dalloc(&h->scan_tmp, scan_tmp_bytes(n), s));
    SCC_TRY(dalloc_t(&h->sources, std::max<int64_t>(n, 64), s));
    SCC_TRY(dalloc_t(&h->fmax, n, s));
    SCC_TRY(dalloc_t(&h->bmax, n, s));
    SCC_TRY(dalloc_t(&h->hit, n, s));
    SCC_TRY(dalloc_t(&h->bits_f, nw, s));
    SCC_TRY(dalloc_t(&h->bits_b, nw, s));
    SCC_TRY(dalloc_t(&h->counters, 4, s));
    SCC_TRY(dalloc_t(&h->flags, 4, s));
    SCC_TRY(dalloc_t(&h->fbits, 2 * nw, s));
    SCC_CUDA(cudaMemsetAsync(h->fbits, 0, sizeof(uint32_t) * (size_t)std::max<int64_t>(2 * nw, 1), s));
    SCC_TRY(dalloc(&h->bgss_ctl, bgss_ctl_bytes(), s));
    SCC_TRY(dalloc_t(&h->rem_pos, n, s));
    SCC_TRY(dalloc_t(&h->rem_v, n, s));
    return SCC_OK;
}

DenseOpts dense_opts(const scc_graph* h, int dir, long long n_active) {
    DenseOpts d;
    d.roff = dir == 0 ? h->toff : h->off;  // in-arcs of the search direction
    d.radj = dir == 0 ? h->tadj : h->adj;
    const int64_t nw = ((int64_t)h->n + 31) / 32;
    d.fbits[0] = h->fbits;
    d.fbits[1] = h->fbits + nw;
    d.n_active = n_active;
    d.frac_inv = h->cfg.dense == 1 ? 20 : h->cfg.dense;
    d.m_active = (long long)h->mt;
    return d;
}

int reserve_table(scc_graph* h, int d, int64_t cap, cudaStream_t s) {
    if (h->tab_alloc[d] >= cap) return SCC_OK;
    dfree(h->tab[d], s);
    h->tab[d] = nullptr;
    h->tab_alloc[d] = 0;
    SCC_TRY(dalloc_t(&h->tab[d], (size_t)cap, s));
    h->tab_alloc[d] = cap;
    return SCC_OK;
}

// at most this many class-trimming passes after the first SCC
constexpr int kClassTrimPasses = 4;

struct EvTimer {
    cudaEvent_t a = nullptr, b = nullptr;
    cudaStream_t s;
    explicit EvTimer(cudaStream_t st) : s(st) {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
    }
    ~EvTimer() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
    void start() { cudaEventRecord(a, s); }
    double stop() {
        cudaEventRecord(b, s);
        cudaEventSynchronize(b);
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        return ms;
    }
};

}  // namespace

// ==================================================================== ABI ====
namespace scc {

// reach_multi with 1..128 sources already on the device: mask2 (device, two
// words per vertex) gets bit j of vertex v (word 2 v + j / 64, bit j % 64) iff
// sources[j] reaches v (dir 0) or v reaches sources[j] (dir 1).
int reach_multi_wide(scc_graph* h, const int32_t* sources_d, int32_t k, int32_t dir,
                          unsigned long long* mask2, cudaStream_t s) {
    if (!h || !sources_d || !mask2 || k < 1 || k > 128 || (dir != 0 && dir != 1)) return SCC_ERR_INVALID_ARG;
    h->last = s;
    const int32_t n = h->n;
    SCC_TRY(reserve_run_state(h, s));
    for (int attempt = 0;; ++attempt) {  // bag too small: restart with twice the buffers
        if (attempt > 8) return SCC_ERR_CAPACITY;
        SCC_CUDA(cudaMemsetAsync(mask2, 0, (size_t)n * 16, s));
        SCC_CUDA(cudaMemsetAsync(h->flags + 1, 0, sizeof(int), s));
        SCC_TRY(launch_mask_init(sources_d, k, n, 2, mask2, h->flags + 1, s));
        int bad = 0;
        SCC_CUDA(cudaMemcpyAsync(&bad, h->flags + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
        SCC_CUDA(cudaStreamSynchronize(s));
        if (bad) return SCC_ERR_INVALID_ARG;
        SCC_TRY(engine_reserve(&h->eb32, 4, ((long long)n + 1024) << attempt, h->cfg.lambda, h->mt, h->di.num_sms, s));
        EngineRun r;
        int rc = run_mask2(dir == 0 ? h->off : h->toff, dir == 0 ? h->adj : h->tadj, n, sources_d, k, mask2, &h->eb32,
                           opts_of(h), &r, s);
        if (rc == SCC_ERR_CAPACITY) continue;
        return rc;
    }
}

}  // namespace scc

extern "C" {

const char* scc_error_string(int code) {
    switch (code) {
        case SCC_OK: return "ok";
        case SCC_ERR_INVALID_ARG: return "invalid argument";
        case SCC_ERR_OOM: return "out of device memory";
        case SCC_ERR_CUDA: return "CUDA error";
        case SCC_ERR_TIMEOUT: return "bounded device wait timed out";
        case SCC_ERR_CAPACITY: return "internal capacity exceeded";
        case SCC_ERR_INTERNAL: return "internal self-check failed";
        default: return "unknown error";
    }
}

int scc_config_default(scc_config* cfg) {
    if (!cfg) return SCC_ERR_INVALID_ARG;
    cfg->tau = 0;
    cfg->beta = 2.0;
    cfg->lambda = 1 << 14;
    cfg->sigma = 50;
    cfg->block = 256;
    cfg->seeds = 32;
    cfg->dense = 1;
    cfg->seed = 0x5CC00ull;
    cfg->ldd_beta = 2.0;
    return SCC_OK;
}

struct CreateEvents {
    cudaEvent_t e[10] = {};
    CreateEvents() {
        for (auto& x : e) cudaEventCreate(&x);
    }
    ~CreateEvents() {
        for (auto& x : e)
            if (x) cudaEventDestroy(x);
    }
    double ms(int a, int b) {
        float t = 0;
        if (cudaEventElapsedTime(&t, e[a], e[b]) == cudaSuccess) return (double)t;
        cudaGetLastError();  // a pass that did not run recorded no events: not an error of later calls
        return 0.0;
    }
};

// The second stream and its events of a chunked intake; on exit the stream's
// work finishes before the call's temporaries are freed on the main stream.
struct ChunkStreams {
    cudaStream_t s2 = nullptr;
    cudaEvent_t cev[9] = {};
    ChunkStreams() = default;
    ChunkStreams(const ChunkStreams&) = delete;
    ChunkStreams& operator=(const ChunkStreams&) = delete;
    ~ChunkStreams() {
        if (s2) {
            cudaStreamSynchronize(s2);
            cudaStreamDestroy(s2);
        }
        for (auto& e : cev)
            if (e) cudaEventDestroy(e);
    }
};

static int graph_create_impl(scc_graph* h, int32_t n, int64_t m, const int32_t* offsets, const int32_t* targets,
                             cudaStream_t s) {
    SCC_TRY(device_info(&h->di));
    CreateEvents ce;
    cudaEventRecord(ce.e[0], s);
    h->n = n;
    h->m_in = m;
    SCC_TRY(dalloc_t(&h->off, (size_t)n + 1, s));
    SCC_TRY(dalloc_t(&h->adj, (size_t)m, s));
    int32_t* const off_in = h->off;
    int32_t* const adj_in = h->adj;
    SCC_TRY(to_device(off_in, offsets, sizeof(int32_t) * ((size_t)n + 1), s));
    // a device target array is copied by the intake pass itself (one read), and
    // so is a page-locked host one (the pass reads it over the host link, so the
    // transfer and the pass are one); a pageable one is staged first
    const int32_t* src = targets;
    bool host_src = false;
    if (m > 0 && !is_device_ptr(targets)) {
        if (const void* mp = mapped_host_ptr(targets)) {
            src = static_cast<const int32_t*>(mp);
            host_src = true;
        } else {
            SCC_TRY(to_device(adj_in, targets, sizeof(int32_t) * (size_t)m, s));
            src = adj_in;
        }
    }
    const int shift = bucket_shift(n);
    const bool bucketed = transpose_bucketed(shift);
    // host input: intake and partition in chunks on two streams, so that each
    // chunk's partition runs while the next chunk crosses the host link
    const int K = bucketed ? transpose_chunks(m, host_src) : 1;
    Scratch tmp(s);  // every temporary below is freed when the call returns
    int* bad = nullptr;
    int32_t* selfrow = nullptr;
    unsigned long long *bcnt = nullptr, *btmp = nullptr;
    unsigned char* stmp = nullptr;
    SCC_TRY(tmp.alloc(&bad, 1));
    SCC_TRY(tmp.alloc(&selfrow, (size_t)n + 1));
    const size_t hist_words = transpose_hist_words(n, shift, K);  // [hist_words - 1]: self-loops found
    SCC_TRY(tmp.alloc(&bcnt, hist_words));
    SCC_TRY(tmp.alloc(&btmp, transpose_tmp_words(n, shift, K)));
    SCC_TRY(tmp.alloc(&stmp, scan_tmp_bytes(n)));
    unsigned long long* self_cnt = bcnt + hist_words - 1;
    SCC_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
    SCC_CUDA(cudaMemsetAsync(selfrow, 0, sizeof(int32_t) * ((size_t)n + 1), s));
    SCC_CUDA(cudaMemsetAsync(bcnt, 0, sizeof(unsigned long long) * hist_words, s));
    // validation before any kernel indexes with these arrays: the offsets, then
    // the targets within the intake pass (copy, range check, histogram); the
    // partition runs only if no target was out of range
    SCC_TRY(launch_validate_offsets(off_in, n, m, bad, s));
    int32_t* trow = nullptr;
    SCC_TRY(tmp.alloc(&trow, tile_rows_count(m)));
    SCC_TRY(launch_tile_rows(off_in, n, m, trow, s));
    int32_t *tmp_u = nullptr, *tmp2_u = nullptr, *ord = nullptr, *tiles = nullptr;
    uint16_t *tmp_lv = nullptr, *tmp2_lv = nullptr;
    int* terr = nullptr;
    ChunkStreams cs;  // declared after tmp: its stream is drained before tmp frees
    if (bucketed) {
        SCC_TRY(tmp.alloc(&tmp_u, (size_t)m + 8));
        SCC_TRY(tmp.alloc(&tmp_lv, (size_t)m + 8));
        SCC_TRY(tmp.alloc(&terr, 1));
        SCC_CUDA(cudaMemsetAsync(terr, 0, sizeof(int), s));
        if (K > 1) {
            SCC_CUDA(cudaStreamCreateWithFlags(&cs.s2, cudaStreamNonBlocking));
            for (int k = 0; k <= K; ++k) SCC_CUDA(cudaEventCreateWithFlags(&cs.cev[k], cudaEventDisableTiming));
        }
        SCC_TRY(launch_intake_partition(src, adj_in, off_in, trow, n, m, shift, K, bcnt, btmp, tmp_u, tmp_lv, selfrow,
                                        self_cnt, bad, terr, h->di.num_sms, s, cs.s2, cs.cev, &ce.e[1]));
    } else {
        cudaEventRecord(ce.e[1], s);
        SCC_TRY(launch_copy_check_hist(src, adj_in, n, m, shift, bcnt, bad, h->di.num_sms, s));
        cudaEventRecord(ce.e[2], s);
    }
    // the range check and (bucketed path) the partition's self-loop count in
    // one host round trip
    int hbad = 0;
    unsigned long long hself0 = 0;
    SCC_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (bucketed) SCC_CUDA(cudaMemcpyAsync(&hself0, self_cnt, sizeof(hself0), cudaMemcpyDeviceToHost, s));
    SCC_CUDA(cudaStreamSynchronize(s));
    tmp.release(bad);
    if (hbad) return SCC_ERR_INVALID_ARG;
    h->mt = m;
    int64_t m_cur = m;
    // forward CSR without its self-loops (selfrow counts them per row)
    auto drop_self_loops = [&](unsigned long long hself) -> int {
        const int64_t mt = m - (int64_t)hself;
        int32_t *cnt = nullptr, *off2 = nullptr, *adj2 = nullptr;
        SCC_TRY(tmp.alloc(&cnt, (size_t)n + 1));
        SCC_TRY(tmp.alloc(&off2, (size_t)n + 1));
        SCC_TRY(tmp.alloc(&adj2, (size_t)mt));
        SCC_TRY(launch_row_nonself(h->off, selfrow, n, cnt, s));
        SCC_TRY(launch_scan(cnt, off2, n, stmp, s));
        SCC_TRY(launch_drop_self_loops(h->off, h->adj, n, m, selfrow, off2, adj2, s));
        tmp.release(cnt);
        dfree(h->off, s);
        dfree(h->adj, s);
        h->off = off2;
        h->adj = adj2;
        tmp.keep(off2);
        tmp.keep(adj2);
        h->mt = mt;
        m_cur = mt;
        SCC_TRY(launch_tile_rows(h->off, n, m_cur, trow, s));  // rows of the new CSR's tiles
        return SCC_OK;
    };
    // G^T: three-level bucketed counting sort by target (direct atomics when n is huge)
    SCC_TRY(dalloc_t(&h->toff, (size_t)n + 1, s));
    SCC_TRY(dalloc_t(&h->tadj, (size_t)m, s));
    if (bucketed) {
        SCC_TRY(tmp.alloc(&tmp2_u, (size_t)m + 8));
        SCC_TRY(tmp.alloc(&tmp2_lv, (size_t)m + 8));
        SCC_TRY(tmp.alloc(&ord, (size_t)transpose_bins(n, shift)));
        SCC_TRY(tmp.alloc(&tiles, transpose_split_tiles(m, n, shift, K)));
        int k_cur = K;
        for (int attempt = 0;; ++attempt) {
            bool self_found = false;
            // the self-loop count of the first attempt is known already
            SCC_TRY(launch_transpose_rest(n, m_cur, shift, k_cur, bcnt, btmp, tmp_u, tmp_lv, tmp2_u, tmp2_lv, ord,
                                          tiles, h->toff, h->tadj, (attempt == 0 && hself0 == 0) ? nullptr : self_cnt,
                                          &self_found, terr, h->di.num_sms, s, &ce.e[5]));
            if (!self_found) break;
            if (attempt > 0) return SCC_ERR_INTERNAL;  // the rebuilt CSR has no self-loops
            // self-loops: rebuild the forward CSR without them and start over
            unsigned long long hself = 0;
            SCC_CUDA(cudaMemcpyAsync(&hself, self_cnt, sizeof(hself), cudaMemcpyDeviceToHost, s));
            SCC_CUDA(cudaStreamSynchronize(s));
            SCC_TRY(drop_self_loops(hself));
            k_cur = 1;
            // histograms and the self-loop count start over
            SCC_CUDA(cudaMemsetAsync(bcnt, 0, sizeof(unsigned long long) * hist_words, s));
            SCC_TRY(launch_intake_partition(h->adj, h->adj, h->off, trow, n, m_cur, shift, 1, bcnt, btmp, tmp_u,
                                            tmp_lv, nullptr, nullptr, nullptr, terr, h->di.num_sms, s, s, nullptr,
                                            &ce.e[1]));
        }
        int herr = 0;
        SCC_CUDA(cudaMemcpyAsync(&herr, terr, sizeof(int), cudaMemcpyDeviceToHost, s));
        SCC_CUDA(cudaStreamSynchronize(s));
        if (herr) return herr;
    } else {
        // self-loops from the row-aware histogram pass, then direct placement
        SCC_CUDA(cudaMemsetAsync(bcnt, 0, sizeof(unsigned long long) * hist_words, s));
        SCC_TRY(launch_bucket_hist(h->off, h->adj, trow, n, m, shift, bcnt, selfrow, self_cnt, h->di.num_sms, s));
        unsigned long long hself = 0;
        SCC_CUDA(cudaMemcpyAsync(&hself, self_cnt, sizeof(hself), cudaMemcpyDeviceToHost, s));
        SCC_CUDA(cudaStreamSynchronize(s));
        if (hself > 0) SCC_TRY(drop_self_loops(hself));
        int32_t* indeg = nullptr;
        SCC_TRY(tmp.alloc(&indeg, (size_t)n + 1));
        SCC_TRY(launch_transpose_direct(h->off, h->adj, trow, n, m_cur, indeg, stmp, h->toff, h->tadj,
                                        h->di.num_sms, s));
    }
    cudaEventRecord(ce.e[9], s);
    SCC_CUDA(cudaStreamSynchronize(s));
    h->create_ms[0] = ce.ms(0, 9);
    h->create_ms[1] = ce.ms(1, 2);
    if (transpose_bucketed(shift) && h->mt > 0) {
        h->create_ms[2] = ce.ms(3, 4);
        h->create_ms[4] = ce.ms(5, 6);
        h->create_ms[3] = ce.ms(7, 8);
    }
    return SCC_OK;
}

static void graph_free(scc_graph* h, cudaStream_t s) {
    dfree(h->off, s);
    dfree(h->adj, s);
    dfree(h->toff, s);
    dfree(h->tadj, s);
    dfree(h->label, s);
    dfree(h->rep, s);
    dfree(h->act, s);
    dfree(h->tmp_a, s);
    dfree(h->tmp_b, s);
    dfree(h->scan_tmp, s);
    dfree(h->sources, s);
    dfree(h->fmax, s);
    dfree(h->bmax, s);
    dfree(h->hit, s);
    dfree(h->bits_f, s);
    dfree(h->bits_b, s);
    dfree(h->counters, s);
    dfree(h->flags, s);
    dfree(h->tab[0], s);
    dfree(h->tab[1], s);
    dfree(h->fbits, s);
    dfree(h->bounds_d, s);
    dfree(h->bgss_ctl, s);
    dfree(h->rem_pos, s);
    dfree(h->rem_v, s);
    engine_release(&h->eb32, s);
    engine_release(&h->eb64, s);
    dfree(h->soff, s);
    dfree(h->sadj, s);
    dfree(h->le_order, s);
    dfree(h->le_off, s);
    dfree(h->le_src, s);
    dfree(h->le_dist, s);
}

int scc_graph_create(int32_t n, int64_t m, const int32_t* offsets, const int32_t* targets, void* stream,
                     scc_handle* out) {
    if (!out) return SCC_ERR_INVALID_ARG;
    *out = nullptr;
    if (n < 0 || n >= INT32_MAX || m < 0 || m > INT32_MAX || !offsets || (m > 0 && !targets))
        return SCC_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    scc_graph* h = new (std::nothrow) scc_graph();
    if (!h) return SCC_ERR_OOM;
    scc_config_default(&h->cfg);
    memset(&h->stats, 0, sizeof(h->stats));
    h->last = s;
    int rc = graph_create_impl(h, n, m, offsets, targets, s);
    if (rc != SCC_OK) {
        graph_free(h, s);
        cudaStreamSynchronize(s);
        delete h;
        return rc;
    }
    *out = h;
    return SCC_OK;
}

int scc_graph_destroy(scc_handle h) {
    if (!h) return SCC_OK;
    graph_free(h, h->last);
    cudaError_t e = cudaStreamSynchronize(h->last);
    delete h;
    return cuda_err(e);
}

int scc_set_config(scc_handle h, const scc_config* cfg) {
    if (!h) return SCC_ERR_INVALID_ARG;
    SCC_TRY(valid_config(cfg));
    h->cfg = *cfg;
    return SCC_OK;
}

int scc_get_stats(scc_handle h, scc_stats* out) {
    if (!h || !out) return SCC_ERR_INVALID_ARG;
    *out = h->stats;
    out->ms_create = h->create_ms[0];
    out->ms_transpose_hist = h->create_ms[1];
    out->ms_transpose_part = h->create_ms[2];
    out->ms_transpose_rows = h->create_ms[3];
    out->ms_transpose_split = h->create_ms[4];
    return SCC_OK;
}

int scc_graph_info(scc_handle h, int32_t* n, int64_t* m, int64_t* m_t) {
    if (!h) return SCC_ERR_INVALID_ARG;
    if (n) *n = h->n;
    if (m) *m = h->m_in;
    if (m_t) *m_t = h->mt;
    return SCC_OK;
}

static int scc_run_impl(scc_graph* h, int32_t* labels_out, cudaStream_t s) {
    const int32_t n = h->n;
    scc_stats& st = h->stats;
    memset(&st, 0, sizeof(st));
    st.tau = opts_of(h).tau;
    if (n == 0) return SCC_OK;
    SCC_TRY(reserve_run_state(h, s));
    EngineOpts o = opts_of(h);

    // ---- trimming (Sec. 4.1) and the active list
    EvTimer t(s);
    t.start();
    SCC_CUDA(cudaMemsetAsync(h->counters, 0, 4 * sizeof(unsigned long long), s));
    SCC_TRY(launch_init_labels(h->off, h->toff, n, h->label, h->rep, &h->counters[0], s));
    SCC_TRY(launch_compact_active(h->label, n, h->scan_tmp, h->act, s));
    unsigned long long hc[4];
    SCC_CUDA(cudaMemcpyAsync(hc, h->counters, sizeof(hc), cudaMemcpyDeviceToHost, s));
    st.ms_trim = t.stop();
    const int64_t N = (int64_t)hc[0];
    st.n_trimmed = (int32_t)(n - N);

    if (N > 0) {
        // ---- prefix-doubling batches over the seeded pivot order (Alg. 1)
        std::vector<int64_t> bounds{0};
        {
            double x = 1.0;
            int64_t pos = 0;
            while (pos < N) {
                int64_t sz;
                if (x >= (double)N) sz = N;
                else {
                    sz = (int64_t)x;
                    if ((double)sz < x) ++sz;
                }
                if (sz < 1) sz = 1;
                pos = (N - pos < sz) ? N : pos + sz;
                bounds.push_back(pos);
                x *= h->cfg.beta;
            }
        }
        const int nb = (int)bounds.size() - 1;

        // ---- first SCC: single-reachability both ways from the first pivot (Sec. 4.2)
        t.start();
        int64_t p0 = feistel_perm_host(0, N, h->cfg.seed);
        int32_t s0 = 0;
        SCC_CUDA(cudaMemcpyAsync(&s0, h->act + p0, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        SCC_CUDA(cudaStreamSynchronize(s));
        // Dense (bottom-up) rounds pay off on low-diameter graphs, whose
        // frontiers grow to a large part of the class; those have a high average
        // degree. Below kDenseDegree arcs per vertex (lattices, k-NN graphs) the
        // forward and backward searches share the rounds of one launch instead.
        const bool both = (h->cfg.dense == 0 || (double)h->mt < kDenseDegree * (double)n) && n < INT32_MAX - 2;
        SCC_TRY(engine_reserve(&h->eb32, 4, (both ? 2 * N : N) + 1024, h->cfg.lambda, h->mt, h->di.num_sms, s));
        SCC_TRY(launch_prefill_bits(h->label, 0, n, h->bits_f, h->bits_b, s));
        EngineRun r0, r1;
        if (both) {
            SCC_TRY(run_single_both(h->off, h->adj, h->toff, h->tadj, n, s0, h->bits_f, h->bits_b, &h->eb32, o, &r0,
                                    s));
        } else {
            SCC_TRY(run_single(h->off, h->adj, n, s0, h->bits_f, dense_opts(h, 0, N), &h->eb32, o, &r0, s));
            SCC_TRY(run_single(h->toff, h->tadj, n, s0, h->bits_b, dense_opts(h, 1, N), &h->eb32, o, &r1, s));
        }
        SCC_TRY(launch_label_first(h->bits_f, h->bits_b, n, s0, h->label, h->rep, &h->counters[1], s));
        SCC_CUDA(cudaMemcpyAsync(hc, h->counters, sizeof(hc), cudaMemcpyDeviceToHost, s));
        st.ms_first_scc = t.stop();
        st.first_scc_size = (int32_t)hc[1];
        st.search_rounds += r0.rounds + r1.rounds;

        // ---- trimming inside the three classes the first SCC leaves: passes
        // while a pass still finishes at least 1/32 of the active vertices
        t.start();
        {
            unsigned long long before = hc[1];
            for (int pass = 0; pass < kClassTrimPasses && (int64_t)before < N; ++pass) {
                SCC_TRY(launch_class_trim(h->act, N, h->off, h->adj, h->toff, h->tadj, h->label, h->rep,
                                          &h->counters[1], s));
                SCC_CUDA(cudaMemcpyAsync(hc, h->counters, sizeof(hc), cudaMemcpyDeviceToHost, s));
                SCC_CUDA(cudaStreamSynchronize(s));
                st.class_trim_passes++;
                const unsigned long long got = hc[1] - before;
                before = hc[1];
                if ((int64_t)got * 32 < N - (int64_t)hc[1]) break;
            }
            st.n_class_trimmed = (int32_t)(hc[1] - (unsigned long long)st.first_scc_size);
        }
        st.ms_class_trim = t.stop();
        for (const EngineRun* r : {&r0, &r1}) {
            if (both && r == &r1) continue;
            st.engine_launches++;
            st.ms_engine += r->ms;
            st.engine_arcs += (int64_t)r->edges;
            st.engine_items += (int64_t)r->items;
        }
        st.batches = 1;

        // ---- multi-reachability batches (Alg. 1; Sec. 4.3-4.5): one device-side loop
        if (nb > 1 && (int64_t)hc[1] < N) {
            if (h->bounds_cap < nb + 1) {
                dfree(h->bounds_d, s);
                h->bounds_d = nullptr;
                h->bounds_cap = 0;
                SCC_TRY(dalloc_t(&h->bounds_d, (size_t)nb + 1, s));
                h->bounds_cap = nb + 1;
            }
            SCC_CUDA(cudaMemcpyAsync(h->bounds_d, bounds.data(), sizeof(long long) * (size_t)(nb + 1),
                                     cudaMemcpyHostToDevice, s));
            long long tab_alloc = std::max<long long>(1 << 14, pow2ceil(4 * (int64_t)std::ceil(0.3 * (double)(N - (int64_t)hc[1]))));
            // the labelling maxima start untagged (only the batches use them)
            SCC_CUDA(cudaMemsetAsync(h->fmax, 0, (size_t)n * 8, s));
            SCC_CUDA(cudaMemsetAsync(h->bmax, 0, (size_t)n * 8, s));
            SCC_CUDA(cudaMemsetAsync(h->hit, 0, (size_t)n * 8, s));
            BgssArgs a;
            a.off = h->off;
            a.adj = h->adj;
            a.toff = h->toff;
            a.tadj = h->tadj;
            a.n = n;
            a.label = h->label;
            a.rep = h->rep;
            a.fmax = h->fmax;
            a.bmax = h->bmax;
            a.hit = h->hit;
            // the pivot positions after the first batch whose vertex is still active
            SCC_TRY(launch_remaining(h->act, N, h->cfg.seed, bounds[1], h->label, h->tmp_a, h->tmp_b, h->scan_tmp,
                                     h->rem_pos, h->rem_v, s));
            int32_t nrem = 0;
            SCC_CUDA(cudaMemcpyAsync(&nrem, h->tmp_b + (N - bounds[1]), sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            SCC_CUDA(cudaStreamSynchronize(s));
            a.rem_pos = h->rem_pos;
            a.rem_v = h->rem_v;
            a.nrem = nrem;
            a.N = N;
            a.bounds = h->bounds_d;
            a.nb = nb;
            a.first = 1;
            a.sources = h->sources;
            a.bgss_ctl = h->bgss_ctl;
            a.ndone = hc[1];
            a.a_prev[0] = a.a_prev[1] = 0;
            a.ka_prev = 0;
            a.o = o;
            // Grid sized to the active vertices (about 2k per block, at least 16
            // blocks): small remainders run on fewer blocks, whose barriers cost
            // less; the launch stops for a smaller grid once it could shrink 4x.
            const int full = bgss_full_grid(h->di.num_sms);
            const int min_grid = std::min(16, full);
            auto grid_for_active = [&](long long b) {
                return (int)std::max<long long>(min_grid, std::min<long long>(full, (b + 2047) / 2048));
            };
            auto plan = [&](long long b) {
                a.grid = grid_for_active(b);
                a.shrink_below = a.grid >= 4 * min_grid ? (long long)(a.grid / 4) * 2048 : 0;
            };
            plan(N - (int64_t)hc[1]);
            bool fresh = true;  // tables (and bag) must be emptied before the next launch
            for (int attempt = 0;; ++attempt) {
                if (attempt > 80) return SCC_ERR_CAPACITY;
                SCC_TRY(reserve_table(h, 0, tab_alloc, s));
                SCC_TRY(reserve_table(h, 1, tab_alloc, s));
                // a search holds at most 3/4 of each of the two tables
                SCC_TRY(engine_reserve(&h->eb64, 8, (long long)(1.5 * (double)tab_alloc) + (1 << 20), h->cfg.lambda,
                                       h->mt, h->di.num_sms, s));
                if (fresh) {  // the kernel keeps both tables empty between batches
                    SCC_CUDA(cudaMemsetAsync(h->tab[0], 0xff, (size_t)tab_alloc * 8, s));
                    SCC_CUDA(cudaMemsetAsync(h->tab[1], 0xff, (size_t)tab_alloc * 8, s));
                    SCC_TRY(engine_reset_slots(&h->eb64, s));
                    fresh = false;
                }
                a.tab[0] = h->tab[0];
                a.tab[1] = h->tab[1];
                a.tab_alloc = tab_alloc;
                a.eb = &h->eb64;
                BgssResult r;
                SCC_TRY(run_bgss_device(a, &r, s));
                st.ms_multi_search += r.ms;
                st.batches += r.batches;
                st.search_rounds += r.rounds;
                st.pairs += (int64_t)r.pairs;
                st.multi_active_sum += (int64_t)r.active_sum;
                st.engine_inserted += (int64_t)r.pairs;
                st.multi_launches++;
                st.multi_arcs += (int64_t)r.edges;
                st.multi_items += (int64_t)r.items;
                hc[1] = r.ndone;
                if (r.status == 0) break;
                if (r.status == 2) {  // stopped between batches: tables and bag are empty
                    a.first = r.batch;
                    a.ndone = r.ndone;
                    a.a_prev[0] = r.a_prev[0];
                    a.a_prev[1] = r.a_prev[1];
                    a.ka_prev = r.ka_prev;
                    a.first_min_cap = 0;
                    plan(N - (int64_t)r.ndone);
                    continue;
                }
                fresh = true;  // stopped inside a batch
                st.table_resizes++;
                tab_alloc = std::max<long long>(tab_alloc, pow2ceil(r.need_cap));
                a.first = r.batch;
                a.first_min_cap = r.need_cap;
                a.ndone = r.ndone;
                a.a_prev[0] = r.a_prev[0];
                a.a_prev[1] = r.a_prev[1];
                a.ka_prev = r.ka_prev;
            }
        }
        if ((int64_t)hc[1] != N) return SCC_ERR_INTERNAL;  // every active vertex must be finished
    }

    // ---- canonical minimum labels
    t.start();
    int32_t* dst = labels_out;
    bool host_out = !is_device_ptr(labels_out);
    if (host_out) dst = h->tmp_a;
    SCC_CUDA(cudaMemsetAsync(h->flags + 1, 0, sizeof(int), s));
    SCC_TRY(launch_canonicalize(h->rep, n, h->tmp_b, dst, h->flags + 1, s));
    if (host_out) SCC_CUDA(cudaMemcpyAsync(labels_out, dst, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToHost, s));
    int bad = 0;
    SCC_CUDA(cudaMemcpyAsync(&bad, h->flags + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    st.ms_label += t.stop();
    if (bad) return SCC_ERR_INTERNAL;
    return SCC_OK;
}

int scc_run(scc_handle h, int32_t* labels_out, void* stream) {
    if (!h || (h->n > 0 && !labels_out)) return SCC_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    h->last = s;
    return scc_run_impl(h, labels_out, s);
}

int reach_multi(scc_handle h, const int32_t* sources, int32_t k, int32_t dir, uint64_t* out, void* stream) {
    if (!h || !sources || !out || k < 1 || k > 64 || (dir != 0 && dir != 1)) return SCC_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    h->last = s;
    const int32_t n = h->n;
    if (!is_device_ptr(sources)) {
        for (int j = 0; j < k; ++j)
            if (sources[j] < 0 || sources[j] >= n) return SCC_ERR_INVALID_ARG;
    }
    SCC_TRY(reserve_run_state(h, s));
    int32_t* dsrc = h->sources;
    SCC_TRY(to_device(dsrc, sources, sizeof(int32_t) * (size_t)k, s));
    bool dev_out = is_device_ptr(out);
    unsigned long long* mask = dev_out ? reinterpret_cast<unsigned long long*>(out) : h->fmax;
    // A vertex re-enters the frontier each time it gains source bits, so a round
    // can hold more than n items; if the bag runs out of room the search restarts
    // from the sources with twice the buffers.
    for (int attempt = 0;; ++attempt) {
        if (attempt > 8) return SCC_ERR_CAPACITY;
        SCC_CUDA(cudaMemsetAsync(mask, 0, (size_t)n * 8, s));
        SCC_CUDA(cudaMemsetAsync(h->flags + 1, 0, sizeof(int), s));
        SCC_TRY(launch_mask_init(dsrc, k, n, 1, mask, h->flags + 1, s));
        int bad = 0;
        SCC_CUDA(cudaMemcpyAsync(&bad, h->flags + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
        SCC_CUDA(cudaStreamSynchronize(s));
        if (bad) return SCC_ERR_INVALID_ARG;
        SCC_TRY(engine_reserve(&h->eb32, 4, ((long long)n + 1024) << attempt, h->cfg.lambda, h->mt, h->di.num_sms, s));
        EngineRun r;
        int rc = run_mask(dir == 0 ? h->off : h->toff, dir == 0 ? h->adj : h->tadj, n, dsrc, k, mask, &h->eb32,
                          opts_of(h), &r, s);
        if (rc == SCC_ERR_CAPACITY) continue;
        SCC_TRY(rc);
        break;
    }
    if (!dev_out) SCC_TRY(from_device(out, mask, (size_t)n * 8, s));
    SCC_CUDA(cudaStreamSynchronize(s));
    // mask mode uses fmax as scratch: the next scc_run clears it
    return SCC_OK;
}

// reach_multi for callers that cannot allocate device memory during the call:
// device buffers only, working memory from the library's fixed device array.
int reach_multi_noalloc(scc_handle h, const int32_t* sources, int32_t k, int32_t dir, uint64_t* out, void* stream) {
    if (!h || !sources || !out || k < 1 || k > 64 || (dir != 0 && dir != 1)) return SCC_ERR_INVALID_ARG;
    if (!is_device_ptr(sources) || !is_device_ptr(out)) return SCC_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    return reach_multi_noalloc_impl(dir == 0 ? h->off : h->toff, dir == 0 ? h->adj : h->tadj, h->n, h->mt,
                                    h->cfg.lambda, opts_of(h), sources, k, out, s);
}

// ----------------------------------------------------------- connectivity --
// Connected components of the undirected graph under G's arcs (Sec. 5.1,
// Alg. 4 LDD-UF-JTB with VGC and the hash bag; steps in cc.cu).

// The symmetric CSR of h (row v = row v of G, then row v of G^T), built on the
// first call and kept with the handle.
static int ensure_sym(scc_graph* h, cudaStream_t s) {
    if (h->soff) return SCC_OK;
    const int32_t n = h->n;
    int32_t *so = nullptr, *sa = nullptr;
    SCC_TRY(dalloc_t(&so, (size_t)n + 1, s));
    if (dalloc_t(&sa, (size_t)std::max<int64_t>(2 * h->mt, 1), s) != SCC_OK) {
        dfree(so, s);
        return SCC_ERR_OOM;
    }
    const int rc = launch_sym_csr(h->off, h->adj, h->toff, h->tadj, n, so, sa, h->di.num_sms, s);
    if (rc != SCC_OK) {
        dfree(so, s);
        dfree(sa, s);
        return rc;
    }
    h->soff = so;
    h->sadj = sa;
    return SCC_OK;
}

static int cc_run_impl(scc_graph* h, int32_t* labels_out, cudaStream_t s) {
    const int32_t n = h->n;
    scc_cc_stats& st = h->cc_stats;
    memset(&st, 0, sizeof(st));
    if (n == 0) return SCC_OK;
    const int num_sms = h->di.num_sms;
    EvTimer tt(s);
    tt.start();
    EvTimer t(s);
    // the symmetric CSR, kept with the handle
    t.start();
    SCC_TRY(ensure_sym(h, s));
    st.ms_sym = t.stop();
    // the seeded order of all vertices and its batches
    Scratch tmp(s);
    int32_t *order = nullptr, *center = nullptr, *parent = nullptr, *root = nullptr, *mn = nullptr, *out = nullptr;
    long long* bounds_d = nullptr;
    unsigned long long* counters = nullptr;
    int* err = nullptr;
    SCC_TRY(tmp.alloc(&order, (size_t)n));
    SCC_TRY(tmp.alloc(&center, (size_t)n));
    SCC_TRY(tmp.alloc(&parent, (size_t)n));
    SCC_TRY(tmp.alloc(&root, (size_t)n));
    SCC_TRY(tmp.alloc(&mn, (size_t)n));
    SCC_TRY(tmp.alloc(&counters, 4));
    SCC_TRY(tmp.alloc(&err, 1));
    const bool dev_out = is_device_ptr(labels_out);
    if (dev_out) out = labels_out;
    else SCC_TRY(tmp.alloc(&out, (size_t)n));
    SCC_CUDA(cudaMemsetAsync(counters, 0, 4 * sizeof(unsigned long long), s));
    SCC_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    std::vector<long long> bounds{0};
    {
        double x = 1.0;
        long long pos = 0;
        while (pos < n) {
            long long sz;
            if (x >= (double)n) sz = n;
            else {
                sz = (long long)x;
                if ((double)sz < x) ++sz;
            }
            if (sz < 1) sz = 1;
            pos = ((long long)n - pos < sz) ? (long long)n : pos + sz;
            bounds.push_back(pos);
            x *= h->cfg.ldd_beta;
        }
    }
    const int nb = (int)bounds.size() - 1;
    SCC_TRY(tmp.alloc(&bounds_d, bounds.size()));
    SCC_CUDA(cudaMemcpyAsync(bounds_d, bounds.data(), sizeof(long long) * bounds.size(), cudaMemcpyHostToDevice, s));
    // ---- LDD (Alg. 4 function LDD)
    t.start();
    SCC_TRY(launch_iota(n, root, num_sms, s));  // the identity list, permuted into the order
    SCC_TRY(launch_pivot_order(root, (int64_t)n, h->cfg.seed, order, s));
    // the visited bitmap and the two frontier bitmaps of the bottom-up rounds
    const size_t nw = ((size_t)n + 31) / 32;
    uint32_t *vbits = nullptr, *fbits = nullptr;
    SCC_TRY(tmp.alloc(&vbits, nw));
    SCC_TRY(tmp.alloc(&fbits, 2 * nw));
    SCC_CUDA(cudaMemsetAsync(fbits, 0, sizeof(uint32_t) * 2 * nw, s));
    SCC_TRY(launch_ldd_setup(order, bounds[1], n, center, vbits, num_sms, s));
    SCC_TRY(engine_reserve(&h->eb32, 4, (long long)n + 1024, h->cfg.lambda, 2 * h->mt, num_sms, s));
    EngineOpts o = opts_of(h);
    EngineRun r;
    // bottom-up rounds when the frontier is large, as for the first SCC's searches
    const int frac_inv = h->cfg.dense == 1 ? 20 : h->cfg.dense;
    SCC_TRY(run_ldd(h->soff, h->sadj, n, 2 * (long long)h->mt, order, bounds_d, bounds[1], nb, center, vbits, fbits,
                    frac_inv, &h->eb32, o, &r, s));
    st.ms_ldd = t.stop();
    st.ldd_rounds = r.rounds;
    st.ldd_batches = nb;
    st.ldd_arcs = (int64_t)r.edges;
    // ---- union-find over the cross arcs (Alg. 4 Union), then the labels
    CreateEvents ev;
    cudaEventRecord(ev.e[0], s);
    const long long big_cap = (long long)(h->mt / 33) + 1;  // rows of more than 32 arcs
    int32_t *big = nullptr, *bdeg = nullptr, *bpre = nullptr;
    unsigned char* stmp = nullptr;
    SCC_TRY(tmp.alloc(&big, (size_t)big_cap));
    SCC_TRY(tmp.alloc(&bdeg, (size_t)big_cap));
    SCC_TRY(tmp.alloc(&bpre, (size_t)big_cap + 1));
    SCC_TRY(tmp.alloc(&stmp, scan_tmp_bytes(big_cap)));
    SCC_TRY(launch_cc_union_label(h->off, h->adj, n, center, parent, root, mn, out, counters, big, bdeg, bpre, stmp,
                                  big_cap, err, num_sms, s, &ev.e[1]));
    if (!dev_out) SCC_TRY(from_device(labels_out, out, sizeof(int32_t) * (size_t)n, s));
    unsigned long long hc[4];
    int herr = 0;
    SCC_CUDA(cudaMemcpyAsync(hc, counters, sizeof(hc), cudaMemcpyDeviceToHost, s));
    SCC_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    SCC_CUDA(cudaStreamSynchronize(s));
    if (herr) return herr;
    st.cross_arcs = (int64_t)hc[0];
    st.clusters = (int32_t)hc[1];
    st.components = (int32_t)hc[2];
    st.ms_union = ev.ms(1, 2);
    st.ms_label = ev.ms(2, 3);
    st.ms_total = tt.stop();
    return SCC_OK;
}

int cc_run(scc_handle h, int32_t* labels_out, void* stream) {
    if (!h || (h->n > 0 && !labels_out)) return SCC_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    h->last = s;
    return cc_run_impl(h, labels_out, s);
}

int cc_get_stats(scc_handle h, scc_cc_stats* out) {
    if (!h || !out) return SCC_ERR_INVALID_ARG;
    *out = h->cc_stats;
    return SCC_OK;
}

// ---------------------------------------------------- least-element lists --
// LE-lists (Sec. 5.2, Alg. 5) of the undirected graph under G's arcs for the
// handle's seeded vertex order (steps in lelists.cu).
static int le_lists_impl(scc_graph* h, int64_t* total, cudaStream_t s, long long init_cap = 0,
                         long long init_log = 0) {
    const int32_t n = h->n;
    scc_le_stats& st = h->le_stats;
    memset(&st, 0, sizeof(st));
    dfree(h->le_off, s);
    dfree(h->le_src, s);
    dfree(h->le_dist, s);
    h->le_off = nullptr;
    h->le_src = h->le_dist = nullptr;
    h->le_total = -1;
    EvTimer t(s);
    t.start();
    SCC_TRY(ensure_sym(h, s));
    if (!h->le_order) SCC_TRY(dalloc_t(&h->le_order, (size_t)std::max(n, 1), s));
    if (n > 0) {
        Scratch tmp(s);
        int32_t* iota = nullptr;
        SCC_TRY(tmp.alloc(&iota, (size_t)n));
        SCC_TRY(launch_iota(n, iota, h->di.num_sms, s));
        SCC_TRY(launch_pivot_order(iota, (int64_t)n, h->cfg.seed, h->le_order, s));
    }
    LeResult r;
    const int rc = le_lists_compute(h->soff, h->sadj, n, h->le_order, h->di.num_sms, &r, s, init_cap, init_log);
    if (rc != SCC_OK) {
        dfree(r.off, s);
        dfree(r.src, s);
        dfree(r.dist, s);
        return rc;
    }
    h->le_off = r.off;
    h->le_src = r.src;
    h->le_dist = r.dist;
    h->le_total = r.total;
    st.entries = r.total;
    st.candidates = r.candidates;
    st.levels = r.levels;
    st.launches = r.launches;
    st.arcs = r.edges;
    st.ms_total = t.stop();
    *total = r.total;
    return SCC_OK;
}

int le_lists_run(scc_handle h, int64_t* total, void* stream) {
    if (!h || !total) return SCC_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    h->last = s;
    *total = 0;
    return le_lists_impl(h, total, s);
}

int le_lists_get(scc_handle h, int32_t* order, int64_t* le_off, int32_t* le_src, int32_t* le_dist, void* stream) {
    if (!h || h->le_total < 0) return SCC_ERR_INVALID_ARG;
    if ((h->n > 0 && (!order || !le_off)) || (h->le_total > 0 && (!le_src || !le_dist))) return SCC_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int32_t n = h->n;
    if (n > 0) {
        SCC_CUDA(cudaMemcpyAsync(order, h->le_order, sizeof(int32_t) * (size_t)n, cudaMemcpyDefault, s));
        SCC_CUDA(cudaMemcpyAsync(le_off, h->le_off, sizeof(int64_t) * ((size_t)n + 1), cudaMemcpyDefault, s));
    } else if (le_off) {
        const int64_t z = 0;
        SCC_CUDA(cudaMemcpyAsync(le_off, &z, sizeof(z), cudaMemcpyDefault, s));
    }
    if (h->le_total > 0) {
        SCC_CUDA(cudaMemcpyAsync(le_src, h->le_src, sizeof(int32_t) * (size_t)h->le_total, cudaMemcpyDefault, s));
        SCC_CUDA(cudaMemcpyAsync(le_dist, h->le_dist, sizeof(int32_t) * (size_t)h->le_total, cudaMemcpyDefault, s));
    }
    SCC_CUDA(cudaStreamSynchronize(s));
    return SCC_OK;
}

int scc_debug_le_lists(scc_handle h, int64_t init_cap, int64_t init_log, int64_t* total, void* stream) {
    if (!h || !total || init_cap < 1 || init_log < 1) return SCC_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    h->last = s;
    *total = 0;
    return le_lists_impl(h, total, s, init_cap, init_log);
}

int le_get_stats(scc_handle h, scc_le_stats* out) {
    if (!h || !out) return SCC_ERR_INVALID_ARG;
    *out = h->le_stats;
    return SCC_OK;
}

// ------------------------------------------------------------ debug hooks --
int scc_debug_csr(scc_handle h, int32_t which, int32_t* off, int32_t* adj, void* stream) {
    if (!h || !off || (h->mt > 0 && !adj) || (which != 0 && which != 1)) return SCC_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    h->last = s;
    SCC_TRY(from_device(off, which ? h->toff : h->off, sizeof(int32_t) * ((size_t)h->n + 1), s));
    SCC_TRY(from_device(adj, which ? h->tadj : h->adj, sizeof(int32_t) * (size_t)h->mt, s));
    SCC_CUDA(cudaStreamSynchronize(s));
    return SCC_OK;
}

int scc_debug_trim(scc_handle h, uint8_t* flags, void* stream) {
    if (!h || (h->n > 0 && !flags)) return SCC_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    h->last = s;
    if (h->n == 0) return SCC_OK;
    Scratch tmp(s);
    uint8_t* d = nullptr;
    SCC_TRY(tmp.alloc(&d, (size_t)h->n));
    int rc = launch_trim(h->off, h->toff, h->n, d, s);
    if (rc == SCC_OK) rc = from_device(flags, d, (size_t)h->n, s);
    if (rc == SCC_OK) rc = cuda_err(cudaStreamSynchronize(s));
    return rc;
}

int scc_debug_pivot_order(scc_handle h, int32_t* order, int32_t* n_active, void* stream) {
    if (!h || !n_active || (h->n > 0 && !order)) return SCC_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    h->last = s;
    *n_active = 0;
    if (h->n == 0) return SCC_OK;
    SCC_TRY(reserve_run_state(h, s));
    SCC_CUDA(cudaMemsetAsync(h->counters, 0, 4 * sizeof(unsigned long long), s));
    SCC_TRY(launch_init_labels(h->off, h->toff, h->n, h->label, h->rep, &h->counters[0], s));
    SCC_TRY(launch_compact_active(h->label, h->n, h->scan_tmp, h->act, s));
    unsigned long long N = 0;
    SCC_CUDA(cudaMemcpyAsync(&N, h->counters, sizeof(N), cudaMemcpyDeviceToHost, s));
    SCC_CUDA(cudaStreamSynchronize(s));
    SCC_TRY(launch_pivot_order(h->act, (int64_t)N, h->cfg.seed, h->sources, s));
    SCC_TRY(from_device(order, h->sources, sizeof(int32_t) * N, s));
    SCC_CUDA(cudaStreamSynchronize(s));
    *n_active = (int32_t)N;
    return SCC_OK;
}

int scc_debug_single_reach(scc_handle h, const int32_t* labels, int32_t src, int32_t dir, uint8_t* visited,
                           void* stream) {
    if (!h || !visited || src < 0 || src >= h->n || (dir != 0 && dir != 1)) return SCC_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    h->last = s;
    SCC_TRY(reserve_run_state(h, s));
    const int32_t n = h->n;
    int32_t L = 0;
    const int32_t* dl = nullptr;
    if (labels) {
        SCC_TRY(to_device(h->label, labels, sizeof(int32_t) * (size_t)n, s));
        dl = h->label;
        SCC_CUDA(cudaMemcpyAsync(&L, h->label + src, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        SCC_CUDA(cudaStreamSynchronize(s));
    }
    uint8_t* d = nullptr;
    SCC_TRY(dalloc_t(&d, (size_t)n, s));
    int rc = SCC_OK;
    if (labels && L < 0) {
        rc = cuda_err(cudaMemsetAsync(d, 0, (size_t)n, s));  // a finished source reaches nothing
    } else {
        rc = launch_prefill_bits(dl, L, n, h->bits_f, nullptr, s);
        if (rc == SCC_OK) rc = engine_reserve(&h->eb32, 4, (long long)n + 1024, h->cfg.lambda, h->mt, h->di.num_sms, s);
        EngineRun r;
        if (rc == SCC_OK)
            rc = run_single(dir == 0 ? h->off : h->toff, dir == 0 ? h->adj : h->tadj, n, src, h->bits_f,
                            dense_opts(h, dir, n), &h->eb32, opts_of(h), &r, s);
        if (rc == SCC_OK) rc = launch_bits_to_bytes(h->bits_f, dl, L, n, d, s);
    }
    if (rc == SCC_OK) rc = from_device(visited, d, (size_t)n, s);
    if (rc == SCC_OK) rc = cuda_err(cudaStreamSynchronize(s));
    dfree(d, s);
    return rc;
}

int scc_debug_reach_multi_wide(scc_handle h, const int32_t* sources, int32_t k, int32_t dir, uint64_t* out,
                               void* stream) {
    if (!h || !sources || !out || k < 1 || k > 128 || (dir != 0 && dir != 1)) return SCC_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    h->last = s;
    const int32_t n = h->n;
    if (!is_device_ptr(sources)) {
        for (int j = 0; j < k; ++j)
            if (sources[j] < 0 || sources[j] >= n) return SCC_ERR_INVALID_ARG;
    }
    SCC_TRY(reserve_run_state(h, s));
    SCC_TRY(to_device(h->sources, sources, sizeof(int32_t) * (size_t)k, s));
    const bool dev_out = is_device_ptr(out);
    unsigned long long* mask2 = reinterpret_cast<unsigned long long*>(out);
    if (!dev_out) SCC_TRY(dalloc_t(&mask2, 2 * (size_t)std::max(n, 1), s));
    int rc = reach_multi_wide(h, h->sources, k, dir, mask2, s);
    if (rc == SCC_OK && !dev_out) rc = from_device(out, mask2, (size_t)n * 16, s);
    if (rc == SCC_OK) rc = cuda_err(cudaStreamSynchronize(s));
    if (!dev_out) dfree(mask2, s);
    return rc;
}

int scc_debug_multi_reach(scc_handle h, const int32_t* labels, const int32_t* sources, int32_t k, int32_t dir,
                          uint64_t* pairs, int64_t cap, int64_t* npairs, int64_t table_cap, void* stream) {
    if (!h || !labels || !sources || k < 1 || k > h->n || (dir != 0 && dir != 1) || !npairs || cap < 0 ||
        (cap > 0 && !pairs))
        return SCC_ERR_INVALID_ARG;
    if (table_cap != 0 && (table_cap < 1024 || (table_cap & (table_cap - 1)))) return SCC_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    h->last = s;
    const int32_t n = h->n;
    SCC_TRY(reserve_run_state(h, s));
    SCC_TRY(to_device(h->label, labels, sizeof(int32_t) * (size_t)n, s));
    SCC_TRY(to_device(h->tmp_a, sources, sizeof(int32_t) * (size_t)k, s));
    // keep only distinct sources in [0,n) whose label is active (finished
    // sources reach nothing); the engine wants valid ids
    SCC_CUDA(cudaMemsetAsync(h->flags, 0, 2 * sizeof(int), s));
    SCC_TRY(launch_filter_sources(h->tmp_a, k, n, h->label, h->sources, &h->flags[0], &h->flags[1], s));
    int hf[2];
    SCC_CUDA(cudaMemcpyAsync(hf, h->flags, sizeof(hf), cudaMemcpyDeviceToHost, s));
    SCC_CUDA(cudaStreamSynchronize(s));
    if (hf[1]) return SCC_ERR_INVALID_ARG;
    const int kk = hf[0];
    *npairs = 0;
    if (kk == 0) return SCC_OK;
    EngineOpts o = opts_of(h);
    int64_t tcap = table_cap ? table_cap : std::max<int64_t>(1024, pow2ceil(std::max<int64_t>((int64_t)(0.3 * n), 2 * kk)));
    const int d = dir;
    int resizes = 0;
    for (int attempt = 0;; ++attempt) {
        if (attempt > 40) return SCC_ERR_CAPACITY;
        SCC_TRY(reserve_table(h, d, tcap, s));
        SCC_CUDA(cudaMemsetAsync(h->tab[d], 0xff, (size_t)tcap * 8, s));
        long long max_ins = (long long)(0.6 * (double)tcap);
        SCC_TRY(engine_reserve(&h->eb64, 8, max_ins + (1 << 20), h->cfg.lambda, h->mt, h->di.num_sms, s));
        EngineRun r;
        int rc = run_pairs(d == 0 ? h->off : h->toff, d == 0 ? h->adj : h->tadj, n, h->label, h->sources, kk,
                           h->tab[d], tcap, max_ins, &h->eb64, o, &r, s);
        if (rc == SCC_ERR_CAPACITY || r.overflow) {
            tcap *= 2;
            ++resizes;
            continue;
        }
        SCC_TRY(rc);
        break;
    }
    h->stats.table_resizes = resizes;
    // gather the table
    Scratch tmp(s);
    unsigned long long* dout = nullptr;
    bool dev_out = is_device_ptr(pairs);
    SCC_CUDA(cudaMemsetAsync(h->counters + 2, 0, sizeof(unsigned long long), s));
    if (dev_out) {
        SCC_TRY(launch_table_gather(h->tab[d], tcap, reinterpret_cast<unsigned long long*>(pairs), cap, h->counters + 2, s));
    } else {
        SCC_TRY(tmp.alloc(&dout, (size_t)std::max<int64_t>(cap, 1)));
        SCC_TRY(launch_table_gather(h->tab[d], tcap, dout, cap, h->counters + 2, s));
    }
    unsigned long long tot = 0;
    SCC_CUDA(cudaMemcpyAsync(&tot, h->counters + 2, sizeof(tot), cudaMemcpyDeviceToHost, s));
    SCC_CUDA(cudaStreamSynchronize(s));
    if (!dev_out) {
        int64_t c = std::min<int64_t>((int64_t)tot, cap);
        SCC_CUDA(cudaMemcpyAsync(pairs, dout, sizeof(uint64_t) * (size_t)c, cudaMemcpyDeviceToHost, s));
        SCC_CUDA(cudaStreamSynchronize(s));
    }
    *npairs = (int64_t)tot;
    return SCC_OK;
}

int64_t scc_debug_launch_count(void) { return launch_count(); }

int scc_debug_barrier_timeout(int32_t absent_block, int64_t limit_ns, int32_t* n_arrived, void* stream) {
    if (!n_arrived || limit_ns < 1000 || limit_ns > 1000000000ll || absent_block < -1) return SCC_ERR_INVALID_ARG;
    int c = 0;
    const int rc = run_barrier_probe(absent_block, limit_ns, &c, (cudaStream_t)stream);
    *n_arrived = c;
    return rc;
}

int scc_debug_hashbag(const int32_t* items, int64_t count, int32_t lambda, int32_t sigma, int32_t* out, int64_t* nout,
                      int32_t* chunks, void* stream) {
    if (!items || !out || !nout || count < 1 || lambda < 1024 || (lambda & (lambda - 1)) || sigma < 1)
        return SCC_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    Scratch tmp(s);
    int32_t *din = nullptr, *dout = nullptr;
    SCC_TRY(tmp.alloc(&din, (size_t)count));
    SCC_TRY(tmp.alloc(&dout, (size_t)count));
    SCC_TRY(to_device(din, items, sizeof(int32_t) * (size_t)count, s));
    int64_t got = 0;
    int ch = 0;
    SCC_TRY(run_bag_only(din, count, lambda, sigma, dout, &got, &ch, s));
    if (got > count) return SCC_ERR_INTERNAL;
    SCC_TRY(from_device(out, dout, sizeof(int32_t) * (size_t)got, s));
    SCC_CUDA(cudaStreamSynchronize(s));
    *nout = got;
    if (chunks) *chunks = ch;
    return SCC_OK;
}

int scc_debug_pair_table(const uint64_t* keys, int64_t count, int64_t init_cap, uint64_t* out, int64_t* nout,
                         int32_t* resizes, void* stream) {
    if (!keys || !out || !nout || count < 1 || init_cap < 1024 || (init_cap & (init_cap - 1)))
        return SCC_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long *dk = nullptr, *tab = nullptr, *cnt = nullptr, *dout = nullptr;
    int* ovf = nullptr;
    Scratch tmp(s);
    SCC_TRY(tmp.alloc(&dk, (size_t)count));
    SCC_TRY(tmp.alloc(&cnt, 2));
    SCC_TRY(tmp.alloc(&ovf, 1));
    SCC_TRY(tmp.alloc(&dout, (size_t)count));
    SCC_TRY(to_device(dk, keys, sizeof(uint64_t) * (size_t)count, s));
    // insert in slices; when a slice pushes the load over 1/2 (or a probe runs
    // too far) the table doubles and every key is rehashed (Sec. 4.5 regrowth)
    int64_t cap = init_cap;
    SCC_TRY(tmp.alloc(&tab, (size_t)cap));
    SCC_CUDA(cudaMemsetAsync(tab, 0xff, (size_t)cap * 8, s));
    SCC_CUDA(cudaMemsetAsync(cnt, 0, 16, s));
    int nres = 0;
    const int64_t slice = 4096;
    for (int64_t b = 0; b < count;) {
        int64_t c = std::min(slice, count - b);
        SCC_CUDA(cudaMemsetAsync(ovf, 0, sizeof(int), s));
        SCC_TRY(launch_table_insert(dk + b, c, tab, cap, ovf, cnt, s));
        unsigned long long hc = 0;
        int hov = 0;
        SCC_CUDA(cudaMemcpyAsync(&hc, cnt, 8, cudaMemcpyDeviceToHost, s));
        SCC_CUDA(cudaMemcpyAsync(&hov, ovf, 4, cudaMemcpyDeviceToHost, s));
        SCC_CUDA(cudaStreamSynchronize(s));
        if (hov || 2 * (int64_t)hc > cap) {
            unsigned long long* t2 = nullptr;
            SCC_TRY(tmp.alloc(&t2, (size_t)cap * 2));
            SCC_CUDA(cudaMemsetAsync(t2, 0xff, (size_t)cap * 16, s));
            SCC_CUDA(cudaMemsetAsync(ovf, 0, sizeof(int), s));
            SCC_TRY(launch_table_rehash(tab, cap, t2, cap * 2, ovf, s));
            tmp.release(tab);
            tab = t2;
            cap *= 2;
            ++nres;
            if (hov) {  // keys of the slice may be missing: insert the slice again
                SCC_CUDA(cudaMemsetAsync(cnt, 0, 8, s));
                continue;
            }
        }
        b += c;
    }
    SCC_CUDA(cudaMemsetAsync(cnt + 1, 0, 8, s));
    SCC_TRY(launch_table_gather(tab, cap, dout, count, cnt + 1, s));
    unsigned long long tot = 0;
    SCC_CUDA(cudaMemcpyAsync(&tot, cnt + 1, 8, cudaMemcpyDeviceToHost, s));
    SCC_CUDA(cudaStreamSynchronize(s));
    if ((int64_t)tot > count) return SCC_ERR_INTERNAL;
    SCC_TRY(from_device(out, dout, sizeof(uint64_t) * (size_t)tot, s));
    SCC_CUDA(cudaStreamSynchronize(s));
    *nout = (int64_t)tot;
    if (resizes) *resizes = nres;
    return SCC_OK;
}

}  // extern "C"
