// Serving SCC and reachability requests with continuous batching (host runtime).
//
// One server thread per handle works in dispatch units (include/scc_serve.h):
// it admits pending requests under the memory cap and starts their uploads on
// a copy stream, then runs the unit of the oldest admitted request on the
// compute stream -- all admitted small SCC requests in one launch of the
// batched kernel (batch.cu), the reachability queries on one resident graph and
// direction in one reach_multi launch, or one large SCC request on the
// full-GPU path -- and completes its requests. Requests that arrive while a
// unit runs are admitted when it ends. Kernels of different units never run at
// the same time (the full-GPU searches are cooperative launches that need every
// SM); uploads of admitted requests overlap the unit that is computing.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "../../include/scc.h"
#include "../../include/scc_serve.h"
#include "common.cuh"
#include "internal.h"

namespace scc {
namespace {

using Clock = std::chrono::steady_clock;

// Sources of one merged reach launch (two mask words per vertex above 64).
constexpr int kMaxMergedSources = 128;

// out[v] = the k <= 64 bits starting at bit `shift` of vertex v's mask, which
// is `words` (1 or 2) 64-bit words, the first holding bits 0..63 (one query's
// share of a merged reach launch)
__global__ void k_split_bits(const unsigned long long* __restrict__ mask, int words, int32_t n, int shift, int k,
                             unsigned long long* __restrict__ out) {
    const unsigned long long lm = k >= 64 ? ~0ull : ((1ull << k) - 1ull);
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long lo = mask[words * v], hi = words > 1 ? mask[words * v + 1] : 0ull;
        unsigned long long x;
        if (shift == 0) x = lo;
        else if (shift < 64) x = (lo >> shift) | (hi << (64 - shift));
        else x = hi >> (shift - 64);
        out[v] = x & lm;
    }
}

// ---------------------------------------------------------------- policy --
// The server's two scheduling decisions as functions of the queue alone, so
// that the host can test them (scc_debug_serve_admission, _unit).

// Admission in arrival order over `count` pending requests: request i is
// admitted when fits(i) holds (fits reserves its bytes); the first request
// that does not fit lets later ones pass while waited_ms(i) <= max_bypass_ms,
// and ends the pass once it has waited longer. Appends the admitted indices,
// in increasing order, to `take`.
template <class Fits, class Waited>
void admission_pass(size_t count, double max_bypass_ms, Fits fits, Waited waited_ms, std::vector<size_t>& take) {
    bool blocked = false;
    for (size_t i = 0; i < count; ++i) {
        if (fits(i)) {
            take.push_back(i);
            continue;
        }
        if (!blocked && waited_ms(i) > max_bypass_ms) break;  // no more passing
        blocked = true;
    }
}

struct UnitItem {
    int kind;       // 0 SCC, 1 reachability
    bool small;     // an SCC request the batched kernel takes
    int32_t graph;  // reachability: resident graph and direction
    int32_t dir;
    int32_t nsrc;   // reachability: sources
};

// The unit of the oldest admitted request q[0], as increasing indices into q:
// a reachability query with every later query on the same graph and direction
// while the sources stay within kMaxMergedSources (merge_reach; otherwise q[0]
// alone); a small SCC request with the next small ones, batch_graphs at most,
// when at least batch_min small SCC requests are admitted (with fewer, q[0]
// alone: it runs on the full-GPU path, which is faster for one graph than one
// block of the batched kernel); a larger SCC request alone.
std::vector<size_t> unit_select(const std::vector<UnitItem>& q, bool merge_reach, int batch_graphs, int batch_min) {
    std::vector<size_t> u;
    if (q.empty()) return u;
    const UnitItem& h = q[0];
    if (h.kind == 1) {
        int k = 0;
        for (size_t i = 0; i < q.size(); ++i) {
            const UnitItem& r = q[i];
            const bool same = r.kind == 1 && r.graph == h.graph && r.dir == h.dir;
            if (same && (u.empty() || (merge_reach && k + r.nsrc <= kMaxMergedSources))) {
                k += r.nsrc;
                u.push_back(i);
            }
            if (!merge_reach) break;
        }
    } else if (h.small) {
        int smalls = 0;
        for (const UnitItem& r : q) smalls += r.kind == 0 && r.small;
        if (smalls < std::max(1, batch_min)) {
            u.push_back(0);
        } else {
            for (size_t i = 0; i < q.size() && (int)u.size() < std::max(1, batch_graphs); ++i)
                if (q[i].kind == 0 && q[i].small) u.push_back(i);
        }
    } else {
        u.push_back(0);
    }
    return u;
}

struct Request {
    int64_t id = 0;
    int kind = 0;  // 0 SCC, 1 reachability
    // SCC
    int32_t n = 0;
    int64_t m = 0;
    const int32_t* off_h = nullptr;
    const int32_t* adj_h = nullptr;
    int32_t* lab_h = nullptr;
    // reachability
    int32_t graph = -1;
    std::vector<int32_t> src;
    int32_t dir = 0;
    uint64_t* out_h = nullptr;
    // runtime
    Clock::time_point t_sub;
    size_t mem = 0;
    int32_t* off_d = nullptr;  // uploaded input (SCC, prefetch)
    int32_t* adj_d = nullptr;
    cudaEvent_t up = nullptr;
};
using ReqPtr = std::shared_ptr<Request>;

struct Resident {
    scc_graph* g = nullptr;
    int32_t n = 0;
    int64_t m = 0;
    size_t bytes = 0;
    int64_t pending = 0;
};

// Device bytes a request may hold while admitted (upper estimates). A full-GPU
// SCC holds its copy of the input, G^T and the transpose's staging, the run
// state (labels, maxima, bitmaps), the pair tables and the hash bags.
size_t plain_bytes(int64_t n, int64_t m) { return (size_t)(18 * m + 360 * n) + ((size_t)64 << 20); }
size_t batched_bytes(int64_t n, int64_t m) { return (size_t)(8 * (n + 1) + 4 * m + 4 * n) + 4096; }
size_t reach_bytes(int64_t n) { return (size_t)(16 * n) + 4096; }

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

double percentile(std::vector<double> v, double q) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = q * (double)(v.size() - 1);
    const size_t i = (size_t)pos;
    const double f = pos - (double)i;
    return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
}

}  // namespace
}  // namespace scc

using namespace scc;

struct scc_server {
    scc_server_config cfg;
    int dev = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<ReqPtr> intake;
    std::unordered_map<int64_t, std::pair<int, double>> done;  // completed, not yet waited for
    std::unordered_set<int64_t> inflight;                       // submitted, not yet completed
    int64_t next_id = 1;
    int64_t outstanding = 0;
    bool stop = false;
    std::thread th;
    // owned by the server thread
    std::deque<ReqPtr> pending, admitted;
    cudaStream_t cs = nullptr, us = nullptr;
    BatchRunner* runner = nullptr;
    // resident graphs (guarded by mu; the map keeps element addresses)
    std::map<int32_t, Resident> graphs;
    int32_t next_graph = 0;
    // memory and statistics (guarded by mu)
    int64_t mem_fixed = 0, mem_in_use = 0, mem_peak = 0;
    int32_t admitted_now = 0;
    scc_server_stats st;
    std::vector<double> lat_all, lat_scc, lat_reach;
};

namespace scc {
namespace {

void finish(scc_server* S, Request& r, int status) {
    const auto t = Clock::now();
    const double lat = ms_between(r.t_sub, t);
    if (r.up) cudaEventDestroy(r.up);
    r.up = nullptr;
    std::lock_guard<std::mutex> lk(S->mu);
    S->done[r.id] = {status, lat};
    S->inflight.erase(r.id);
    S->outstanding--;
    S->mem_in_use -= (int64_t)r.mem;
    S->admitted_now--;
    S->st.completed++;
    if (status != SCC_OK) S->st.failed++;
    S->lat_all.push_back(lat);
    (r.kind == 0 ? S->lat_scc : S->lat_reach).push_back(lat);
    if (r.kind == 1) {
        auto it = S->graphs.find(r.graph);
        if (it != S->graphs.end()) it->second.pending--;
    }
    S->cv_done.notify_all();
}

void release_inputs(scc_server* S, Request& r) {
    dfree(r.off_d, S->cs);
    dfree(r.adj_d, S->cs);
    r.off_d = r.adj_d = nullptr;
}

bool is_small(const scc_server* S, const Request& r) {
    return S->runner && r.kind == 0 && S->cfg.batch_vertices > 0 && r.n <= S->cfg.batch_vertices &&
           r.m <= 32ll * S->cfg.batch_vertices && batch_runner_fits(S->runner, r.n, r.m);
}

size_t request_bytes(scc_server* S, const Request& r) {
    if (r.kind == 1) {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->graphs.find(r.graph);
        return reach_bytes(it == S->graphs.end() ? 0 : it->second.n);
    }
    return is_small(S, r) ? batched_bytes(r.n, r.m) : plain_bytes(r.n, r.m);
}

// Start the upload of an SCC request's input on the copy stream.
int upload(scc_server* S, Request& r) {
    SCC_TRY(dalloc_t(&r.off_d, (size_t)r.n + 1, S->us));
    SCC_TRY(dalloc_t(&r.adj_d, (size_t)std::max<int64_t>(r.m, 1), S->us));
    SCC_CUDA(cudaMemcpyAsync(r.off_d, r.off_h, sizeof(int32_t) * ((size_t)r.n + 1), cudaMemcpyDefault, S->us));
    if (r.m > 0)
        SCC_CUDA(cudaMemcpyAsync(r.adj_d, r.adj_h, sizeof(int32_t) * (size_t)r.m, cudaMemcpyDefault, S->us));
    SCC_CUDA(cudaEventCreateWithFlags(&r.up, cudaEventDisableTiming));
    SCC_CUDA(cudaEventRecord(r.up, S->us));
    return SCC_OK;
}

// Moves q[idx[0]], q[idx[1]], ... (increasing indices) into out, in that
// order, and erases them from q.
void take_indices(std::deque<ReqPtr>& q, const std::vector<size_t>& idx, std::vector<ReqPtr>& out) {
    std::deque<ReqPtr> rest;
    size_t j = 0;
    for (size_t i = 0; i < q.size(); ++i) {
        if (j < idx.size() && idx[j] == i) {
            out.push_back(std::move(q[i]));
            ++j;
        } else {
            rest.push_back(std::move(q[i]));
        }
    }
    q.swap(rest);
}

// Admission in arrival order; a request that does not fit waits while later
// ones that fit pass it, until it has waited max_bypass_ms. The admitted
// requests' uploads start on the copy stream in arrival order.
void admit(scc_server* S) {
    const auto now = Clock::now();
    std::vector<size_t> take;
    admission_pass(
        S->pending.size(), S->cfg.max_bypass_ms,
        [&](size_t i) {
            Request& r = *S->pending[i];
            const size_t need = request_bytes(S, r);
            std::lock_guard<std::mutex> lk(S->mu);
            if (S->mem_in_use + (int64_t)need > S->cfg.mem_cap_bytes) return false;
            S->mem_in_use += (int64_t)need;
            S->mem_peak = std::max(S->mem_peak, S->mem_in_use);
            S->admitted_now++;
            S->st.max_admitted = std::max(S->st.max_admitted, S->admitted_now);
            r.mem = need;
            return true;
        },
        [&](size_t i) { return ms_between(S->pending[i]->t_sub, now); }, take);
    std::vector<ReqPtr> adm;
    take_indices(S->pending, take, adm);
    for (auto& p : adm) {
        if (p->kind == 0 && S->cfg.prefetch) {
            const int rc = upload(S, *p);
            if (rc != SCC_OK) {
                release_inputs(S, *p);
                finish(S, *p, rc);
                continue;
            }
        }
        S->admitted.push_back(p);
    }
}

// ---------------------------------------------------------------- units --
void run_reach(scc_server* S, std::vector<ReqPtr>& u) {
    Resident* R = nullptr;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->graphs.find(u[0]->graph);
        if (it != S->graphs.end()) R = &it->second;
    }
    if (!R) {
        for (auto& r : u) finish(S, *r, SCC_ERR_INVALID_ARG);
        return;
    }
    const int32_t n = R->n;
    std::vector<int32_t> all;
    for (auto& r : u) all.insert(all.end(), r->src.begin(), r->src.end());
    const int32_t K = (int32_t)all.size();
    const int words = K > 64 ? 2 : 1;  // above 64 sources: the two-word search
    int32_t* src_d = nullptr;
    unsigned long long* mask_d = nullptr;
    unsigned long long* part_d = nullptr;
    int rc = dalloc_t(&src_d, (size_t)K, S->cs);
    if (rc == SCC_OK) rc = dalloc_t(&mask_d, (size_t)words * std::max(n, 1), S->cs);
    if (rc == SCC_OK && u.size() > 1) rc = dalloc_t(&part_d, (size_t)std::max(n, 1), S->cs);
    if (rc == SCC_OK) rc = cuda_err(cudaMemcpyAsync(src_d, all.data(), sizeof(int32_t) * K, cudaMemcpyHostToDevice, S->cs));
    if (rc == SCC_OK)
        rc = words == 1 ? reach_multi(R->g, src_d, K, u[0]->dir, reinterpret_cast<uint64_t*>(mask_d), S->cs)
                        : reach_multi_wide(R->g, src_d, K, u[0]->dir, mask_d, S->cs);
    if (rc == SCC_OK) {
        int shift = 0;
        for (auto& r : u) {
            const int k = (int)r->src.size();
            if (u.size() == 1) {
                rc = cuda_err(cudaMemcpyAsync(r->out_h, mask_d, sizeof(uint64_t) * (size_t)n, cudaMemcpyDefault,
                                              S->cs));
            } else {
                k_split_bits<<<std::max(1, std::min(4096, (n + 255) / 256)), 256, 0, S->cs>>>(mask_d, words, n, shift,
                                                                                                k, part_d);
                count_launch();
                rc = cuda_err(cudaGetLastError());
                if (rc == SCC_OK)
                    rc = cuda_err(cudaMemcpyAsync(r->out_h, part_d, sizeof(uint64_t) * (size_t)n, cudaMemcpyDefault,
                                                  S->cs));
                // the next split reuses part_d: let this copy finish first
                if (rc == SCC_OK) rc = cuda_err(cudaStreamSynchronize(S->cs));
            }
            if (rc != SCC_OK) break;
            shift += k;
        }
    }
    if (rc == SCC_OK) rc = cuda_err(cudaStreamSynchronize(S->cs));
    dfree(src_d, S->cs);
    dfree(mask_d, S->cs);
    dfree(part_d, S->cs);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->st.reach_launches++;
        if (u.size() > 1) S->st.reach_shared += (int64_t)u.size();
    }
    for (auto& r : u) finish(S, *r, rc);
}

int plain_one(scc_server* S, Request& r) {
    const int32_t* off = r.off_d ? r.off_d : r.off_h;
    const int32_t* adj = r.adj_d ? r.adj_d : r.adj_h;
    if (r.up) SCC_CUDA(cudaStreamWaitEvent(S->cs, r.up, 0));
    scc_handle g = nullptr;
    SCC_TRY(scc_graph_create(r.n, r.m, off, adj, S->cs, &g));
    int rc = scc_run(g, r.lab_h, S->cs);
    if (rc == SCC_OK) rc = cuda_err(cudaStreamSynchronize(S->cs));
    const int rc2 = scc_graph_destroy(g);
    return rc != SCC_OK ? rc : rc2;
}

void run_plain(scc_server* S, Request& r) {
    const int rc = plain_one(S, r);
    release_inputs(S, r);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->st.plain_scc++;
    }
    finish(S, r, rc);
}

void run_batched(scc_server* S, std::vector<ReqPtr>& u) {
    const int32_t G = (int32_t)u.size();
    std::vector<long long> vb(G + 1, 0), eb(G + 1, 0);
    for (int32_t g = 0; g < G; ++g) {
        vb[g + 1] = vb[g] + u[g]->n;
        eb[g + 1] = eb[g] + u[g]->m;
    }
    long long *vb_d = nullptr, *eb_d = nullptr;
    int32_t *off_d = nullptr, *adj_d = nullptr, *ord_d = nullptr, *lab_d = nullptr;
    int* err_h = nullptr;
    int* bad_d = nullptr;
    std::vector<int> bad(G, 0);
    int rc = dalloc_t(&vb_d, (size_t)G + 1, S->cs);
    if (rc == SCC_OK) rc = dalloc_t(&eb_d, (size_t)G + 1, S->cs);
    if (rc == SCC_OK) rc = dalloc_t(&off_d, (size_t)(vb[G] + G) + 1, S->cs);
    if (rc == SCC_OK) rc = dalloc_t(&adj_d, (size_t)eb[G] + 1, S->cs);
    if (rc == SCC_OK) rc = dalloc_t(&ord_d, (size_t)G, S->cs);
    if (rc == SCC_OK) rc = dalloc_t(&lab_d, (size_t)vb[G] + 1, S->cs);
    if (rc == SCC_OK) rc = dalloc_t(&bad_d, (size_t)G, S->cs);
    if (rc == SCC_OK) rc = cuda_err(cudaMallocHost(&err_h, sizeof(int)));
    if (rc == SCC_OK) rc = cuda_err(cudaMemcpyAsync(vb_d, vb.data(), 8 * ((size_t)G + 1), cudaMemcpyHostToDevice, S->cs));
    if (rc == SCC_OK) rc = cuda_err(cudaMemcpyAsync(eb_d, eb.data(), 8 * ((size_t)G + 1), cudaMemcpyHostToDevice, S->cs));
    // pack the inputs (uploaded at admission, or straight from the host)
    for (int32_t g = 0; g < G && rc == SCC_OK; ++g) {
        Request& r = *u[g];
        if (r.up) rc = cuda_err(cudaStreamWaitEvent(S->cs, r.up, 0));
        const int32_t* so = r.off_d ? r.off_d : r.off_h;
        const int32_t* sa = r.adj_d ? r.adj_d : r.adj_h;
        if (rc == SCC_OK)
            rc = cuda_err(cudaMemcpyAsync(off_d + vb[g] + g, so, 4 * ((size_t)r.n + 1), cudaMemcpyDefault, S->cs));
        if (rc == SCC_OK && r.m > 0)
            rc = cuda_err(cudaMemcpyAsync(adj_d + eb[g], sa, 4 * (size_t)r.m, cudaMemcpyDefault, S->cs));
    }
    // malformed graphs are left out of the launch (and fail on their own)
    if (rc == SCC_OK) rc = batch_validate_each(G, vb_d, eb_d, off_d, adj_d, bad_d, S->cs);
    if (rc == SCC_OK) rc = cuda_err(cudaMemcpyAsync(bad.data(), bad_d, sizeof(int) * G, cudaMemcpyDeviceToHost, S->cs));
    if (rc == SCC_OK) rc = cuda_err(cudaStreamSynchronize(S->cs));
    std::vector<int32_t> order;
    for (int32_t g = 0; g < G; ++g)
        if (!bad[g]) order.push_back(g);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
        return (u[a]->m + u[a]->n) > (u[b]->m + u[b]->n);
    });
    const int32_t nvalid = (int32_t)order.size();
    if (rc == SCC_OK && nvalid > 0)
        rc = cuda_err(cudaMemcpyAsync(ord_d, order.data(), 4 * (size_t)nvalid, cudaMemcpyHostToDevice, S->cs));
    if (rc == SCC_OK && nvalid > 0)
        rc = batch_runner_enqueue(S->runner, G, vb_d, eb_d, off_d, adj_d, ord_d, nvalid, lab_d, S->cs);
    if (rc == SCC_OK && nvalid == 0) *err_h = SCC_OK;
    else if (rc == SCC_OK)
        rc = cuda_err(cudaMemcpyAsync(err_h, batch_runner_err(S->runner), sizeof(int), cudaMemcpyDeviceToHost, S->cs));
    for (int32_t g = 0; g < G && rc == SCC_OK; ++g)
        if (u[g]->n > 0 && !bad[g])
            rc = cuda_err(cudaMemcpyAsync(u[g]->lab_h, lab_d + vb[g], 4 * (size_t)u[g]->n, cudaMemcpyDefault, S->cs));
    if (rc == SCC_OK) rc = cuda_err(cudaStreamSynchronize(S->cs));
    const int kerr = (rc == SCC_OK && err_h) ? *err_h : SCC_OK;
    dfree(vb_d, S->cs);
    dfree(eb_d, S->cs);
    dfree(off_d, S->cs);
    dfree(adj_d, S->cs);
    dfree(ord_d, S->cs);
    dfree(lab_d, S->cs);
    dfree(bad_d, S->cs);
    if (err_h) cudaFreeHost(err_h);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->st.batched_launches++;
        S->st.batched_graphs += G;
    }
    for (int32_t g = 0; g < G; ++g) {
        auto& r = u[g];
        int st = rc;
        if (st == SCC_OK && bad[g]) st = SCC_ERR_INVALID_ARG;
        // the batched kernel could not finish (its working memory ran out for
        // one of them): serve every request of the launch on the full-GPU path
        if (st == SCC_OK && kerr != SCC_OK && !bad[g]) st = plain_one(S, *r);
        release_inputs(S, *r);
        finish(S, *r, st);
    }
}

// The unit of the oldest admitted request, run to completion.
void run_unit(scc_server* S) {
    std::vector<UnitItem> q;
    q.reserve(S->admitted.size());
    for (const ReqPtr& r : S->admitted)
        q.push_back({r->kind, is_small(S, *r), r->graph, r->dir, (int32_t)r->src.size()});
    const std::vector<size_t> pick =
        unit_select(q, S->cfg.merge_reach != 0, S->cfg.batch_graphs, S->cfg.batch_min);
    std::vector<ReqPtr> u;
    take_indices(S->admitted, pick, u);
    const auto t0 = Clock::now();
    double* busy = nullptr;
    if (q[0].kind == 1) {
        run_reach(S, u);
        busy = &S->st.busy_reach_ms;
    } else if (q[0].small && (int)pick.size() >= std::max(1, S->cfg.batch_min)) {
        run_batched(S, u);
        busy = &S->st.busy_batched_ms;
    } else {
        run_plain(S, *u[0]);
        busy = &S->st.busy_plain_ms;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    S->st.units++;
    *busy += ms_between(t0, Clock::now());
}

void server_main(scc_server* S) {
    cudaSetDevice(S->dev);
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] {
                return S->stop || !S->intake.empty() || !S->pending.empty() || !S->admitted.empty();
            });
            if (S->stop && S->intake.empty() && S->pending.empty() && S->admitted.empty()) break;
            while (!S->intake.empty()) {
                S->pending.push_back(S->intake.front());
                S->intake.pop_front();
            }
        }
        admit(S);
        if (S->admitted.empty()) {
            // nothing admitted and nothing holds memory that could be freed: the
            // oldest pending request can never fit
            if (!S->pending.empty()) {
                ReqPtr r = S->pending.front();
                S->pending.pop_front();
                {
                    std::lock_guard<std::mutex> lk(S->mu);
                    S->admitted_now++;
                }
                finish(S, *r, SCC_ERR_OOM);
            }
            continue;
        }
        run_unit(S);
    }
}

int submit(scc_server* S, ReqPtr r, int64_t* id) {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) return SCC_ERR_INVALID_ARG;
    r->id = S->next_id++;
    S->inflight.insert(r->id);
    r->t_sub = Clock::now();
    S->outstanding++;
    S->st.submitted++;
    (r->kind == 0 ? S->st.scc_requests : S->st.reach_requests)++;
    S->intake.push_back(r);
    *id = r->id;
    S->cv_work.notify_one();
    return SCC_OK;
}

}  // namespace
}  // namespace scc

extern "C" {

SCC_API int scc_server_config_default(scc_server_config* cfg) {
    if (!cfg) return SCC_ERR_INVALID_ARG;
    cfg->mem_cap_bytes = 120000000000ll;
    cfg->batch_vertices = 262144;
    cfg->batch_graphs = 512;
    cfg->merge_reach = 1;
    cfg->prefetch = 1;
    cfg->max_bypass_ms = 50.0;
    cfg->batch_min = 4;
    return SCC_OK;
}

SCC_API int scc_server_create(const scc_server_config* cfg, scc_server_handle* out) {
    if (!out) return SCC_ERR_INVALID_ARG;
    *out = nullptr;
    scc_server_config c;
    if (cfg) c = *cfg;
    else scc_server_config_default(&c);
    if (c.mem_cap_bytes <= 0 || c.batch_vertices < 0 || c.batch_graphs < 1 || !(c.max_bypass_ms >= 0) ||
        c.batch_min < 1 || c.batch_min > c.batch_graphs)
        return SCC_ERR_INVALID_ARG;
    scc_server* S = new (std::nothrow) scc_server();
    if (!S) return SCC_ERR_OOM;
    S->cfg = c;
    memset(&S->st, 0, sizeof(S->st));
    auto fail = [&](int rc) {
        if (S->runner) batch_runner_destroy(S->runner, 0);
        if (S->cs) cudaStreamDestroy(S->cs);
        if (S->us) cudaStreamDestroy(S->us);
        delete S;
        return rc;
    };
    if (cudaGetDevice(&S->dev) != cudaSuccess) return fail(SCC_ERR_CUDA);
    if (cudaStreamCreateWithFlags(&S->cs, cudaStreamNonBlocking) != cudaSuccess) return fail(SCC_ERR_CUDA);
    if (cudaStreamCreateWithFlags(&S->us, cudaStreamNonBlocking) != cudaSuccess) return fail(SCC_ERR_CUDA);
    if (c.batch_vertices > 0) {
        // working memory of the batched kernel for graphs up to batch_vertices,
        // at most a quarter of the cap
        const int rc = batch_runner_create(nullptr, c.batch_vertices, 32ll * c.batch_vertices, c.batch_graphs,
                                           (size_t)(c.mem_cap_bytes / 4), S->cs, &S->runner);
        if (rc != SCC_OK) return fail(rc);
        if (cudaStreamSynchronize(S->cs) != cudaSuccess) return fail(SCC_ERR_CUDA);
        S->mem_fixed = (int64_t)batch_runner_bytes(S->runner);
    }
    S->mem_in_use = S->mem_fixed;
    S->mem_peak = S->mem_in_use;
    S->th = std::thread(server_main, S);
    *out = S;
    return SCC_OK;
}

SCC_API int scc_server_destroy(scc_server_handle S) {
    if (!S) return SCC_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->cv_work.notify_all();
    }
    if (S->th.joinable()) S->th.join();
    for (auto& kv : S->graphs) scc_graph_destroy(kv.second.g);
    S->graphs.clear();
    if (S->runner) batch_runner_destroy(S->runner, S->cs);
    cudaStreamSynchronize(S->cs);
    cudaStreamSynchronize(S->us);
    cudaStreamDestroy(S->cs);
    cudaStreamDestroy(S->us);
    delete S;
    return SCC_OK;
}

SCC_API int scc_server_add_graph(scc_server_handle S, int32_t n, int64_t m, const int32_t* offsets,
                                 const int32_t* targets, int32_t* graph_id) {
    if (!S || !graph_id || n < 0 || m < 0 || m > INT32_MAX) return SCC_ERR_INVALID_ARG;
    const size_t bytes = plain_bytes(n, m);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->mem_in_use + (int64_t)bytes > S->cfg.mem_cap_bytes) return SCC_ERR_OOM;
        S->mem_in_use += (int64_t)bytes;  // reserved while the graph is built
        S->mem_fixed += (int64_t)bytes;
        S->mem_peak = std::max(S->mem_peak, S->mem_in_use);
    }
    cudaStream_t s = nullptr;
    int rc = cuda_err(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    scc_handle g = nullptr;
    if (rc == SCC_OK) rc = scc_graph_create(n, m, offsets, targets, s, &g);
    if (rc == SCC_OK) rc = cuda_err(cudaStreamSynchronize(s));
    if (s) cudaStreamDestroy(s);
    std::lock_guard<std::mutex> lk(S->mu);
    if (rc != SCC_OK) {
        if (g) scc_graph_destroy(g);
        S->mem_in_use -= (int64_t)bytes;
        S->mem_fixed -= (int64_t)bytes;
        return rc;
    }
    Resident R;
    R.g = g;
    R.n = n;
    R.m = m;
    R.bytes = bytes;
    const int32_t id = S->next_graph++;
    S->graphs[id] = R;
    *graph_id = id;
    return SCC_OK;
}

SCC_API int scc_server_remove_graph(scc_server_handle S, int32_t graph_id) {
    if (!S) return SCC_ERR_INVALID_ARG;
    scc_graph* g = nullptr;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->graphs.find(graph_id);
        if (it == S->graphs.end() || it->second.pending > 0) return SCC_ERR_INVALID_ARG;
        g = it->second.g;
        S->mem_in_use -= (int64_t)it->second.bytes;
        S->mem_fixed -= (int64_t)it->second.bytes;
        S->graphs.erase(it);
    }
    return scc_graph_destroy(g);
}

SCC_API int scc_server_submit_scc(scc_server_handle S, int32_t n, int64_t m, const int32_t* offsets,
                                  const int32_t* targets, int32_t* labels_out, int64_t* request_id) {
    if (!S || !request_id || n < 0 || m < 0 || m > INT32_MAX || !offsets || (m > 0 && !targets) ||
        (n > 0 && !labels_out))
        return SCC_ERR_INVALID_ARG;
    auto r = std::make_shared<Request>();
    r->kind = 0;
    r->n = n;
    r->m = m;
    r->off_h = offsets;
    r->adj_h = targets;
    r->lab_h = labels_out;
    {
        // a request that could not fit even alone is refused at once
        const size_t need = is_small(S, *r) ? batched_bytes(n, m) : plain_bytes(n, m);
        std::lock_guard<std::mutex> lk(S->mu);
        if ((int64_t)need + S->mem_fixed > S->cfg.mem_cap_bytes) return SCC_ERR_OOM;
    }
    return submit(S, r, request_id);
}

SCC_API int scc_server_submit_reach(scc_server_handle S, int32_t graph_id, const int32_t* sources, int32_t k,
                                    int32_t dir, uint64_t* out, int64_t* request_id) {
    if (!S || !request_id || !sources || !out || k < 1 || k > 64 || (dir != 0 && dir != 1))
        return SCC_ERR_INVALID_ARG;
    auto r = std::make_shared<Request>();
    r->kind = 1;
    r->graph = graph_id;
    r->src.assign(sources, sources + k);
    r->dir = dir;
    r->out_h = out;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->graphs.find(graph_id);
        if (it == S->graphs.end()) return SCC_ERR_INVALID_ARG;
        for (int32_t s : r->src)
            if (s < 0 || s >= it->second.n) return SCC_ERR_INVALID_ARG;
        it->second.pending++;
    }
    const int rc = submit(S, r, request_id);
    if (rc != SCC_OK) {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->graphs.find(graph_id);
        if (it != S->graphs.end()) it->second.pending--;
    }
    return rc;
}

SCC_API int scc_server_wait(scc_server_handle S, int64_t request_id, int32_t* status, double* latency_ms) {
    if (!S) return SCC_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    if (request_id <= 0 || request_id >= S->next_id) return SCC_ERR_INVALID_ARG;
    S->cv_done.wait(lk, [&] { return S->done.count(request_id) > 0 || S->inflight.count(request_id) == 0; });
    auto it = S->done.find(request_id);
    if (it == S->done.end()) return SCC_ERR_INVALID_ARG;  // collected by an earlier wait
    if (status) *status = it->second.first;
    if (latency_ms) *latency_ms = it->second.second;
    S->done.erase(it);
    return SCC_OK;
}

SCC_API int scc_server_drain(scc_server_handle S) {
    if (!S) return SCC_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    S->cv_done.wait(lk, [&] { return S->outstanding == 0; });
    return SCC_OK;
}

SCC_API int scc_server_get_stats(scc_server_handle S, scc_server_stats* out) {
    if (!S || !out) return SCC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    *out = S->st;
    out->mem_in_use = S->mem_in_use;
    out->mem_peak = S->mem_peak;
    out->mem_cap = S->cfg.mem_cap_bytes;
    out->resident_graphs = (int32_t)S->graphs.size();
    out->p50_ms = percentile(S->lat_all, 0.50);
    out->p99_ms = percentile(S->lat_all, 0.99);
    out->scc_p50_ms = percentile(S->lat_scc, 0.50);
    out->scc_p99_ms = percentile(S->lat_scc, 0.99);
    out->reach_p50_ms = percentile(S->lat_reach, 0.50);
    out->reach_p99_ms = percentile(S->lat_reach, 0.99);
    return SCC_OK;
}

SCC_API int scc_server_reset_stats(scc_server_handle S) {
    if (!S) return SCC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    memset(&S->st, 0, sizeof(S->st));
    S->lat_all.clear();
    S->lat_scc.clear();
    S->lat_reach.clear();
    S->mem_peak = S->mem_in_use;
    return SCC_OK;
}


SCC_API int scc_debug_serve_admission(int32_t count, const int64_t* need, const double* waited_ms, int64_t in_use,
                                      int64_t cap, double max_bypass_ms, int32_t* admitted, int32_t* nadmitted) {
    if (count < 0 || !nadmitted || (count > 0 && (!need || !waited_ms || !admitted)) || !(max_bypass_ms >= 0))
        return SCC_ERR_INVALID_ARG;
    for (int32_t i = 0; i < count; ++i)
        if (need[i] < 0) return SCC_ERR_INVALID_ARG;
    std::vector<size_t> take;
    admission_pass(
        (size_t)count, max_bypass_ms,
        [&](size_t i) {
            if (in_use + need[i] > cap) return false;
            in_use += need[i];
            return true;
        },
        [&](size_t i) { return waited_ms[i]; }, take);
    for (size_t j = 0; j < take.size(); ++j) admitted[j] = (int32_t)take[j];
    *nadmitted = (int32_t)take.size();
    return SCC_OK;
}

SCC_API int scc_debug_serve_unit(int32_t count, const int32_t* kind, const int32_t* small, const int32_t* graph,
                                 const int32_t* dir, const int32_t* nsrc, int32_t merge_reach, int32_t batch_graphs,
                                 int32_t batch_min, int32_t* unit, int32_t* nunit) {
    if (count < 0 || !nunit || (count > 0 && (!kind || !small || !graph || !dir || !nsrc || !unit)))
        return SCC_ERR_INVALID_ARG;
    std::vector<UnitItem> q((size_t)count);
    for (int32_t i = 0; i < count; ++i) {
        if ((kind[i] != 0 && kind[i] != 1) || nsrc[i] < 0) return SCC_ERR_INVALID_ARG;
        q[i] = {kind[i], kind[i] == 0 && small[i] != 0, graph[i], dir[i], nsrc[i]};
    }
    const std::vector<size_t> u = unit_select(q, merge_reach != 0, batch_graphs, batch_min);
    for (size_t j = 0; j < u.size(); ++j) unit[j] = (int32_t)u[j];
    *nunit = (int32_t)u.size();
    return SCC_OK;
}

}  // extern "C"
