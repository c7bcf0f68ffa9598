// Host-side declarations shared by the library's translation units.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/scc.h"
#include "../../include/scc_batch.h"

namespace scc {

struct EngineCtl;

// ------------------------------------------------------------------ errors --
inline int cuda_err(cudaError_t e) {
    if (e == cudaSuccess) return SCC_OK;
    if (e == cudaErrorMemoryAllocation) return SCC_ERR_OOM;
    return SCC_ERR_CUDA;
}
#define SCC_TRY(expr)                         \
    do {                                      \
        int _rc = (expr);                     \
        if (_rc != SCC_OK) return _rc;        \
    } while (0)
#define SCC_CUDA(expr) SCC_TRY(::scc::cuda_err(expr))
// Kernel launches issued by the library since it was loaded (every launch site
// goes through SCC_LAUNCH or count_launch).
void count_launch();
long long launch_count();
#define SCC_LAUNCH()                                      \
    do {                                                  \
        ::scc::count_launch();                            \
        SCC_TRY(::scc::cuda_err(cudaGetLastError()));     \
    } while (0)

// Stream-ordered device allocation from the library's memory pool on the
// current device (the device's default pool if that cannot be created).
int dalloc(void** p, size_t bytes, cudaStream_t s);
void dfree(void* p, cudaStream_t s);
template <class T>
inline int dalloc_t(T** p, size_t count, cudaStream_t s) {
    return dalloc(reinterpret_cast<void**>(p), count * sizeof(T), s);
}

// The device temporaries of one host call: every allocation made through it is
// freed (stream-ordered on s) when the call returns, on error paths too, unless
// it was freed earlier (release) or handed to a longer-lived owner (keep).
class Scratch {
  public:
    explicit Scratch(cudaStream_t s) : s_(s) {}
    Scratch(const Scratch&) = delete;
    Scratch& operator=(const Scratch&) = delete;
    ~Scratch() {
        for (int i = 0; i < n_; ++i) dfree(p_[i], s_);
    }
    template <class T>
    int alloc(T** p, size_t count) {
        *p = nullptr;
        int slot = -1;  // a slot freed by release or keep, else a new one
        for (int i = 0; i < n_ && slot < 0; ++i)
            if (!p_[i]) slot = i;
        if (slot < 0) {
            if (n_ == kMax) return SCC_ERR_INTERNAL;
            slot = n_++;
        }
        const int rc = dalloc_t(p, count, s_);
        if (rc == SCC_OK) p_[slot] = *p;
        return rc;
    }
    void release(const void* p) {
        for (int i = 0; i < n_; ++i)
            if (p && p_[i] == p) {
                dfree(p_[i], s_);
                p_[i] = nullptr;
            }
    }
    void keep(const void* p) {
        for (int i = 0; i < n_; ++i)
            if (p && p_[i] == p) p_[i] = nullptr;
    }

  private:
    static constexpr int kMax = 48;
    cudaStream_t s_;
    void* p_[kMax] = {};
    int n_ = 0;
};

// True when p is device (or managed) memory.
bool is_device_ptr(const void* p);
const void* mapped_host_ptr(const void* p);

struct DeviceInfo {
    int dev = -1;
    int num_sms = 0;
};
int device_info(DeviceInfo* out);

// --------------------------------------------------------- graph building --
// Validate CSR offsets on the device (off[0] = 0, off[n] = m, non-decreasing);
// *bad (device int) becomes nonzero if malformed.
int launch_validate_offsets(const int32_t* off, int32_t n, int64_t m, int* bad, cudaStream_t s);
// Transposed CSR (transpose.cu). bucket_shift(n): vertices per coarse bucket
// = 2^shift, at most 512 buckets.
int bucket_shift(int32_t n);
// trow[t] = row of arc t * step (t < T), trow[T] = row of the last arc; the
// table has tile_rows_count(m) entries and drives the arc passes below.
size_t tile_rows_count(int64_t m);
int launch_tile_rows(const int32_t* off, int32_t n, int64_t m, int32_t* trow, cudaStream_t s);
// Sub-bucket bins of the histogram (at most 16384): the transpose's finest
// level, up to 32 per bucket.
int transpose_bins(int32_t n, int shift);
// Intake of the target array: dst = src (no copy when equal), targets outside
// [0, n) set *bad, bucket_cnt[f] += arcs into sub-bucket f (transpose_bins
// bins; self-loops included).
int launch_copy_check_hist(const int32_t* src, int32_t* dst, int32_t n, int64_t m, int shift,
                           unsigned long long* bucket_cnt, int* bad, int num_sms, cudaStream_t s);
// bucket_cnt[b] += non-self arcs into bucket b; selfrow[u] += self-loops of u.
int launch_bucket_hist(const int32_t* off, const int32_t* adj, const int32_t* trow, int32_t n, int64_t m, int shift,
                       unsigned long long* bucket_cnt, int32_t* selfrow, unsigned long long* nself, int num_sms,
                       cudaStream_t s);
// G^T of the CSR (off, adj) with m arcs by the three-level bucketed counting
// sort (when transpose_bucketed(shift)), in two calls:
//  * launch_intake_partition: in K chunks of whole tiles (transpose_chunks:
//    1 unless `overlap`), the intake of the targets (src -> adj, no copy when
//    equal; targets outside [0, n) set *bad) with a per-chunk sub-bucket
//    histogram (hist: K x transpose_bins words), then the chunk's partition
//    into its buckets (skipped once *bad is set). With K > 1 the partitions run
//    on s2 after each chunk's intake on s (events cev[0..K]), so a chunk's
//    partition overlaps the next chunk's intake; s waits for the last one.
//    selfrow == nullptr: self-loops are kept (not counted).
//  * launch_transpose_rest: sub-bucket offsets, the split into sub-buckets and
//    the rows. With nself != nullptr, self-loops found by the partition are
//    reported (*self_found; nothing is written to toff/tadj) after a host read;
//    with nullptr nothing is read back (the launches can be captured).
// bucket_tmp: transpose_tmp_words; tmp_u, tmp2_u, tmp_lv, tmp2_lv: m + 8
// entries (the padding is read, never used); order_tmp: transpose_bins
// entries; tile_tmp: transpose_split_tiles entries. Events: ev[0..3] around
// the intakes (s) and the partitions (their stream); around the split and the
// rows.
bool transpose_bucketed(int shift);
int transpose_chunks(int64_t m, bool overlap);
size_t transpose_hist_words(int32_t n, int shift, int K);
size_t transpose_tmp_words(int32_t n, int shift, int K);
size_t transpose_split_tiles(int64_t m, int32_t n, int shift, int K);
int launch_intake_partition(const int32_t* src, int32_t* adj, const int32_t* off, const int32_t* trow, int32_t n,
                            int64_t m, int shift, int K, unsigned long long* hist, unsigned long long* bucket_tmp,
                            int32_t* tmp_u, uint16_t* tmp_lv, int32_t* selfrow, unsigned long long* nself, int* bad,
                            int* err, int num_sms, cudaStream_t s, cudaStream_t s2, cudaEvent_t* cev, cudaEvent_t* ev);
int launch_transpose_rest(int32_t n, int64_t mt, int shift, int K, const unsigned long long* hist,
                          unsigned long long* bucket_tmp, const int32_t* tmp_u, const uint16_t* tmp_lv, int32_t* tmp2_u,
                          uint16_t* tmp2_lv, int32_t* order_tmp, int32_t* tile_tmp, int32_t* toff, int32_t* tadj,
                          const unsigned long long* nself, bool* self_found, int* err, int num_sms, cudaStream_t s,
                          cudaEvent_t* ev);
// G^T without host synchronisation for packed groups of graphs (batch.cu):
// self-loops are kept (they change no reachability), targets must be valid.
struct TransposeScratch {
    unsigned long long *bcnt, *btmp;
    int32_t *tmp_u, *tmp2_u, *order, *tiles, *trow;
    uint16_t *tmp_lv, *tmp2_lv;
    int *bad, *err;
};
size_t transpose_scratch_bytes(int64_t m_max);
void transpose_scratch_carve(unsigned char* base, int64_t m_max, TransposeScratch* ts);
int launch_transpose_keep_self(const int32_t* off, const int32_t* adj, int32_t n, int64_t m, const TransposeScratch& ts,
                               int32_t* toff, int32_t* tadj, int num_sms, cudaStream_t s);
int transpose_set_attributes();
// Direct G^T for very large n: global atomics. indeg: n + 1.
int launch_transpose_direct(const int32_t* off, const int32_t* adj, const int32_t* trow, int32_t n, int64_t m,
                            int32_t* indeg, void* scan_tmp, int32_t* toff, int32_t* tadj, int num_sms,
                            cudaStream_t s);
// Exclusive scan of int32 counts: out[0..n] with out[n] = total. tmp: scan_tmp_bytes(n).
size_t scan_tmp_bytes(int64_t n);
int launch_scan(const int32_t* in, int32_t* out, int64_t n, void* tmp, cudaStream_t s);
// Copy G without self-loops: off2 already scanned from per-row non-self counts.
int launch_drop_self_loops(const int32_t* off, const int32_t* adj, int32_t n, int64_t m, const int32_t* selfrow,
                           const int32_t* off2, int32_t* adj2, cudaStream_t s);
// cnt[u] = out-arcs of u that are not self-loops.
int launch_row_nonself(const int32_t* off, const int32_t* selfrow, int32_t n, int32_t* cnt, cudaStream_t s);

// ------------------------------------------------------------- SCC steps --
// trimmed flags from the self-loop-free CSRs (Sec. 4.1).
int launch_trim(const int32_t* off, const int32_t* toff, int32_t n, uint8_t* flags, cudaStream_t s);
// label[v] = trimmed ? kDone : 0, rep[v] = trimmed ? v : -1; counts active into *nact.
int launch_init_labels(const int32_t* off, const int32_t* toff, int32_t n, int32_t* label, int32_t* rep,
                       unsigned long long* nact, cudaStream_t s);
// act = increasing list of v with label[v] >= 0 (scan-based, order preserving).
int launch_compact_active(const int32_t* label, int32_t n, void* scan_tmp, int32_t* act, cudaStream_t s);
// Pivot positions p in [p0, N) whose vertex act[pi(p)] is still active, in
// increasing p: rem_pos[j] = p, rem_v[j] = the vertex; their number is
// pos_tmp[N - p0] after the call (exclusive scan of the flags).
int launch_remaining(const int32_t* act, int64_t N, uint64_t seed, int64_t p0, const int32_t* label,
                     int32_t* flags_tmp, int32_t* pos_tmp, void* scan_tmp, int32_t* rem_pos, int32_t* rem_v,
                     cudaStream_t s);
// order[p] = act[pi(p)] for p < N (debug hook).
int launch_pivot_order(const int32_t* act, int64_t N, uint64_t seed, int32_t* order, cudaStream_t s);

// Host copy of the Feistel permutation, for the first pivot (identical definition).
int64_t feistel_perm_host(int64_t p, int64_t N, uint64_t seed);

// bitmap bit v = (label == NULL ? done-free : label[v] != L)  (pre-set "not in class")
int launch_prefill_bits(const int32_t* label, int32_t L, int32_t n, uint32_t* bits, uint32_t* bits2, cudaStream_t s);
// visited[v] = bit v of bits AND label[v] == L (undo the prefill) -> uint8
int launch_bits_to_bytes(const uint32_t* bits, const int32_t* label, int32_t L, int32_t n, uint8_t* out,
                         cudaStream_t s);

// Round-0 labelling from the two visited bitmaps of pivot s (Alg. 1 label step
// with one source). Adds the number of finished vertices to *ndone.
int launch_class_trim(const int32_t* act, int64_t N, const int32_t* off, const int32_t* adj, const int32_t* toff,
                      const int32_t* tadj, int32_t* label, int32_t* rep, unsigned long long* ndone, cudaStream_t s);
int launch_label_first(const uint32_t* bf, const uint32_t* bb, int32_t n, int32_t s, int32_t* label, int32_t* rep,
                       unsigned long long* ndone, cudaStream_t s_);

// Labelling after a multi-reachability round (Alg. 1; Sec. 4.4).
// labels_out[v] = min{u : rep[u] == rep[v]} (canonical minimum).
int launch_canonicalize(const int32_t* rep, int32_t n, int32_t* minid, int32_t* labels_out, int* bad,
                        cudaStream_t s);

// mask[sources[j]] |= 1 << j; *bad = 1 if a source is outside [0, n).
int launch_mask_init(const int32_t* sources, int32_t k, int32_t n, int words, unsigned long long* mask, int* bad,
                     cudaStream_t s);
// out = the sources with label >= 0 (count in *cnt); *bad = 1 if one is outside [0, n).
int launch_filter_sources(const int32_t* in, int32_t k, int32_t n, const int32_t* label, int32_t* out, int* cnt,
                          int* bad, cudaStream_t s);

// Gather pair-table contents (non-empty keys) into out; *count (device) total.
int launch_table_gather(const unsigned long long* tab, int64_t cap, unsigned long long* out, int64_t out_cap,
                        unsigned long long* count, cudaStream_t s);
// Rehash every key of src (capacity src_cap) into dst (capacity dst_cap, empty).
int launch_table_rehash(const unsigned long long* src, int64_t src_cap, unsigned long long* dst, int64_t dst_cap,
                        int* overflow, cudaStream_t s);
// Insert keys (debug): dst table capacity cap.
int launch_table_insert(const unsigned long long* keys, int64_t count, unsigned long long* tab, int64_t cap,
                        int* overflow, unsigned long long* inserted, cudaStream_t s);

// ---------------------------------------------------------------- engine --
// Buffers of one engine instance (item type = 4 or 8 bytes): two hash-bag slot
// arrays and two hub lists, alternating between rounds.
struct EngineBuf {
    int item_bytes = 0;
    void* slots[2] = {nullptr, nullptr};
    long long nslots = 0;
    long long items = 0;  // items per round the buffers were sized for
    void* hub_item[2] = {nullptr, nullptr};
    int32_t* hub_beg[2] = {nullptr, nullptr};
    int32_t* hub_deg[2] = {nullptr, nullptr};
    long long* hub_segbase[2] = {nullptr, nullptr};
    int hub_cap = 0;
    int32_t* segmap[2] = {nullptr, nullptr};
    long long segmap_cap = 0;
    EngineCtl* ctl = nullptr;
    int lambda = 0;
    void* init = nullptr;  // staging of the initial items
    size_t init_bytes = 0;
};
// Empty both slot arrays (after a search that stopped early).
int engine_reset_slots(EngineBuf* b, cudaStream_t s);
// Allocate (or keep, if large enough) buffers for at most `items` items per round.
// One cooperative launch whose blocks meet at a grid barrier with a limit of
// limit_ns, block `absent` (< 0: none) never arriving; returns the device's
// error flag (SCC_ERR_TIMEOUT when a wait ran out) and the blocks that passed.
int run_barrier_probe(int absent, int64_t limit_ns, int* n_arrived, cudaStream_t st);
int engine_reserve(EngineBuf* b, int item_bytes, long long items, int lambda, int64_t m, int num_sms, cudaStream_t s);
void engine_release(EngineBuf* b, cudaStream_t s);

struct EngineRun {
    float ms = 0;  // kernel duration (CUDA events on the launching stream)
    int err = 0;
    int overflow = 0;
    int rounds = 0;
    int max_chunk = 0;
    unsigned long long edges = 0;
    unsigned long long inserted = 0;
    unsigned long long items = 0;  // items expanded (adjacency rows read)
};

struct EngineOpts {
    int tau = 512;
    int seeds = 32;
    int sigma = 50;
    int block = 256;
    int num_sms = 0;
    // average degree of at least 8: most targets of a mask search already
    // carry the sources, and a plain read before each atomic saves atomics
    bool high_degree = false;
};

// Dense-round inputs of a single-reachability search (Sec. 4.2 dense mode):
// the reverse CSR, a zeroed frontier bitmap, the class size and the graph's
// arcs; frac_inv = 0 disables dense rounds.
struct DenseOpts {
    const int32_t* roff = nullptr;
    const int32_t* radj = nullptr;
    uint32_t* fbits[2] = {nullptr, nullptr};
    long long n_active = 0;
    int frac_inv = 0;
    long long m_active = 0;
};
// Single reachability from `s` over (off, adj) with the bitmap (already prefilled).
// Forward (off/adj, marks bits_f) and backward (toff/tadj, marks bits_b)
// single-reachability from s in one search, without dense rounds.
int run_single_both(const int32_t* off, const int32_t* adj, const int32_t* toff, const int32_t* tadj, int32_t n,
                    int32_t s, uint32_t* bits_f, uint32_t* bits_b, EngineBuf* b, const EngineOpts& o, EngineRun* out,
                    cudaStream_t st);
int run_single(const int32_t* off, const int32_t* adj, int32_t n, int32_t s, uint32_t* bits, const DenseOpts& dn,
               EngineBuf* b, const EngineOpts& o, EngineRun* out, cudaStream_t st);
// Multi reachability: init pairs (s,s) from sources (device int32[k]); pairs into table.
int run_pairs(const int32_t* off, const int32_t* adj, int32_t n, const int32_t* label, const int32_t* sources,
              int32_t k, unsigned long long* table, int64_t cap, long long max_inserted, EngineBuf* b,
              const EngineOpts& o, EngineRun* out, cudaStream_t st);
// Mask reachability: mask already holds the source bits; init = sources.
// mask2: two words per vertex, k <= 128
int run_mask2(const int32_t* off, const int32_t* adj, int32_t n, const int32_t* sources, int32_t k,
              unsigned long long* mask2, EngineBuf* b, const EngineOpts& o, EngineRun* out, cudaStream_t st);
int run_mask(const int32_t* off, const int32_t* adj, int32_t n, const int32_t* sources, int32_t k,
             unsigned long long* mask, EngineBuf* b, const EngineOpts& o, EngineRun* out, cudaStream_t st);

// Device-side loop over the multi-reachability batches (bgss.cu).
struct BgssArgs {
    const int32_t *off, *adj, *toff, *tadj;
    int32_t n;
    int32_t* label;
    int32_t* rep;
    unsigned long long *fmax, *bmax, *hit;
    const int32_t* rem_pos;   // remaining active pivot positions (increasing) and their vertices
    const int32_t* rem_v;
    long long nrem;
    long long N;              // active vertices after trimming (pivot positions)
    const long long* bounds;  // device, nb + 1 entries
    int nb;
    int first;
    long long first_min_cap = 0;
    long long shrink_below = 0;  // return with status 2 once fewer vertices are active
    int grid = 0;                // blocks of the cooperative launch (0 = all co-resident)
    int32_t* sources;
    unsigned long long* tab[2];
    long long tab_alloc;
    EngineBuf* eb;
    void* bgss_ctl;  // device, bgss_ctl_bytes()
    unsigned long long ndone;
    unsigned long long a_prev[2];
    int ka_prev = 0;  // sources of the batch whose pairs a_prev holds (0: unknown)
    EngineOpts o;
};
struct BgssResult {
    float ms = 0;
    int status = 0;  // 0 finished; 1 grow to need_cap and resume at batch; 2 resume with a smaller grid
    int batch = 0;
    long long need_cap = 0;
    unsigned long long ndone = 0;
    unsigned long long a_prev[2] = {0, 0};
    int ka_prev = 0;
    unsigned long long pairs = 0;
    int batches = 0;
    int rounds = 0;
    unsigned long long edges = 0, items = 0;
    unsigned long long active_sum = 0;  // active vertices summed over the launch's batches
};
size_t bgss_ctl_bytes();
int bgss_full_grid(int num_sms);
int run_bgss_device(const BgssArgs& a, BgssResult* res, cudaStream_t st);

// Batched SCC kernel on caller-owned packed device arrays (batch.cu), working
// memory allocated once: for a serving loop. budget 0: half the free memory,
// at most 96 GiB.
struct BatchRunner;
int batch_runner_create(const scc_batch_config* cfg, long long n_max, long long m_max, long long gcap, size_t budget,
                        cudaStream_t s, BatchRunner** out);
void batch_runner_destroy(BatchRunner* r, cudaStream_t s);
bool batch_runner_fits(const BatchRunner* r, long long n, long long m);
size_t batch_runner_bytes(const BatchRunner* r);
const int* batch_runner_err(const BatchRunner* r);  // device error flag of the last launch
// bad[g] (device int[G]) = 1 when graph g of a packed batch is malformed
int batch_validate_each(int32_t G, const long long* vbase, const long long* ebase, const int32_t* offsets,
                        const int32_t* targets, int* bad, cudaStream_t s);
int batch_runner_enqueue(BatchRunner* r, int32_t G, const long long* vbase, const long long* ebase,
                         const int32_t* offsets, const int32_t* targets, const int32_t* order, int32_t norder,
                         int32_t* out, cudaStream_t s);

// Mask reachability on fixed buffers (no allocation, no events).
// Low-diameter decomposition (Sec. 5.1, Alg. 4) on the symmetric CSR: batch i
// of the seeded order is order[bounds_d[i] .. bounds_d[i + 1]) (nbatches
// batches; the first, of `first` vertices, already centres itself in center[]
// and in the visited bitmap `bits`, whose bits past n are set); on return
// center[v] is the centre of v's cluster. fbits: two zeroed frontier bitmaps
// of ceil(n / 32) words (zero again on return); a round whose frontier holds
// n / frac_inv vertices, or arcs numbering soff_arcs / frac_inv, or more runs
// bottom-up (frac_inv = 0: never).
int run_ldd(const int32_t* soff, const int32_t* sadj, int32_t n, long long soff_arcs, const int32_t* order,
            const long long* bounds_d, long long first, int nbatches, int32_t* center, uint32_t* bits, uint32_t* fbits,
            int frac_inv, EngineBuf* b, const EngineOpts& o, EngineRun* out, cudaStream_t st);
// Connectivity steps (cc.cu): the symmetric CSR (soff[v] = off[v] + toff[v],
// row v = row v of G then row v of G^T); center[] = -1 with the first `first`
// vertices of order centring themselves; then union-find over the arcs of G
// joining two clusters and out[v] = the smallest vertex id of v's component
// (counters[0] += cross arcs, counters[1] += centres, counters[2] += components;
// err: a bounded union-find loop ran out). launch_iota: a[v] = v. Events ev[0..2]: after the union-find set-up, after the
// unions, after the labels.
int launch_sym_csr(const int32_t* off, const int32_t* adj, const int32_t* toff, const int32_t* tadj, int32_t n,
                   int32_t* soff, int32_t* sadj, int num_sms, cudaStream_t s);
int launch_iota(int32_t n, int32_t* a, int num_sms, cudaStream_t s);
int launch_ldd_setup(const int32_t* order, long long first, int32_t n, int32_t* center, uint32_t* bits, int num_sms,
                     cudaStream_t s);
// counters: [0] cross arcs [1] clusters [2] components [3] rows of more than 32
// arcs (big, bdeg: big_cap >= m / 33 + 1 entries; bpre: big_cap + 1; scan_tmp:
// scan_tmp_bytes(big_cap))
int launch_cc_union_label(const int32_t* off, const int32_t* adj, int32_t n, const int32_t* center, int32_t* parent,
                          int32_t* root, int32_t* mn, int32_t* out, unsigned long long* counters, int32_t* big,
                          int32_t* bdeg, int32_t* bpre, void* scan_tmp, long long big_cap, int* err, int num_sms,
                          cudaStream_t s, cudaEvent_t* ev);
// Least-element lists (lelists.cu, Sec. 5.2 Alg. 5) of the symmetric CSR for
// the vertex order `order`: on success res->off (int64[n+1]), res->src and
// res->dist (int32[total]) are device allocations the caller frees (dfree);
// candidates = pairs logged before the per-vertex filter.
struct LeResult {
    int64_t* off = nullptr;
    int32_t* src = nullptr;
    int32_t* dist = nullptr;
    long long total = 0, candidates = 0, edges = 0;
    int levels = 0, launches = 0;
};
// init_cap / init_log > 0: the first table capacity and log length (tests of
// the growth path); 0: sized from n.
int le_lists_compute(const int32_t* soff, const int32_t* sadj, int32_t n, const int32_t* order, int num_sms,
                     LeResult* res, cudaStream_t s, long long init_cap = 0, long long init_log = 0);
int run_mask_fixed(const int32_t* off, const int32_t* adj, int32_t n, const int32_t* sources, int32_t k,
                   unsigned long long* mask, const EngineBuf* b, const EngineOpts& o, EngineRun* out,
                   cudaStream_t st);
// reach_multi with 1..128 device sources into two mask words per vertex (api.cu).
int reach_multi_wide(scc_graph* h, const int32_t* sources_d, int32_t k, int32_t dir, unsigned long long* mask2,
                     cudaStream_t s);
// reach_multi on the library's fixed device scratch array (noalloc.cu).
int reach_multi_noalloc_impl(const int32_t* off, const int32_t* adj, int32_t n, int64_t mt, int lambda,
                             const EngineOpts& o, const int32_t* sources, int32_t k, uint64_t* out,
                             cudaStream_t s);

// Debug: hash bag alone (vertex items).
int run_bag_only(const int32_t* items, int64_t count, int lambda, int sigma, int32_t* out, int64_t* nout,
                 int* chunks, cudaStream_t st);

}  // namespace scc
