/*
 * scc.h -- C ABI of the GB300 (sm_103a) strongly-connected-components library.
 *
 * Method: the BGSS reachability-based SCC algorithm as engineered in Wang, Dong,
 * Gu, Sun, "Parallel Strong Connectivity Based on Faster Reachability"
 * (SIGMOD 2023): trimming (Sec. 4.1), a first SCC from one pivot by forward and
 * backward single-reachability (Sec. 4.2), then forward and backward
 * multi-reachability searches over prefix-doubling batches of random pivots
 * (Alg. 1; Sec. 4.3), labelling/partitioning by reachability signature
 * (Alg. 1; Sec. 4.4). Every reachability search uses vertical granularity control
 * (bounded multi-hop local searches, Sec. 3.1-3.2) and a hash-bag frontier
 * (Sec. 3.3). All of it runs in hand-written CUDA kernels on one GPU.
 *
 * Conventions shared by every entry point:
 *  - Graphs are int32 CSR: row v of targets is targets[offsets[v] .. offsets[v+1]),
 *    the out-neighbours of v; 0 <= targets[e] < n, offsets[0] = 0,
 *    offsets[n] = m, offsets non-decreasing; m <= INT32_MAX. Self-loops and
 *    duplicate arcs are accepted (they never change an SCC).
 *  - Pointers marked "host or device" may point to either; the library asks the
 *    driver (cudaPointerGetAttributes) which one it is. Pointers marked "device"
 *    must be device (or managed) memory of the current CUDA device.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream). Work is stream-ordered on it. Calls return after enqueueing, except
 *    where a call says it synchronises `stream`.
 *  - Every call returns SCC_OK (0) or a negative SCC_ERR_* code and never
 *    throws. On failure, outputs are undefined. A handle is not thread-safe: one
 *    host thread at a time per handle.
 *  - Memory: the library allocates its device buffers stream-ordered
 *    (cudaMallocFromPoolAsync) from a memory pool of its own on the current
 *    device (the device's default pool if that cannot be created), whose release
 *    threshold keeps freed memory for reuse by later calls. A handle's buffers
 *    are freed in its destroy call; a call's temporaries are freed
 *    (stream-ordered) when it returns, on error paths too.
 */
#ifndef SCC_GB300_SCC_H
#define SCC_GB300_SCC_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SCC_API __attribute__((visibility("default")))
#else
#define SCC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- errors ---- */
#define SCC_OK 0
#define SCC_ERR_INVALID_ARG (-1) /* bad size, CSR not well formed, id out of range, bad k/dir */
#define SCC_ERR_OOM (-2)         /* a device allocation failed */
#define SCC_ERR_CUDA (-3)        /* a CUDA runtime call or kernel launch failed */
#define SCC_ERR_TIMEOUT (-4)     /* a bounded device-side wait gave up (kernel returned early) */
#define SCC_ERR_CAPACITY (-5)    /* an internal table/bag could not grow far enough */
#define SCC_ERR_INTERNAL (-6)    /* a self-check of the library failed */

/* Static string describing an error code (never NULL). */
SCC_API const char* scc_error_string(int code);

/* ---------------------------------------------------------------- config ---- */
/*
 * Tunables. None of them changes any result: labels and reachability masks are
 * identical for every valid configuration and seed.
 *   tau         VGC edge budget of one local search (Sec. 3.2 "Control of
 *               Granularity"): a warp task stops expanding after visiting about
 *               tau arcs; vertices with more than tau out-arcs are expanded by
 *               many warps in parallel instead. 1..2^20, or 0 (the default):
 *               chosen per graph, 128 when the average degree is at least 8,
 *               2048 below. The paper's 2^9 = 512 is the middle of that range;
 *               on the GPU a round's time is set by its longest local search,
 *               which on a graph of high degree grows faster with tau than the
 *               rounds it saves, and on a lattice or k-NN graph more slowly.
 *   beta        prefix-doubling multiplier in (1, 64] (Alg. 1 doubles the batches, the
 *               experiments use 1.5). Default 2: a batch costs rounds whose
 *               time on the GPU is set by memory latency more than by the pairs
 *               they visit, so fewer and larger batches are faster here.
 *   lambda      first hash-bag chunk size in slots, a power of two in [1024, 2^24]
 *               (Sec. 3.3; chunks grow lambda, 2*lambda, ...). Default 16384.
 *   sigma       hash-bag samples per chunk before it is declared full (Sec. 3.3),
 *               1..2^20, default 50; 0 replaces the sampled hash bag by a
 *               reservation bag (one counter hands out 32-slot segments in
 *               order) as the comparison point of the paper's bag design.
 *   block       threads per block of the search kernels (256; other values are
 *               rejected with SCC_ERR_INVALID_ARG).
 *   seeds       frontier items one warp takes per task, 1..32 (default 32).
 *   dense       0: the first-SCC single-reachability never switches to the dense
 *               (bottom-up) mode of Sec. 4.2; 1: it does once a round's frontier
 *               holds 1/20 of the searched class (the default); k in [2, 1024]:
 *               once it holds 1/k of it.
 *   seed        seed of the pivot permutation (default 0x5CC00).
 *   ldd_beta    growth factor of the centre batches of cc_run's low-diameter
 *               decomposition, in (1, 64] (Sec. 5.1 uses 1.2). Default 2: each
 *               batch adds a round whose time on the GPU is mostly barrier and
 *               memory latency, so fewer and larger batches are faster here
 *               (R-MAT 24: 83 -> 24 rounds); the components do not change.
 * Out-of-range values are rejected with SCC_ERR_INVALID_ARG.
 */
typedef struct scc_config {
    int32_t tau;
    double beta;
    int32_t lambda;
    int32_t sigma;
    int32_t block;
    int32_t seeds;
    int32_t dense;
    uint64_t seed;
    double ldd_beta;
} scc_config;

/* Fill *cfg with the defaults listed above. */
SCC_API int scc_config_default(scc_config* cfg);

/* ----------------------------------------------------------------- graphs ---- */
typedef struct scc_graph* scc_handle; /* opaque, owned by the library */

/*
 * Copy a CSR graph to the device and build what every later call needs: the
 * self-loop-free forward CSR and its transpose G^T (Sec. 2: a backward search is a
 * forward search on G^T). G^T is a counting sort of the arcs by target in three
 * levels (buckets, sub-buckets of at most 1024 targets, rows), each pass reading
 * and writing whole tiles; within a row of G^T the sources are in no set order.
 * Page-locked host targets are read over the host link by the first pass itself,
 * in chunks whose later passes overlap the next chunk's transfer.
 *   n        number of vertices, 0 <= n < 2^31 - 1.
 *   m        number of arcs, 0 <= m <= INT32_MAX.
 *   offsets  host or device int32[n+1]; targets host or device int32[m]. Both are
 *            only read; the caller keeps ownership and may free them when the
 *            call returns.
 *   out      receives the handle.
 * Synchronises `stream` (it validates the CSR and returns SCC_ERR_INVALID_ARG if
 * it is not well formed).
 */
SCC_API int scc_graph_create(int32_t n, int64_t m, const int32_t* offsets, const int32_t* targets,
                     void* stream, scc_handle* out);

/* Release every buffer of h (stream-ordered on the stream of the last call). NULL is ok. */
SCC_API int scc_graph_destroy(scc_handle h);

/* Replace the configuration of h (validated; SCC_ERR_INVALID_ARG if out of range). */
SCC_API int scc_set_config(scc_handle h, const scc_config* cfg);

/* ------------------------------------------------------------------- SCC ---- */
/*
 * Strongly connected components (Sec. 1 problem statement, computed by Alg. 1):
 * labels_out[v] = the smallest vertex id u with u ~> v and v ~> u. The result is
 * deterministic and independent of the configuration and seed.
 *   labels_out  host or device int32[n], written.
 * Host-driven rounds: the call synchronises `stream` a few times per round and
 * before returning.
 */
SCC_API int scc_run(scc_handle h, int32_t* labels_out, void* stream);

/* -------------------------------------------------------------- reach ---- */
/*
 * Multi-source reachability (Sec. 2 "Reachability Search"): for j < k,
 * bit j of out[v] is 1 iff sources[j] ~> v (dir = 0, forward on G) or
 * v ~> sources[j] (dir = 1, backward: forward on G^T). Plain reachability: no
 * label classes. Duplicate sources are allowed; bit j always refers to
 * sources[j].
 *   sources  host or device int32[k], 1 <= k <= 64, each in [0, n).
 *   out      host or device uint64[n], written.
 * Synchronises `stream` before returning.
 */
SCC_API int reach_multi(scc_handle h, const int32_t* sources, int32_t k, int32_t dir, uint64_t* out,
                void* stream);

/*
 * reach_multi without device allocation. The paper has no counterpart. Some
 * callers may not call cudaMalloc, or any routine that allocates device
 * memory, at the point where they need a reachability result: latency-critical
 * loops that forbid allocator calls (an allocation can block or synchronise
 * the device), and hosts whose device memory belongs to their own allocator (a
 * framework's caching allocator or a fixed arena), where an allocation by a
 * library would bypass the owner's accounting. This entry point computes
 * exactly what reach_multi computes, with the same engine kernel, and
 * allocates nothing: the caller passes the sources and the output, and the
 * search's working memory comes from one fixed device array of 32 MiB that the
 * library keeps on every device it has run on, until the process exits.
 *   sources  DEVICE int32[k], 1 <= k <= 64, each in [0, n).
 *   out      DEVICE uint64[n], written. (Host pointers are rejected.)
 * Returns SCC_ERR_INVALID_ARG when the graph's working space does not fit the
 * array (about 500 thousand vertices for sparse graphs) or a source is out of
 * range, SCC_ERR_CAPACITY when a search needs more frontier space than the
 * array holds.
 * Every call shares the array and finds the previous call's contents in it, so
 * a call clears what must start empty; calls whose work overlaps on the GPU
 * (for instance on two streams) race on it and must be serialised by the
 * caller. Every call looks the array's device address up on the current
 * device (after a cudaDeviceReset the array is a new one, zeroed, and the
 * handles made before the reset are gone). Synchronises `stream`.
 */
SCC_API int reach_multi_noalloc(scc_handle h, const int32_t* sources, int32_t k, int32_t dir, uint64_t* out,
                                void* stream);

/* ------------------------------------------------------------ statistics ---- */
/*
 * Counters of the last scc_run on h, in the paper's cost categories (Sec. 4,
 * Fig. 8), and of the handle's construction: times in milliseconds measured
 * with CUDA events on the stream of the call.
 */
typedef struct scc_stats {
    int32_t n_trimmed;         /* vertices removed by trimming */
    int32_t first_scc_size;    /* size of the SCC found from the first pivot */
    int32_t batches;           /* prefix-doubling batches run (including the first) */
    int32_t search_rounds;     /* reachability rounds (frontier swaps), all searches */
    int64_t pairs;             /* reachability pairs inserted by multi-reachability */
    int32_t table_resizes;     /* pair-table regrowths */
    int32_t engine_launches;   /* launches of the reachability engine kernel */
    double ms_trim, ms_first_scc, ms_multi_search, ms_resize, ms_label;
    double ms_engine;          /* summed duration of the first-SCC engine launches */
    int64_t engine_arcs;       /* arcs examined by the first-SCC engine launches */
    int64_t engine_items;      /* items they expanded (adjacency rows read) */
    int64_t engine_inserted;   /* reachability pairs inserted by multi-reachability */
    /* graph construction (scc_graph_create of this handle), CUDA events on the
       creating stream: total; the intake pass (copy and range check of the
       targets with the sub-bucket histogram of the transpose); the passes that
       build the transpose: bucket partition, per-sub-bucket rows (and the split
       of buckets into sub-buckets, ms_transpose_split below) */
    double ms_create, ms_transpose_hist, ms_transpose_part, ms_transpose_rows;
    /* trimming inside the classes left by the first SCC: vertices with no arc
       from or no arc to a vertex of their own class are singleton SCCs */
    int32_t n_class_trimmed;   /* vertices finished this way */
    int32_t class_trim_passes; /* passes run */
    double ms_class_trim;
    /* the launches of the device-side batch loop (multi-reachability) */
    int32_t multi_launches;
    int64_t multi_arcs;        /* arcs examined */
    int64_t multi_items;       /* items expanded */
    int32_t tau;               /* the VGC edge budget used (config tau, or the automatic one) */
    double ms_transpose_split; /* transpose: buckets cut into sub-buckets (ms_transpose_rows: their rows) */
    int64_t multi_active_sum;  /* active vertices summed over the multi-reachability batches */
} scc_stats;

SCC_API int scc_get_stats(scc_handle h, scc_stats* out);

/* ---------------------------------------------------------- connectivity ---- */
/*
 * Connected components (Sec. 5.1, Alg. 4: LDD-UF-JTB, with the hash bag and
 * VGC applied to the low-diameter decomposition) of the undirected graph under
 * the arcs of h: u and v are in one component iff a path joins them when every
 * arc may be taken in either direction (the paper symmetrises directed inputs
 * for connectivity; for a directed graph these are its weakly connected
 * components). labels_out[v] = the smallest vertex id of v's component.
 *   labels_out  host or device int32[n], written.
 * The first call on h builds the symmetric CSR (each vertex's out-arcs then
 * its in-arcs, 2 m_t entries) and keeps it with the handle until it is
 * destroyed. The decomposition takes its centres from h's seeded order in
 * batches growing by the configuration's ldd_beta (default 2; the paper's
 * choice is 1.2); the result depends on neither the seed nor ldd_beta. Returns SCC_ERR_INTERNAL if a bounded union-find loop
 * ran out (never expected). Synchronises `stream` before returning.
 */
SCC_API int cc_run(scc_handle h, int32_t* labels_out, void* stream);

/* Counters of the last cc_run on h (times in milliseconds, CUDA events on the
   stream of the call). */
typedef struct scc_cc_stats {
    int32_t components;   /* connected components found */
    int32_t clusters;     /* clusters of the low-diameter decomposition (centres) */
    int32_t ldd_rounds;   /* rounds of the decomposition's search */
    int32_t ldd_batches;  /* batches of candidate centres */
    int64_t ldd_arcs;     /* arcs examined by the decomposition's search */
    int64_t cross_arcs;   /* arcs of G joining two clusters (the union-find's work) */
    double ms_sym;        /* building the symmetric CSR (0 when it was kept from an earlier call) */
    double ms_ldd, ms_union, ms_label, ms_total;
} scc_cc_stats;

SCC_API int cc_get_stats(scc_handle h, scc_cc_stats* out);

/* --------------------------------------------------- least-element lists ---- */
/*
 * Least-element lists (Sec. 5.2, Alg. 5: the BGSS LE-lists algorithm with the
 * frontier of each level kept packed and a hash table of visited
 * (vertex, source) pairs) of the undirected graph under the arcs of h,
 * unweighted: for the vertex order order[0..n) (the seeded permutation of h's
 * pivot seed over all vertices), source order[j] is in L(v) iff its hop
 * distance to v is smaller than the distance from v to every earlier source.
 * L(v) lists those sources in order; their distances strictly decrease and
 * the last entry is v itself at distance 0.
 * le_lists_run computes the lists and keeps them with the handle (replacing
 * earlier ones); *total (host) receives the number of entries. The first call
 * on h builds the symmetric CSR that cc_run also uses. Synchronises `stream`.
 */
SCC_API int le_lists_run(scc_handle h, int64_t* total, void* stream);
/*
 * Copies the lists of the last le_lists_run out:
 *   order            host or device int32[n]: the vertex order used.
 *   le_off           host or device int64[n + 1]: L(v) = entries le_off[v] .. le_off[v+1] - 1.
 *   le_src, le_dist  host or device int32[total]: each entry's source and distance.
 * SCC_ERR_INVALID_ARG if no lists were computed. Synchronises `stream`.
 */
SCC_API int le_lists_get(scc_handle h, int32_t* order, int64_t* le_off, int32_t* le_src, int32_t* le_dist,
                         void* stream);

/* Counters of the last le_lists_run on h. */
typedef struct scc_le_stats {
    int64_t entries;     /* entries of all lists */
    int64_t candidates;  /* (vertex, source) pairs found before the per-vertex filter */
    int64_t arcs;        /* arcs examined by the multi-source BFS */
    int32_t levels;      /* BFS levels run, all batches */
    int32_t launches;    /* cooperative launches (more than one when a buffer had to grow) */
    double ms_total;
} scc_le_stats;

SCC_API int le_get_stats(scc_handle h, scc_le_stats* out);

#ifdef __cplusplus
}
#endif
#endif /* SCC_GB300_SCC_H */
