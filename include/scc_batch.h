/*
 * Batched SCC: the strongly connected components of many independent graphs
 * in one persistent launch.
 *
 * The paper (Wang, Dong, Gu, Sun, SIGMOD 2023) computes the SCCs of one graph
 * (Alg. 1 with the reachability of Sec. 3 and the implementation of Sec. 4).
 * This entry point runs that same method -- trimming, the first SCC by
 * forward and backward single-reachability, prefix-doubling batches of
 * multi-reachability with VGC local searches and a hash-bag frontier, the
 * labelling step of Alg. 1, and the canonical minimum label -- on every graph
 * of a batch. There is no counterpart in the paper: batching is how a serving
 * system amortises launches over thousands of small graphs.
 *
 * Single-pivot steps: the next pivots of the order take the first pivot's
 * single-reachability step too, while the last such step left at least 1/8
 * of the active vertices reached one way only (at most 8 steps); and the
 * sources of a batch of at most 16 that overflows its pair tables are taken
 * one such step each. Sources that reach much of the graph (a pivot that
 * missed a giant SCC) cost one bitmap search each this way, not pair-table
 * searches that fill up and rerun. On a graph of high or skewed degree (at
 * least 8 arcs per vertex, or a row of at least 16 times the mean degree) a
 * step runs its forward and backward searches one after the other with the
 * dense rounds of Sec. 4.2; on the others both directions share each round.
 * The labels never depend on these choices.
 *
 * Execution: one persistent kernel; each thread block takes the next graph from
 * a device work queue (largest graphs first) and runs its whole SCC alone, with
 * block-level synchronisation between rounds, then takes the next graph. The
 * host is not involved until every graph is done, so a run is one CUDA graph
 * (captured once per configuration and output buffer, then replayed).
 *
 * Packed input (one int32 CSR for all graphs, per-graph int64 bases):
 *   vbase[g], g = 0..G: first vertex of graph g in the packed vertex space;
 *     n_g = vbase[g + 1] - vbase[g] (vbase[0] = 0, non-decreasing).
 *   ebase[g], g = 0..G: first arc of graph g in `targets`; m_g = ebase[g + 1] -
 *     ebase[g] (ebase[0] = 0, non-decreasing).
 *   offsets: graph g's n_g + 1 local row offsets start at offsets[vbase[g] + g]
 *     (so offsets has vbase[G] + G entries); local offsets start at 0 and end
 *     at m_g.
 *   targets: graph g's arcs at targets[ebase[g] .. ebase[g + 1]), local vertex
 *     ids in [0, n_g). Self-loops and duplicate arcs are allowed.
 * Output: labels_out[vbase[g] + v] = the smallest local vertex id of v's SCC in
 * graph g (int32, vbase[G] entries).
 *
 * Limits: n_g <= 2^30, m_g <= 2^31 - 1, G >= 0. Every pointer may be host or
 * device memory; the library copies the input at creation and keeps it.
 * Errors: the codes of scc.h; SCC_ERR_INVALID_ARG for a malformed batch (the
 * handle is not created), SCC_ERR_OOM when the device memory for the inputs
 * and the per-block working memory is not available.
 */
#ifndef SCC_BATCH_H
#define SCC_BATCH_H

#include <stdint.h>

#include "scc.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Tunables of the batched kernel (results never depend on them). Defaults:
 * tau 0, block 1024, lambda 256, sigma 50, seeds 32, beta 2, blocks_per_sm 0.
 *   tau     VGC edge budget of a warp's local search (Sec. 3.2), 1..65536, or 0
 *           (the default): chosen per graph, 128 for a graph with at least 8
 *           arcs per vertex or a row of at least 16 times the mean degree
 *           (hubs), 2048 otherwise (lattices, k-NN-like graphs).
 *   block   threads per block, 128, 256, 512 or 1024 (one block runs one
 *           graph; the kernel takes 64 registers a thread, one SM holds
 *           1,024 threads).
 *   lambda  first hash-bag chunk, a power of two in [256, 65536] (Sec. 3.3).
 *           Every round of a search reads at least the first chunk, and one
 *           block's rounds are short, so the default is the smallest, 256.
 *   sigma   hash-bag samples per chunk (Sec. 3.3), >= 1.
 *   seeds   frontier items one warp takes per task, 1..32.
 *   beta    prefix-doubling multiplier in (1, 64] (Alg. 1).
 *   blocks_per_sm  resident blocks per SM, 0..16 (0: as many as registers,
 *           shared memory and the working-memory budget allow).
 *   seed    seed of the pivot permutation.
 */
typedef struct scc_batch_config {
    int32_t tau;
    int32_t block;
    int32_t lambda;
    int32_t sigma;
    int32_t seeds;
    double beta;
    int32_t blocks_per_sm;
    uint64_t seed;
} scc_batch_config;

SCC_API int scc_batch_config_default(scc_batch_config* cfg);

typedef struct scc_batch* scc_batch_handle;

/* Validate and copy a packed batch (layout above) to the device, stream-ordered
   on `stream`, and return a handle. G = 0 is allowed. */
SCC_API int scc_batch_create(int32_t G, const int64_t* vbase, const int64_t* ebase, const int32_t* offsets,
                             const int32_t* targets, void* stream, scc_batch_handle* out);
/* Free every buffer of h (the call synchronises the device first). NULL is ok. */
SCC_API int scc_batch_destroy(scc_batch_handle h);
/* SCC_ERR_INVALID_ARG for out-of-range values (the configuration is unchanged). */
SCC_API int scc_batch_set_config(scc_batch_handle h, const scc_batch_config* cfg);
SCC_API int scc_batch_get_config(scc_batch_handle h, scc_batch_config* cfg);

/*
 * Labels of every graph into labels_out (int32[vbase[G]], host or device). The
 * work is one CUDA-graph replay on `stream` followed by a read of the error
 * flag (the call synchronises `stream`). A first run with a configuration or a
 * device output buffer not seen before allocates working memory and captures
 * the graph first.
 */
SCC_API int scc_batch_run(scc_batch_handle h, int32_t* labels_out, void* stream);

/*
 * Autotuner: runs the batched kernel on a sample of about `sample` graphs
 * (spread over the size range; all graphs when sample <= 0 or >= G) for the
 * handle's configuration and for every configuration of the grid tau in
 * {16, 64, 256, 1024, 4096} x block in {128, 256, 512, 1024} x lambda in
 * {256, 1024, 4096, 16384}. It scores each by the sample's total block time
 * (the sum over the sampled graphs of the time a block spent on each, which is
 * what a full batch's time follows), keeps the best in the handle if it beats
 * the handle's configuration by more than 3% (the handle's otherwise), and
 * returns it and the sample's launch time in milliseconds when the pointers
 * are not NULL. Synchronises `stream`.
 */
SCC_API int scc_batch_autotune(scc_batch_handle h, int32_t sample, void* stream, scc_batch_config* best,
                               double* best_ms);

typedef struct scc_batch_stats {
    int32_t graphs;
    int64_t vertices;        /* vbase[G] */
    int64_t arcs;            /* ebase[G] */
    int32_t max_vertices;    /* largest n_g */
    int64_t max_arcs;        /* largest m_g */
    int32_t blocks;          /* blocks of the persistent launch */
    int64_t workspace_bytes; /* device working memory, all blocks */
    double ms_last_run;      /* CUDA-event time of the last replay */
    int32_t captures;        /* CUDA graphs captured so far */
    int32_t replays;         /* CUDA graph replays so far */
} scc_batch_stats;

SCC_API int scc_batch_get_stats(scc_batch_handle h, scc_batch_stats* out);

#ifdef __cplusplus
}
#endif

#endif /* SCC_BATCH_H */
