/*
 * Serving SCC and reachability requests with continuous batching.
 *
 * There is no counterpart in the paper (Wang, Dong, Gu, Sun, SIGMOD 2023),
 * which computes one SCC at a time; this is the request loop a service puts
 * around the same method (Alg. 1; Sec. 3-4) and its reachability searches.
 *
 * A server owns one thread that works in dispatch units:
 *   - admission: pending requests are admitted in arrival order while the
 *     device memory they need fits under the cap next to what is already held
 *     (resident graphs, the batched kernel's working memory, admitted
 *     requests); a request that does not fit yet waits while later ones that
 *     fit pass it, unless it has waited for `max_bypass_ms`. The inputs of every
 *     admitted request are uploaded at once on a copy stream, overlapping the
 *     compute of earlier units.
 *   - units, oldest request first: every admitted SCC request small enough for
 *     the batched kernel (scc_batch.h: one block per graph) joins one launch;
 *     reachability queries on the same resident graph and direction share one
 *     reachability launch (up to 128 sources: above 64 the search carries two
 *     mask words per vertex; each query's bits are split out on the device); a
 *     larger SCC request runs the full-GPU path (scc.h).
 *     Requests that arrive while a unit runs are admitted when it ends.
 * Results are identical whether a request runs alone or in any mix.
 *
 * Host buffers passed to the submit calls stay owned by the caller and must
 * stay valid until the request has completed (scc_server_wait). Pinned host
 * memory makes the copies asynchronous.
 */
#ifndef SCC_SERVE_H
#define SCC_SERVE_H

#include <stdint.h>

#include "scc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct scc_server_config {
    int64_t mem_cap_bytes;  /* device memory the server may hold (default 120e9) */
    int32_t batch_vertices; /* SCC requests with at most this many vertices and at most
                               32x as many arcs share batched launches (default 262144;
                               0: every SCC request runs alone on the full-GPU path) */
    int32_t batch_graphs;   /* at most this many SCC requests per batched launch (default 512) */
    int32_t merge_reach;    /* 1: queries on the same graph and direction share launches (default 1) */
    int32_t prefetch;       /* 1: upload the inputs of every admitted request at admission
                               (default 1); 0: upload each request's input when its unit runs */
    double max_bypass_ms;   /* a waiting request stops later ones from passing it after this
                               long (default 50) */
    int32_t batch_min;      /* a batched launch needs at least this many small SCC requests
                               admitted (default 4, at most batch_graphs); with fewer, the
                               oldest runs alone on the full-GPU path, which finishes one graph
                               sooner than one block of the batched kernel does (1: every
                               small request goes to a batched launch) */
} scc_server_config;

SCC_API int scc_server_config_default(scc_server_config* cfg);

typedef struct scc_server* scc_server_handle;

/* Start a server on the current device. */
SCC_API int scc_server_create(const scc_server_config* cfg, scc_server_handle* out);
/* Complete every submitted request, then stop the server and free everything.
   NULL is ok. */
SCC_API int scc_server_destroy(scc_server_handle h);

/* A resident graph for reachability queries: its CSR and G^T stay on the
   device until removed. The call returns when the graph is built. */
SCC_API int scc_server_add_graph(scc_server_handle h, int32_t n, int64_t m, const int32_t* offsets,
                                 const int32_t* targets, int32_t* graph_id);
/* Remove a resident graph once no submitted query on it is pending. */
SCC_API int scc_server_remove_graph(scc_server_handle h, int32_t graph_id);

/* SCC labels of a graph given with the request (host CSR in, host labels out,
   int32[n], the smallest vertex id of each SCC). SCC_ERR_OOM if the request
   alone would exceed the memory cap. */
SCC_API int scc_server_submit_scc(scc_server_handle h, int32_t n, int64_t m, const int32_t* offsets,
                                  const int32_t* targets, int32_t* labels_out, int64_t* request_id);
/* reach_multi (scc.h) on a resident graph: out (host uint64[n]) gets bit j of
   vertex v set iff sources[j] reaches v (dir 0) or v reaches sources[j] (dir 1). */
SCC_API int scc_server_submit_reach(scc_server_handle h, int32_t graph_id, const int32_t* sources, int32_t k,
                                    int32_t dir, uint64_t* out, int64_t* request_id);

/* Block until the request has completed; its status (SCC_OK or an error code)
   and latency (submission to results in host memory, milliseconds). A result
   is collected once: a later wait for the same id returns SCC_ERR_INVALID_ARG
   at once, as does an id that was never returned by a submit call. */
SCC_API int scc_server_wait(scc_server_handle h, int64_t request_id, int32_t* status, double* latency_ms);
/* Block until every submitted request has completed. */
SCC_API int scc_server_drain(scc_server_handle h);

typedef struct scc_server_stats {
    int64_t submitted, completed, failed;
    int64_t scc_requests, reach_requests;
    int64_t units;            /* dispatch units run */
    int64_t batched_launches; /* launches of the batched SCC kernel */
    int64_t batched_graphs;   /* SCC requests they served */
    int64_t plain_scc;        /* SCC requests served by the full-GPU path */
    int64_t reach_launches;   /* reach_multi launches */
    int64_t reach_shared;     /* queries that shared their launch with another query */
    int64_t mem_in_use, mem_peak, mem_cap;
    int32_t max_admitted;     /* most requests admitted at the same time */
    int32_t resident_graphs;
    double p50_ms, p99_ms;    /* latency percentiles of the completed requests */
    double scc_p50_ms, scc_p99_ms, reach_p50_ms, reach_p99_ms;
    double busy_reach_ms, busy_batched_ms, busy_plain_ms;  /* server-thread time in each kind of unit */
} scc_server_stats;

SCC_API int scc_server_get_stats(scc_server_handle h, scc_server_stats* out);
/* Forget the recorded latencies and counters (the memory figures stay). */
SCC_API int scc_server_reset_stats(scc_server_handle h);

#ifdef __cplusplus
}
#endif

#endif /* SCC_SERVE_H */
