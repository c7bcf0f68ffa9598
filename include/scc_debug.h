/*
 * scc_debug.h -- step-level entry points of the SCC library, for parity tests.
 *
 * Each call runs ONE step of the hot path in the same kernels scc_run uses, so a
 * test can compare that step's output with a CPU restatement. Conventions
 * (errors, streams, host-or-device pointers) are those of scc.h. Every call here
 * synchronises `stream` before returning.
 */
#ifndef SCC_GB300_SCC_DEBUG_H
#define SCC_GB300_SCC_DEBUG_H

#include "scc.h"

#ifdef __cplusplus
extern "C" {
#endif

/* n, m of the input and m_t = arcs of the self-loop-free graph (= arcs of G^T). */
SCC_API int scc_graph_info(scc_handle h, int32_t* n, int64_t* m, int64_t* m_t);

/*
 * Copy the library's self-loop-free CSR of G (which = 0) or of G^T (which = 1)
 * (Sec. 2; G^T row v lists the in-neighbours of v, one entry per arc, in an
 * unspecified order).
 *   off  host or device int32[n+1]; adj host or device int32[m_t].
 */
SCC_API int scc_debug_csr(scc_handle h, int32_t which, int32_t* off, int32_t* adj, void* stream);

/*
 * Trimming (Sec. 4.1): flags[v] = 1 iff v has no arc to or no arc from another
 * vertex. flags: host or device uint8[n].
 */
SCC_API int scc_debug_trim(scc_handle h, uint8_t* flags, void* stream);

/*
 * Pivot order (Alg. 1 random batches; Sec. 2 prefix doubling): order[p] =
 * act[pi(p)], act the increasing list of untrimmed vertices and pi the seeded
 * Feistel bijection of [0, N) with cycle walking (Black & Rogaway, CT-RSA 2002)
 * under h's config seed. order: host or device int32[n] (first N entries
 * written); *n_active (host) receives N.
 */
SCC_API int scc_debug_pivot_order(scc_handle h, int32_t* order, int32_t* n_active, void* stream);

/*
 * Single-reachability with the first-SCC engine (Alg. 3 with VGC, Sec. 3;
 * dense mode per config, Sec. 4.2): visited[v] = 1 iff s reaches v over arcs
 * whose endpoints both carry label[s] (labels NULL: one class).
 *   labels  host or device int32[n] or NULL; a negative label means finished.
 *   dir     0 forward on G, 1 backward on G^T.
 *   visited host or device uint8[n].
 */
SCC_API int scc_debug_single_reach(scc_handle h, const int32_t* labels, int32_t s, int32_t dir,
                           uint8_t* visited, void* stream);

/*
 * Multi-reachability (Alg. 1 MultiReach with VGC and a hash-bag frontier,
 * Sec. 3, and the pair table of Sec. 4.3/4.5): the set of pairs
 * (v, s), s in sources, s ~> v (dir 0) or v ~> s (dir 1) inside s's label class.
 *   labels   host or device int32[n] (negative = finished: no pairs).
 *   sources  host or device int32[k], k >= 1.
 *   pairs    host or device uint64[cap]; receives v << 32 | s, unordered, when
 *            the total fits.
 *   *npairs  (host) total number of pairs (may exceed cap).
 *   table_cap  initial pair-table capacity (power of two >= 1024, or 0 = by the
 *            paper's sizing heuristic); small values exercise regrowth.
 */
SCC_API int scc_debug_multi_reach(scc_handle h, const int32_t* labels, const int32_t* sources, int32_t k,
                          int32_t dir, uint64_t* pairs, int64_t cap, int64_t* npairs,
                          int64_t table_cap, void* stream);

/*
 * reach_multi (scc.h) with up to 128 sources, as the serving loop runs it when
 * it merges queries (Sec. 2 reachability; the wider mask has no counterpart in
 * the paper): out[2 v + j / 64] gets bit j % 64 set iff sources[j] reaches v
 * (dir 0) or v reaches sources[j] (dir 1).
 *   sources  host or device int32[k], 1 <= k <= 128, each in [0, n).
 *   out      host or device uint64[2 n].
 * SCC_ERR_INVALID_ARG for k or a source out of range.
 */
SCC_API int scc_debug_reach_multi_wide(scc_handle h, const int32_t* sources, int32_t k, int32_t dir, uint64_t* out,
                                       void* stream);

/*
 * Hash bag (Sec. 3.3, Fig. 5): insert items[0..count) from many warps
 * concurrently (each warp claims random 32-slot segments of the current chunk by
 * CAS, with sampled chunk advance), then ExtractAll by warp-aggregated
 * compaction. out receives the extracted multiset (unordered), *nout (host) its
 * size, *chunks (host, may be NULL) the number of chunks in use at extraction.
 *   items  host or device int32[count], each in [0, 2^31 - 1).
 *   out    host or device int32[count].
 */
SCC_API int scc_debug_hashbag(const int32_t* items, int64_t count, int32_t lambda, int32_t sigma,
                      int32_t* out, int64_t* nout, int32_t* chunks, void* stream);

/*
 * Pair table (Sec. 4.3 phase-concurrent table, with the regrowth of Sec. 4.5):
 * insert keys[0..count) (duplicates allowed) into a table of initial capacity
 * init_cap; out receives the distinct keys (unordered), *nout (host) their number,
 * *resizes (host, may be NULL) how often the table grew.
 *   keys  host or device uint64[count], each != UINT64_MAX.
 *   out   host or device uint64[count].
 */
SCC_API int scc_debug_pair_table(const uint64_t* keys, int64_t count, int64_t init_cap, uint64_t* out,
                         int64_t* nout, int32_t* resizes, void* stream);

/* Number of kernel launches the library has issued since it was loaded. */
SCC_API int64_t scc_debug_launch_count(void);

/*
 * The failure path of the grid barrier that separates the rounds of every
 * cooperative search (the bounded device wait behind SCC_ERR_TIMEOUT; the paper
 * has no counterpart). One cooperative launch of two blocks per SM meets at one
 * grid barrier whose wait is limited to limit_ns (1e3 .. 1e9 ns); block
 * absent_block (-1: none) returns without arriving, so every other block's
 * wait runs out and the launch ends with SCC_ERR_TIMEOUT instead of hanging.
 *   *n_arrived (host) receives the number of blocks whose wait ended because
 *   every block arrived (all of them with absent_block = -1, none otherwise).
 * Returns SCC_OK when every block passed, SCC_ERR_TIMEOUT when a wait ran out,
 * SCC_ERR_INVALID_ARG for a limit out of range or absent_block >= the grid.
 */
SCC_API int scc_debug_barrier_timeout(int32_t absent_block, int64_t limit_ns, int32_t* n_arrived, void* stream);

/*
 * le_lists_run (scc.h; Sec. 5.2, Alg. 5) starting from a visited-pair table of
 * init_cap slots (rounded up to a power of two, at least 1024) and a candidate
 * log of init_log entries instead of the sizes taken from n, so that tests can
 * make both grow (a batch that overflows either is run again after the buffer
 * doubles). The lists are kept with the handle as by le_lists_run.
 */
SCC_API int scc_debug_le_lists(scc_handle h, int64_t init_cap, int64_t init_log, int64_t* total, void* stream);

/* Batched SCC (scc_batch.h): for every graph g of the last scc_batch_run,
   out[11g .. 11g + 5] = device globaltimer (ns) at its start and at the end of
   the transpose, the single-pivot steps, the class trimming, the batches and
   the labels; out[11g + 6] = the block that ran it; out[11g + 7 .. 11g + 10]
   = engine rounds of its batches, pair searches, pair searches that stopped
   because a table or the bag filled up (the batch then reruns or takes its
   sources one single-pivot step each), batches labelled. out: host
   uint64[11 * G]. */
SCC_API int scc_debug_batch_times(struct scc_batch* h, uint64_t* out);

/*
 * The grouping of a batched run's G^T passes (scc_batch.h; host only, no
 * device work): graphs are taken in packed order, as many consecutive ones per
 * group as fit in max_vertices vertices and max_arcs arcs; a graph larger than
 * either limit ends the current group and is in none (its block builds its
 * G^T); groups without vertices are dropped. The library uses 2^24 vertices
 * and 2^27 arcs.
 *   vbase, ebase  host int64[G + 1], non-decreasing (scc_batch.h layout).
 *   groups        host int32[2 G]: group k is graphs [groups[2k], groups[2k+1]).
 *   *ngroups      (host) the number of groups.
 */
SCC_API int scc_debug_batch_groups(int32_t G, const int64_t* vbase, const int64_t* ebase, int64_t max_vertices,
                                   int64_t max_arcs, int32_t* groups, int32_t* ngroups);

/*
 * The serving loop's scheduling decisions (scc_serve.h) on a described queue,
 * host only (no device work). No counterpart in the paper.
 *
 * Admission: count pending requests in arrival order, request i needing
 * need[i] bytes and having waited waited_ms[i]; in_use bytes are held of cap.
 * Request i is admitted when in_use + need[i] <= cap (in_use then grows by
 * need[i]); the first request that does not fit lets later ones pass while it
 * has waited at most max_bypass_ms, and ends the pass once it has waited
 * longer. admitted (int32[count]) receives the admitted indices in increasing
 * order, *nadmitted their number.
 */
SCC_API int scc_debug_serve_admission(int32_t count, const int64_t* need, const double* waited_ms, int64_t in_use,
                                      int64_t cap, double max_bypass_ms, int32_t* admitted, int32_t* nadmitted);
/*
 * Unit selection: count admitted requests in arrival order; kind[i] 0 (SCC;
 * small[i] != 0 when the batched kernel takes it) or 1 (reachability on
 * resident graph graph[i], direction dir[i], with nsrc[i] sources). The unit
 * of request 0, as increasing indices into unit (int32[count]), *nunit their
 * number: a reachability query with every later query on the same graph and
 * direction while the sources stay within 128 (merge_reach != 0; otherwise
 * request 0 alone); a small SCC request with the next small ones, batch_graphs
 * at most, when at least batch_min small SCC requests are admitted (with fewer,
 * request 0 alone, for the full-GPU path); a larger SCC request alone.
 * count = 0 gives an empty unit.
 */
SCC_API int scc_debug_serve_unit(int32_t count, const int32_t* kind, const int32_t* small, const int32_t* graph,
                                 const int32_t* dir, const int32_t* nsrc, int32_t merge_reach, int32_t batch_graphs,
                                 int32_t batch_min, int32_t* unit, int32_t* nunit);

#ifdef __cplusplus
}
#endif
#endif /* SCC_GB300_SCC_DEBUG_H */
