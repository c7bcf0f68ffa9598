/*
 * CPU ORACLE -- test infrastructure only.
 *
 * Plain, slow, obviously-correct host C for what the GPU path computes. It is
 * used only by tests/, by the package's smoke check and by the benchmark's
 * cpu_baseline / reference leg. It shares no code with the CUDA path.
 *
 * Contents (paper: Wang, Dong, Gu, Sun, "Parallel Strong Connectivity Based on
 * Faster Reachability", SIGMOD 2023):
 *   or_scc_tarjan      SCC labels, label[v] = min{u : u ~> v and v ~> u}
 *                      (problem statement, Sec. 1; Tarjan's sequential algorithm,
 *                      the paper's SEQ baseline, Sec. 6), iterative.
 *   or_transpose       G^T: every arc (u,v), u != v, becomes (v,u) (Sec. 2,
 *                      "backward reachability search ... on the transpose graph").
 *   or_trim            vertices with zero in- or out-degree (self-loops not
 *                      counted) are singleton SCCs (Sec. 4.1).
 *   or_reach_set       single-source reachability restricted to the source's
 *                      label class (Sec. 2 "Reachability Search"; Alg. 1 note that
 *                      MultiReach skips an arc (u,v) with L(u) != L(v)).
 *   or_multi_reach     the pair set {(v,s) : s ~> v inside s's class} (Sec. 2;
 *                      Alg. 1 forward/backward MultiReach).
 *   or_reach_mask      plain multi-source reachability as a 64-bit mask per vertex.
 *   or_pivot_order     the seeded pivot permutation (Feistel network with cycle
 *                      walking) and or_batch_bounds the prefix-doubling batch
 *                      bounds (Alg. 1; Sec. 2 "The BGSS Algorithm", beta > 1).
 *   or_cc_labels       connected components of the undirected graph under the
 *                      arcs, label = smallest vertex id of the component: what
 *                      the connectivity algorithm of Sec. 5.1 (Alg. 4, LDD-UF-JTB)
 *                      computes, by its plain definition (sequential union-find).
 *   or_le_lists        least-element lists of the undirected graph under the arcs
 *                      for a given vertex order (Sec. 5.2): the sequential
 *                      pruned BFS, one source at a time in order (the batches of
 *                      Alg. 5 with one source each).
 *
 * Parity pins (tests/test_oracle_*.py): brute-force transitive closure on every
 * digraph with n <= 4 and on random digraphs, closed forms (cycles, chains,
 * complete digraphs, tori with all arcs), invariants (partition, canonical min,
 * acyclic condensation) and the paper's Table 2 statistics for its REC/REC'
 * lattices.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_API __attribute__((visibility("default")))

/* ----------------------------------------------------------- Tarjan ---- */
/*
 * Iterative Tarjan SCC on the CSR (off[n+1], adj[m]). Writes
 * label[v] = smallest vertex id of v's SCC. Returns the number of SCCs, or -1 if
 * memory could not be allocated.
 */
OR_API int64_t or_scc_tarjan(int64_t n, const int32_t* off, const int32_t* adj, int32_t* label) {
    if (n == 0) return 0;
    int64_t* index = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    int64_t* low = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    char* onstack = (char*)calloc((size_t)n, 1);
    int32_t* comp = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);   /* Tarjan's vertex stack */
    int32_t* cs_v = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);   /* DFS call stack: vertex */
    int64_t* cs_e = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);   /* DFS call stack: next arc */
    if (!index || !low || !onstack || !comp || !cs_v || !cs_e) {
        free(index); free(low); free(onstack); free(comp); free(cs_v); free(cs_e);
        return -1;
    }
    for (int64_t v = 0; v < n; ++v) index[v] = -1;
    int64_t next_index = 0, ncomp = 0, sp = 0, csp = 0;
    for (int64_t root = 0; root < n; ++root) {
        if (index[root] >= 0) continue;
        index[root] = low[root] = next_index++;
        comp[sp++] = (int32_t)root; onstack[root] = 1;
        cs_v[csp] = (int32_t)root; cs_e[csp] = off[root]; ++csp;
        while (csp > 0) {
            int64_t v = cs_v[csp - 1];
            int64_t e = cs_e[csp - 1];
            if (e < off[v + 1]) {
                cs_e[csp - 1] = e + 1;
                int64_t w = adj[e];
                if (index[w] < 0) {                       /* tree arc: descend */
                    index[w] = low[w] = next_index++;
                    comp[sp++] = (int32_t)w; onstack[w] = 1;
                    cs_v[csp] = (int32_t)w; cs_e[csp] = off[w]; ++csp;
                } else if (onstack[w] && index[w] < low[v]) {
                    low[v] = index[w];                   /* arc back into the stack */
                }
            } else {                                      /* v finished */
                --csp;
                if (low[v] == index[v]) {                 /* v is the root of an SCC */
                    int64_t top = sp;
                    do { --sp; } while (comp[sp] != v);
                    int32_t mn = comp[sp];
                    for (int64_t i = sp; i < top; ++i) if (comp[i] < mn) mn = comp[i];
                    for (int64_t i = sp; i < top; ++i) { label[comp[i]] = mn; onstack[comp[i]] = 0; }
                    ++ncomp;
                }
                if (csp > 0) {
                    int64_t u = cs_v[csp - 1];
                    if (low[v] < low[u]) low[u] = low[v];
                }
            }
        }
    }
    free(index); free(low); free(onstack); free(comp); free(cs_v); free(cs_e);
    return ncomp;
}

/* -------------------------------------------------------- transpose ---- */
/*
 * G^T without self-loops: row v of (toff, tadj) lists every u != v with an arc
 * u -> v, in increasing u (one entry per arc, so duplicate arcs stay duplicated).
 * tadj must hold m entries. Returns the number of arcs written.
 */
OR_API int64_t or_transpose(int64_t n, const int32_t* off, const int32_t* adj, int32_t* toff, int32_t* tadj) {
    int64_t* cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    if (!cnt) return -1;
    for (int64_t u = 0; u < n; ++u)
        for (int64_t e = off[u]; e < off[u + 1]; ++e)
            if (adj[e] != u) cnt[adj[e] + 1]++;
    for (int64_t v = 0; v < n; ++v) cnt[v + 1] += cnt[v];
    for (int64_t v = 0; v <= n; ++v) toff[v] = (int32_t)cnt[v];
    for (int64_t u = 0; u < n; ++u)
        for (int64_t e = off[u]; e < off[u + 1]; ++e)
            if (adj[e] != u) tadj[cnt[adj[e]]++] = (int32_t)u;
    int64_t mt = toff[n];
    free(cnt);
    return mt;
}

/* ------------------------------------------------------------- trim ---- */
/*
 * flag[v] = 1 iff v has no out-arc or no in-arc to/from another vertex
 * (self-loops are not counted). Such a v is a singleton SCC. Returns the number
 * of flagged vertices.
 */
OR_API int64_t or_trim(int64_t n, const int32_t* off, const int32_t* adj, uint8_t* flag) {
    int64_t* indeg = (int64_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
    int64_t* outdeg = (int64_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
    if (!indeg || !outdeg) { free(indeg); free(outdeg); return -1; }
    for (int64_t u = 0; u < n; ++u)
        for (int64_t e = off[u]; e < off[u + 1]; ++e)
            if (adj[e] != u) { outdeg[u]++; indeg[adj[e]]++; }
    int64_t c = 0;
    for (int64_t v = 0; v < n; ++v) { flag[v] = (outdeg[v] == 0 || indeg[v] == 0); c += flag[v]; }
    free(indeg); free(outdeg);
    return c;
}

/* ------------------------------------------------------ reachability ---- */
/*
 * BFS from s inside its label class: a vertex w is entered over an arc (u,w)
 * only when label[w] == label[s]; a source with label[s] < 0 (finished) reaches
 * nothing. label == NULL means every vertex is in one class. (off, adj) is G for
 * a forward search, G^T for a backward one. queue must hold n entries; stamp[]
 * marks visited vertices with the value `mark`. Returns the number visited.
 */
static int64_t bfs_class(int64_t n, const int32_t* off, const int32_t* adj, const int32_t* label,
                         int32_t s, int32_t* queue, int32_t* stamp, int32_t mark) {
    (void)n;
    if (label && label[s] < 0) return 0;
    int32_t L = label ? label[s] : 0;
    int64_t head = 0, tail = 0;
    if (stamp[s] == mark) return 0;
    stamp[s] = mark; queue[tail++] = s;
    while (head < tail) {
        int32_t u = queue[head++];
        for (int64_t e = off[u]; e < off[u + 1]; ++e) {
            int32_t w = adj[e];
            if (stamp[w] == mark) continue;
            if (label && label[w] != L) continue;
            stamp[w] = mark; queue[tail++] = w;
        }
    }
    return tail;
}

/* visited[v] = 1 iff s reaches v inside s's label class. Returns the count. */
OR_API int64_t or_reach_set(int64_t n, const int32_t* off, const int32_t* adj, const int32_t* label,
                            int32_t s, uint8_t* visited) {
    int32_t* q = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t* st = (int32_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
    if (!q || !st) { free(q); free(st); return -1; }
    int64_t c = (s >= 0 && s < n) ? bfs_class(n, off, adj, label, s, q, st, 1) : 0;
    for (int64_t v = 0; v < n; ++v) visited[v] = (st[v] == 1);
    free(q); free(st);
    return c;
}

/*
 * The reachability pair set of a (forward or backward) multi-reachability search:
 * every (v, s) with s in sources[0..k) and s ~> v inside s's class. Pairs are
 * written as (uint64)v << 32 | s into pairs[] when the total fits in cap, each
 * source contributing its pairs in BFS order (duplicate sources contribute once).
 * Returns the total number of pairs (which may exceed cap), or -1 on allocation
 * failure.
 */
OR_API int64_t or_multi_reach(int64_t n, const int32_t* off, const int32_t* adj, const int32_t* label,
                              const int32_t* sources, int64_t k, uint64_t* pairs, int64_t cap) {
    int32_t* q = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t* st = (int32_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
    uint8_t* seen_src = (uint8_t*)calloc((size_t)(n > 0 ? n : 1), 1);
    if (!q || !st || !seen_src) { free(q); free(st); free(seen_src); return -1; }
    int64_t total = 0;
    for (int64_t j = 0; j < k; ++j) {
        int32_t s = sources[j];
        if (s < 0 || s >= n || seen_src[s]) continue;
        seen_src[s] = 1;
        int64_t c = bfs_class(n, off, adj, label, s, q, st, (int32_t)(j + 1));
        for (int64_t i = 0; i < c; ++i) {
            if (total < cap) pairs[total] = ((uint64_t)(uint32_t)q[i] << 32) | (uint32_t)s;
            ++total;
        }
    }
    free(q); free(st); free(seen_src);
    return total;
}

/*
 * Plain multi-source reachability (no classes): out[v] bit j = 1 iff sources[j]
 * reaches v in the given CSR (G for forward, G^T for backward), 1 <= k <= 64.
 */
OR_API int64_t or_reach_mask(int64_t n, const int32_t* off, const int32_t* adj,
                             const int32_t* sources, int64_t k, uint64_t* out) {
    if (k < 1 || k > 64) return -1;
    int32_t* q = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t* st = (int32_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
    if (!q || !st) { free(q); free(st); return -1; }
    memset(out, 0, sizeof(uint64_t) * (size_t)n);
    for (int64_t j = 0; j < k; ++j) {
        int32_t s = sources[j];
        if (s < 0 || s >= n) { free(q); free(st); return -1; }
        int64_t c = bfs_class(n, off, adj, NULL, s, q, st, (int32_t)(j + 1));
        for (int64_t i = 0; i < c; ++i) out[q[i]] |= (uint64_t)1 << j;
    }
    free(q); free(st);
    return 0;
}

/* --------------------------------------------------- pivot permutation ---- */
/*
 * SplitMix64 finaliser (Steele, Lea & Flood, OOPSLA 2014), used as the Feistel
 * round function. Keys: key_r = mix(seed + (r+1) * golden), r = 0..3.
 */
static uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
OR_API uint64_t or_mix64(uint64_t z) { return mix64(z); }

/*
 * A bijection of [0, N) (Black & Rogaway, "Ciphers with arbitrary finite
 * domains", CT-RSA 2002: a balanced Feistel network on the smallest even bit
 * width b >= 2 with 2^b >= N, applied repeatedly until the value falls in
 * [0, N) -- "cycle walking"). Four rounds; the round function for round r on the
 * right half R is the low b/2 bits of mix64(key_r ^ R).
 */
static uint64_t feistel_once(uint64_t x, int half, const uint64_t key[4]) {
    uint64_t mask = (half >= 64) ? ~0ull : ((1ull << half) - 1);
    uint64_t L = x >> half, R = x & mask;
    for (int r = 0; r < 4; ++r) {
        uint64_t F = mix64(key[r] ^ R) & mask;
        uint64_t nl = R, nr = L ^ F;
        L = nl; R = nr;
    }
    return (L << half) | R;
}

static int feistel_half_bits(uint64_t N) {
    int b = 2;
    while (b < 62 && (1ull << b) < N) b += 2;
    return b / 2;
}

/*
 * order[p] = act[pi(p)] for p in [0, N), where act is the increasing list of
 * vertices v with active[v] != 0 and pi the seeded bijection above. Returns N.
 */
OR_API int64_t or_pivot_order(int64_t n, const uint8_t* active, uint64_t seed, int32_t* order) {
    int32_t* act = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!act) return -1;
    int64_t N = 0;
    for (int64_t v = 0; v < n; ++v) if (active[v]) act[N++] = (int32_t)v;
    uint64_t key[4];
    for (int r = 0; r < 4; ++r) key[r] = mix64(seed + (uint64_t)(r + 1) * 0x9E3779B97F4A7C15ull);
    int half = feistel_half_bits((uint64_t)N);
    for (int64_t p = 0; p < N; ++p) {
        uint64_t y = feistel_once((uint64_t)p, half, key);
        while (y >= (uint64_t)N) y = feistel_once(y, half, key);
        order[p] = act[y];
    }
    free(act);
    return N;
}

/*
 * Prefix-doubling batch bounds over N permuted positions with multiplier beta:
 * batch i covers positions [bounds[i], bounds[i+1]) with size ceil(x_i), where
 * x_0 = 1 and x_{i+1} = x_i * beta in IEEE double; the last batch is clipped at
 * N. Writes at most maxb+1 bounds and returns the number of batches.
 */
OR_API int64_t or_batch_bounds(int64_t N, double beta, int64_t* bounds, int64_t maxb) {
    int64_t nb = 0, pos = 0;
    double x = 1.0;
    if (nb <= maxb) bounds[0] = 0;
    while (pos < N) {
        double c = x;
        int64_t sz;
        if (c >= (double)N) sz = N;       /* also keeps the cast in range */
        else { sz = (int64_t)c; if ((double)sz < c) ++sz; }  /* ceil */
        if (sz < 1) sz = 1;
        pos = (N - pos < sz) ? N : pos + sz;
        ++nb;
        if (nb <= maxb) bounds[nb] = pos;
        x *= beta;
    }
    return nb;
}

/* ------------------------------------------------- connected components ---- */
/*
 * Connectivity (Sec. 5.1, Alg. 4 output): the components of the undirected
 * graph in which every arc (u, v) of the CSR joins u and v (the paper
 * symmetrises directed inputs for connectivity). A sequential union-find over
 * the arcs: a union hooks the larger root under the smaller one, so the root of
 * a component is its smallest vertex id; finds halve the path. Writes
 * label[v] = smallest vertex id of v's component; returns the number of
 * components (-1 if memory could not be allocated).
 */
static int32_t uf_find(int32_t* parent, int32_t x) {
    while (parent[x] != x) {
        parent[x] = parent[parent[x]];
        x = parent[x];
    }
    return x;
}

OR_API int64_t or_cc_labels(int64_t n, const int32_t* off, const int32_t* adj, int32_t* label) {
    if (n == 0) return 0;
    int32_t* parent = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    if (!parent) return -1;
    for (int64_t v = 0; v < n; ++v) parent[v] = (int32_t)v;
    for (int64_t u = 0; u < n; ++u)
        for (int64_t e = off[u]; e < off[u + 1]; ++e) {
            int32_t a = uf_find(parent, (int32_t)u), b = uf_find(parent, adj[e]);
            if (a == b) continue;
            if (a < b) parent[b] = a;
            else parent[a] = b;
        }
    int64_t comps = 0;
    for (int64_t v = 0; v < n; ++v) {
        label[v] = uf_find(parent, (int32_t)v);
        if (label[v] == (int32_t)v) ++comps;
    }
    free(parent);
    return comps;
}

/* ---------------------------------------------------- least-element lists ---- */
/*
 * LE-lists (Sec. 5.2) of the undirected graph in which every arc (u, v) joins u
 * and v, for the vertex order order[0..n): source order[j] is in L(u) iff its
 * BFS distance d to u is smaller than the distance from u to every earlier
 * source. Sources are taken one at a time in order; a BFS from s expands a
 * vertex u first reached at distance d only if d < delta(u) (the smallest
 * distance from u to an earlier source), and then appends (s, d) to L(u) and
 * sets delta(u) = d -- Alg. 5 with batches of one source. Each list is in
 * source order, so its distances strictly decrease.
 * Output in CSR form: le_off[n + 1], entries le_src / le_dist (cap of them).
 * Returns the number of entries (written only if it is at most cap), or -1 if
 * memory could not be allocated.
 */
OR_API int64_t or_le_lists(int64_t n, const int32_t* off, const int32_t* adj, const int32_t* order, int64_t* le_off,
                           int32_t* le_src, int32_t* le_dist, int64_t cap) {
    if (n == 0) {
        le_off[0] = 0;
        return 0;
    }
    int64_t m = off[n];
    /* symmetric adjacency: out-arcs and in-arcs of every vertex */
    int64_t* so = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    int32_t* sa = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * m > 0 ? 2 * m : 1));
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    int32_t* delta = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    int32_t* dist = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    int64_t* stamp = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    int32_t* queue = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    int64_t tcap = 4 * n + 16, tn = 0;
    int32_t* tu = (int32_t*)malloc(sizeof(int32_t) * (size_t)tcap);
    int32_t* ts = (int32_t*)malloc(sizeof(int32_t) * (size_t)tcap);
    int32_t* td = (int32_t*)malloc(sizeof(int32_t) * (size_t)tcap);
    int64_t ret = -1;
    if (!so || !sa || !fill || !delta || !dist || !stamp || !queue || !tu || !ts || !td) goto done;
    for (int64_t u = 0; u < n; ++u)
        for (int64_t e = off[u]; e < off[u + 1]; ++e) {
            ++so[u + 1];
            ++so[adj[e] + 1];
        }
    for (int64_t u = 0; u < n; ++u) so[u + 1] += so[u];
    for (int64_t u = 0; u < n; ++u) fill[u] = so[u];
    for (int64_t u = 0; u < n; ++u)
        for (int64_t e = off[u]; e < off[u + 1]; ++e) {
            sa[fill[u]++] = adj[e];
            sa[fill[adj[e]]++] = (int32_t)u;
        }
    for (int64_t u = 0; u < n; ++u) {
        delta[u] = INT32_MAX;
        stamp[u] = -1;
    }
    for (int64_t j = 0; j < n; ++j) {
        int32_t s = order[j];
        int64_t qh = 0, qt = 0;
        queue[qt++] = s;
        stamp[s] = j;
        dist[s] = 0;
        while (qh < qt) {
            int32_t u = queue[qh++];
            int32_t d = dist[u];
            if (d >= delta[u]) continue; /* an earlier source is as close: pruned */
            delta[u] = d;
            if (tn == tcap) {
                int64_t nc = 2 * tcap;
                int32_t* a = (int32_t*)realloc(tu, sizeof(int32_t) * (size_t)nc);
                if (!a) goto done;
                tu = a;
                a = (int32_t*)realloc(ts, sizeof(int32_t) * (size_t)nc);
                if (!a) goto done;
                ts = a;
                a = (int32_t*)realloc(td, sizeof(int32_t) * (size_t)nc);
                if (!a) goto done;
                td = a;
                tcap = nc;
            }
            tu[tn] = u;
            ts[tn] = s;
            td[tn] = d;
            ++tn;
            for (int64_t e = so[u]; e < so[u + 1]; ++e) {
                int32_t w = sa[e];
                if (stamp[w] == j) continue;
                stamp[w] = j;
                dist[w] = d + 1;
                queue[qt++] = w;
            }
        }
    }
    ret = tn;
    if (tn <= cap) {
        /* group by vertex, keeping the order in which entries were found */
        for (int64_t u = 0; u <= n; ++u) le_off[u] = 0;
        for (int64_t i = 0; i < tn; ++i) ++le_off[tu[i] + 1];
        for (int64_t u = 0; u < n; ++u) le_off[u + 1] += le_off[u];
        for (int64_t u = 0; u < n; ++u) fill[u] = le_off[u];
        for (int64_t i = 0; i < tn; ++i) {
            int64_t p = fill[tu[i]]++;
            le_src[p] = ts[i];
            le_dist[p] = td[i];
        }
    }
done:
    free(so); free(sa); free(fill); free(delta); free(dist); free(stamp); free(queue);
    free(tu); free(ts); free(td);
    return ret;
}
