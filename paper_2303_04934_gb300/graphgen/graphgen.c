/*
 * Seeded synthetic directed-graph generators (host C, OpenMP).
 *
 * This module produces INPUTS only: int32 CSR graphs (offsets[n+1], targets[m],
 * rows sorted by source). It contains none of the SCC method's arithmetic and is
 * shared by the CUDA path's tests/benchmark and by the CPU oracle's tests.
 *
 * Every random draw is a counter-based SplitMix64 value (Steele, Lea & Flood,
 * "Fast splittable pseudorandom number generators", OOPSLA 2014; finaliser
 * constants as published there), so a graph depends only on (parameters, seed),
 * never on the thread count or the machine.
 *
 * Families (paper Sec. 6 "Setup" describes the lattice models; the other
 * families are stand-ins for the paper's social/web and k-NN graphs):
 *   - torus lattices in 2D / 3D where each of the 2*dims neighbour arcs of every
 *     vertex is present independently with probability p (rows/columns circular);
 *   - the paper's SQR/REC model (each vertex draws, for each of its 4 neighbours,
 *     one arc in a random direction; duplicates removed) and SQR'/REC' model (each
 *     of the two arcs between adjacent vertices present independently w.p. 0.3);
 *   - R-MAT (Chakrabarti, Zhan & Faloutsos, SDM 2004) with self-loops and
 *     duplicate arcs removed and vertex ids randomly permuted;
 *   - directed k-NN graphs of points drawn from a mixture of isotropic 3D
 *     Gaussians (exact k nearest neighbours, self excluded, squared float32
 *     distance, ties to the smaller index).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <omp.h>

#define GG_API __attribute__((visibility("default")))

/* ---------------------------------------------------------------- RNG ---- */
static inline uint64_t sm64(uint64_t seed, uint64_t ctr) {
    uint64_t z = seed + (ctr + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
/* stream separation: each family/purpose hashes its own stream id into the seed */
static inline uint64_t stream_seed(uint64_t seed, uint64_t stream) {
    return sm64(seed ^ 0xD1B54A32D192ED03ull, stream);
}
static inline double u01(uint64_t x) { return (double)(x >> 11) * (1.0 / 9007199254740992.0); }

static void set_threads(int threads) {
    if (threads > 0) omp_set_num_threads(threads);
}

/* exclusive scan of cnt[0..n) into off[0..n], returns total */
static int64_t scan_counts(const int64_t* cnt, int32_t* off, int64_t n) {
    int64_t s = 0;
    for (int64_t i = 0; i < n; ++i) { off[i] = (int32_t)s; s += cnt[i]; }
    off[n] = (int32_t)s;
    return s;
}

/* ------------------------------------------------------- torus lattices ---- */
/* neighbour of v=(x,y,z) in direction d: d = 2*axis + (0:+1, 1:-1) */
static inline int64_t torus_nb(int64_t v, int d, int64_t X, int64_t Y, int64_t Z) {
    int64_t x = v % X, y = (v / X) % Y, z = v / (X * Y);
    int axis = d >> 1, neg = d & 1;
    if (axis == 0) x = neg ? (x + X - 1) % X : (x + 1) % X;
    else if (axis == 1) y = neg ? (y + Y - 1) % Y : (y + 1) % Y;
    else z = neg ? (z + Z - 1) % Z : (z + 1) % Z;
    return (z * Y + y) * X + x;
}

/*
 * Torus with independent arcs: every vertex v and direction d in [0, 2*dims)
 * carries the arc v -> nb(v,d) with probability p. dims is 2 (Z must be 1) or 3.
 * adj must hold 2*dims*n entries. Returns m, or -1 on bad arguments.
 */
GG_API int64_t gg_torus(int dims, int64_t X, int64_t Y, int64_t Z, double p, uint64_t seed,
                        int32_t* off, int32_t* adj, int threads) {
    if (dims < 1 || dims > 3 || X < 1 || Y < 1 || Z < 1) return -1;
    if (dims < 3 && Z != 1) return -1;
    if (dims < 2 && Y != 1) return -1;
    int64_t n = X * Y * Z;
    if (n > 2147483647ll / (2 * dims)) return -1;
    set_threads(threads);
    const int nd = 2 * dims;
    const uint64_t ss = stream_seed(seed, 0x70125ull + (uint64_t)dims);
    int64_t* cnt = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    #pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < n; ++v) {
        int64_t c = 0;
        for (int d = 0; d < nd; ++d) c += u01(sm64(ss, (uint64_t)v * nd + d)) < p;
        cnt[v] = c;
    }
    int64_t m = scan_counts(cnt, off, n);
    #pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < n; ++v) {
        int64_t o = off[v];
        for (int d = 0; d < nd; ++d)
            if (u01(sm64(ss, (uint64_t)v * nd + d)) < p) adj[o++] = (int32_t)torus_nb(v, d, X, Y, Z);
    }
    free(cnt);
    return m;
}

/*
 * The paper's 2D lattice models on an X-by-Y torus (Sec. 6, "Setup").
 * model 0 (SQR/REC): vertex u, for each of its 4 neighbours v, adds u->v with
 *   probability 0.5 and v->u otherwise; duplicates are then removed. Every
 *   adjacent pair is therefore drawn twice (once from each end).
 * model 1 (SQR'/REC'): each of the two arcs u->v and v->u of every adjacent
 *   pair is present independently with probability 0.3. (The paper's wording
 *   lists 0.3 / 0.3 / 0.4 outcomes; the independent reading is the one whose
 *   arc count, m = 0.6 * 2n, and SCC count agree with its table of SCC running times (Table 2).)
 * adj must hold 4*n entries. Returns m.
 */
GG_API int64_t gg_paper_lattice(int64_t X, int64_t Y, int model, uint64_t seed,
                                int32_t* off, int32_t* adj, int threads) {
    if (X < 3 || Y < 3 || (model != 0 && model != 1)) return -1;
    int64_t n = X * Y;
    if (n > 2147483647ll / 4) return -1;
    set_threads(threads);
    const uint64_t ss = stream_seed(seed, 0x5A11ull + (uint64_t)model);
    int64_t* cnt = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    /* out-arc u->w for neighbour w = nb(u,d), computed locally from the draws
       that concern the pair {u,w}. */
    #define LATTICE_ARC(u, d, res)                                                        \
        do {                                                                           \
            int64_t w_ = torus_nb((u), (d), X, Y, 1);                                  \
            int dop_ = (d) ^ 1; /* direction from w back to u */                       \
            if (model == 0) {                                                          \
                /* draw of u for neighbour w: <0.5 gives u->w; draw of w for u: */     \
                /* >=0.5 gives (w's "v->u" case) u->w                              */  \
                int a_ = u01(sm64(ss, (uint64_t)(u) * 4 + (d))) < 0.5;                 \
                int b_ = !(u01(sm64(ss, (uint64_t)w_ * 4 + dop_)) < 0.5);              \
                (res) = a_ | b_;                                                       \
            } else {                                                                   \
                (res) = u01(sm64(ss, (uint64_t)(u) * 4 + (d))) < 0.3;                   \
            }                                                                          \
        } while (0)
    #pragma omp parallel for schedule(static)
    for (int64_t u = 0; u < n; ++u) {
        int64_t c = 0;
        for (int d = 0; d < 4; ++d) { int r; LATTICE_ARC(u, d, r); c += r; }
        cnt[u] = c;
    }
    int64_t m = scan_counts(cnt, off, n);
    #pragma omp parallel for schedule(static)
    for (int64_t u = 0; u < n; ++u) {
        int64_t o = off[u];
        for (int d = 0; d < 4; ++d) {
            int r; LATTICE_ARC(u, d, r);
            if (r) adj[o++] = (int32_t)torus_nb(u, d, X, Y, 1);
        }
    }
    #undef LATTICE_ARC
    free(cnt);
    return m;
}

/* ---------------------------------------------------- parallel radix sort ---- */
/* LSD radix sort of 64-bit keys on the low `bits` bits; result in keys. */
static void radix_sort_u64(uint64_t* keys, uint64_t* tmp, int64_t n, int bits) {
    const int R = 11, B = 1 << R;
    int nth = omp_get_max_threads();
    int64_t* hist = (int64_t*)malloc(sizeof(int64_t) * (size_t)nth * B);
    uint64_t* src = keys; uint64_t* dst = tmp;
    int passes = (bits + R - 1) / R;
    for (int ps = 0; ps < passes; ++ps) {
        int sh = ps * R;
        memset(hist, 0, sizeof(int64_t) * (size_t)nth * B);
        #pragma omp parallel num_threads(nth)
        {
            int t = omp_get_thread_num();
            int64_t lo = n * t / nth, hi = n * (t + 1) / nth;
            int64_t* h = hist + (int64_t)t * B;
            for (int64_t i = lo; i < hi; ++i) h[(src[i] >> sh) & (B - 1)]++;
        }
        int64_t s = 0;
        for (int d = 0; d < B; ++d)
            for (int t = 0; t < nth; ++t) { int64_t c = hist[(int64_t)t * B + d]; hist[(int64_t)t * B + d] = s; s += c; }
        #pragma omp parallel num_threads(nth)
        {
            int t = omp_get_thread_num();
            int64_t lo = n * t / nth, hi = n * (t + 1) / nth;
            int64_t* h = hist + (int64_t)t * B;
            for (int64_t i = lo; i < hi; ++i) { uint64_t k = src[i]; dst[h[(k >> sh) & (B - 1)]++] = k; }
        }
        uint64_t* x = src; src = dst; dst = x;
    }
    if (src != keys) memcpy(keys, src, sizeof(uint64_t) * (size_t)n);
    free(hist);
}

/* CSR from sorted (src<<32|dst) keys with duplicates removed. Returns m. */
static int64_t csr_from_sorted_keys(const uint64_t* keys, int64_t M, int64_t n, int32_t* off, int32_t* adj) {
    int nth = omp_get_max_threads();
    int64_t* uc = (int64_t*)calloc((size_t)nth + 1, sizeof(int64_t));
    #pragma omp parallel num_threads(nth)
    {
        int t = omp_get_thread_num();
        int64_t lo = M * t / nth, hi = M * (t + 1) / nth, c = 0;
        for (int64_t i = lo; i < hi; ++i) c += (i == 0 || keys[i] != keys[i - 1]);
        uc[t + 1] = c;
    }
    for (int t = 0; t < nth; ++t) uc[t + 1] += uc[t];
    #pragma omp parallel num_threads(nth)
    {
        int t = omp_get_thread_num();
        int64_t lo = M * t / nth, hi = M * (t + 1) / nth, o = uc[t];
        for (int64_t i = lo; i < hi; ++i)
            if (i == 0 || keys[i] != keys[i - 1]) adj[o++] = (int32_t)(keys[i] & 0xffffffffu);
    }
    int64_t m = uc[nth];
    /* offsets: first unique index of each source row */
    int64_t* cnt = (int64_t*)calloc((size_t)n, sizeof(int64_t));
    #pragma omp parallel num_threads(nth)
    {
        int t = omp_get_thread_num();
        int64_t lo = M * t / nth, hi = M * (t + 1) / nth;
        for (int64_t i = lo; i < hi; ++i)
            if (i == 0 || keys[i] != keys[i - 1]) {
                int64_t u = (int64_t)(keys[i] >> 32);
                __atomic_fetch_add(&cnt[u], 1, __ATOMIC_RELAXED);
            }
    }
    scan_counts(cnt, off, n);
    free(cnt); free(uc);
    return m;
}

/*
 * R-MAT: nsamples arcs drawn by recursive quadrant choice over `scale` levels with
 * probabilities (a, b, c, 1-a-b-c); self-loops dropped, duplicates removed. If
 * `permute`, vertex ids are relabelled by a seeded uniform permutation
 * (Fisher-Yates) before the CSR is built. adj must hold nsamples entries.
 * Returns m.
 */
GG_API int64_t gg_rmat(int scale, int64_t nsamples, double a, double b, double c, uint64_t seed,
                       int permute, int32_t* off, int32_t* adj, int threads) {
    if (scale < 1 || scale > 30 || nsamples < 0 || a < 0 || b < 0 || c < 0 || a + b + c > 1.0) return -1;
    set_threads(threads);
    int64_t n = (int64_t)1 << scale;
    const uint64_t ss = stream_seed(seed, 0x12A7ull);
    const uint64_t sp = stream_seed(seed, 0x9E57ull);
    const double ab = a + b, abc = a + b + c;
    uint32_t* perm = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) perm[i] = (uint32_t)i;
    if (permute)
        for (int64_t i = n - 1; i > 0; --i) {
            uint64_t j = sm64(sp, (uint64_t)i) % (uint64_t)(i + 1);
            uint32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
        }
    uint64_t* keys = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(nsamples > 0 ? nsamples : 1));
    int64_t* kept = (int64_t*)calloc((size_t)omp_get_max_threads() + 1, sizeof(int64_t));
    int nth = omp_get_max_threads();
    /* draw samples; each thread keeps its non-self-loop samples compacted in place
       within its own index range, then ranges are concatenated */
    #pragma omp parallel num_threads(nth)
    {
        int t = omp_get_thread_num();
        int64_t lo = nsamples * t / nth, hi = nsamples * (t + 1) / nth, o = lo;
        for (int64_t i = lo; i < hi; ++i) {
            uint64_t u = 0, v = 0, r = 0;
            for (int l = 0; l < scale; ++l) {
                if ((l & 1) == 0) r = sm64(ss, (uint64_t)i * 16 + (uint64_t)(l >> 1));
                uint32_t half = (l & 1) ? (uint32_t)(r >> 32) : (uint32_t)r;
                double x = (double)half * (1.0 / 4294967296.0);
                int bu, bv;
                if (x < a) { bu = 0; bv = 0; }
                else if (x < ab) { bu = 0; bv = 1; }
                else if (x < abc) { bu = 1; bv = 0; }
                else { bu = 1; bv = 1; }
                u = (u << 1) | (uint64_t)bu; v = (v << 1) | (uint64_t)bv;
            }
            uint64_t pu = perm[u], pv = perm[v];
            if (pu != pv) keys[o++] = (pu << 32) | pv;
        }
        kept[t + 1] = o - lo;
    }
    int64_t M = 0;
    for (int t = 0; t < nth; ++t) {
        int64_t lo = nsamples * t / nth;
        if (M != lo) memmove(keys + M, keys + lo, sizeof(uint64_t) * (size_t)kept[t + 1]);
        M += kept[t + 1];
    }
    uint64_t* tmp = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(M > 0 ? M : 1));
    radix_sort_u64(keys, tmp, M, 32 + scale);
    free(tmp);
    int64_t m = csr_from_sorted_keys(keys, M, n, off, adj);
    free(keys); free(perm); free(kept);
    return m;
}

/* ----------------------------------------------------------------- k-NN ---- */
typedef struct { float d; int32_t j; } cand_t;

static inline int cand_less(float d, int32_t j, const cand_t* c) {
    return d < c->d || (d == c->d && j < c->j);
}

/*
 * Directed k-NN graph over n points drawn from `clusters` isotropic Gaussians
 * (standard deviation sigma per axis) whose centres are uniform in the unit
 * cube; every point picks a cluster uniformly. Arc i -> j for each of the k
 * nearest points j != i under squared float32 distance, ties to the smaller j.
 * Exact search over a uniform grid with ring expansion. adj must hold k*n entries;
 * pts (optional, 3n floats) receives the coordinates. Returns m = k*n.
 */
GG_API int64_t gg_knn(int64_t n, int clusters, double sigma, int k, uint64_t seed,
                      int32_t* off, int32_t* adj, float* pts_out, int threads) {
    if (n < 0 || clusters < 1 || k < 1 || k > 64 || (n > 0 && k >= n) || n * k > 2147483647ll) return -1;
    set_threads(threads);
    const uint64_t sc = stream_seed(seed, 0xC1u), sp = stream_seed(seed, 0x9075u);
    float* P = pts_out ? pts_out : (float*)malloc(sizeof(float) * 3 * (size_t)(n > 0 ? n : 1));
    double* cen = (double*)malloc(sizeof(double) * 3 * (size_t)clusters);
    for (int c = 0; c < clusters * 3; ++c) cen[c] = u01(sm64(sc, (uint64_t)c));
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        uint64_t base = (uint64_t)i * 8;
        int c = (int)(sm64(sp, base) % (uint64_t)clusters);
        for (int ax = 0; ax < 3; ++ax) {
            /* Box-Muller from two uniforms in (0,1] and [0,1) */
            double u1 = 1.0 - u01(sm64(sp, base + 1 + 2 * ax));
            double u2 = u01(sm64(sp, base + 2 + 2 * ax));
            double g = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
            P[3 * i + ax] = (float)(cen[3 * c + ax] + sigma * g);
        }
    }
    free(cen);
    for (int64_t i = 0; i <= n; ++i) off[i] = (int32_t)(i * k);
    if (n == 0) { if (!pts_out) free(P); return 0; }
    /* grid */
    float lo[3] = {P[0], P[1], P[2]}, hi[3] = {P[0], P[1], P[2]};
    for (int64_t i = 0; i < n; ++i)
        for (int ax = 0; ax < 3; ++ax) {
            float x = P[3 * i + ax];
            if (x < lo[ax]) lo[ax] = x;
            if (x > hi[ax]) hi[ax] = x;
        }
    double ext = 0;
    for (int ax = 0; ax < 3; ++ax) if (hi[ax] - lo[ax] > ext) ext = hi[ax] - lo[ax];
    if (ext <= 0) ext = 1;
    int64_t G = (int64_t)ceil(cbrt((double)n * 2.0));
    if (G < 1) G = 1;
    if (G > 1024) G = 1024;
    double cs = ext / (double)G * (1.0 + 1e-9);
    int64_t NC = G * G * G;
    int32_t* cell = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    int64_t* cstart = (int64_t*)calloc((size_t)NC + 1, sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) {
        int64_t ci[3];
        for (int ax = 0; ax < 3; ++ax) {
            int64_t q = (int64_t)((P[3 * i + ax] - lo[ax]) / cs);
            ci[ax] = q < 0 ? 0 : (q >= G ? G - 1 : q);
        }
        cell[i] = (int32_t)((ci[2] * G + ci[1]) * G + ci[0]);
        cstart[cell[i] + 1]++;
    }
    for (int64_t c = 0; c < NC; ++c) cstart[c + 1] += cstart[c];
    int32_t* order = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    {
        int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)NC);
        memcpy(fill, cstart, sizeof(int64_t) * (size_t)NC);
        for (int64_t i = 0; i < n; ++i) order[fill[cell[i]]++] = (int32_t)i;
        free(fill);
    }
    #pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t i = 0; i < n; ++i) {
        cand_t best[64];
        int nb = 0;
        const float xi = P[3 * i], yi = P[3 * i + 1], zi = P[3 * i + 2];
        int64_t c0 = cell[i];
        int64_t cx = c0 % G, cy = (c0 / G) % G, cz = c0 / (G * G);
        for (int64_t r = 0;; ++r) {
            for (int64_t z = cz - r; z <= cz + r; ++z) {
                if (z < 0 || z >= G) continue;
                for (int64_t y = cy - r; y <= cy + r; ++y) {
                    if (y < 0 || y >= G) continue;
                    int onshell_zy = (z == cz - r || z == cz + r || y == cy - r || y == cy + r);
                    for (int64_t x = cx - r; x <= cx + r; ++x) {
                        if (x < 0 || x >= G) continue;
                        if (!onshell_zy && x != cx - r && x != cx + r) continue;
                        int64_t cc = (z * G + y) * G + x;
                        for (int64_t q = cstart[cc]; q < cstart[cc + 1]; ++q) {
                            int32_t j = order[q];
                            if (j == i) continue;
                            float dx = xi - P[3 * j], dy = yi - P[3 * j + 1], dz = zi - P[3 * j + 2];
                            float d = dx * dx + dy * dy + dz * dz;
                            if (nb < k) {
                                int p = nb++;
                                while (p > 0 && cand_less(d, j, &best[p - 1])) { best[p] = best[p - 1]; --p; }
                                best[p].d = d; best[p].j = j;
                            } else if (cand_less(d, j, &best[k - 1])) {
                                int p = k - 1;
                                while (p > 0 && cand_less(d, j, &best[p - 1])) { best[p] = best[p - 1]; --p; }
                                best[p].d = d; best[p].j = j;
                            }
                        }
                    }
                }
            }
            /* lower bound on the distance to any point outside the searched block */
            if (cx - r <= 0 && cy - r <= 0 && cz - r <= 0 && cx + r >= G - 1 && cy + r >= G - 1 && cz + r >= G - 1)
                break; /* searched everything */
            if (nb == k) {
                double bnd = 1e300;
                const float pi[3] = {xi, yi, zi};
                const int64_t cc3[3] = {cx, cy, cz};
                for (int ax = 0; ax < 3; ++ax) {
                    double blo = lo[ax] + (double)(cc3[ax] - r) * cs;     /* block lower face */
                    double bhi = lo[ax] + (double)(cc3[ax] + r + 1) * cs; /* block upper face */
                    if (cc3[ax] - r > 0) { double g = pi[ax] - blo; if (g < bnd) bnd = g; }
                    if (cc3[ax] + r < G - 1) { double g = bhi - pi[ax]; if (g < bnd) bnd = g; }
                }
                /* stop only when every unseen point is strictly farther than the
                   k-th candidate (with a relative margin for float rounding) */
                if (bnd > 0 && bnd * bnd > (double)best[k - 1].d * (1.0 + 1e-5) + 1e-30) break;
            }
        }
        for (int t = 0; t < k; ++t) adj[i * k + t] = best[t].j;
    }
    free(order); free(cstart); free(cell);
    if (!pts_out) free(P);
    return n * k;
}

/* Uniform random digraph (Erdos-Renyi G(n,p) over ordered pairs, self-loops
   optional), for small test graphs. adj must hold n*n entries. Returns m. */
GG_API int64_t gg_gnp(int64_t n, double p, int allow_self, uint64_t seed, int32_t* off, int32_t* adj) {
    if (n < 0 || n > 46340) return -1;
    const uint64_t ss = stream_seed(seed, 0x6A9ull);
    int64_t o = 0;
    for (int64_t u = 0; u < n; ++u) {
        off[u] = (int32_t)o;
        for (int64_t v = 0; v < n; ++v) {
            if (u == v && !allow_self) continue;
            if (u01(sm64(ss, (uint64_t)(u * n + v))) < p) adj[o++] = (int32_t)v;
        }
    }
    off[n] = (int32_t)o;
    return o;
}
