// Labelling after a forward and a backward multi-reachability search
// (Alg. 1 label step; Sec. 4.4), as grid-stride device functions of the
// device-side batch loop.
//
// T_out holds pairs (v, s) with s ~> v, T_in pairs (v, s) with v ~> s, both as
// keys v << 32 | s in open-addressed tables. For every touched vertex v:
//   fmax[v] = max s over T_out, bmax[v] = max s over T_in,
//   hit[v]  = max s over T_out n T_in  (= max of R1 n R2 in Alg. 1).
// All three are 64-bit maxima tagged with the batch index in the high word, so
// they never need clearing between batches. Then exactly one table entry per
// vertex (the one carrying fmax, or bmax when v is not in T_out) rewrites v's
// label: finished (label kDone, rep = hit) when R1 n R2 is not empty, else the
// hash of its old class and its two maxima.
#pragma once
#include "common.cuh"
#include "engine.cuh"

namespace scc {

// Both passes walk the two tables as one index space of 16-byte entry pairs
// (capacities are powers of two >= 2, the tables 16-byte aligned), four pairs
// per thread per iteration with their loads issued together, so each thread
// keeps eight table entries in flight instead of one.
constexpr int kLabelUnroll = 4;

__device__ __forceinline__ ulonglong2 load_pair(const unsigned long long* tf, long long nf,
                                                const unsigned long long* tb, long long tot, long long j) {
    if (j < nf) return reinterpret_cast<const ulonglong2*>(tf)[j];
    if (j < tot) return reinterpret_cast<const ulonglong2*>(tb)[j - nf];
    return make_ulonglong2(~0ull, ~0ull);
}

__device__ __forceinline__ void label_scan(long long i0, long long stride, const unsigned long long* __restrict__ tf,
                                           long long capf, const PairTable& tb, unsigned long long tag,
                                           unsigned long long* fmax, unsigned long long* bmax,
                                           unsigned long long* hit) {
    constexpr int U = kLabelUnroll;
    const long long nf = capf / 2, tot = nf + (long long)(tb.mask + 1) / 2;
    for (long long i = i0; i < tot; i += U * stride) {
        unsigned long long key[2 * U];
        bool fw[2 * U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long long j = i + u * stride;
            const ulonglong2 e = load_pair(tf, nf, tb.keys, tot, j);
            key[2 * u] = e.x;
            key[2 * u + 1] = e.y;
            fw[2 * u] = fw[2 * u + 1] = j < nf;
        }
        // first probe of every forward key in T_in, issued together
        unsigned long long h[2 * U], c[2 * U];
#pragma unroll
        for (int k = 0; k < 2 * U; ++k) {
            h[k] = PairTable::hash(key[k]) & tb.mask;
            c[k] = (fw[k] && key[k] != ~0ull) ? tb.keys[h[k]] : ~0ull;
        }
#pragma unroll
        for (int k = 0; k < 2 * U; ++k) {
            if (key[k] == ~0ull) continue;
            const uint32_t v = (uint32_t)(key[k] >> 32), s = (uint32_t)key[k];
            if (!fw[k]) {
                atomicMax(&bmax[v], tag | s);
                continue;
            }
            atomicMax(&fmax[v], tag | s);
            bool in = c[k] == key[k];
            if (!in && c[k] != ~0ull) in = tb.contains_from((h[k] + 1) & tb.mask, key[k]);
            if (in) atomicMax(&hit[v], tag | s);
        }
    }
}

__device__ __forceinline__ void finalize_vertex(uint32_t v, unsigned long long tag, const unsigned long long* fmax,
                                                const unsigned long long* bmax, const unsigned long long* hit,
                                                int32_t* label, int32_t* rep, unsigned long long& c) {
    const unsigned long long h = hit[v], f = fmax[v], b = bmax[v];
    if ((h & 0xffffffff00000000ull) == tag) {
        label[v] = kDone;
        rep[v] = (int32_t)(uint32_t)h;
        ++c;
    } else {
        const int32_t a = (f & 0xffffffff00000000ull) == tag ? (int32_t)(uint32_t)f : -1;
        const int32_t bb = (b & 0xffffffff00000000ull) == tag ? (int32_t)(uint32_t)b : -1;
        label[v] = class_hash(label[v], a, bb);
    }
}

// Returns how many vertices this thread finished. With `clear`, every entry is
// reset to empty once used (each entry is read by exactly one thread here), so
// the tables are empty again for the next batch.
__device__ __forceinline__ unsigned long long label_finalize(long long i0, long long stride,
                                                             unsigned long long* __restrict__ tf, long long capf,
                                                             unsigned long long* __restrict__ tb, long long capb,
                                                             unsigned long long tag, const unsigned long long* fmax,
                                                             const unsigned long long* bmax,
                                                             const unsigned long long* hit, int32_t* label,
                                                             int32_t* rep, bool clear) {
    constexpr int U = kLabelUnroll;
    constexpr unsigned long long kHi = 0xffffffff00000000ull;
    const long long nf = capf / 2, tot = nf + capb / 2;
    unsigned long long c = 0;
    for (long long i = i0; i < tot; i += U * stride) {
        unsigned long long key[2 * U];
        bool fw[2 * U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long long j = i + u * stride;
            const ulonglong2 e = load_pair(tf, nf, tb, tot, j);
            key[2 * u] = e.x;
            key[2 * u + 1] = e.y;
            fw[2 * u] = fw[2 * u + 1] = j < nf;
        }
        if (clear) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const long long j = i + u * stride;
                if (key[2 * u] == ~0ull && key[2 * u + 1] == ~0ull) continue;
                ulonglong2* p = j < nf ? reinterpret_cast<ulonglong2*>(tf) + j
                                       : reinterpret_cast<ulonglong2*>(tb) + (j - nf);
                *p = make_ulonglong2(~0ull, ~0ull);
            }
        }
        unsigned long long f[2 * U];
#pragma unroll
        for (int k = 0; k < 2 * U; ++k) f[k] = key[k] != ~0ull ? fmax[(uint32_t)(key[k] >> 32)] : 0ull;
#pragma unroll
        for (int k = 0; k < 2 * U; ++k) {
            if (key[k] == ~0ull) continue;
            const uint32_t v = (uint32_t)(key[k] >> 32), s = (uint32_t)key[k];
            // the entry that carries fmax owns v; when v is not in T_out, the one
            // carrying bmax does
            const bool owner = fw[k] ? f[k] == (tag | s) : ((f[k] & kHi) != tag && bmax[v] == (tag | s));
            if (owner) finalize_vertex(v, tag, fmax, bmax, hit, label, rep, c);
        }
    }
    return c;
}

}  // namespace scc
