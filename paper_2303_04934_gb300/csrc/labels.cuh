// Labelling after a forward and a backward multi-reachability search
// (Alg. 1 label step; Sec. 4.4), as grid-stride device functions shared by the
// host-launched kernels and the device-side batch loop.
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

__device__ __forceinline__ void label_scan(long long i0, long long stride, const unsigned long long* __restrict__ tf,
                                           long long capf, const PairTable& tb, unsigned long long tag,
                                           unsigned long long* fmax, unsigned long long* bmax,
                                           unsigned long long* hit) {
    const long long capb = (long long)tb.mask + 1;
    for (long long i = i0; i < capf + capb; i += stride) {
        if (i < capf) {
            const unsigned long long key = tf[i];
            if (key == ~0ull) continue;
            const uint32_t v = (uint32_t)(key >> 32), s = (uint32_t)key;
            atomicMax(&fmax[v], tag | s);
            if (tb.contains(key)) atomicMax(&hit[v], tag | s);
        } else {
            const unsigned long long key = tb.keys[i - capf];
            if (key == ~0ull) continue;
            atomicMax(&bmax[(uint32_t)(key >> 32)], tag | (uint32_t)key);
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
    unsigned long long c = 0;
    for (long long i = i0; i < capf + capb; i += stride) {
        const bool fw = i < capf;
        const unsigned long long key = fw ? tf[i] : tb[i - capf];
        if (key == ~0ull) continue;
        if (clear) {
            if (fw) tf[i] = ~0ull;
            else tb[i - capf] = ~0ull;
        }
        const uint32_t v = (uint32_t)(key >> 32), s = (uint32_t)key;
        const unsigned long long f = fmax[v];
        const bool owner = fw ? f == (tag | s)
                              : ((f & 0xffffffff00000000ull) != tag && bmax[v] == (tag | s));
        if (owner) finalize_vertex(v, tag, fmax, bmax, hit, label, rep, c);
    }
    return c;
}

}  // namespace scc
