// Device helpers shared by the SCC kernels (sm_103a).
#pragma once
#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

#include "../../include/scc.h"

namespace scc {

constexpr int kWarp = 32;
constexpr uint32_t kFull = 0xffffffffu;

// Finished vertices carry this label; active classes are >= 0 (Alg. 1 keeps the
// finished set V \ V' implicit; here it is a reserved label value).
constexpr int32_t kDone = -1;

// ---------------------------------------------------------------- hashing --
// SplitMix64 finaliser (Steele, Lea & Flood, OOPSLA 2014).
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// New class id of an unfinished vertex (Alg. 1 "hash(L[i], R1, R2)"): a 31-bit
// hash of the old class and the largest source reaching it / reached by it
// (-1 for none). Equal inputs give equal ids, so an SCC is never split; an
// (improbable) collision only merges classes, which costs work but never
// changes a result.
__host__ __device__ __forceinline__ int32_t class_hash(int32_t old_label, int32_t max_from, int32_t max_to) {
    uint64_t z = ((uint64_t)(uint32_t)old_label << 32) | (uint32_t)max_from;
    z = mix64(z + 0x9E3779B97F4A7C15ull);
    z ^= (uint64_t)(uint32_t)max_to * 0xD6E8FEB86659FD93ull;
    z = mix64(z);
    return (int32_t)(z >> 33);
}

// ------------------------------------------------------------ warp helpers --
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}
__device__ __forceinline__ int warp_incl_scan(int x) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        int y = __shfl_up_sync(kFull, x, d);
        if (lane_id() >= d) x += y;
    }
    return x;
}
__device__ __forceinline__ uint32_t shfl_any(uint32_t v, int src) { return __shfl_sync(kFull, v, src); }
__device__ __forceinline__ uint64_t shfl_any(uint64_t v, int src) {
    return (uint64_t)__shfl_sync(kFull, (unsigned long long)v, src);
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <class T>
__device__ __forceinline__ T ld_volatile(const T* p) {
    return *(const volatile T*)p;
}

// ---------------------------------------------------------- grid barrier --
// Sense-by-generation barrier for a cooperative (co-resident) grid. The spin
// has a time limit: past it the block records SCC_ERR_TIMEOUT in *err and
// returns false, so a kernel can never hang the GPU.
struct GridBarrier {
    unsigned int count;
    unsigned int gen;
};

constexpr uint64_t kBarrierTimeoutNs = 4000000000ull;  // 4 s

__device__ __forceinline__ bool grid_sync_limit(GridBarrier* b, int* err, uint64_t limit_ns) {
    if (gridDim.x == 1) {  // a one-block grid needs no global arrival counter
        __threadfence_block();
        __syncthreads();
        return true;
    }
    __syncthreads();
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        int ok = 1;
        unsigned int g = ld_volatile(&b->gen);
        __threadfence();
        unsigned int arrived = atomicAdd(&b->count, 1u) + 1u;
        if (arrived == gridDim.x) {
            atomicExch(&b->count, 0u);
            __threadfence();
            atomicExch(&b->gen, g + 1u);
        } else {
            uint64_t t0 = globaltimer_ns();
            while (ld_volatile(&b->gen) == g) {
                __nanosleep(64);
                if (globaltimer_ns() - t0 > limit_ns) {
                    atomicCAS(err, 0, SCC_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}
__device__ __forceinline__ bool grid_sync(GridBarrier* b, int* err) { return grid_sync_limit(b, err, kBarrierTimeoutNs); }

// ---------------------------------------------------------- pivot order --
// Seeded bijection of [0, N): 4-round balanced Feistel network on the smallest
// even bit width b >= 2 with 2^b >= N, round function low(b/2) bits of
// mix64(key_r ^ R), key_r = mix64(seed + (r + 1) * golden), then cycle walking
// into [0, N) (Black & Rogaway, CT-RSA 2002).
struct Feistel {
    uint64_t key[4];
    int half;
    uint64_t mask;
    __host__ __device__ void init(uint64_t seed, uint64_t N) {
        for (int r = 0; r < 4; ++r) key[r] = mix64(seed + (uint64_t)(r + 1) * 0x9E3779B97F4A7C15ull);
        int b = 2;
        while (b < 62 && (1ull << b) < N) b += 2;
        half = b / 2;
        mask = (1ull << half) - 1;
    }
    __host__ __device__ uint64_t once(uint64_t x) const {
        uint64_t L = x >> half, R = x & mask;
        for (int r = 0; r < 4; ++r) {
            uint64_t F = mix64(key[r] ^ R) & mask;
            uint64_t t = L ^ F;
            L = R;
            R = t;
        }
        return (L << half) | R;
    }
    __host__ __device__ uint64_t perm(uint64_t p, uint64_t N) const {
        uint64_t y = once(p);
        while (y >= N) y = once(y);
        return y;
    }
};

// ------------------------------------------------------------ misc helpers --
__host__ __device__ __forceinline__ int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace scc
