// Warp-level sorting helpers on 64-bit keys (one key per lane).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace erq {

__device__ __forceinline__ uint64_t ws_shfl_xor(uint64_t x, int m) {
    const uint32_t lo = __shfl_xor_sync(0xffffffffu, (uint32_t)x, m);
    const uint32_t hi = __shfl_xor_sync(0xffffffffu, (uint32_t)(x >> 32), m);
    return ((uint64_t)hi << 32) | lo;
}
__device__ __forceinline__ uint64_t ws_shfl(uint64_t x, int src) {
    const uint32_t lo = __shfl_sync(0xffffffffu, (uint32_t)x, src);
    const uint32_t hi = __shfl_sync(0xffffffffu, (uint32_t)(x >> 32), src);
    return ((uint64_t)hi << 32) | lo;
}
// Ascending bitonic sort of the warp's 32 keys (lane i ends with the i-th smallest).
__device__ __forceinline__ uint64_t ws_sort32(uint64_t v, int lane) {
#pragma unroll
    for (int size = 2; size <= 32; size <<= 1)
#pragma unroll
        for (int d = size >> 1; d > 0; d >>= 1) {
            const uint64_t p = ws_shfl_xor(v, d);
            const bool asc = size == 32 || (lane & size) == 0;
            const bool keep_min = ((lane & d) == 0) == asc;
            v = keep_min ? (p < v ? p : v) : (p > v ? p : v);
        }
    return v;
}
// The 32 smallest keys of two ascending sorted warp lists, ascending: the
// elementwise minimum of one list and the other reversed is bitonic, and a
// half-cleaner cascade sorts it.
__device__ __forceinline__ uint64_t ws_merge32(uint64_t list, uint64_t sorted_cand, int lane) {
    const uint64_t r = ws_shfl(sorted_cand, 31 - lane);
    uint64_t m = list < r ? list : r;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        const uint64_t q = ws_shfl_xor(m, d);
        m = (lane & d) == 0 ? (q < m ? q : m) : (q > m ? q : m);
    }
    return m;
}

// Insert every key of this lane whose `pass` is set into the warp's ascending
// 32-entry list, keeping the 32 smallest; th becomes the list's (kp-1)-th key.
// Cost per inserted key is a ballot and a few shuffles, so it suits chunks where
// few keys pass.
__device__ __forceinline__ void ws_insert_each(uint64_t& list, uint64_t& th, uint64_t key, bool pass, int kp,
                                               int lane) {
    uint32_t m = __ballot_sync(0xffffffffu, pass);
    while (m) {
        const int src = __ffs(m) - 1;
        m &= m - 1;
        const uint64_t k = ws_shfl(key, src);
        if (!(k < th)) continue;                       // warp-uniform
        const int pos = __popc(__ballot_sync(0xffffffffu, list < k));
        const uint32_t lo = __shfl_up_sync(0xffffffffu, (uint32_t)list, 1);
        const uint32_t hi = __shfl_up_sync(0xffffffffu, (uint32_t)(list >> 32), 1);
        const uint64_t up = ((uint64_t)hi << 32) | lo;
        list = lane < pos ? list : (lane == pos ? k : up);
        th = ws_shfl(list, kp - 1);
    }
}

}  // namespace erq
