// Philox4x64-10 on the device (Salmon, Moraes, Dror, Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC'11): ten rounds of two 64x64 -> 128-bit
// products with the published multipliers, a word permutation and a key
// xor; the key advances by the published Weyl increments between rounds.
// The host planner draws with the same definition.
#pragma once

#include <stdint.h>

namespace tusq {

__device__ __forceinline__ void philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3, uint64_t k0,
                                              uint64_t k1, uint64_t out[4]) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint64_t m0 = 0xD2E7470EE14C6C93ull, m1 = 0xCA5A826395121157ull;
        const uint64_t hi0 = __umul64hi(m0, c0), lo0 = m0 * c0;
        const uint64_t hi1 = __umul64hi(m1, c2), lo1 = m1 * c2;
        const uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B97F4A7C15ull;
        k1 += 0xBB67AE8584CAA73Bull;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

}  // namespace tusq
