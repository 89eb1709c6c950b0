// The permutations pi_t of the layout hash (Sec. III-A draws them at random
// and leaves the generator open).
//
// A set is built either with the caller's permutation table (rows of m
// entries) or with permutations the library computes on the fly from a 64-bit
// seed, so that no table is uploaded or gathered:
//
//   * round keys: SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) started from
//     the seed; table t takes outputs 4t .. 4t+3, low 32 bits each;
//   * one pass E_t: a balanced four-round Feistel network on b bits, b the
//     smallest even number >= max(2, ceil(log2 m)); each round maps
//     (L, R) -> (R, L ^ (fmix32(R ^ k) & mask)), fmix32 being MurmurHash3's
//     32-bit finalizer (Appleby);
//   * pi_t(x): cycle walking, E_t applied to x until the value is below m
//     (a Feistel network is a bijection of [0, 2^b); walking along x's cycle
//     to the first value in [0, m) gives a bijection of [0, m); the expected
//     number of passes is 2^b / m < 4).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bm {

constexpr int PERM_MAX_TABLES = 5;  // d + 1 <= 5 (up to 4-of-5 BatMaps)

struct PermView {
    const uint32_t *table;  // caller's rows pi_0.. of m entries each, or nullptr: computed
    uint32_t m;
    uint32_t half;          // b / 2
    uint32_t mask;          // 2^half - 1
    uint32_t pad;
    uint4 key[PERM_MAX_TABLES];  // round keys of table t

    __host__ __device__ __forceinline__ static uint32_t fmix32(uint32_t z) {
        z ^= z >> 16;
        z *= 0x85EBCA6Bu;
        z ^= z >> 13;
        z *= 0xC2B2AE35u;
        z ^= z >> 16;
        return z;
    }

    __host__ __device__ __forceinline__ uint32_t pass(const uint4 &k, uint32_t v) const {
        uint32_t l = v >> half, r = v & mask;
        uint32_t f;
        f = l ^ (fmix32(r ^ k.x) & mask); l = r; r = f;
        f = l ^ (fmix32(r ^ k.y) & mask); l = r; r = f;
        f = l ^ (fmix32(r ^ k.z) & mask); l = r; r = f;
        f = l ^ (fmix32(r ^ k.w) & mask); l = r; r = f;
        return (l << half) | r;
    }

    // pi_t(x) for x < m and t < PERM_MAX_TABLES (t < d + 1 of the set).
    __device__ __forceinline__ uint32_t operator()(uint32_t t, uint32_t x) const {
        if (table) return __ldg(&table[(uint64_t)t * m + x]);
        const uint4 k = t == 0 ? key[0] : t == 1 ? key[1] : t == 2 ? key[2] : t == 3 ? key[3] : key[4];
        uint32_t v = pass(k, x);
        while (v >= m) v = pass(k, v);  // ends: x's own cycle returns below m
        return v;
    }
};

// The computed permutations of [0, m) for `seed` (table == nullptr), or a view
// of the caller's table.
PermView make_perm_view(const uint32_t *table, uint32_t m, uint64_t seed);

}  // namespace bm
