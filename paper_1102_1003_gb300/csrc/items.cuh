// Element-level build machinery shared by the 2-of-3 build (build.cu) and the
// d-of-(d+1) build (witness.cu): per-block element chunks, input validation,
// the failed-insertion CSR and the cached placement scratch.
#pragma once

#include <algorithm>
#include <mutex>

#include "common.cuh"

namespace bm {

constexpr uint32_t EMPTY = 0xFFFFFFFFu;  // empty slot of the uint32 placement tables
constexpr int TPB = 256;
constexpr int PER_THREAD = 16;
constexpr int CHUNK = TPB * PER_THREAD;  // elements handled by one block

// Per-item view for the element kernels (original item order).
struct ItemView {
    const uint64_t *off;     // CSR offsets [n+1]
    const uint32_t *tids;    // CSR tids
    const uint64_t *base;    // [n] first slot (byte) of item i in the BatMap array
    const uint32_t *rlog;    // [n] log2 r_i
    const uint32_t *ch_item; // [chunks] item of chunk b
    const uint64_t *ch_start;// [chunks] first element of chunk b
};

__device__ __forceinline__ void chunk_range(const ItemView &v, uint32_t b, uint32_t *item,
                                            uint64_t *e0, uint64_t *e1) {
    uint32_t i = v.ch_item[b];
    uint64_t s = v.ch_start[b];
    uint64_t end = v.off[i + 1];
    *item = i;
    *e0 = s;
    *e1 = s + CHUNK < end ? s + CHUNK : end;
}

// err <- 1 when a tidlist is not strictly increasing or holds a tid >= m.
__global__ void k_validate_tids(ItemView v, uint32_t m, int *err);
// err <- 2 when one of the `rows` permutation rows of length m is not a
// bijection of [0, m); bits: rows * ceil(m/32) zeroed words.
__global__ void k_validate_perm(const uint32_t *perm, uint32_t m, uint32_t rows, uint32_t *bits, int *err);
// f_off[i] = first failure of item i in the (item, tid)-sorted list.
__global__ void k_fail_offsets(const uint32_t *f_item, uint64_t nfail, uint32_t n, uint64_t *f_off);

// log2 r_i: the smallest power of two >= (num/den) |S_i|, at least r_0 = 2^shift.
inline uint32_t log2_range(uint64_t size, uint32_t num, uint32_t den, uint32_t shift) {
    uint64_t need = (num * std::max<uint64_t>(size, 1) + den - 1) / den;
    uint32_t lg = 0;
    while ((1ull << lg) < need) lg++;
    return std::max(lg, shift);
}

inline unsigned grid_for(uint64_t work, unsigned tpb = 256) {
    uint64_t g = (work + tpb - 1) / tpb;
    return (unsigned)std::min<uint64_t>(std::max<uint64_t>(g, 1), 1u << 20);
}

extern std::mutex g_scratch_mu;             // held for the duration of a build
DevBuf<uint32_t> &scratch_table(uint64_t slots);

}  // namespace bm
