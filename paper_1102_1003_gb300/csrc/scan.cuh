// Block- and device-level prefix sums used for ordered stream compaction
// (failed-insertion lists, frequent-pair output) and bitmap ranks.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bm {

constexpr int SCAN_TPB = 256;

// Exclusive prefix of `v` over the threads of a 256-thread block, in thread
// order.  Returns the prefix; *total receives the block sum.  All threads of
// the block must call it (contains __syncthreads).
__device__ __forceinline__ uint64_t block_exclusive_scan(uint64_t v, uint64_t *total) {
    __shared__ uint64_t warp_sums[SCAN_TPB / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint64_t y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint64_t w = lane < SCAN_TPB / 32 ? warp_sums[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            uint64_t y = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= d) w += y;
        }
        if (lane < SCAN_TPB / 32) warp_sums[lane] = w;
    }
    __syncthreads();
    uint64_t warp_prefix = warp ? warp_sums[warp - 1] : 0;
    *total = warp_sums[SCAN_TPB / 32 - 1];
    __syncthreads();
    return warp_prefix + x - v;
}

// In-place exclusive scan of a[0..count) by ONE block of 256 threads; writes
// the grand total to *total (device) and a[count] if with_tail.
__global__ void k_scan_single_block(uint64_t *a, uint64_t count, uint64_t *total, int with_tail);

// Exclusive scan of a uint64 array on `stream`: a[i] <- sum_{j<i} a[j];
// *d_total <- sum.  Uses one block (adequate for up to a few million values).
void scan_exclusive(uint64_t *d_a, uint64_t count, uint64_t *d_total, cudaStream_t stream);

}  // namespace bm
