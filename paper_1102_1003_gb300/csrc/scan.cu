#include "common.cuh"
#include "scan.cuh"

namespace bm {

__global__ void k_scan_single_block(uint64_t *a, uint64_t count, uint64_t *total, int with_tail) {
    constexpr int PER = 8;  // values per thread per tile
    uint64_t carry = 0;
    for (uint64_t base = 0; base < count; base += (uint64_t)SCAN_TPB * PER) {
        uint64_t v[PER];
        uint64_t sum = 0;
        uint64_t i0 = base + (uint64_t)threadIdx.x * PER;
#pragma unroll
        for (int q = 0; q < PER; q++) {
            v[q] = (i0 + q < count) ? a[i0 + q] : 0;
            sum += v[q];
        }
        uint64_t tile_total;
        uint64_t pre = block_exclusive_scan(sum, &tile_total) + carry;
#pragma unroll
        for (int q = 0; q < PER; q++) {
            if (i0 + q < count) a[i0 + q] = pre;
            pre += v[q];
        }
        carry += tile_total;
    }
    if (threadIdx.x == 0) {
        if (total) *total = carry;
        if (with_tail) a[count] = carry;
    }
}

void scan_exclusive(uint64_t *d_a, uint64_t count, uint64_t *d_total, cudaStream_t stream) {
    k_scan_single_block<<<1, SCAN_TPB, 0, stream>>>(d_a, count, d_total, 0);
    BM_CHECK_LAUNCH();
}

}  // namespace bm
