// Failure correction and support-threshold compaction (Sec. III-C; Sec. I
// problem statement: report the pairs with support at least s).
//
// Supports live in a packed row-major upper triangle indexed by ORIGINAL item
// ids, so lexicographic (i, j) order is plain array order and the frequent
// pairs come out of an ordered stream compaction: per-block counts, one
// exclusive scan of the block counts, then a write pass in which each block
// ranks its qualifying pairs with warp ballots and a block scan.
#include <algorithm>

#include "common.cuh"
#include "scan.cuh"

namespace bm {

constexpr int CTPB = 256;
constexpr int CPER = 16;
constexpr uint64_t CCHUNK = (uint64_t)CTPB * CPER;

__global__ void k_apply_corrections(const uint32_t *__restrict__ corr, uint64_t ncorr, uint64_t n,
                                    uint32_t n_a, uint32_t *__restrict__ C) {
    for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < ncorr;
         k += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t i = corr[2 * k], j = corr[2 * k + 1];
        if (n_a && !(i < n_a && j >= n_a)) continue;  // cross mode: A x B pairs only
        atomicAdd(&C[support_index(i, j, n, n_a)], 1u);
    }
}

// Row of packed index L: the largest i with i*n - i(i+1)/2 <= L.
__device__ __forceinline__ uint64_t row_of(uint64_t L, uint64_t n) {
    uint64_t lo = 0, hi = n - 1;  // answer in [0, n-2]
    while (hi - lo > 1) {
        uint64_t mid = (lo + hi) >> 1;
        uint64_t start = mid * n - mid * (mid + 1) / 2;
        if (start <= L) lo = mid; else hi = mid;
    }
    return lo;
}

template <bool WRITE>
__global__ void k_threshold(const uint32_t *__restrict__ C, uint64_t npairs, uint64_t n, uint32_t n_a, uint32_t s,
                            uint64_t *__restrict__ blocksums, uint32_t *__restrict__ out, uint64_t cap) {
    const uint64_t base = blockIdx.x * CCHUNK;
    uint64_t running = WRITE ? blocksums[blockIdx.x] : 0;
    for (int j = 0; j < CPER; j++) {
        const uint64_t L = base + (uint64_t)j * CTPB + threadIdx.x;
        uint32_t v = 0;
        bool keep = false;
        if (L < npairs) {
            v = C[L];
            keep = v >= s;
        }
        uint64_t tot;
        uint64_t rank = block_exclusive_scan(keep ? 1 : 0, &tot);
        if (WRITE && keep) {
            uint64_t idx = running + rank;
            if (idx < cap) {
                uint64_t i, jj;
                if (n_a) {  // rectangular: (A item, B item numbered from 0)
                    i = L / (n - n_a);
                    jj = L - i * (n - n_a);
                } else {
                    i = row_of(L, n);
                    jj = L - (i * n - i * (i + 1) / 2) + i + 1;
                }
                out[3 * idx] = (uint32_t)i;
                out[3 * idx + 1] = (uint32_t)jj;
                out[3 * idx + 2] = v;
            }
        }
        running += tot;
    }
    if (!WRITE && threadIdx.x == 0) blocksums[blockIdx.x] = running;
}

// Allocates the compaction scratch of a set ahead of stream capture.
void prepare_compaction(batmap_set *S) {
    const uint64_t npairs = S->npairs();
    if (npairs) S->d_blocksums.ensure((npairs + CCHUNK - 1) / CCHUNK + 1);
}

// Enqueues the correction and the compaction of one set: adds the correction
// entries into C, writes the frequent pairs (at most cap) and stores their
// number at d_total.  No host synchronisation.
void enqueue_correct_compact(batmap_set *S, uint32_t *C, uint32_t s, uint32_t *d_pairs, uint64_t cap,
                             uint64_t *d_total, cudaStream_t st) {
    const uint64_t n = S->n;
    const uint64_t npairs = S->npairs();
    if (S->n_corr) {
        uint64_t g = std::min<uint64_t>((S->n_corr + 255) / 256, 1u << 16);
        k_apply_corrections<<<(unsigned)g, 256, 0, st>>>(S->d_corr.p, S->n_corr, n, S->n_a, C);
        BM_CHECK_LAUNCH();
    }
    if (npairs == 0) {
        BM_CUDA(cudaMemsetAsync(d_total, 0, sizeof(uint64_t), st));
        return;
    }
    const uint64_t nblk = (npairs + CCHUNK - 1) / CCHUNK;
    prepare_compaction(S);
    k_threshold<false><<<(unsigned)nblk, CTPB, 0, st>>>(C, npairs, n, S->n_a, s, S->d_blocksums.p, nullptr, 0);
    BM_CHECK_LAUNCH();
    scan_exclusive(S->d_blocksums.p, nblk, d_total, st);
    if (cap && d_pairs) {
        k_threshold<true><<<(unsigned)nblk, CTPB, 0, st>>>(C, npairs, n, S->n_a, s, S->d_blocksums.p, d_pairs, cap);
        BM_CHECK_LAUNCH();
    }
}

// Number of block counts the threshold compaction of n items needs.
uint64_t threshold_blocks(uint64_t n) {
    const uint64_t npairs = n * (n > 0 ? n - 1 : 0) / 2;
    return (npairs + CCHUNK - 1) / CCHUNK;
}

// Threshold compaction of a packed support triangle that no set owns, with
// block counts in blocksums[0 .. threshold_blocks(n)) provided by the caller;
// allocates nothing.
void enqueue_threshold_into(const uint32_t *C, uint64_t n, uint32_t s, uint32_t *d_pairs, uint64_t cap,
                            uint64_t *blocksums, uint64_t *d_total, cudaStream_t st) {
    const uint64_t npairs = n * (n > 0 ? n - 1 : 0) / 2;
    if (npairs == 0) {
        BM_CUDA(cudaMemsetAsync(d_total, 0, sizeof(uint64_t), st));
        return;
    }
    const uint64_t nblk = threshold_blocks(n);
    k_threshold<false><<<(unsigned)nblk, CTPB, 0, st>>>(C, npairs, n, 0, s, blocksums, nullptr, 0);
    BM_CHECK_LAUNCH();
    scan_exclusive(blocksums, nblk, d_total, st);
    if (cap && d_pairs) {
        k_threshold<true><<<(unsigned)nblk, CTPB, 0, st>>>(C, npairs, n, 0, s, blocksums, d_pairs, cap);
        BM_CHECK_LAUNCH();
    }
}

// The same for the dense path, block counts in a buffer the library grows.
void enqueue_threshold(const uint32_t *C, uint64_t n, uint32_t s, uint32_t *d_pairs, uint64_t cap,
                       DevBuf<uint64_t> *blocksums, uint64_t *d_total, cudaStream_t st) {
    blocksums->ensure(threshold_blocks(n) + 1);
    enqueue_threshold_into(C, n, s, d_pairs, cap, blocksums->p, d_total, st);
}

}  // namespace bm
