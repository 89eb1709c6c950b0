// pair_threshold_noalloc: the support-threshold compaction for callers that
// cannot allocate device memory.
//
// Some callers must not call cudaMalloc: a serving loop that runs inside a
// fixed, pre-partitioned memory budget, or latency-critical code that cannot
// afford the implicit device synchronisation cudaMalloc and cudaFree may
// perform.  This entry point takes the packed supports (the d_full output of
// pair_support_all) and writes the frequent pairs exactly like the
// compaction inside pair_support_all, but its only scratch -- per-block
// counts and their prefix sums -- lives in a fixed device array declared in
// this file.  The array is created when the library is loaded on a device and
// stays resident until the process exits.
#include <mutex>

#include "common.cuh"
#include "scan.cuh"

namespace bm {

// Capacity of the fixed scratch: one 64-bit count per block of 4096 pairs.
constexpr uint64_t NOALLOC_BLOCK_PAIRS = 4096;
constexpr uint64_t NOALLOC_MAX_BLOCKS = 65536;  // 2^28 pairs, n <= 23,170 items
constexpr uint64_t NOALLOC_MAX_PAIRS = NOALLOC_BLOCK_PAIRS * NOALLOC_MAX_BLOCKS;

// [0, NOALLOC_MAX_BLOCKS): block counts, then their exclusive prefix sums;
// [NOALLOC_MAX_BLOCKS]: the number of qualifying pairs.  512 KiB + 8 B.
static __device__ __align__(256) uint64_t g_noalloc_scratch[NOALLOC_MAX_BLOCKS + 1];

constexpr int NA_TPB = 256;
constexpr int NA_PER = (int)(NOALLOC_BLOCK_PAIRS / NA_TPB);

__device__ __forceinline__ uint64_t na_row_of(uint64_t L, uint64_t n) {
    uint64_t lo = 0, hi = n - 1;
    while (hi - lo > 1) {
        uint64_t mid = (lo + hi) >> 1;
        if (mid * n - mid * (mid + 1) / 2 <= L) lo = mid; else hi = mid;
    }
    return lo;
}

// Count (WRITE = false) or write (WRITE = true) the pairs of one block of
// 4096 packed positions whose support is at least s, in position order.
template <bool WRITE>
__global__ void k_threshold_noalloc(const uint32_t *__restrict__ C, uint64_t npairs, uint64_t n, uint32_t s,
                                    uint64_t *__restrict__ scratch, uint32_t *__restrict__ out, uint64_t cap) {
    const uint64_t base = blockIdx.x * NOALLOC_BLOCK_PAIRS;
    uint64_t running = WRITE ? scratch[blockIdx.x] : 0;
    for (int j = 0; j < NA_PER; j++) {
        const uint64_t L = base + (uint64_t)j * NA_TPB + threadIdx.x;
        uint32_t v = 0;
        bool keep = false;
        if (L < npairs) {
            v = C[L];
            keep = v >= s;
        }
        uint64_t tot;
        const uint64_t rank = block_exclusive_scan(keep ? 1 : 0, &tot);
        if (WRITE && keep) {
            const uint64_t idx = running + rank;
            if (idx < cap) {
                const uint64_t i = na_row_of(L, n);
                out[3 * idx] = (uint32_t)i;
                out[3 * idx + 1] = (uint32_t)(L - (i * n - i * (i + 1) / 2) + i + 1);
                out[3 * idx + 2] = v;
            }
        }
        running += tot;
    }
    if (!WRITE && threadIdx.x == 0) scratch[blockIdx.x] = running;
}

// Device address of g_noalloc_scratch, looked up once per device.
static std::mutex g_na_mu;
static uint64_t *g_na_ptr[64] = {};

static uint64_t *noalloc_scratch_for_current_device() {
    int dev = 0;
    BM_CUDA(cudaGetDevice(&dev));
    BM_REQUIRE(dev >= 0 && dev < 64, BATMAP_ERR_INTERNAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_na_mu);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            throw Error{BATMAP_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e)};
        g_na_ptr[dev] = static_cast<uint64_t *>(p);
    }
    return g_na_ptr[dev];
}

void threshold_noalloc(const uint32_t *d_full, uint32_t n, uint32_t s, uint32_t *d_pairs, uint64_t cap,
                       uint64_t *n_out, cudaStream_t st) {
    BM_REQUIRE(n_out != nullptr, BATMAP_ERR_ARG, "n_out is NULL");
    BM_REQUIRE(cap == 0 || d_pairs != nullptr, BATMAP_ERR_ARG, "d_pairs is NULL with cap > 0");
    const uint64_t npairs = (uint64_t)n * (n > 0 ? n - 1 : 0) / 2;
    BM_REQUIRE(npairs <= NOALLOC_MAX_PAIRS, BATMAP_ERR_CAPACITY,
               "pair_threshold_noalloc supports at most 2^28 pairs (n <= 23170); use pair_support_all");
    BM_REQUIRE(npairs == 0 || d_full != nullptr, BATMAP_ERR_ARG, "d_full is NULL");
    uint64_t *scratch = noalloc_scratch_for_current_device();
    uint64_t *d_total = scratch + NOALLOC_MAX_BLOCKS;
    if (npairs == 0) {
        BM_CUDA(cudaMemsetAsync(d_total, 0, sizeof(uint64_t), st));
    } else {
        const uint64_t nblk = (npairs + NOALLOC_BLOCK_PAIRS - 1) / NOALLOC_BLOCK_PAIRS;
        k_threshold_noalloc<false><<<(unsigned)nblk, NA_TPB, 0, st>>>(d_full, npairs, n, s, scratch, nullptr, 0);
        BM_CHECK_LAUNCH();
        k_scan_single_block<<<1, SCAN_TPB, 0, st>>>(scratch, nblk, d_total, 0);
        BM_CHECK_LAUNCH();
        if (cap) {
            k_threshold_noalloc<true><<<(unsigned)nblk, NA_TPB, 0, st>>>(d_full, npairs, n, s, scratch, d_pairs,
                                                                        cap);
            BM_CHECK_LAUNCH();
        }
    }
    uint64_t total = 0;
    BM_CUDA(cudaMemcpyAsync(&total, d_total, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    BM_CUDA(cudaStreamSynchronize(st));
    *n_out = total;
    if (total > cap)
        throw Error{BATMAP_ERR_CAPACITY, "d_pairs too small: " + std::to_string(total) + " pairs qualify"};
}

}  // namespace bm

extern "C" batmap_status pair_threshold_noalloc(const uint32_t *d_full, uint32_t n, uint32_t s, uint32_t *d_pairs,
                                                uint64_t cap, uint64_t *n_out, cudaStream_t stream) {
    try {
        bm::threshold_noalloc(d_full, n, s, d_pairs, cap, n_out, stream);
        return BATMAP_OK;
    } catch (const bm::Error &e) {
        bm::set_error(e.msg);
        return e.code;
    } catch (...) {
        bm::set_error("unexpected internal error");
        return BATMAP_ERR_INTERNAL;
    }
}
