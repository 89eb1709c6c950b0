// pair_threshold_noalloc: the support-threshold compaction for callers that
// cannot allocate device memory.
//
// Some callers must not call cudaMalloc: a serving loop that runs inside a
// fixed, pre-partitioned memory budget, or latency-critical code that cannot
// afford the implicit device synchronisation cudaMalloc and cudaFree may
// perform.  This entry point takes the packed supports (the d_full output of
// pair_support_all) and writes the frequent pairs with the same kernels as
// the compaction inside pair_support_all, but its only scratch -- per-block
// counts and their prefix sums -- lives in a fixed device array declared in
// this file.  With lazy module loading (the CUDA default) the array's memory
// is reserved when this file's module is first loaded on a device, which is
// the first call's address lookup; a caller that must not see that happen
// during its critical section makes one call beforehand.  The array then
// stays resident until the process exits.
#include <mutex>

#include "common.cuh"

namespace bm {

// Compaction of compact.cu: block counts of 4096 packed positions each.
uint64_t threshold_blocks(uint64_t n);
void enqueue_threshold_into(const uint32_t *C, uint64_t n, uint32_t s, uint32_t *d_pairs, uint64_t cap,
                            uint64_t *blocksums, uint64_t *d_total, cudaStream_t st);

// Capacity of the fixed scratch: one 64-bit count per block of 4096 pairs.
constexpr uint64_t NOALLOC_BLOCK_PAIRS = 4096;
constexpr uint64_t NOALLOC_MAX_BLOCKS = 65536;  // 2^28 pairs, n <= 23,170 items
constexpr uint64_t NOALLOC_MAX_PAIRS = NOALLOC_BLOCK_PAIRS * NOALLOC_MAX_BLOCKS;

// [0, NOALLOC_MAX_BLOCKS): block counts, then their exclusive prefix sums;
// [NOALLOC_MAX_BLOCKS]: the number of qualifying pairs.  512 KiB + 8 B.
static __device__ __align__(256) uint64_t g_noalloc_scratch[NOALLOC_MAX_BLOCKS + 1];

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
    BM_REQUIRE(threshold_blocks(n) <= NOALLOC_MAX_BLOCKS, BATMAP_ERR_INTERNAL, "block size mismatch");
    enqueue_threshold_into(d_full, n, s, d_pairs, cap, scratch, d_total, st);
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
