// Shared helpers of the CUDA path: error plumbing, device utilities, layout
// arithmetic (Sec. III-A) and the internal representation of a built set.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "batmap.h"
#include "perm.cuh"

namespace bm {

// ---- error plumbing ---------------------------------------------------------

void set_error(const std::string &msg);

struct Error {
    batmap_status code;
    std::string msg;
};

#define BM_CUDA(call)                                                                       \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            throw ::bm::Error{e_ == cudaErrorMemoryAllocation ? BATMAP_ERR_NOMEM            \
                                                              : BATMAP_ERR_CUDA,            \
                              std::string(#call) + ": " + cudaGetErrorString(e_)};         \
        }                                                                                   \
    } while (0)

void count_launch();
#define BM_CHECK_LAUNCH()             \
    do {                              \
        BM_CUDA(cudaGetLastError());  \
        ::bm::count_launch();         \
    } while (0)

#define BM_REQUIRE(cond, code, msg)                                                         \
    do {                                                                                    \
        if (!(cond)) throw ::bm::Error{(code), (msg)};                                      \
    } while (0)

// RAII device buffer (cudaMalloc / cudaFree).
template <typename T>
struct DevBuf {
    T *p = nullptr;
    size_t n = 0;
    DevBuf() = default;
    explicit DevBuf(size_t count) { alloc(count); }
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    DevBuf(DevBuf &&o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
    DevBuf &operator=(DevBuf &&o) noexcept {
        if (this != &o) { release(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
        return *this;
    }
    ~DevBuf() { release(); }
    void alloc(size_t count) {
        release();
        if (count) BM_CUDA(cudaMalloc(&p, count * sizeof(T)));
        n = count;
    }
    void ensure(size_t count) { if (count > n) alloc(count); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    size_t bytes() const { return n * sizeof(T); }
};

// The BatMap array of a built set comes from a small cache: a freed set's
// array (after a device synchronisation, as cudaFree would do) is kept for the
// next build, at most two arrays, reused when no larger than twice the request
// plus 64 MiB, so repeated builds do not map and unmap hundreds of MB each.
uint8_t *bm_buffer_take(size_t bytes, size_t *capacity);
void bm_buffer_give(uint8_t *p, size_t capacity);
void bm_buffer_release_all();

struct BmBuf {
    uint8_t *p = nullptr;
    size_t n = 0, cap = 0;
    BmBuf() = default;
    BmBuf(const BmBuf &) = delete;
    BmBuf &operator=(const BmBuf &) = delete;
    ~BmBuf() { release(); }
    void alloc(size_t bytes) {
        release();
        if (bytes) p = bm_buffer_take(bytes, &cap);
        n = bytes;
    }
    void release() {
        if (p) bm_buffer_give(p, cap);
        p = nullptr;
        n = cap = 0;
    }
};

// Events bracketing phases of a call on its stream.
struct PhaseEvents {
    static constexpr int N = 8;
    cudaEvent_t ev[N] = {};
    bool ok = false;
    void create() {
        if (ok) return;
        for (int i = 0; i < N; i++) BM_CUDA(cudaEventCreate(&ev[i]));
        ok = true;
    }
    void record(int i, cudaStream_t st) { BM_CUDA(cudaEventRecord(ev[i], st)); }
    float ms(int a, int b) const {
        float t = 0.f;
        if (ok && cudaEventElapsedTime(&t, ev[a], ev[b]) != cudaSuccess) {
            cudaGetLastError();
            t = 0.f;
        }
        return t;
    }
    ~PhaseEvents() {
        if (ok)
            for (int i = 0; i < N; i++) cudaEventDestroy(ev[i]);
    }
};

// ---- layout arithmetic (Sec. III-A) ----------------------------------------

// Slot of pi = pi_t(x) in table t of a BatMap with range r (power of two,
// >= r0 = 2^shift): |B_0| floor((pi mod r)/r0) + (pi mod r0) + t r0.
__host__ __device__ __forceinline__ uint64_t slot_of(uint32_t t, uint32_t pi, uint32_t r,
                                                    uint32_t shift) {
    uint32_t r0 = 1u << shift;
    uint32_t h = pi & (r - 1u);
    return 3ull * r0 * (uint64_t)(h >> shift) + (h & (r0 - 1u)) + (uint64_t)t * r0;
}

// 8-bit element: indicator in bit 7, code (pi >> shift) + 1 in bits 0..6.
__host__ __device__ __forceinline__ uint32_t element_byte(uint32_t pi, uint32_t shift,
                                                         uint32_t ind) {
    return (ind << 7) | ((pi >> shift) + 1u);
}

// ---- compare work units ----------------------------------------------------

// One unit of the all-pairs compare: rows [r0, r1) x columns [c0, c1) of the
// width-sorted item order, word range [k0, k0 + klen) of the column width.
// Rows are never wider than columns; columns of a unit share one width.
struct WorkUnit {
    uint32_t r0, r1, c0, c1;
    uint32_t k0, klen;
    uint32_t inst;   // instance index (batched launches), 0 otherwise
    uint32_t shape;  // tile shape index (0-based) | UNIT_WHOLE_K if [k0, k0+klen) is the whole width
};
constexpr uint32_t UNIT_WHOLE_K = 0x100u;  // the unit owns its pairs: plain stores, no atomics
constexpr uint32_t UNIT_SHAPE_MASK = 0xFFu;
static_assert(sizeof(WorkUnit) == 32, "WorkUnit layout");

// Per-instance device view used by the compare kernel (batched form indexes
// an array of these by WorkUnit::inst).
struct InstView {
    const uint4 *bm;          // BatMap bytes of this instance, as 16-byte chunks
    const uint32_t *line_off; // [n] sorted order: byte offset / 128 of each BatMap
    const uint32_t *wshift;   // [n] sorted order: e with |B|/4 words = 3 * 2^e
    const uint32_t *order;    // [n] sorted position -> original item id
    uint32_t *C;              // supports: packed upper triangle (original ids), or n_a x (n - n_a) in cross mode
    uint32_t n;
    uint32_t n_a;             // 0: all pairs i < j; else cross pairs of items [0, n_a) with [n_a, n)
    uint32_t shift;           // s: r_0 = 2^s, codes (pi >> s) + 1 (the probe route decodes slots)
};

// Index of the support of the pair of original items (oi, oj) in C.
__device__ __forceinline__ uint64_t support_index(uint32_t oi, uint32_t oj, uint64_t n, uint32_t n_a) {
    const uint64_t lo = oi < oj ? oi : oj, hi = oi < oj ? oj : oi;
    if (n_a) return lo * (n - n_a) + (hi - n_a);
    return lo * n - lo * (lo + 1) / 2 + (hi - lo - 1);
}

}  // namespace bm

// The library-owned handle behind the opaque C type.
struct batmap_set {
    batmap_params params{};
    uint32_t m = 0, n = 0, shift = 0, r0 = 0;

    // number of supports (pairs) the set reports
    uint64_t npairs() const { return n_a ? (uint64_t)n_a * (n - n_a) : (uint64_t)n * (n > 0 ? n - 1 : 0) / 2; }
    uint64_t n_elements = 0, bytes = 0, n_failed = 0, n_corr = 0;
    double word_pairs = 0.0;
    double probe_word_pairs = 0.0;  // part of word_pairs counted by the probe route (scan-equivalent words)
    double probe_words = 0.0;       // words the probe route reads: rows' widths x columns per unit
    uint32_t n_a = 0;            // cross mode: items [0, n_a) x [n_a, n); 0 = all pairs
    uint32_t d = 2;              // copies per element: 2 (2-of-3 BatMaps) or 3 (3-of-4, k-way witnesses)
    uint64_t gen = 0;            // unique build id (batch plans key on it)
    bool skip_schedule = false;  // pool builds need no all-pairs schedule
    cudaStream_t stream = nullptr;

    // host metadata
    std::vector<uint32_t> range;          // r_i, original order
    std::vector<uint32_t> order;          // sorted position -> original id
    std::vector<uint32_t> rank;           // original id -> sorted position
    std::vector<uint64_t> byte_off;       // byte offset of BatMap, sorted order
    std::vector<uint32_t> wshift_sorted;  // e per sorted position
    std::vector<uint32_t> class_begin;    // sorted positions where a width class starts (+ n)
    std::vector<bm::WorkUnit> units;      // compare schedule, longest first

    // device data
    bm::BmBuf d_bm;                       // all BatMaps, width-sorted order
    bm::DevBuf<uint32_t> d_line_off;      // [n] sorted
    bm::DevBuf<uint32_t> d_wshift;        // [n] sorted
    bm::DevBuf<uint32_t> d_order;         // [n]
    bm::DevBuf<bm::WorkUnit> d_units;
    bm::DevBuf<uint32_t> d_corr;          // [2 * n_corr] (i, j) original ids, i < j
    bm::DevBuf<uint64_t> d_fail_off;      // [n+1] failed tids per item (CSR)
    bm::DevBuf<uint32_t> d_fail_tid;      // [n_failed], sorted per item
    // 3-of-4 sets (original item order): byte offsets, log2 r_i, own copy of pi_0..pi_3
    bm::DevBuf<uint64_t> d_base;          // [n+1]
    bm::DevBuf<uint32_t> d_rlog;          // [n]
    bm::DevBuf<uint32_t> d_perm;          // [4 m] copy of the caller's table, if one was given
    bm::PermView perm{};                  // the set's pi_t (table view or computed)

    // timing of the most recent calls
    bm::PhaseEvents build_ev, pairs_ev;
    batmap_timing timing{};

    // scratch reused across pair_support_all calls
    bm::DevBuf<uint32_t> d_C;             // packed upper triangle when no d_full
    bm::DevBuf<uint32_t> d_counters;      // work-queue counter
    bm::DevBuf<bm::InstView> d_view;      // device copy of this set's InstView
    bm::DevBuf<uint64_t> d_blocksums;     // compaction block counts / offsets
    bm::DevBuf<uint64_t> d_total;         // compaction total
};
