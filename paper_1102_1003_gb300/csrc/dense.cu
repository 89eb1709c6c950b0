// Dense-bitmap comparison path (Sec. I-A / Sec. I-B: the bitmap vertical
// representation of PBI-GPU, m*n bits, AND + popcount).  Support counting over
// bitmaps is the dense boolean contraction C = M M^T with M in {0,1}^(n x m)
// (items x transactions), so it runs on the 5th-generation tensor cores:
//
//   * M stays packed in HBM, one bit per (item, transaction), rows padded to
//     a multiple of 128 bits (n m / 8 bytes: 4.3 GB at n = 8,192, m = 2^22);
//   * a CTA computes a 256 x 256 block as two 128 x 256 tiles sharing their B
//     operand; per K step of 128 transactions, TMA loads the 512 rows' bits
//     (8 KiB) into a 3-stage ring, sixteen expander warps turn them into e4m3
//     {0, 1} bytes (1.0 = 0x38) in the 128-byte-swizzled layout the MMA reads
//     (64 KiB, 3-stage ring) and publish each stage after a proxy fence;
//   * one thread issues tcgen05.mma.cta_group::1.kind::f8f6f4 (M = 128,
//     N = 256, K = 32) into two FP32 accumulators that fill the 512 columns
//     of tensor memory;
//   * four epilogue warps read both accumulators with tcgen05.ld, convert to
//     integers and add them into the packed upper triangle.
//
// Exactness: every product is exactly 0 or 1 and every partial sum an integer
// below 2^24, which the FP32 accumulator represents exactly (the tests check
// bit-exactness at supports up to 10^6); INT8 MMA (kind::i8) is not available
// on sm_103a.  Split-K partial sums are added with integer atomics (exact in
// any order).  Only blocks that hold a pair i < j are computed.
//
// Every mbarrier wait is bounded; on timeout the kernel records an error
// flag, stops issuing work, waits (bounded) for what it issued, frees its
// tensor memory and returns.  A test hook (batmap_test_dense_timeout) runs
// one launch whose producer issues no loads and whose waits are short, so
// that every wait gives up with nothing in flight.
#include <cuda.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "scan.cuh"

namespace bm {

void enqueue_threshold(const uint32_t *C, uint64_t n, uint32_t s, uint32_t *d_pairs, uint64_t cap,
                       DevBuf<uint64_t> *blocksums, uint64_t *d_total, cudaStream_t st);

namespace dense {

constexpr int BM = 128, BN = 256, BK = 128, STAGES = 3, UMMA_K = 32;
constexpr uint32_t A_BYTES = BM * BK;          // 16 KiB per A tile (two per stage)
constexpr uint32_t B_BYTES = BN * BK;          // 32 KiB
constexpr uint32_t STAGE_BYTES = 2 * A_BYTES + B_BYTES;
constexpr uint32_t TMEM_COLS = 512;            // two FP32 accumulators of 128 lanes x 256 columns
constexpr int XW = 16;                             // expander warps 2 .. 2 + XW - 1
constexpr int THREADS = 64 + 32 * XW;              // warp 0 TMA, warp 1 MMA, warps 2.. expand (2..5: epilogue)
constexpr int SB = 3;                              // stages of the packed-bit ring
constexpr uint32_t BITS_ROW = BK / 8;              // 16 bytes of bits per row and K step
constexpr uint32_t BITS_STAGE = (2 * BM + BN) * BITS_ROW;  // 8 KiB: rows of A0, A1, B
constexpr size_t SMEM = (size_t)STAGES * STAGE_BYTES + (size_t)SB * BITS_STAGE + 1024 /*align*/ + 256;
constexpr uint32_t SPIN_LIMIT = 1u << 26;          // bounded waits (tens of ms per wait)

struct Tile {
    uint32_t bp, bj;  // row blocks 2 bp and 2 bp + 1 (128 rows each), column block bj (256 columns)
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// Bounded wait for the phase with the given parity (at most `limit` polls);
// false on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint32_t limit) {
    for (uint32_t it = 0; it < limit; it++) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\n"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            "selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, uint32_t bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
        ::"r"(dst), "l"(map), "r"(bar), "r"(x), "r"(y)
        : "memory");
}

// Shared-memory matrix descriptor of a K-major operand tile stored with the
// 128-byte swizzle: rows of 128 bytes, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);  // start address
    d |= (uint64_t)1 << 16;                    // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;          // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;                    // descriptor version
    d |= (uint64_t)2 << 61;                    // 128-byte swizzle
    return d;
}

// Instruction descriptor: D = F32, A = B = E4M3, both K-major, M = 128, N = 256.
constexpr uint32_t IDESC = (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void umma_e4m3(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(tmem_d), "l"(da), "l"(db), "r"(IDESC), "r"(accumulate));
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// The low four bits of v to four bytes, byte j = 0x38 (1.0 in e4m3) iff bit j
// is set: the multiply by 1 + 2^7 + 2^14 + 2^21 copies the nibble to offsets
// 0, 7, 14, 21 (disjoint bit ranges, so no carries), which puts bit j at the
// low bit of byte j; the mask keeps those four bits.
__device__ __forceinline__ uint32_t spread4(uint32_t v) {
    return (((v & 15u) * 0x00204081u) & 0x01010101u) * 0x38u;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// One CTA per 256 x 256 block (two 128 x 256 tiles sharing B) over one K
// range.  The operands stay packed in HBM (one bit per transaction): warp 0
// loads the K step's bits of the 512 rows (8 KiB) with TMA into a 3-stage
// ring; eight expander warps turn them into e4m3 {0, 1} bytes in the
// 128-byte-swizzled layout the MMA reads (64 KiB per step, 3-stage ring) and
// hand each stage to the MMA warp after a proxy fence; warp 1 issues the
// tcgen05 MMAs; warps 2..5 then read the accumulators.
__global__ void __launch_bounds__(THREADS, 1)
k_dense_mmt(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
            const Tile *__restrict__ tiles, uint32_t ksplit, uint32_t kblocks, uint32_t n,
            uint32_t *__restrict__ C, int *__restrict__ err, uint32_t spin, uint32_t no_loads) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *bits = smem + STAGES * STAGE_BYTES;
    uint64_t *bars = reinterpret_cast<uint64_t *>(bits + SB * BITS_STAGE);
    // bars: [0, SB) bits full (TMA), [SB, 2 SB) bits empty (expanders), [2 SB, 2 SB + S) bytes full
    // (expanders), [2 SB + S, 2 SB + 2 S) bytes empty (MMA commit), [2 SB + 2 S] accumulators ready
    constexpr int BF = 0, BE = SB, YF = 2 * SB, YE = 2 * SB + STAGES, ACC = 2 * SB + 2 * STAGES;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + ACC + 1);
    __shared__ volatile int s_abort;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const Tile tile = tiles[blockIdx.x / ksplit];
    const uint32_t split = blockIdx.x % ksplit;
    const uint32_t kb0 = (uint32_t)((uint64_t)kblocks * split / ksplit);
    const uint32_t kb1 = (uint32_t)((uint64_t)kblocks * (split + 1) / ksplit);
    const uint32_t nk = kb1 - kb0;

    if (threadIdx.x == 0) {
        s_abort = 0;
        for (int i = 0; i <= ACC; i++)
            mbar_init(smem_addr(&bars[i]), (i >= BE && i < BE + SB) || (i >= YF && i < YF + STAGES) ? XW : 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_addr(tmem_slot)), "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // TMA producer of the packed bits (no_loads: the timeout test issues nothing)
        uint32_t it = 0;
        for (; it < nk && !s_abort && !no_loads; it++) {
            const uint32_t sb = it % SB, ph = it / SB;
            if (ph > 0 && !mbar_wait(smem_addr(&bars[BE + sb]), (ph - 1) & 1, spin)) {
                atomicExch(err, 1);
                s_abort = 1;
                break;
            }
            const uint32_t full = smem_addr(&bars[BF + sb]);
            uint8_t *dst = bits + sb * BITS_STAGE;
            mbar_expect_tx(full, BITS_STAGE);  // rows past the matrix are zero-filled and counted
            const int kx = (int)((kb0 + it) * BITS_ROW);
            tma_load_2d(smem_addr(dst), &tmA, full, kx, (int)(2 * tile.bp * BM));
            tma_load_2d(smem_addr(dst + BM * BITS_ROW), &tmA, full, kx, (int)((2 * tile.bp + 1) * BM));
            tma_load_2d(smem_addr(dst + 2 * BM * BITS_ROW), &tmB, full, kx, (int)(tile.bj * BN));
        }
        if (s_abort) {
            // wait (bounded) for the last load issued into every bits stage
            for (uint32_t sb = 0; sb < (uint32_t)SB && sb < it; sb++) {
                const uint32_t last = sb + SB * ((it - 1 - sb) / SB);
                mbar_wait(smem_addr(&bars[BF + sb]), (last / SB) & 1, spin);
            }
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        for (uint32_t it = 0; it < nk; it++) {
            const uint32_t st = it % STAGES;
            if (s_abort || !mbar_wait(smem_addr(&bars[YF + st]), (it / STAGES) & 1, spin)) {
                atomicExch(err, 1);
                s_abort = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_addr(smem + st * STAGE_BYTES);
            const uint64_t da0 = smem_desc(a0), da1 = smem_desc(a0 + A_BYTES), db = smem_desc(a0 + 2 * A_BYTES);
#pragma unroll
            for (int k = 0; k < BK / UMMA_K; k++) {
                // advance 32 e4m3 = 32 bytes along K inside the swizzled 128-byte rows
                const uint32_t acc = (it > 0 || k > 0) ? 1u : 0u;
                umma_e4m3(tmem, da0 + (uint64_t)(k * 2), db + (uint64_t)(k * 2), acc);
                umma_e4m3(tmem + (uint32_t)BN, da1 + (uint64_t)(k * 2), db + (uint64_t)(k * 2), acc);
            }
            umma_commit(smem_addr(&bars[YE + st]));  // frees the byte stage when the MMAs have read it
        }
        umma_commit(smem_addr(&bars[ACC]));  // accumulators ready (or nothing issued)
    } else if (warp >= 2) {
        // expanders: thread t owns rows t, t + 32 XW, .. of the 512 rows (A0 0..127, A1 128..255,
        // B 256..511); row r of the byte stage starts at r * 128, 16-byte chunk c at c ^ (r & 7)
        const uint32_t t = (uint32_t)threadIdx.x - 64;
        for (uint32_t it = 0; it < nk; it++) {
            const uint32_t sb = it % SB, st = it % STAGES;
            bool ok = !s_abort && mbar_wait(smem_addr(&bars[BF + sb]), (it / SB) & 1, spin);
            if (ok && it >= (uint32_t)STAGES) ok = mbar_wait(smem_addr(&bars[YE + st]), ((it / STAGES) - 1) & 1, spin);
            if (!ok) {
                atomicExch(err, 1);
                s_abort = 1;
                break;
            }
            const uint8_t *src = bits + sb * BITS_STAGE;
            uint8_t *dst = smem + st * STAGE_BYTES;
#pragma unroll
            for (uint32_t r = t; r < 2 * BM + BN; r += 32 * XW) {
                const uint4 w = *reinterpret_cast<const uint4 *>(src + r * BITS_ROW);
                const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
                uint8_t *row = dst + r * 128u;
#pragma unroll
                for (int c = 0; c < 8; c++) {
                    const uint32_t h = ws[c >> 1] >> (16 * (c & 1));
                    const uint4 o = make_uint4(spread4(h), spread4(h >> 4), spread4(h >> 8), spread4(h >> 12));
                    *reinterpret_cast<uint4 *>(row + ((((uint32_t)c) ^ (r & 7u)) << 4)) = o;
                }
            }
            // generic-proxy writes become visible to the tensor core's reads
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(smem_addr(&bars[YF + st]));
                mbar_arrive(smem_addr(&bars[BE + sb]));
            }
        }
        if (warp < 6) {
            // epilogue: TMEM lanes 32*(warp % 4) .. +31 hold tile rows of that quarter
            const uint32_t q = warp & 3;
            bool ready = false;
            for (int rep = 0; rep < 16 && !ready; rep++) ready = mbar_wait(smem_addr(&bars[ACC]), 0, spin);
            if (!ready) {
                atomicExch(err, 1);
                s_abort = 1;
            } else if (!s_abort && nk > 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint64_t nn = n;
#pragma unroll 1
                for (int h = 0; h < 2; h++) {
                    const uint32_t gi = (2 * tile.bp + h) * BM + q * 32 + lane;
#pragma unroll 1
                    for (int c0 = 0; c0 < BN; c0 += 32) {
                        uint32_t v[32];
                        asm volatile(
                            "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                            "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                              "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
                              "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
                              "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
                              "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
                              "=r"(v[31])
                            : "r"(tmem + ((q * 32u) << 16) + (uint32_t)(h * BN + c0)));
                        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                        if (gi < n) {
#pragma unroll
                            for (int c = 0; c < 32; c++) {
                                const uint32_t gj = tile.bj * BN + c0 + c;
                                const uint32_t cnt = __float2uint_rn(__uint_as_float(v[c]));
                                if (gi < gj && gj < n && cnt)
                                    atomicAdd(&C[(uint64_t)gi * nn - (uint64_t)gi * (gi + 1) / 2 + (gj - gi - 1)],
                                              cnt);
                            }
                        }
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
    }
}

// Scatter the tidlists into the zeroed bit matrix (row i, bit x = transaction x).
__global__ void k_bitmap(const uint64_t *__restrict__ off, const uint32_t *__restrict__ tids, uint32_t n,
                         uint32_t m, uint64_t ldw, uint32_t *__restrict__ M, int *__restrict__ err) {
    for (uint32_t i = blockIdx.y; i < n; i += gridDim.y) {
        const uint64_t b = off[i], e = off[i + 1];
        for (uint64_t k = b + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < e;
             k += (uint64_t)gridDim.x * blockDim.x) {
            const uint32_t x = tids[k];
            if (x >= m) {
                atomicExch(err, 2);
                continue;
            }
            atomicOr(&M[(uint64_t)i * ldw + (x >> 5)], 1u << (x & 31));
        }
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        BM_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
        BM_REQUIRE(p && q == cudaDriverEntryPointSuccess, BATMAP_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
        fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// Packed bit rows viewed as bytes: box of BITS_ROW bytes (one K step) x box_rows rows.
static CUtensorMap make_map(void *base, uint64_t rows, uint64_t row_bytes, uint32_t box_rows) {
    CUtensorMap map;
    std::memset(&map, 0, sizeof(map));
    cuuint64_t dims[2] = {row_bytes, rows};
    cuuint64_t strides[1] = {row_bytes};
    cuuint32_t box[2] = {(cuuint32_t)BITS_ROW, box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = encode_fn()(&map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, base, dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    BM_REQUIRE(r == CUDA_SUCCESS, BATMAP_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    return map;
}

}  // namespace dense

// Workspace kept across calls (bitmap, supports, tile list, scratch).
struct DenseWork {
    DevBuf<uint32_t> bitmap;  // packed bit rows, ld bits each
    DevBuf<uint32_t> C;
    DevBuf<dense::Tile> tiles;
    DevBuf<int> err;
    DevBuf<uint64_t> blocksums, total;
    PhaseEvents ev;
    batmap_timing timing{};
};

static std::mutex g_dense_mu;
static DenseWork *g_dense = nullptr;
static std::atomic<uint32_t> g_dense_timeout_test{0};  // one-shot spin limit of the timeout test

void set_dense_timeout_test(uint32_t spin_limit) { g_dense_timeout_test.store(spin_limit); }

void release_dense_workspace() {
    std::lock_guard<std::mutex> lock(g_dense_mu);
    delete g_dense;
    g_dense = nullptr;
}

void run_dense(uint32_t m, uint32_t n, const uint64_t *d_off, const uint32_t *d_tids, uint32_t s,
               uint32_t *d_pairs, uint64_t cap, uint64_t *n_out, uint32_t *d_full, batmap_timing *tout,
               cudaStream_t st) {
    using namespace dense;
    BM_REQUIRE(n_out, BATMAP_ERR_ARG, "n_out is NULL");
    BM_REQUIRE(cap == 0 || d_pairs, BATMAP_ERR_ARG, "d_pairs is NULL with cap > 0");
    BM_REQUIRE(m >= 1 && m <= (1u << 24), BATMAP_ERR_ARG, "dense path needs 1 <= m <= 2^24 (exact FP32 sums)");
    BM_REQUIRE(n == 0 || d_off, BATMAP_ERR_ARG, "d_offsets is NULL");
    std::lock_guard<std::mutex> lock(g_dense_mu);
    if (!g_dense) g_dense = new DenseWork();
    DenseWork &W = *g_dense;
    W.ev.create();
    W.ev.record(0, st);
    const uint64_t npairs = (uint64_t)n * (n > 0 ? n - 1 : 0) / 2;
    const uint64_t ld = (m + BK - 1) / BK * BK;  // padded row length (bits)
    const uint64_t ldw = ld / 32;                 // 32-bit words per row
    const uint64_t nrows = std::max<uint64_t>(n, 1);
    uint32_t *C = d_full;
    if (!C) {
        W.C.ensure(std::max<uint64_t>(npairs, 1));
        C = W.C.p;
    }
    W.err.ensure(1);
    BM_CUDA(cudaMemsetAsync(W.err.p, 0, sizeof(int), st));
    W.bitmap.ensure(nrows * ldw);
    BM_CUDA(cudaMemsetAsync(W.bitmap.p, 0, nrows * ldw * 4, st));
    if (n) {
        dim3 grid((unsigned)std::min<uint64_t>((m + 255) / 256, 64), std::min<uint32_t>(n, 65535u));
        k_bitmap<<<grid, 256, 0, st>>>(d_off, d_tids, n, m, ldw, W.bitmap.p, W.err.p);
        BM_CHECK_LAUNCH();
    }
    W.ev.record(1, st);
    if (npairs) BM_CUDA(cudaMemsetAsync(C, 0, npairs * sizeof(uint32_t), st));
    // upper-triangle blocks: row blocks 2 bp, 2 bp + 1 (128 rows each) hold a pair i < j with
    // column block bj (256) iff bp <= bj; the second row block may lie past n (zero rows)
    std::vector<Tile> tl;
    const uint32_t nbp = (n + 2 * BM - 1) / (2 * BM), nbj = (n + BN - 1) / BN;
    for (uint32_t bj = 0; bj < nbj; bj++)
        for (uint32_t bp = 0; bp < nbp && bp <= bj; bp++) tl.push_back({bp, bj});
    const uint32_t kblocks = (uint32_t)(ld / BK);
    if (!tl.empty()) {
        int dev = 0, nsm = 0;
        BM_CUDA(cudaGetDevice(&dev));
        BM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        // K split: one CTA per SM at a time, so choose the split whose CTA count fills its last
        // wave best (whole waves of equal CTAs), preferring fewer splits; each K range keeps
        // at least 64 K steps
        const uint32_t ntiles = (uint32_t)tl.size();
        uint32_t ksplit = 1;
        double best = -1.0;
        for (uint32_t k = 1; k <= 16 && (k == 1 || 64u * k <= kblocks); k++) {
            const uint64_t u = (uint64_t)ntiles * k, waves = (u + nsm - 1) / nsm;
            const double score = (double)u / (double)(waves * (uint64_t)nsm) - 0.01 * k;
            if (score > best) {
                best = score;
                ksplit = k;
            }
        }
        W.tiles.ensure(tl.size());
        BM_CUDA(cudaMemcpyAsync(W.tiles.p, tl.data(), tl.size() * sizeof(Tile), cudaMemcpyHostToDevice, st));
        CUtensorMap mA = make_map(W.bitmap.p, nrows, ld / 8, BM);
        CUtensorMap mB = make_map(W.bitmap.p, nrows, ld / 8, BN);
        static bool attr = false;
        if (!attr) {
            BM_CUDA(cudaFuncSetAttribute(k_dense_mmt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM));
            attr = true;
        }
        const uint32_t test_spin = g_dense_timeout_test.exchange(0);
        k_dense_mmt<<<(unsigned)(tl.size() * ksplit), THREADS, SMEM, st>>>(
            mA, mB, W.tiles.p, ksplit, kblocks, n, C, W.err.p, test_spin ? test_spin : SPIN_LIMIT,
            test_spin ? 1u : 0u);
        BM_CHECK_LAUNCH();
    }
    W.ev.record(2, st);
    W.total.ensure(1);
    enqueue_threshold(C, n, s, d_pairs, cap, &W.blocksums, W.total.p, st);
    W.ev.record(3, st);
    int err = 0;
    uint64_t total = 0;
    BM_CUDA(cudaMemcpyAsync(&err, W.err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    BM_CUDA(cudaMemcpyAsync(&total, W.total.p, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    BM_CUDA(cudaStreamSynchronize(st));
    W.timing.build_ms = W.ev.ms(0, 1);
    W.timing.compare_ms = W.ev.ms(1, 2);
    W.timing.compact_ms = W.ev.ms(2, 3);
    W.timing.pairs_ms = W.ev.ms(0, 3);
    W.timing.place_ms = W.timing.finalize_ms = 0.f;
    if (tout) *tout = W.timing;
    BM_REQUIRE(err != 2, BATMAP_ERR_ARG, "tids must be < m");
    BM_REQUIRE(err != 1, BATMAP_ERR_TIMEOUT, "dense tensor-core kernel: a bounded pipeline wait timed out");
    *n_out = total;
    if (total > cap)
        throw Error{BATMAP_ERR_CAPACITY, "d_pairs too small: " + std::to_string(total) + " pairs qualify"};
}

}  // namespace bm

extern "C" void batmap_test_dense_timeout(uint32_t spin_limit) { bm::set_dense_timeout_test(spin_limit); }

extern "C" batmap_status pair_support_dense(uint32_t m, uint32_t n, const uint64_t *d_offsets, const uint32_t *d_tids,
                                            uint32_t s, uint32_t *d_pairs, uint64_t cap, uint64_t *n_out,
                                            uint32_t *d_full, batmap_timing *timing, cudaStream_t stream) {
    try {
        bm::run_dense(m, n, d_offsets, d_tids, s, d_pairs, cap, n_out, d_full, timing, stream);
        return BATMAP_OK;
    } catch (const bm::Error &e) {
        bm::set_error(e.msg);
        return e.code;
    } catch (...) {
        bm::set_error("unexpected internal error");
        return BATMAP_ERR_INTERNAL;
    }
}
