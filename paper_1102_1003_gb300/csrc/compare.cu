// The all-pairs BatMap compare kernel and its schedule (Sec. III-A/B/C).
//
// Counting rule (Sec. II, Fig. 3): a slot counts iff the 7 element bits of
// the two bytes agree and at least one indicator bit is set; the bottom byte
// 0x00 never counts.  Four slots are compared per 32-bit word:
//     L = (x ^ y) & 0x7F7F7F7F      element bits equal  <=>  lane of L == 0
//     t = L + 0x7F7F7F7F            lane bit 7 = [element bits differ]; no
//                                   carry leaves a lane (0x7F + 0x7F < 0x100)
//     q = ~t & (xi | yi)            xi, yi = indicator bits (x & 0x80808080)
//     acc += dp4a(q, 0x01010101)    adds 128 per counted slot
// This equals the paper's p / p' formulation (Sec. III-A) lane by lane; the
// indicator masks xi, yi are formed once per loaded word and reused across
// the 8 partners of the register tile.
//
// Sizes of different width (Sec. II, Fig. 1): the BatMap of the narrower row
// item i is compared cyclically, word k of the wider column item j against
// word k mod (|B_i|/4) of item i.  Widths are 3 * 2^e words, so the wrap is
// ((k >> e) % 3) << e | (k & (2^e - 1)).
//
// Work decomposition (GB300 design, replacing the paper's 16 x 16 work groups
// and host-side k x k blocks, Sec. III-B/C): items are sorted by width; the
// columns of a tile come from ONE width class, the rows are any items before
// them in sorted order; each (tile, word range) is a work unit; a persistent
// grid pulls units (longest first) from an atomic counter and adds its
// partial counts into the packed upper triangle with atomics (integer sums
// are exact in any order).
#include <algorithm>
#include <cmath>

#include "compare.cuh"

namespace bm {

// Shapes 1..6 and 14..16 stage tiles through shared memory (cp.async ring);
// shapes 7..13 stream operands from global memory into registers.  The efficiency
// column is the prior relative throughput per padded word pair used when no
// autotuned table is available: on the m = 10^6, n = 2,000 Zipf workload, the
// rate each shape reaches on the width classes it serves there (shapes 1, 2,
// 3, 10, 13; unit timings), else batmap_autotune's measurement with the
// shape forced on every width class.
const ShapeDesc SHAPES[NUM_SHAPES] = {
    {1, 128, 128, 8, 32, 3, 1.000},  {2, 256, 64, 8, 32, 3, 0.981},
    {3, 512, 32, 8, 32, 2, 0.946},   {4, 1024, 16, 8, 16, 2, 0.818},
    {5, 2048, 8, 8, 8, 2, 0.567},    {6, 2048, 4, 4, 8, 2, 0.367},
    {7, 128, 128, 8, 4, 0, 0.845},   {8, 256, 64, 8, 4, 0, 0.789},
    {9, 512, 32, 8, 4, 0, 0.834},    {10, 1024, 16, 8, 4, 0, 0.811},
    {11, 2048, 8, 8, 4, 0, 0.827},   {12, 2048, 4, 4, 4, 0, 0.689},
    {13, 1024, 12, 12, 4, 0, 0.912},
    // one column per thread, few rows: for width classes of small instances
    // (priors from batmap_autotune on 1,024 instances with m in [1e3, 1e5], n in [50, 400])
    {14, 256, 8, 1, 32, 3, 0.545},   {15, 128, 16, 1, 32, 3, 0.599},
    {16, 64, 32, 1, 32, 3, 0.619},
    // 12 column-staged columns over 256 or 512 rows (1 or 2 rows per thread):
    // the near-width rows that the probe route leaves to the scan in classes
    // of few wide items (priors from unit timings on the m = 10^6, n = 2,000
    // Zipf workload)
    {17, 256, 12, 12, 4, 0, 0.65},   {18, 512, 12, 12, 4, 0, 0.80},
};

int device_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        BM_CUDA(cudaGetDevice(&dev));
        BM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    }
    return sms;
}

// ---- device helpers -----------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src),
                 "r"(valid ? 16 : 0));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// The memory clobber keeps the compiler from moving shared-memory reads of the
// copied data above the wait.
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

__device__ __forceinline__ uint32_t wrap_word(uint32_t k, uint32_t e) {
    uint32_t q = k >> e;
    return ((q % 3u) << e) | (k & ((1u << e) - 1u));
}

__device__ __forceinline__ uint32_t lane_word(const uint4 &v, int kk) {
    return kk == 0 ? v.x : kk == 1 ? v.y : kk == 2 ? v.z : v.w;
}

// One 32-bit word pair: adds 128 per counted slot to acc.  Written as
// explicit three-input logic operations (lop3) so that each boolean step is
// one instruction: LUT 0x28 = (a ^ b) & c, LUT 0x0E = ~a & (b | c).
__device__ __forceinline__ uint32_t swar_step(uint32_t acc, uint32_t x, uint32_t xi, uint32_t y,
                                              uint32_t yi) {
    uint32_t l, t, q;
    asm("lop3.b32 %0, %1, %2, 0x7F7F7F7F, 0x28;" : "=r"(l) : "r"(x), "r"(y));
    asm("add.u32 %0, %1, 0x7F7F7F7F;" : "=r"(t) : "r"(l));
    asm("lop3.b32 %0, %1, %2, %3, 0x0E;" : "=r"(q) : "r"(t), "r"(xi), "r"(yi));
    asm("dp4a.u32.u32 %0, %1, 0x01010101, %0;" : "+r"(acc) : "r"(q));
    return acc;
}

template <int TR_T, int TC_T, int MC, int KC, int STAGES>
struct Tile {
    static constexpr int MR = 8;
    static constexpr int NT = TR_T * TC_T;
    static constexpr int TR = MR * TR_T;
    static constexpr int TC = MC * TC_T;
    static constexpr int CPR = KC / 4;  // 16-byte chunks per row per stage
    static constexpr int SWB = CPR < 8 ? CPR : 8;
    static constexpr int SWS = CPR >= 8 ? 0 : (CPR == 4 ? 1 : (CPR == 2 ? 2 : 3));
    static constexpr int ROW_CHUNKS = TR * CPR;
    static constexpr int COL_CHUNKS = TC * CPR;
    static constexpr int STAGE_CHUNKS = ROW_CHUNKS + COL_CHUNKS;
    // Shapes with three stages keep a second, masked copy of two stages
    // (indicator bits only, x & 0x80808080), written once per stage: the
    // compare loop reads the masks instead of forming them for every
    // register-tile word, which takes (8 + MC) / (8 MC) logic instructions
    // per word pair off the ALU pipe.
    static constexpr bool MASKED = STAGES >= 3;
    static constexpr int MASK_BUFS = MASKED ? 2 : 0;
    static constexpr size_t SMEM = (size_t)(STAGES + MASK_BUFS) * STAGE_CHUNKS * 16;
    static_assert(NT == 256, "256 threads per CTA");

    __device__ static __forceinline__ int sw(int r, int kq) {
        return r * CPR + (kq ^ ((r >> SWS) & (SWB - 1)));
    }
};

// Processes one work unit with tile shape <TR_T, TC_T, MC, KC, STAGES>.
template <int TR_T, int TC_T, int MC, int KC, int STAGES>
__device__ __forceinline__ void process_unit(uint4 *smem, const InstView &V, const WorkUnit &wu) {
    using T = Tile<TR_T, TC_T, MC, KC, STAGES>;
    const int tid = threadIdx.x;
    const int tc = tid % TC_T;
    const int tr = tid / TC_T;
    const uint32_t nst = wu.klen / KC;

    auto fill = [&](uint32_t stage, int buf) {
        uint4 *rows = smem + (size_t)buf * T::STAGE_CHUNKS;
        uint4 *cols = rows + T::ROW_CHUNKS;
        const uint32_t kbase = wu.k0 + stage * KC;
        for (int q = tid; q < T::ROW_CHUNKS; q += T::NT) {
            const int r = q / T::CPR, kq = q % T::CPR;
            const uint32_t g = wu.r0 + r;
            const bool ok = g < wu.r1;
            const uint4 *src = V.bm;
            if (ok) {
                uint32_t w = wrap_word(kbase + 4u * kq, __ldg(&V.wshift[g]));
                src = V.bm + (size_t)__ldg(&V.line_off[g]) * 8u + (w >> 2);
            }
            cp_async16(smem_u32(rows + T::sw(r, kq)), src, ok);
        }
        for (int q = tid; q < T::COL_CHUNKS; q += T::NT) {
            const int c = q / T::CPR, kq = q % T::CPR;
            const uint32_t g = wu.c0 + c;
            const bool ok = g < wu.c1;
            const uint4 *src = V.bm;
            if (ok) src = V.bm + (size_t)__ldg(&V.line_off[g]) * 8u + ((kbase >> 2) + kq);
            cp_async16(smem_u32(cols + T::sw(c, kq)), src, ok);
        }
    };

    uint32_t acc[8][MC];
#pragma unroll
    for (int a = 0; a < 8; a++)
#pragma unroll
        for (int b = 0; b < MC; b++) acc[a][b] = 0;

    // masked copy of stage `stage` (same positions as its raw copy)
    uint4 *const mring = smem + (size_t)STAGES * T::STAGE_CHUNKS;
    auto mask_stage = [&](uint32_t stage) {
        const uint4 *src = smem + (size_t)(stage % STAGES) * T::STAGE_CHUNKS;
        uint4 *dst = mring + (size_t)(stage & 1u) * T::STAGE_CHUNKS;
        for (int q = tid; q < T::STAGE_CHUNKS; q += T::NT) {
            const uint4 v = src[q];
            dst[q] = make_uint4(v.x & 0x80808080u, v.y & 0x80808080u, v.z & 0x80808080u, v.w & 0x80808080u);
        }
    };

    // Copy groups: one per stage.  Unmasked: stage s is waited for in
    // iteration s.  Masked: stage s+1 is waited for in iteration s, which then
    // masks it (into mask buffer (s+1) & 1) while stage s is compared; the
    // barrier of iteration s publishes stage s+1 and the masks of stage s, and
    // retires every read of stage s-1 (whose raw buffer the fill of stage s+2
    // and whose mask buffer the masks of stage s+1 overwrite).
#pragma unroll
    for (int s = 0; s < STAGES - 1; s++) {
        if ((uint32_t)s < nst) fill(s, s);
        cp_async_commit();
    }
    if constexpr (T::MASKED) {
        cp_async_wait<STAGES - 2>();
        __syncthreads();
        if (nst) mask_stage(0);
    }
    for (uint32_t s = 0; s < nst; s++) {
        if constexpr (T::MASKED) cp_async_wait<0>(); else cp_async_wait<STAGES - 2>();
        __syncthreads();
        {
            uint32_t nxt = s + STAGES - 1;
            if (nxt < nst) fill(nxt, nxt % STAGES);
            cp_async_commit();
        }
        if constexpr (T::MASKED) {
            if (s + 1 < nst) mask_stage(s + 1);
        }
        const uint4 *rows = smem + (size_t)(s % STAGES) * T::STAGE_CHUNKS;
        const uint4 *cols = rows + T::ROW_CHUNKS;
        const uint4 *mrows = mring + (size_t)(s & 1u) * T::STAGE_CHUNKS;
        const uint4 *mcols = mrows + T::ROW_CHUNKS;
#pragma unroll 1
        for (int kq = 0; kq < T::CPR; kq++) {
            uint4 X[8], Y[MC], XI[T::MASKED ? 8 : 1], YI[T::MASKED ? MC : 1];
#pragma unroll
            for (int a = 0; a < 8; a++) {
                X[a] = rows[T::sw(tr + TR_T * a, kq)];
                if constexpr (T::MASKED) XI[a] = mrows[T::sw(tr + TR_T * a, kq)];
            }
#pragma unroll
            for (int b = 0; b < MC; b++) {
                Y[b] = cols[T::sw(tc + TC_T * b, kq)];
                if constexpr (T::MASKED) YI[b] = mcols[T::sw(tc + TC_T * b, kq)];
            }
#pragma unroll
            for (int kk = 0; kk < 4; kk++) {
                uint32_t yw[MC], yi[MC];
#pragma unroll
                for (int b = 0; b < MC; b++) {
                    yw[b] = lane_word(Y[b], kk);
                    if constexpr (T::MASKED) yi[b] = lane_word(YI[b], kk);
                    else yi[b] = yw[b] & 0x80808080u;
                }
#pragma unroll
                for (int a = 0; a < 8; a++) {
                    const uint32_t xw = lane_word(X[a], kk);
                    uint32_t xi;
                    if constexpr (T::MASKED) xi = lane_word(XI[a], kk);
                    else xi = xw & 0x80808080u;
#pragma unroll
                    for (int b = 0; b < MC; b++) acc[a][b] = swar_step(acc[a][b], xw, xi, yw[b], yi[b]);
                }
            }
        }
    }
    cp_async_wait<0>();
    __syncthreads();

    // epilogue: partial supports into the packed upper triangle (original ids)
    const uint64_t n = V.n;
#pragma unroll
    for (int a = 0; a < 8; a++) {
        const uint32_t gi = wu.r0 + tr + TR_T * a;
        if (gi >= wu.r1) continue;
        const uint32_t oi = __ldg(&V.order[gi]);
#pragma unroll
        for (int b = 0; b < MC; b++) {
            const uint32_t gj = wu.c0 + tc + TC_T * b;
            const uint32_t v = acc[a][b] >> 7;
            if (gj < wu.c1 && (V.n_a || gi < gj) && v) {
                uint32_t *dst = &V.C[support_index(oi, __ldg(&V.order[gj]), n, V.n_a)];
                if (wu.shape & UNIT_WHOLE_K) *dst = v; else atomicAdd(dst, v);
            }
        }
    }
}

// Register-streaming variant for narrow column tiles, where a staged row word
// would have only a few partners.  Every thread streams its own MR row chunks
// per 4-word step into a private DEPTH-deep shared-memory ring with cp.async
// and waits only for its own copy groups.  The tile's TC column chunks are
// staged COL_CK steps at a time into a COL_STAGES-deep shared ring (laid out
// [step][column], so the TC_T distinct columns a warp reads are adjacent and
// conflict-free); one block barrier per COL_CK steps publishes a column stage
// and frees the oldest.  The wrap of a narrower row is an incremental index
// reset.
// Per-thread row ring depth (16-byte chunks, DEPTH-1 steps ahead): as deep as
// the shared memory allows, 6 steps for 8 rows per thread (192 KiB), 8 for 4.
constexpr int DEPTH_MR8 = 6, DEPTH_MR4 = 8;
constexpr int direct_depth(int MR) { return MR >= 8 ? DEPTH_MR8 : DEPTH_MR4; }
constexpr int COL_CK = 32;       // column chunks per stage (128 words)
constexpr int COL_STAGES = 3;    // column stages in flight
static_assert(2 * COL_CK >= DEPTH_MR8 && 2 * COL_CK >= DEPTH_MR4,
              "column copies must retire before their stage is read");

template <int TR_T, int TC_T, int MC, int MR, bool STAGE_COLS>
struct DirectTile {
    static constexpr int TC = TC_T * MC;
    static constexpr int DEPTH = direct_depth(MR);
    static constexpr int ROW_CHUNKS = DEPTH * MR * 256;
    static constexpr int COL_STAGE = COL_CK * TC;
    static constexpr int FILL = STAGE_COLS ? (COL_STAGE + 255) / 256 : 1;  // column chunks copied per thread
    // the dynamic shared memory of the kernel is the maximum over shapes and
    // is taken from L1, which the unstaged column loads go through
    static constexpr size_t SMEM = (size_t)(ROW_CHUNKS + (STAGE_COLS ? COL_STAGES * COL_STAGE : 0)) * 16;
};

template <int TR_T, int TC_T, int MC, int MR, bool STAGE_COLS>
__device__ __forceinline__ void process_unit_direct(uint4 *smem, const InstView &V, const WorkUnit &wu) {
    using T = DirectTile<TR_T, TC_T, MC, MR, STAGE_COLS>;
    const int tid = threadIdx.x;
    const int tc = tid % TC_T;
    const int tr = tid / TC_T;
    const uint32_t q0 = wu.k0 >> 2;  // first 16-byte chunk of the column range
    const uint32_t nq = wu.klen >> 2;
    const uint32_t nstage = (nq + COL_CK - 1) / COL_CK;
    const uint4 *__restrict__ bm = V.bm;
    uint4 *const cring = smem + T::ROW_CHUNKS;

    // row state: chunk index of the row start, current chunk, row length (chunks)
    uint32_t rbase[MR], rcur[MR], rlen[MR];
#pragma unroll
    for (int a = 0; a < MR; a++) {
        const uint32_t g = wu.r0 + tr + TR_T * a;
        if (g < wu.r1) {
            const uint32_t e = __ldg(&V.wshift[g]);
            rbase[a] = __ldg(&V.line_off[g]) * 8u;
            rlen[a] = 3u << (e - 2);
            rcur[a] = wrap_word(wu.k0, e) >> 2;
        } else {
            rbase[a] = 0xFFFFFFFFu;  // marks an empty row slot
            rlen[a] = 1;
            rcur[a] = 0;
        }
    }
    // the column chunks this thread copies in every stage: slot f = tid + 256 i
    // holds (step f / TC, tile column f % TC)
    uint32_t fbase[T::FILL];
#pragma unroll
    for (int i = 0; i < T::FILL; i++) {
        const uint32_t f = tid + 256u * i, c = f % T::TC;
        fbase[i] = (STAGE_COLS && f < (uint32_t)T::COL_STAGE && wu.c0 + c < wu.c1)
                       ? __ldg(&V.line_off[wu.c0 + c]) * 8u + q0
                       : 0xFFFFFFFFu;
    }
    // without column staging: the thread's own column chunks, loaded from
    // global memory (through L1) one step ahead into registers
    uint32_t cbase[MC];
#pragma unroll
    for (int b = 0; b < MC; b++) {
        const uint32_t g = wu.c0 + tc + TC_T * b;
        cbase[b] = (!STAGE_COLS && g < wu.c1) ? __ldg(&V.line_off[g]) * 8u + q0 : 0xFFFFFFFFu;
    }
    auto fill_cols = [&](uint32_t st) {
#pragma unroll
        for (int i = 0; i < T::FILL; i++) {
            const uint32_t f = tid + 256u * i;
            if (f < (uint32_t)T::COL_STAGE) {
                const uint32_t q = st * COL_CK + f / T::TC;
                const bool ok = fbase[i] != 0xFFFFFFFFu && q < nq;
                cp_async16(smem_u32(cring + (st % COL_STAGES) * T::COL_STAGE + f),
                           ok ? (const void *)(bm + (size_t)fbase[i] + q) : (const void *)bm, ok);
            }
        }
    };

    uint32_t acc[MR][MC];
#pragma unroll
    for (int a = 0; a < MR; a++)
#pragma unroll
        for (int b = 0; b < MC; b++) acc[a][b] = 0;

    auto issue_rows = [&](uint32_t step) {
        uint4 *slot = smem + (size_t)(step % T::DEPTH) * MR * 256 + tid;
#pragma unroll
        for (int a = 0; a < MR; a++) {
            const bool ok = rbase[a] != 0xFFFFFFFFu;
            cp_async16(smem_u32(slot + a * 256), ok ? (const void *)(bm + (size_t)rbase[a] + rcur[a]) : (const void *)bm,
                       ok);
            rcur[a] = (rcur[a] + 1 == rlen[a]) ? 0 : rcur[a] + 1;
        }
    };
    // Copy groups: the prologue commits DEPTH-1 groups (the first also holds
    // column stages 0 .. COL_STAGES-2); step q commits one group (rows of step
    // q+DEPTH-1, plus column stage s+COL_STAGES-1 when q = s*COL_CK).  Waiting
    // until DEPTH-1 groups are pending retires the rows of step q and every
    // column stage issued at least 2*COL_CK >= DEPTH steps earlier.
    if constexpr (STAGE_COLS) {
#pragma unroll
        for (int st = 0; st < COL_STAGES - 1; st++)
            if ((uint32_t)st < nstage) fill_cols(st);
    }
#pragma unroll
    for (int d = 0; d < T::DEPTH - 1; d++) {
        if ((uint32_t)d < nq) issue_rows(d);
        cp_async_commit();
    }

    const uint4 zero = make_uint4(0, 0, 0, 0);
    uint4 Y[MC];
    if constexpr (!STAGE_COLS) {
#pragma unroll
        for (int b = 0; b < MC; b++) Y[b] = (cbase[b] != 0xFFFFFFFFu && nq) ? __ldg(bm + (size_t)cbase[b]) : zero;
    }

#pragma unroll 1
    for (uint32_t q = 0; q < nq; q++) {
        if constexpr (STAGE_COLS) {
            // waiting with DEPTH-2 groups pending before this step's commit is
            // the same retirement point as DEPTH-1 after it
            const uint32_t s = q / COL_CK, kq = q % COL_CK;
            if (kq == 0) {
                cp_async_wait<T::DEPTH - 2>();
                __syncthreads();  // column stage s is complete; stage s-1 is no longer read
                if (s + COL_STAGES - 1 < nstage) fill_cols(s + COL_STAGES - 1);
            }
            // the column words are read before the row copies are issued, so
            // their latency overlaps the copy issue and the wait
            const uint4 *cs = cring + (s % COL_STAGES) * T::COL_STAGE + kq * T::TC + tc;
#pragma unroll
            for (int b = 0; b < MC; b++) Y[b] = cs[TC_T * b];
        }
        if (q + T::DEPTH - 1 < nq) issue_rows(q + T::DEPTH - 1);
        cp_async_commit();
        uint4 Yn[MC];
        if constexpr (!STAGE_COLS) {
            const bool more = q + 1 < nq;
#pragma unroll
            for (int b = 0; b < MC; b++)
                Yn[b] = (more && cbase[b] != 0xFFFFFFFFu) ? __ldg(bm + (size_t)cbase[b] + q + 1) : zero;
        }
        cp_async_wait<T::DEPTH - 1>();
        uint4 X[MR];
        const uint4 *slot = smem + (size_t)(q % T::DEPTH) * MR * 256 + tid;
#pragma unroll
        for (int a = 0; a < MR; a++) X[a] = slot[a * 256];
#pragma unroll
        for (int kk = 0; kk < 4; kk++) {
            uint32_t yw[MC], yi[MC];
#pragma unroll
            for (int b = 0; b < MC; b++) {
                yw[b] = lane_word(Y[b], kk);
                yi[b] = yw[b] & 0x80808080u;
            }
#pragma unroll
            for (int a = 0; a < MR; a++) {
                const uint32_t xw = lane_word(X[a], kk);
                const uint32_t xi = xw & 0x80808080u;
#pragma unroll
                for (int b = 0; b < MC; b++) acc[a][b] = swar_step(acc[a][b], xw, xi, yw[b], yi[b]);
            }
        }
        if constexpr (!STAGE_COLS) {
#pragma unroll
            for (int b = 0; b < MC; b++) Y[b] = Yn[b];
        }
    }
    cp_async_wait<0>();

    const uint64_t n = V.n;
#pragma unroll
    for (int a = 0; a < MR; a++) {
        const uint32_t gi = wu.r0 + tr + TR_T * a;
        if (gi >= wu.r1) continue;
        const uint32_t oi = __ldg(&V.order[gi]);
#pragma unroll
        for (int b = 0; b < MC; b++) {
            const uint32_t gj = wu.c0 + tc + TC_T * b;
            const uint32_t v = acc[a][b] >> 7;
            if (gj < wu.c1 && (V.n_a || gi < gj) && v) {
                uint32_t *dst = &V.C[support_index(oi, __ldg(&V.order[gj]), n, V.n_a)];
                if (wu.shape & UNIT_WHOLE_K) *dst = v; else atomicAdd(dst, v);
            }
        }
    }
}

#define BM_SHAPE_LIST(X)          \
    X(0, 16, 16, 8, 32, 3)        \
    X(1, 32, 8, 8, 32, 3)         \
    X(2, 64, 4, 8, 32, 2)         \
    X(3, 128, 2, 8, 16, 2)        \
    X(4, 256, 1, 8, 8, 2)         \
    X(5, 256, 1, 4, 8, 2)

// One column per thread (shapes 14..16), staged like shapes 1..6.
#define BM_SMALL_LIST(X)          \
    X(13, 32, 8, 1, 32, 3)        \
    X(14, 16, 16, 1, 32, 3)       \
    X(15, 8, 32, 1, 32, 3)

// Column-staged streaming shapes with few rows per thread (shapes 17, 18),
// run by the small-shape kernel.
#define BM_DIRECT_SMALL_LIST(X)  \
    X(16, 256, 1, 12, 1, true)   \
    X(17, 256, 1, 12, 2, true)

#define BM_DIRECT_LIST(X)      \
    X(6, 16, 16, 8, 8, false)    \
    X(7, 32, 8, 8, 8, false)     \
    X(8, 64, 4, 8, 8, false)     \
    X(9, 128, 2, 8, 8, false)    \
    X(10, 256, 1, 8, 8, false)   \
    X(11, 256, 1, 4, 8, false)   \
    X(12, 256, 1, 12, 4, true)

size_t compare_smem_bytes(uint32_t shape_idx) {
#define X(i, a, b, c, d, e) if (shape_idx == i) return Tile<a, b, c, d, e>::SMEM;
    BM_SHAPE_LIST(X)
    BM_SMALL_LIST(X)
#undef X
    return 0;
}

static size_t max_smem_bytes() {
    size_t m = 0;
#define X(i, a, b, c, d, e) m = std::max(m, DirectTile<a, b, c, d, e>::SMEM);
    BM_DIRECT_LIST(X)
#undef X
    for (uint32_t s = 0; s < NUM_SHAPES; s++)
        if (!small_shape(s)) m = std::max(m, compare_smem_bytes(s));
    return m;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Optional span stamps of a launch (nullptr: none): stamps[0] <- earliest CTA
// start, stamps[1] <- latest CTA end, in globaltimer nanoseconds.
__device__ __forceinline__ void stamp_start(unsigned long long *stamps) {
    if (stamps && threadIdx.x == 0) atomicMin(&stamps[0], (unsigned long long)global_ns());
}
__device__ __forceinline__ void stamp_end(unsigned long long *stamps) {
    if (stamps && threadIdx.x == 0) atomicMax(&stamps[1], (unsigned long long)global_ns());
}

// Persistent compare kernel: each CTA pulls units (longest first) from the
// queue until it is empty.  Every unit names its tile shape and instance.
__global__ void __launch_bounds__(256, 1)
k_compare(const InstView *__restrict__ views, const WorkUnit *__restrict__ units, uint32_t count,
          uint32_t *__restrict__ counter, unsigned long long *stamps) {
    extern __shared__ __align__(16) uint4 smem[];
    __shared__ uint32_t s_unit;
    stamp_start(stamps);
    for (;;) {
        if (threadIdx.x == 0) s_unit = atomicAdd(counter, 1u);
        __syncthreads();
        const uint32_t u = s_unit;
        __syncthreads();
        if (u >= count) break;
        const WorkUnit wu = units[u];
        const InstView V = views[wu.inst];
        switch (wu.shape & UNIT_SHAPE_MASK) {
#define X(i, a, b, c, d, e) case i: process_unit<a, b, c, d, e>(smem, V, wu); break;
            BM_SHAPE_LIST(X)
#undef X
#define X(i, a, b, c, d, e) case i: process_unit_direct<a, b, c, d, e>(smem, V, wu); break;
            BM_DIRECT_LIST(X)
#undef X
            default: break;
        }
    }
    stamp_end(stamps);
}

// The one-column-per-thread shapes 14..16 and the few-rows streaming shapes
// 17, 18 run in a kernel of their own (after the main one, on its own
// counter), so that they leave the register allocation of the main shapes'
// loops untouched.
__global__ void __launch_bounds__(256, 1)
k_compare_small(const InstView *__restrict__ views, const WorkUnit *__restrict__ units, uint32_t count,
                uint32_t *__restrict__ counter, unsigned long long *stamps) {
    extern __shared__ __align__(16) uint4 smem[];
    __shared__ uint32_t s_unit;
    stamp_start(stamps);
    for (;;) {
        if (threadIdx.x == 0) s_unit = atomicAdd(counter, 1u);
        __syncthreads();
        const uint32_t u = s_unit;
        __syncthreads();
        if (u >= count) break;
        const WorkUnit wu = units[u];
        const InstView V = views[wu.inst];
        switch (wu.shape & UNIT_SHAPE_MASK) {
#define X(i, a, b, c, d, e) case i: process_unit<a, b, c, d, e>(smem, V, wu); break;
            BM_SMALL_LIST(X)
#undef X
#define X(i, a, b, c, d, e) case i: process_unit_direct<a, b, c, d, e>(smem, V, wu); break;
            BM_DIRECT_SMALL_LIST(X)
#undef X
            default: break;
        }
    }
    stamp_end(stamps);
}

// ---- probe route for width-skewed pairs (Sec. V: look up the smaller set) ----
//
// A nonempty slot of row item i in table t at byte h holds a copy of some x
// with pi_t(x) = ((code - 1) << s) | (h mod r_0): the code carries the bits
// above s and the slot the bits below (r_0 = 2^s divides every range).  The
// cyclic scan pairs that slot with the r_j / r_i slots of column item j that
// share its table and its position modulo r_i; of those, only the slot of
// pi_t(x) in j, 3 r_0 floor((pi_t(x) mod r_j) / r_0) + t r_0 + (h mod r_0),
// can carry the same code (equal code and equal low bits mean equal pi_t,
// and pi_t is a bijection).  Reading that one byte and applying the counting
// rule (equal element bits, an indicator set) therefore adds the same count
// as the scan, r_j / r_i times fewer comparisons, at the price of one random
// byte read per nonempty row slot and column.

// One warp: every row of the unit against its (at most PROBE_COLS) columns.
// Lanes read 16-byte chunks of the row, pack the nonempty slots (slot index
// within the 32 chunks << 8 | byte) into shared memory by a warp prefix
// sum, then take whole slots, each decoded once and probed in every column.
__device__ __forceinline__ void probe_unit(const InstView &V, const WorkUnit &wu, uint32_t *ent, uint32_t lane) {
    const uint32_t s = V.shift, r0m = (1u << s) - 1u;
    const uint32_t nc = wu.c1 - wu.c0;
    const uint32_t rcm = (4u << __ldg(&V.wshift[wu.c0])) - 1u;  // r_j - 1 for the column class
    const uint8_t *bytes = reinterpret_cast<const uint8_t *>(V.bm);
    const uint8_t *col[PROBE_COLS];
#pragma unroll
    for (uint32_t b = 0; b < PROBE_COLS; b++)
        col[b] = bytes + (size_t)__ldg(&V.line_off[wu.c0 + (b < nc ? b : 0)]) * 128u;
    const uint64_t n = V.n;
    for (uint32_t q = wu.r0; q < wu.r1; q++) {
        const uint32_t nchunks = 3u << (__ldg(&V.wshift[q]) - 2u);  // 3 r_i bytes / 16
        const uint4 *row = V.bm + (size_t)__ldg(&V.line_off[q]) * 8u;
        uint32_t cnt[PROBE_COLS];
#pragma unroll
        for (uint32_t b = 0; b < PROBE_COLS; b++) cnt[b] = 0;
        for (uint32_t base = 0; base < nchunks; base += 32) {
            const uint32_t k = base + lane;
            const uint4 v = k < nchunks ? __ldg(row + k) : make_uint4(0, 0, 0, 0);
            const uint32_t vw[4] = {v.x, v.y, v.z, v.w};
            uint32_t cntw = 0;
#pragma unroll
            for (int j = 0; j < 16; j++) cntw += ((vw[j >> 2] >> (8 * (j & 3))) & 0x7Fu) ? 1u : 0u;
            uint32_t incl = cntw;  // inclusive prefix sum over the warp
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t o = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= (uint32_t)d) incl += o;
            }
            const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
            uint32_t pos = incl - cntw;
#pragma unroll
            for (int j = 0; j < 16; j++) {
                const uint32_t byte = (vw[j >> 2] >> (8 * (j & 3))) & 0xFFu;
                if (byte & 0x7Fu) ent[pos++] = ((lane * 16u + (uint32_t)j) << 8) | byte;
            }
            __syncwarp();
            for (uint32_t e = lane; e < total; e += 32) {
                const uint32_t x = ent[e], byte = x & 0xFFu;
                const uint32_t h = base * 16u + (x >> 8);  // byte offset in the row's BatMap
                const uint32_t hs = h >> s, t = hs % 3u, low = h & r0m;
                const uint32_t pi = (((byte & 0x7Fu) - 1u) << s) | low;
                const uint64_t hj = ((uint64_t)(3u * ((pi & rcm) >> s) + t) << s) | low;
#pragma unroll
                for (uint32_t b = 0; b < PROBE_COLS; b++) {
                    if (b < nc) {
                        const uint32_t y = __ldg(col[b] + hj);
                        cnt[b] += (((y ^ byte) & 0x7Fu) == 0u) & ((y | byte) >> 7);
                    }
                }
            }
            __syncwarp();
        }
#pragma unroll
        for (uint32_t b = 0; b < PROBE_COLS; b++)
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) cnt[b] += __shfl_xor_sync(0xffffffffu, cnt[b], d);
        uint32_t mine = 0;
#pragma unroll
        for (uint32_t b = 0; b < PROBE_COLS; b++)
            if (lane == b) mine = cnt[b];
        if (lane < nc) {
            const uint32_t oi = __ldg(&V.order[q]), oj = __ldg(&V.order[wu.c0 + lane]);
            V.C[support_index(oi, oj, n, V.n_a)] = mine;  // the unit owns these pairs
        }
    }
}

// Probe kernel: every warp pulls probe units from the queue until it is empty.
__global__ void __launch_bounds__(256, 3)
k_pair_probe(const InstView *__restrict__ views, const WorkUnit *__restrict__ units, uint32_t count,
             uint32_t *__restrict__ counter, unsigned long long *stamps) {
    __shared__ uint32_t s_ent[8][512];
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t *ent = s_ent[threadIdx.x >> 5];
    if (stamps && lane == 0) atomicMin(&stamps[0], (unsigned long long)global_ns());
    for (;;) {
        uint32_t u = 0;
        if (lane == 0) u = atomicAdd(counter, 1u);
        u = __shfl_sync(0xffffffffu, u, 0);
        if (u >= count) break;
        const WorkUnit wu = units[u];
        probe_unit(views[wu.inst], wu, ent, lane);
    }
    if (stamps && lane == 0) atomicMax(&stamps[1], (unsigned long long)global_ns());
}

static size_t g_compare_smem = 0, g_small_smem = 0;

void prepare_compare() {
    if (!g_compare_smem) {
        size_t smem = max_smem_bytes();
        BM_CUDA(cudaFuncSetAttribute(k_compare, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        g_compare_smem = smem;
        size_t small = 0;
#define X(i, a, b, c, d, e) small = std::max(small, Tile<a, b, c, d, e>::SMEM);
        BM_SMALL_LIST(X)
#undef X
#define X(i, a, b, c, d, e) small = std::max(small, DirectTile<a, b, c, d, e>::SMEM);
        BM_DIRECT_SMALL_LIST(X)
#undef X
        BM_CUDA(cudaFuncSetAttribute(k_compare_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)small));
        g_small_smem = small;
    }
}

bool small_shape(uint32_t shape) {
    const uint32_t k = shape & UNIT_SHAPE_MASK;
    return k >= 13 && k < (uint32_t)NUM_SHAPES;
}
bool probe_shape(uint32_t shape) { return (shape & UNIT_SHAPE_MASK) == PROBE_SHAPE; }

void launch_compare(const InstView *d_views, const WorkUnit *d_units, UnitParts parts, uint32_t *d_counters,
                    cudaStream_t st, unsigned long long *d_stamps, cudaEvent_t probe_start) {
    prepare_compare();
    const uint32_t sms = (uint32_t)device_sms();
    if (parts.main) {
        k_compare<<<std::min(parts.main, sms), 256, g_compare_smem, st>>>(d_views, d_units, parts.main, d_counters,
                                                                         d_stamps);
        BM_CHECK_LAUNCH();
    }
    if (parts.small) {
        k_compare_small<<<std::min(parts.small, sms), 256, g_small_smem, st>>>(
            d_views, d_units + parts.main, parts.small, d_counters + 1, d_stamps);
        BM_CHECK_LAUNCH();
    }
    if (probe_start) BM_CUDA(cudaEventRecord(probe_start, st));
    if (parts.probe) {
        const uint32_t warps = 3u * 8u * sms;  // three 256-thread blocks per SM
        const uint32_t blocks = (std::min(parts.probe, warps) + 7u) / 8u;
        k_pair_probe<<<blocks, 256, 0, st>>>(d_views, d_units + parts.main + parts.small, parts.probe,
                                             d_counters + 2, d_stamps);
        BM_CHECK_LAUNCH();
    }
}

// ---- schedule ------------------------------------------------------------------

// Width in words of sorted item q.
static inline uint64_t words_of(const batmap_set *S, uint32_t q) {
    return 3ull << S->wshift_sorted[q];
}

struct Tile2 {
    uint32_t r0, r1, c0, c1;
    uint32_t shape;  // 0-based shape index
};

// Tiles of the column class [cb, ce) with primary shape `s`.  All pairs: the
// rows are every earlier item from row_lo on, [row_lo, c1 - 1) (rows below
// row_lo are probed).  Cross mode: the rows are the given range [row_lo,
// row_hi) of the other family (items no wider than the columns).  Tiles are
// listed in groups of TILE_GROUP column strips, row strip by row strip inside
// a group, so the tiles that run at the same time (consecutive in the queue)
// share row and column strips and read them through L2 instead of each from
// DRAM.  A column tile's last, partial row strip may instead be covered by
// tiles of a shorter-row shape of the same column width (`shorter`, each with
// its cost per padded row), whichever pads least per unit of cost.
constexpr uint32_t TILE_GROUP = 12;
struct RowOption {
    uint32_t shape, TR;
    double cost_per_row;  // 1 / shape efficiency
};
static void class_tiles(uint32_t cb, uint32_t ce, uint32_t s, const std::vector<RowOption> &shorter,
                        double primary_cost_per_row, std::vector<Tile2> *out, bool cross = false,
                        uint32_t row_lo = 0, uint32_t row_hi = 0) {
    const ShapeDesc &sh = SHAPES[s];
    for (uint32_t g0 = cb; g0 < ce; g0 += TILE_GROUP * sh.TC) {
        const uint32_t g1 = std::min(ce, g0 + TILE_GROUP * sh.TC);
        const uint32_t lo = row_lo, top = cross ? row_hi : g1 - 1;
        for (uint32_t r0 = lo; r0 < top; r0 += sh.TR)
            for (uint32_t c0 = g0; c0 < g1; c0 += sh.TC) {
                const uint32_t c1 = std::min(ce, c0 + sh.TC);
                const uint32_t hi = cross ? row_hi : c1 - 1;
                if (r0 >= hi) continue;
                const uint32_t r1 = std::min(hi, r0 + sh.TR), rows = r1 - r0;
                // cheapest cover of a partial strip: the primary tile or k shorter tiles
                uint32_t best = s, best_tr = sh.TR;
                double best_cost = primary_cost_per_row * sh.TR;
                if (rows < sh.TR)
                    for (const RowOption &o : shorter) {
                        const double c = (double)((rows + o.TR - 1) / o.TR) * o.TR * o.cost_per_row;
                        if (c < best_cost) {
                            best_cost = c;
                            best = o.shape;
                            best_tr = o.TR;
                        }
                    }
                for (uint32_t a = r0; a < r1; a += best_tr) out->push_back({a, std::min(r1, a + best_tr), c0, c1, best});
            }
    }
}

// Cross mode, items sorted family first then by width: rows for a column
// class in family B are the A items with width <= the class width; for a
// class in family A, the B items strictly narrower (equal widths are taken
// once, from the B side).
static void cross_rows(const batmap_set *S, uint32_t cb, uint32_t *lo, uint32_t *hi) {
    const uint32_t e = S->wshift_sorted[cb];
    if (cb >= S->n_a) {
        uint32_t r = 0;
        while (r < S->n_a && S->wshift_sorted[r] <= e) r++;
        *lo = 0;
        *hi = r;
    } else {
        uint32_t r = S->n_a;
        while (r < S->n && S->wshift_sorted[r] < e) r++;
        *lo = S->n_a;
        *hi = r;
    }
}

uint32_t probe_log_of(const batmap_params &p) {
    if (p.probe_log >= 32) return 0;
    return p.probe_log ? p.probe_log : PROBE_LOG_DEFAULT;
}

// Probe units of one column class: rows [lo, p) (all narrower than the
// columns by 2^probe_log or more) against column chunks of at most
// PROBE_COLS, widest rows first inside a chunk; rows are grouped into units
// of about `target` probed words (row words x columns).
static void probe_units(const batmap_set *S, uint32_t cb, uint32_t ce, uint32_t lo, uint32_t p, double target,
                        std::vector<WorkUnit> *out) {
    if (p <= lo || ce <= cb) return;
    const uint32_t nc = ce - cb, nchunk = (nc + PROBE_COLS - 1) / PROBE_COLS, per = (nc + nchunk - 1) / nchunk;
    for (uint32_t c0 = cb; c0 < ce; c0 += per) {
        const uint32_t c1 = std::min(ce, c0 + per);
        uint32_t r1 = p;
        while (r1 > lo) {
            uint32_t r0 = r1;
            double cost = 0.0;
            while (r0 > lo && (r0 == r1 || cost < target)) {
                r0--;
                cost += (double)words_of(S, r0) * (c1 - c0);
            }
            out->push_back({r0, r1, c0, c1, 0, 0, 0, PROBE_SHAPE | UNIT_WHOLE_K});
            r1 = r0;
        }
    }
}

// Cost of probing one row word against one column, in the scheduler's
// cost unit (a padded word pair of the 128 x 128 tile, shape efficiency 1):
// on the m = 10^6, n = 2,000 Zipf workload the probe kernel reads 2.5e11 to
// 3.4e11 row words (times columns) per second where the 128 x 128 tile
// compares about 7e12 word pairs per second.
constexpr double PROBE_WORD_COST = 24.0;

void schedule_units(const batmap_set *S, uint32_t force_shape, const double *shape_eff,
                    double target_cost, std::vector<WorkUnit> *out) {
    const uint32_t ncls = (uint32_t)S->class_begin.size() - 1;
    // Width-skewed rows of each class may go to the probe route (never when
    // a shape is forced: the autotuner and the shape tests time the scan).
    // Rows are sorted by width, so the probed rows are a prefix [lo, p) of
    // the class's rows; p is chosen among the width boundaries of the rows
    // eligible by probe_log so that probe cost + scan cost is least.
    const uint32_t plog = force_shape ? 0 : probe_log_of(S->params);
    std::vector<double> prefix(S->n + 1, 0.0);  // row words, sorted order
    for (uint32_t q = 0; q < S->n; q++) prefix[q + 1] = prefix[q] + (double)words_of(S, q);
    struct Pick {
        uint32_t shape;
        std::vector<Tile2> tiles;
        uint64_t K;
    };
    std::vector<Pick> picks;
    struct ProbeRange {
        uint32_t cb, ce, lo, p;
    };
    std::vector<ProbeRange> probes;
    double total = 0.0, probe_total = 0.0;
    for (uint32_t c = 0; c < ncls; c++) {
        uint32_t cb = S->class_begin[c], ce = S->class_begin[c + 1];
        uint64_t K = words_of(S, cb);
        uint32_t lo = 0, hi = cb;
        if (S->n_a) cross_rows(S, cb, &lo, &hi);
        uint32_t pmax = lo;
        if (plog)
            while (pmax < hi && S->wshift_sorted[pmax] + plog <= S->wshift_sorted[cb]) pmax++;
        Pick best{0, {}, K};
        double best_cost = INFINITY, best_scan = 0.0, best_probe = 0.0;
        uint32_t best_p = lo;
        auto allowed = [&](uint32_t s) {
            if (force_shape) return s + 1 == force_shape;
            if (S->params.shape_mask && !((S->params.shape_mask >> s) & 1u)) return false;
            return K % SHAPES[s].KC == 0;
        };
        auto eff_of = [&](uint32_t s) { return shape_eff ? shape_eff[s] : SHAPES[s].eff; };
        for (uint32_t p = lo; p <= pmax; p++) {
            if (p > lo && p < pmax && S->wshift_sorted[p] == S->wshift_sorted[p - 1]) continue;
            const double probe_cost = PROBE_WORD_COST * (double)(ce - cb) * (prefix[p] - prefix[lo]);
            for (uint32_t s = 0; s < (uint32_t)NUM_SHAPES; s++) {
                if (!allowed(s)) continue;
                std::vector<RowOption> shorter;  // same column width, fewer rows (never when forced)
                for (uint32_t f = 0; f < (uint32_t)NUM_SHAPES && !force_shape; f++)
                    if (allowed(f) && SHAPES[f].TC == SHAPES[s].TC && SHAPES[f].TR < SHAPES[s].TR)
                        shorter.push_back({f, SHAPES[f].TR, 1.0 / eff_of(f)});
                std::vector<Tile2> tiles;
                class_tiles(cb, ce, s, shorter, 1.0 / eff_of(s), &tiles, S->n_a != 0, p, hi);
                double scan_cost = 0.0;
                for (const Tile2 &t : tiles)
                    scan_cost += (double)SHAPES[t.shape].TR * SHAPES[t.shape].TC * (double)K / eff_of(t.shape);
                if (scan_cost + probe_cost < best_cost) {
                    best_cost = scan_cost + probe_cost;
                    best_scan = scan_cost;
                    best_probe = probe_cost;
                    best_p = p;
                    best = Pick{s, std::move(tiles), K};
                }
            }
        }
        if (best_p > lo) {
            probes.push_back({cb, ce, lo, best_p});
            probe_total += best_probe / PROBE_WORD_COST;
        }
        if (!best.tiles.empty()) {
            total += best_scan;
            picks.push_back(std::move(best));
        }
    }
    // about 32 units per SM: with equal units (one width class) the last round
    // of the queue then idles under 1% of the SMs' time instead of a few percent
    if (target_cost <= 0.0) target_cost = total / (32.0 * device_sms());
    for (auto &p : picks) {
        // the K split of each shape in the pick: units of about target_cost
        uint64_t klen_of[NUM_SHAPES] = {};
        for (const Tile2 &t : p.tiles) {
            if (klen_of[t.shape]) continue;
            const ShapeDesc &sh = SHAPES[t.shape];
            const double tile_cost = (double)sh.TR * sh.TC * (double)p.K;
            uint64_t nk = (uint64_t)std::ceil(tile_cost / std::max(target_cost, 1.0));
            nk = std::max<uint64_t>(1, std::min<uint64_t>(nk, p.K / sh.KC));
            if (picks.size() == 1 && p.tiles.size() > 1) {
                // one width class, all units equal: the last round of the queue keeps
                // ceil(u) - u of a round idle (u = units per SM); among nk .. 2 nk
                // splits take the one that idles least
                const double G = (double)device_sms(), T = (double)p.tiles.size();
                double best_idle = 2.0;
                uint64_t best_nk = nk;
                for (uint64_t k = nk; k <= 2 * nk && k <= p.K / sh.KC; k++) {
                    const double u = T * (double)k / G, idle = (std::ceil(u) - u) / std::ceil(u);
                    if (idle < best_idle - 1e-3) {
                        best_idle = idle;
                        best_nk = k;
                    }
                }
                nk = best_nk;
            }
            uint64_t klen = (p.K + nk - 1) / nk;
            klen = (klen + sh.KC - 1) / sh.KC * sh.KC;
            klen_of[t.shape] = std::min<uint64_t>(klen, 1ull << 22);  // 128 * 4 * klen < 2^32
        }
        // K piece by K piece, each over the tiles in their grouped order, so that the
        // units running at the same time are neighbouring tiles over the same words
        // (they share row and column strips through L2)
        for (uint64_t piece = 0;; piece++) {
            bool any = false;
            for (const Tile2 &t : p.tiles) {
                const uint64_t klen = klen_of[t.shape], k0 = piece * klen;
                if (k0 >= p.K) continue;
                any = true;
                out->push_back({t.r0, t.r1, t.c0, t.c1, (uint32_t)k0,
                                (uint32_t)std::min<uint64_t>(klen, p.K - k0), 0,
                                t.shape | (klen >= p.K ? UNIT_WHOLE_K : 0u)});
            }
            if (!any) break;
        }
    }
    // probe units: widest column classes first, about 8 units per warp of
    // the probe kernel (three 256-thread blocks per SM)
    const double probe_target = probe_total / (8.0 * 24.0 * device_sms());
    for (auto it = probes.rbegin(); it != probes.rend(); ++it)
        probe_units(S, it->cb, it->ce, it->lo, it->p, probe_target, out);
    sort_units(out);
}

double unit_cost(const WorkUnit &u) {
    if (probe_shape(u.shape)) return 0.0;
    const ShapeDesc &sh = SHAPES[u.shape & UNIT_SHAPE_MASK];
    return (double)sh.TR * sh.TC * (double)u.klen / sh.eff;
}

void sort_units(std::vector<WorkUnit> *units) {
    // probe units last, in the order they were listed; the rest longest first,
    // the main shapes before the one-column shapes
    auto mid = std::stable_partition(units->begin(), units->end(),
                                     [](const WorkUnit &u) { return !probe_shape(u.shape); });
    std::stable_sort(units->begin(), mid,
                     [](const WorkUnit &a, const WorkUnit &b) { return unit_cost(a) > unit_cost(b); });
    std::stable_partition(units->begin(), mid, [](const WorkUnit &u) { return !small_shape(u.shape); });
}

UnitParts unit_parts(const std::vector<WorkUnit> &units) {
    UnitParts p;
    size_t k = 0;
    while (k < units.size() && !small_shape(units[k].shape) && !probe_shape(units[k].shape)) k++;
    p.main = (uint32_t)k;
    while (k < units.size() && small_shape(units[k].shape)) k++;
    p.small = (uint32_t)k - p.main;
    p.probe = (uint32_t)(units.size() - k);
    return p;
}

// Algorithmic work of the probe route in a unit list of one set: the
// scan-equivalent word pairs it takes over (rows x columns x column words)
// and the row words it reads (row words x columns).
static void probe_stats(const batmap_set *S, const std::vector<WorkUnit> &units, double *word_pairs,
                        double *words) {
    double wp = 0.0, w = 0.0;
    for (const WorkUnit &u : units) {
        if (!probe_shape(u.shape)) continue;
        const double nc = u.c1 - u.c0;
        wp += (double)(u.r1 - u.r0) * nc * (double)words_of(S, u.c0);
        for (uint32_t q = u.r0; q < u.r1; q++) w += (double)words_of(S, q) * nc;
    }
    *word_pairs = wp;
    *words = w;
}

bool tuned_shape_eff(double *eff);  // batch.cu

void build_schedule(batmap_set *S) {
    S->units.clear();
    double eff[NUM_SHAPES];
    const bool tuned = tuned_shape_eff(eff);
    schedule_units(S, S->params.tile, tuned ? eff : nullptr, 0.0, &S->units);
    probe_stats(S, S->units, &S->probe_word_pairs, &S->probe_words);
    S->d_units.alloc(S->units.size());
    if (!S->units.empty())
        BM_CUDA(cudaMemcpyAsync(S->d_units.p, S->units.data(), S->units.size() * sizeof(WorkUnit),
                                cudaMemcpyHostToDevice, S->stream));
}

}  // namespace bm
