// d-of-(d+1) BatMaps and k-way supports (the generalisation that closes
// Sec. V), and frequent itemsets of sizes 3 and 4 (the problem of Sec. I
// beyond pairs, by the Apriori join-and-prune steps).
//
// d = 4 (4-of-5) follows the same pattern with five tables (block 5 r_0),
// four copies per element, the missing table in bits 7..5 and a five-bit
// code (m <= 31 * 2^s); the k-way rule (k <= 4) is witness_word5.
//
// Layout (d = 3): the BatMap of item i has four tables of r_i byte slots,
// interleaved in blocks of r_0 as Sec. III-A interleaves three (block size
// 4 r_0); slot h_t(x) = 4 r_0 floor((pi_t(x) mod r_i) / r_0)
// + (pi_t(x) mod r_0) + t r_0; width 4 r_i bytes = r_i words.  Every stored
// element has copies in exactly three tables; each copy's byte holds the
// fourth (missing) table in bits 7..6 and the code (pi_t(x) >> s) + 1 in bits
// 5..0; 0x00 is empty and s is the smallest shift >= min_shift with
// m <= 63 * 2^s.
//
// Witness rule: k <= 3 sets that all hold x miss at most three of the four
// tables, so at least one table holds all k copies (pigeonhole); the slot of
// table t counts iff the six code bits agree and are nonzero and t is the
// smallest table that none of the k sets misses.  Exactly one table
// satisfies this for every common element, and the rule reads only the k
// bytes of the slot and t.
//
// Failed insertions (elements left with fewer than three copies) are deleted
// and listed in F_i; a k-way support adds the common elements that failed in
// at least one of the k sets, each once.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "items.cuh"
#include "scan.cuh"

namespace bm {
namespace wit {

constexpr uint32_t TABLES = 4;  // d + 1
constexpr uint32_t COPIES = 3;  // d
constexpr uint32_t CODE_MASK = 0x3Fu;

// Field widths of a d-of-(d+1) byte over NT = d + 1 tables: the missing table
// in the top bits, the code (pi >> s) + 1 in the rest (six code bits for four
// tables, five for five).
template <uint32_t NT>
struct Fmt {
    static constexpr uint32_t COPIES = NT - 1;
    static constexpr uint32_t CODE_BITS = NT <= 4 ? 6u : 5u;
    static constexpr uint32_t CODE_MASK = (1u << CODE_BITS) - 1u;
    static constexpr uint32_t CODE_MAX = CODE_MASK;
};

// Slot of pi in table t: NT tables interleaved in blocks of r_0.
template <uint32_t NT>
__host__ __device__ __forceinline__ uint64_t slot_nt(uint32_t t, uint32_t pi, uint32_t r, uint32_t shift) {
    const uint32_t r0 = 1u << shift;
    const uint32_t h = pi & (r - 1u);
    return (uint64_t)NT * r0 * (uint64_t)(h >> shift) + (h & (r0 - 1u)) + (uint64_t)t * r0;
}

__host__ __device__ __forceinline__ uint64_t slot4(uint32_t t, uint32_t pi, uint32_t r, uint32_t shift) {
    return slot_nt<4>(t, pi, r, shift);
}

__device__ __forceinline__ uint32_t code6(uint32_t pi, uint32_t shift) { return (pi >> shift) + 1u; }

// ---- build ------------------------------------------------------------------

// Parallel INSERT with d = NT - 1 copies: copy c of every element starts in
// table c; a copy is swapped into its slot and the evicted occupant continues
// in the next table (0, 1, .., NT - 1, 0, ...).  Swapping with another copy
// of the same element leaves the slot unchanged and the element moves on, so
// copies of one element never share a table.  A chain longer than max_moves
// drops the copy it holds (the element then fails).
template <uint32_t NT>
__global__ void k_place(ItemView v, const PermView P, uint32_t shift, uint32_t max_moves,
                        uint32_t *__restrict__ table) {
    constexpr uint32_t NC = Fmt<NT>::COPIES;
    const uint32_t m = P.m;
    uint32_t item;
    uint64_t e0, e1;
    chunk_range(v, blockIdx.x / NC, &item, &e0, &e1);
    const uint32_t copy = blockIdx.x % NC;
    const uint64_t base = v.base[item];
    const uint32_t r = 1u << v.rlog[item];
    for (uint64_t e = e0 + threadIdx.x; e < e1; e += TPB) {
        uint32_t x = v.tids[e];
        if (x >= m) continue;  // rejected by validation; never index past perm
        uint32_t t = copy;
        for (uint32_t mv = 0; mv < max_moves; mv++) {
            const uint32_t pi = P(t, x);
            const uint32_t old = atomicExch(&table[base + slot_nt<NT>(t, pi, r, shift)], x);
            if (old == EMPTY) break;
            x = old;
            t = (t + 1u == NT) ? 0u : t + 1u;
        }
    }
}

template <uint32_t NT>
struct CopiesN {
    uint32_t pi[NT];
    uint64_t pos[NT];
    uint32_t has;  // bit t: a copy sits in table t
};

template <uint32_t NT>
__device__ __forceinline__ CopiesN<NT> find_copies(uint32_t x, uint64_t base, uint32_t r, uint32_t shift,
                                                   const PermView &P, const uint32_t *__restrict__ table) {
    CopiesN<NT> c;
    c.has = 0;
#pragma unroll
    for (uint32_t t = 0; t < NT; t++) {
        c.pi[t] = P(t, x);
        c.pos[t] = base + slot_nt<NT>(t, c.pi[t], r, shift);
        if (table[c.pos[t]] == x) c.has |= 1u << t;
    }
    return c;
}

// Bytes of every element stored d times; failures counted per block.
template <uint32_t NT>
__global__ void k_finalize(ItemView v, const PermView P, uint32_t shift, const uint32_t *__restrict__ table,
                           uint8_t *__restrict__ out, uint64_t *__restrict__ blocksums) {
    const uint32_t m = P.m;
    __shared__ uint32_t s_fail;
    if (threadIdx.x == 0) s_fail = 0;
    __syncthreads();
    uint32_t item;
    uint64_t e0, e1;
    chunk_range(v, blockIdx.x, &item, &e0, &e1);
    const uint64_t base = v.base[item];
    const uint32_t r = 1u << v.rlog[item];
    uint32_t fails = 0;
    for (uint64_t e = e0 + threadIdx.x; e < e1; e += TPB) {
        const uint32_t x = v.tids[e];
        if (x >= m) continue;
        const CopiesN<NT> c = find_copies<NT>(x, base, r, shift, P, table);
        if (__popc(c.has) != (int)Fmt<NT>::COPIES) {
            fails++;
            continue;
        }
        const uint32_t missing = __ffs(~c.has & ((1u << NT) - 1u)) - 1;
#pragma unroll
        for (uint32_t t = 0; t < NT; t++)
            if (c.has & (1u << t))
                out[c.pos[t]] = (uint8_t)((missing << Fmt<NT>::CODE_BITS) | code6(c.pi[t], shift));
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) fails += __shfl_xor_sync(0xffffffffu, fails, d);
    if ((threadIdx.x & 31) == 0 && fails) atomicAdd(&s_fail, fails);
    __syncthreads();
    if (threadIdx.x == 0) blocksums[blockIdx.x] = s_fail;
}

// Failed insertions in (item, tid) order: block offsets come from the scan
// of the finalize counts.
template <uint32_t NT>
__global__ void k_failures(ItemView v, const PermView P, uint32_t shift, const uint32_t *__restrict__ table,
                           const uint64_t *blocksums, uint32_t *f_item, uint32_t *f_tid) {
    const uint32_t m = P.m;
    uint32_t item;
    uint64_t e0, e1;
    chunk_range(v, blockIdx.x, &item, &e0, &e1);
    uint64_t running = blocksums[blockIdx.x];
    if (blocksums[blockIdx.x + 1] == running) return;  // no failure in this block
    const uint64_t base = v.base[item];
    const uint32_t r = 1u << v.rlog[item];
    for (int j = 0; j < PER_THREAD; j++) {
        const uint64_t e = e0 + (uint64_t)j * TPB + threadIdx.x;
        bool fail = false;
        uint32_t x = 0;
        if (e < e1) {
            x = v.tids[e];
            fail = x < m && __popc(find_copies<NT>(x, base, r, shift, P, table).has) != (int)Fmt<NT>::COPIES;
        }
        uint64_t tot;
        const uint64_t rank = block_exclusive_scan(fail ? 1 : 0, &tot);
        if (fail) {
            f_item[running + rank] = item;
            f_tid[running + rank] = x;
        }
        running += tot;
    }
}

// Smallest s >= min_shift with m <= code_max * 2^s (codes 1..code_max, 0 = empty).
static uint32_t shift_bits_codes(uint32_t m, uint32_t min_shift, uint32_t code_max) {
    uint32_t s = min_shift;
    while ((uint64_t)m > (uint64_t)code_max << s) s++;
    return s;
}

template <uint32_t NT>
void build_witness_impl(batmap_set *S, const uint64_t *d_offsets, const uint32_t *d_tids, const uint32_t *d_perm) {
    constexpr uint32_t TABLES = NT, COPIES = Fmt<NT>::COPIES;
    std::lock_guard<std::mutex> scratch_lock(g_scratch_mu);
    const uint32_t m = S->m, n = S->n;
    cudaStream_t st = S->stream;
    const batmap_params &P = S->params;
    PhaseEvents &E = S->build_ev;
    E.create();
    E.record(0, st);

    std::vector<uint64_t> off(n + 1, 0);
    if (n) {
        BM_REQUIRE(d_offsets != nullptr, BATMAP_ERR_ARG, "d_offsets is NULL");
        BM_CUDA(cudaMemcpyAsync(off.data(), d_offsets, (n + 1) * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
        BM_CUDA(cudaStreamSynchronize(st));
    }
    BM_REQUIRE(off[0] == 0, BATMAP_ERR_ARG, "offsets[0] must be 0");
    for (uint32_t i = 0; i < n; i++)
        BM_REQUIRE(off[i + 1] >= off[i], BATMAP_ERR_ARG, "offsets must be non-decreasing");
    const uint64_t T = off[n];
    S->n_elements = T;
    BM_REQUIRE(T == 0 || d_tids != nullptr, BATMAP_ERR_ARG, "d_tids is NULL");

    // ---- sizes: four tables of r_i slots; items keep their original order ----
    S->shift = shift_bits_codes(m, P.min_shift, Fmt<NT>::CODE_MAX);
    S->r0 = 1u << S->shift;
    std::vector<uint32_t> rlog(n);
    std::vector<uint64_t> base(n + 1, 0);
    S->range.resize(n);
    for (uint32_t i = 0; i < n; i++) {
        rlog[i] = log2_range(off[i + 1] - off[i], P.load_num, P.load_den, S->shift);
        BM_REQUIRE(rlog[i] <= 30, BATMAP_ERR_ARG, "hash range exceeds 2^30");
        S->range[i] = 1u << rlog[i];
        base[i + 1] = base[i] + ((uint64_t)TABLES << rlog[i]);
    }
    S->bytes = base[n];
    S->order.resize(n);
    S->rank.resize(n);
    S->byte_off.assign(base.begin(), base.begin() + n);
    for (uint32_t i = 0; i < n; i++) S->order[i] = S->rank[i] = i;
    S->word_pairs = 0.0;

    S->d_bm.alloc(S->bytes);
    S->d_base.alloc(n + 1);
    S->d_rlog.alloc(n);
    if (d_perm) S->d_perm.alloc((uint64_t)TABLES * m);  // the caller's table is kept; computed ones need none
    if (n) {
        BM_CUDA(cudaMemcpyAsync(S->d_base.p, base.data(), (n + 1) * 8ull, cudaMemcpyHostToDevice, st));
        BM_CUDA(cudaMemcpyAsync(S->d_rlog.p, rlog.data(), n * 4ull, cudaMemcpyHostToDevice, st));
    }
    if (d_perm) BM_CUDA(cudaMemcpyAsync(S->d_perm.p, d_perm, (uint64_t)TABLES * m * 4, cudaMemcpyDeviceToDevice, st));
    S->perm = make_perm_view(d_perm ? S->d_perm.p : nullptr, m, P.perm_seed);
    const PermView PV = S->perm;
    if (S->bytes) BM_CUDA(cudaMemsetAsync(S->d_bm.p, 0, S->bytes, st));
    S->d_fail_off.alloc(n + 1);

    std::vector<uint32_t> ch_item;
    std::vector<uint64_t> ch_start;
    for (uint32_t i = 0; i < n; i++)
        for (uint64_t s0 = off[i]; s0 < off[i + 1]; s0 += CHUNK) {
            ch_item.push_back(i);
            ch_start.push_back(s0);
        }
    const uint32_t nch = (uint32_t)ch_item.size();
    DevBuf<uint32_t> d_ch_item(nch);
    DevBuf<uint64_t> d_ch_start(nch);
    if (nch) {
        BM_CUDA(cudaMemcpyAsync(d_ch_item.p, ch_item.data(), nch * 4ull, cudaMemcpyHostToDevice, st));
        BM_CUDA(cudaMemcpyAsync(d_ch_start.p, ch_start.data(), nch * 8ull, cudaMemcpyHostToDevice, st));
    }
    ItemView v{d_offsets, d_tids, S->d_base.p, S->d_rlog.p, d_ch_item.p, d_ch_start.p};

    if (P.validate) {
        DevBuf<int> d_err(1);
        DevBuf<uint32_t> d_bits(d_perm ? (uint64_t)TABLES * ((m + 31) / 32) : 0);
        BM_CUDA(cudaMemsetAsync(d_err.p, 0, sizeof(int), st));
        if (d_perm) BM_CUDA(cudaMemsetAsync(d_bits.p, 0, d_bits.bytes(), st));
        if (nch) {
            k_validate_tids<<<nch, TPB, 0, st>>>(v, m, d_err.p);
            BM_CHECK_LAUNCH();
        }
        if (d_perm) {  // computed permutations are bijections by construction
            k_validate_perm<<<grid_for((uint64_t)TABLES * m), 256, 0, st>>>(d_perm, m, TABLES, d_bits.p, d_err.p);
            BM_CHECK_LAUNCH();
        }
        int err = 0;
        BM_CUDA(cudaMemcpyAsync(&err, d_err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        BM_CUDA(cudaStreamSynchronize(st));
        BM_REQUIRE(err != 1, BATMAP_ERR_ARG, "tids must be strictly increasing per item and < m");
        BM_REQUIRE(err != 2, BATMAP_ERR_ARG, "each permutation row must be a bijection of [0, m)");
    }

    S->n_failed = 0;
    if (nch) {
        DevBuf<uint32_t> &table = scratch_table(S->bytes);
        BM_CUDA(cudaMemsetAsync(table.p, 0xFF, S->bytes * sizeof(uint32_t), st));
        const uint32_t max_moves = TABLES * std::max<uint32_t>(P.max_loop, 1u);
        E.record(2, st);
        k_place<NT><<<COPIES * nch, TPB, 0, st>>>(v, PV, S->shift, max_moves, table.p);
        BM_CHECK_LAUNCH();
        E.record(3, st);
        DevBuf<uint64_t> bs(nch + 1), d_tot(1);
        k_finalize<NT><<<nch, TPB, 0, st>>>(v, PV, S->shift, table.p, S->d_bm.p, bs.p);
        BM_CHECK_LAUNCH();
        k_scan_single_block<<<1, SCAN_TPB, 0, st>>>(bs.p, nch, d_tot.p, 1);
        BM_CHECK_LAUNCH();
        uint64_t nfail = 0;
        BM_CUDA(cudaMemcpyAsync(&nfail, d_tot.p, 8, cudaMemcpyDeviceToHost, st));
        BM_CUDA(cudaStreamSynchronize(st));
        S->n_failed = nfail;
        DevBuf<uint32_t> f_item(nfail);
        S->d_fail_tid.alloc(nfail);
        if (nfail) {
            k_failures<NT><<<nch, TPB, 0, st>>>(v, PV, S->shift, table.p, bs.p, f_item.p,
                                            S->d_fail_tid.p);
            BM_CHECK_LAUNCH();
        }
        k_fail_offsets<<<(n + 1 + 255) / 256, 256, 0, st>>>(f_item.p, nfail, n, S->d_fail_off.p);
        BM_CHECK_LAUNCH();
        E.record(4, st);
    } else {
        BM_CUDA(cudaMemsetAsync(S->d_fail_off.p, 0, (n + 1) * sizeof(uint64_t), st));
        E.record(2, st);
        E.record(3, st);
        E.record(4, st);
    }
    E.record(1, st);
    BM_CUDA(cudaStreamSynchronize(st));
    S->timing.build_ms = E.ms(0, 1);
    S->timing.place_ms = E.ms(2, 3);
    S->timing.finalize_ms = E.ms(3, 4);
}

}  // namespace wit

// d-of-(d+1) build for d = 3 (3-of-4) and d = 4 (4-of-5).
void build_witness_set(batmap_set *S, const uint64_t *d_offsets, const uint32_t *d_tids, const uint32_t *d_perm) {
    if (S->d == 4) wit::build_witness_impl<5>(S, d_offsets, d_tids, d_perm);
    else wit::build_witness_impl<4>(S, d_offsets, d_tids, d_perm);
}

namespace wit {

// ---- k-way supports ------------------------------------------------------------

struct View {
    const uint32_t *bm;     // BatMap bytes as 32-bit words
    const uint64_t *base;   // [n+1] byte offset of item i
    const uint32_t *rlog;   // [n] log2 r_i (r_i words per BatMap)
    PermView perm;          // pi_0 .. pi_3
    const uint64_t *f_off;  // [n+1] failed insertions (CSR, sorted tids)
    const uint32_t *f_tid;
    uint32_t m, n, shift;
};

// Counted slots among the four lanes of one word of each of K BatMaps, all in
// table t.  Bit 6 of lane q of (v & 0x3F..) + 0x3F.. is set iff the lane's
// six low bits are nonzero (0x3F + 0x3F < 0x80: no carry leaves a lane).
template <int K>
__device__ __forceinline__ uint32_t witness_word(const uint32_t (&x)[K], uint32_t t) {
    constexpr uint32_t C6 = 0x3F3F3F3Fu, B6 = 0x40404040u;
    uint32_t diff = 0;
#pragma unroll
    for (int j = 1; j < K; j++) diff |= x[0] ^ x[j];
    const uint32_t ne = ((diff & C6) + C6) & B6;   // codes differ somewhere
    const uint32_t nz = ((x[0] & C6) + C6) & B6;   // slot not empty
    uint32_t ok = nz & ~ne;
    if (t == 0) return __popc(ok);
    // e_u (bit 6 of each lane): some set misses table u
    uint32_t e0 = 0, e1 = 0, e2 = 0;
#pragma unroll
    for (int j = 0; j < K; j++) {
        const uint32_t hi = (x[j] >> 1) & B6, lo = x[j] & B6;
        e0 |= ~(hi | lo) & B6;
        e1 |= ~hi & lo;
        e2 |= hi & ~lo;
    }
    ok &= e0;
    if (t >= 2) ok &= e1;
    if (t >= 3) ok &= e2;
    return __popc(ok);
}

// The same rule over five tables (d = 4): five code bits, the missing table
// in bits 7..5.  A lane counts iff the K codes agree and are nonzero and
// every table u < t is missed by some set (then t, which the K copies occupy,
// is the smallest table missed by none).
template <int K>
__device__ __forceinline__ uint32_t witness_word5(const uint32_t (&x)[K], uint32_t t) {
    constexpr uint32_t C5 = 0x1F1F1F1Fu, K7 = 0x7F7F7F7Fu, H7 = 0x80808080u, M3 = 0xE0E0E0E0u;
    uint32_t diff = 0;
#pragma unroll
    for (int j = 1; j < K; j++) diff |= x[0] ^ x[j];
    // bit 7 of (v + 0x7F..) flags a nonzero lane of v <= 0x1F (no carry leaves a lane)
    const uint32_t ne = ((diff & C5) + K7) & H7;  // codes differ somewhere
    const uint32_t nz = ((x[0] & C5) + K7) & H7;  // slot not empty
    uint32_t ok = nz & ~ne;
    for (uint32_t u = 0; u < t; u++) {
        const uint32_t U = u * 0x20202020u;  // u in bits 7..5 of every lane
        uint32_t e = 0;                       // bit 7: some set misses table u
#pragma unroll
        for (int j = 0; j < K; j++) e |= ~((((x[j] ^ U) & M3) >> 5) + K7);
        ok &= e;
    }
    return __popc(ok & H7);
}

// x is stored in item's BatMap: a copy sits in table 0 or table 1 (d of the
// d + 1 tables hold one), recognised by its code at h_t(x).
template <uint32_t NT>
__device__ __forceinline__ bool stored_in(const View &V, uint32_t item, uint32_t x) {
    const uint32_t r = 1u << V.rlog[item];
    const uint8_t *b = reinterpret_cast<const uint8_t *>(V.bm) + V.base[item];
#pragma unroll
    for (uint32_t t = 0; t < 2; t++) {
        const uint32_t pi = V.perm(t, x);
        if ((b[slot_nt<NT>(t, pi, r, V.shift)] & Fmt<NT>::CODE_MASK) == code6(pi, V.shift)) return true;
    }
    return false;
}

__device__ __forceinline__ bool failed_in(const View &V, uint32_t item, uint32_t x) {
    uint64_t lo = V.f_off[item], hi = V.f_off[item + 1];
    while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        const uint32_t y = V.f_tid[mid];
        if (y == x) return true;
        if (y < x) lo = mid + 1; else hi = mid;
    }
    return false;
}

// The lane's share of the failed common elements of the K sets: x from F of
// set j counts unless an earlier set i < j also failed it (then it is
// counted from set i's list).
template <int K, uint32_t NT>
__device__ __forceinline__ uint32_t failed_common(const View &V, const uint32_t (&it)[K], uint32_t lane) {
    uint32_t cnt = 0;
#pragma unroll
    for (int j = 0; j < K; j++) {
        const uint64_t f1 = V.f_off[it[j] + 1];
        for (uint64_t f = V.f_off[it[j]] + lane; f < f1; f += 32) {
            const uint32_t x = V.f_tid[f];
            bool all = true;
#pragma unroll
            for (int i = 0; i < K; i++) {
                if (i == j || !all) continue;
                const bool fi = failed_in(V, it[i], x);
                if (i < j && fi) all = false;
                else all = fi || stored_in<NT>(V, it[i], x);
            }
            cnt += all ? 1u : 0u;
        }
    }
    return cnt;
}

// One warp per query of K item ids on a set of NT = d + 1 tables.  Lane l
// reads word w = w0 + l of every BatMap, the narrower ones cyclically (w mod
// the width NT r_i / 4 words: block-wise, Fig. 1); 32 consecutive words lie
// in one table because a table block is r_0 >= 128 bytes.
// Width-skewed tuples go to a probe kernel instead of the scan: when the
// widest of the BatMaps is at least 2^PROBE_LOG times the narrowest, the scan
// (which runs over the widest) costs more than visiting the narrowest one's
// slots and probing the others (a same-box sweep of the frequent-triples
// step put the best threshold at 8x).
constexpr uint32_t PROBE_LOG = 3;
// On 4-of-5 sets the scan alternative is the one-warp-per-candidate kernel, so
// the probe pays from a width ratio of 2 on (same-box sweep of the frequent
// quadruples step on the Zipf triples workload: 2x 106.7 ms, 4x 110.5 ms,
// 8x 144.8 ms).
constexpr uint32_t PROBE_LOG5 = 1;
template <int K, uint32_t NT>
__device__ __forceinline__ bool probe_route_k(const uint32_t (&lg)[K]) {
    uint32_t lo = lg[0], hi = lg[0];
#pragma unroll
    for (int j = 1; j < K; j++) {
        lo = min(lo, lg[j]);
        hi = max(hi, lg[j]);
    }
    return hi - lo >= (NT == 5 ? PROBE_LOG5 : PROBE_LOG);
}

// skip_routed: leave the width-skewed queries (probe_route_k) to
// k_witness_probe_k, which writes their supports.
template <int K, uint32_t NT>
__global__ void __launch_bounds__(256) k_witness(View V, const uint32_t *__restrict__ items, uint64_t nq,
                                                 uint32_t *__restrict__ out, uint32_t skip_routed) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x / 32);
    for (uint64_t q = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) / 32; q < nq; q += nwarps) {
        uint32_t it[K], e[K], lg[K];
        uint64_t wb[K];
        uint32_t wmax = 0;
#pragma unroll
        for (int j = 0; j < K; j++) {
            it[j] = __ldg(&items[q * K + j]);
            lg[j] = V.rlog[it[j]];
            e[j] = lg[j] - 2;  // 2^e words per table segment of a block run
            wb[j] = V.base[it[j]] >> 2;
            wmax = max(wmax, NT << e[j]);
        }
        if (skip_routed && probe_route_k<K, NT>(lg)) continue;
        const uint32_t tshift = V.shift - 2;  // words per table block = r_0 / 4
        uint32_t cnt = 0;
        for (uint32_t w = lane; w < wmax; w += 32) {
            uint32_t x[K];
#pragma unroll
            for (int j = 0; j < K; j++) {
                const uint32_t wj = ((w >> e[j]) % NT) << e[j] | (w & ((1u << e[j]) - 1u));
                x[j] = __ldg(&V.bm[wb[j] + wj]);
            }
            const uint32_t t = (w >> tshift) % NT;
            if constexpr (NT == 4) cnt += witness_word<K>(x, t);
            else cnt += witness_word5<K>(x, t);
        }
        cnt += failed_common<K, NT>(V, it, lane);
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, d);
        if (lane == 0) out[q] = cnt;
    }
}

// Indices of the queries of K items routed to the probe kernel (any order).
template <int K, uint32_t NT>
__global__ void k_route_probe_k(const uint32_t *__restrict__ items, uint64_t nq, const uint32_t *__restrict__ rlog,
                                uint32_t *__restrict__ list, unsigned long long *__restrict__ count) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < nq; i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t lg[K];
#pragma unroll
        for (int j = 0; j < K; j++) lg[j] = rlog[items[K * i + j]];
        if (probe_route_k<K, NT>(lg)) list[atomicAdd(count, 1ull)] = (uint32_t)i;
    }
}

// Supports of K-tuples by probing (the second k-way idea of Sec. V: look up the
// elements of the smallest set in the others) on a set of NT = d + 1 tables,
// for any K <= d.  A nonempty slot of the narrowest BatMap in table t at byte h
// holds a copy of some x with pi_t(x) = ((code - 1) << s) | (h mod r_0); each
// other set holds x in table t iff the byte at its slot for pi_t(x) carries
// the same code.  The copy in t is counted only where all K sets hold x there
// and t is the smallest table none of them misses (the witness), which counts
// every element stored in all K sets once, as the scan's witness rule does;
// elements failed in any of them come from their F lists.  One warp per routed
// query; lanes take the narrowest BatMap's slots after a warp compaction.
template <int K, uint32_t NT>
__global__ void __launch_bounds__(256) k_witness_probe_k(View V, const uint32_t *__restrict__ items,
                                                         const uint32_t *__restrict__ list,
                                                         const unsigned long long *__restrict__ count,
                                                         uint32_t *__restrict__ out) {
    constexpr uint32_t CM = Fmt<NT>::CODE_MASK, CB = Fmt<NT>::CODE_BITS;
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x / 32);
    const uint64_t np = *count;
    const uint32_t s = V.shift, r0m = (1u << s) - 1u;
    const uint8_t *bytes = reinterpret_cast<const uint8_t *>(V.bm);
    __shared__ uint32_t s_slots[8][512];  // per warp: the nonempty slots of 32 chunks
    uint32_t *slots = s_slots[threadIdx.x >> 5];
    for (uint64_t q = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) / 32; q < np; q += nwarps) {
        const uint32_t i = list[q];
        uint32_t it[K], lg[K];
        uint32_t nj = 0, n_it = 0, n_lg = 0xFFFFFFFFu;  // the narrowest set (first of the narrowest)
#pragma unroll
        for (int j = 0; j < K; j++) {
            it[j] = items[(uint64_t)K * i + j];
            lg[j] = V.rlog[it[j]];
            if (lg[j] < n_lg) {
                n_lg = lg[j];
                n_it = it[j];
                nj = j;
            }
        }
        // the other K - 1 sets, in order (selects keep every index static)
        const uint8_t *ob[K - 1];
        uint32_t orr[K - 1];
#pragma unroll
        for (int o = 0; o < K - 1; o++) {
            const bool after = (uint32_t)o >= nj;
            ob[o] = bytes + V.base[after ? it[o + 1] : it[o]];
            orr[o] = 1u << (after ? lg[o + 1] : lg[o]);
        }
        const uint32_t *w0 = V.bm + (V.base[n_it] >> 2);
        const uint32_t chunks = (NT << n_lg) / 16;  // NT r bytes of the narrowest BatMap
        uint32_t cnt = 0;
        const uint4 *c0 = reinterpret_cast<const uint4 *>(w0);
        for (uint32_t base = 0; base < chunks; base += 32) {
            const uint32_t k = base + lane;
            const uint4 v = k < chunks ? __ldg(&c0[k]) : make_uint4(0, 0, 0, 0);
            const uint32_t vw[4] = {v.x, v.y, v.z, v.w};
            uint32_t n = 0;
#pragma unroll
            for (int j = 0; j < 16; j++) n += ((vw[j >> 2] >> (8 * (j & 3))) & CM) ? 1u : 0u;
            uint32_t incl = n;  // inclusive prefix sum over the warp
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t o = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= (uint32_t)d) incl += o;
            }
            const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
            uint32_t pos = incl - n;
#pragma unroll
            for (int j = 0; j < 16; j++) {
                const uint32_t byte = (vw[j >> 2] >> (8 * (j & 3))) & 0xFFu;
                if (byte & CM) slots[pos++] = ((lane * 16u + (uint32_t)j) << 8) | byte;
            }
            __syncwarp();
            for (uint32_t e = lane; e < total; e += 32) {
                const uint32_t ent = slots[e], byte = ent & 0xFFu, code = byte & CM;
                const uint32_t h = base * 16u + (ent >> 8);  // byte offset in the narrowest BatMap
                const uint32_t t = (h >> s) % NT;
                const uint32_t pi = ((code - 1u) << s) | (h & r0m);
                uint32_t missed = 1u << (byte >> CB);  // tables missed by some set (each misses one)
                bool all = true;
#pragma unroll
                for (int o = 0; o < K - 1; o++) {
                    const uint32_t y = __ldg(&ob[o][slot_nt<NT>(t, pi, orr[o], s)]);
                    all = all && (y & CM) == code;
                    missed |= 1u << (y >> CB);
                }
                cnt += all && (uint32_t)(__ffs(~missed) - 1) == t ? 1u : 0u;
            }
            __syncwarp();
        }
        cnt += failed_common<K, NT>(V, it, lane);
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, d);
        if (lane == 0) out[i] = cnt;
    }
}

__global__ void k_check_ids(const uint32_t *ids, uint64_t count, uint32_t n, int *err) {
    for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < count;
         k += (uint64_t)gridDim.x * blockDim.x)
        if (ids[k] >= n) atomicExch(err, 1);
}

// ---- grouped triple supports ------------------------------------------------------
//
// The candidates of the frequent pair p = (a, b) are contiguous
// (cand_off[p] .. cand_off[p+1]).  A work unit is up to GROUP of them: the
// warp reads a's and b's chunks once and every c of the unit against them.
// Lanes read 16-byte chunks; a table block is r_0 >= 128 bytes (8 chunks), so
// a chunk lies in one table.  The warp takes the four tables one after the
// other (chunk k of table t is q = 4 * 2^tq * (k >> tq) + t * 2^tq + (k mod
// 2^tq), 2^tq chunks per table block), so the witness requirement is a
// compile-time case of each pass.
constexpr uint32_t GROUP = 8;
constexpr uint32_t WG_TPB = 128;  // threads per block of k_witness_group
static_assert(GROUP <= 8, "a unit's slot order is kept in four bits per slot of one word");

// Width-skewed candidates go to the probe kernel instead of the grouped scan
// (the same PROBE_LOG rule as probe_route_k).
__device__ __forceinline__ bool probe_route(uint32_t la, uint32_t lb, uint32_t lc) {
    return max(max(la, lb), lc) - min(min(la, lb), lc) >= PROBE_LOG;
}

// Indices of the candidates routed to the probe kernel (any order).
__global__ void k_route_probe(const uint32_t *__restrict__ cand, uint64_t nc, const uint32_t *__restrict__ rlog,
                              uint32_t *__restrict__ list, unsigned long long *__restrict__ count) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < nc; i += (uint64_t)gridDim.x * blockDim.x)
        if (probe_route(rlog[cand[3 * i]], rlog[cand[3 * i + 1]], rlog[cand[3 * i + 2]]))
            list[atomicAdd(count, 1ull)] = (uint32_t)i;
}

// Triple supports by probing (the second k-way idea of Sec. V: look up the
// elements of the smallest set in the others), on 3-of-4 BatMaps.  A
// nonempty slot of the narrowest BatMap in table t at byte h holds a copy of
// some x with pi_t(x) = ((code - 1) << s) | (h mod r_0): the code gives the
// bits above s and the slot the bits below.  The other two sets hold x in
// table t iff the byte at their slot for pi_t(x) carries the same code (slot
// and code together fix pi_t(x), and pi_t is a bijection).  Counting the copy
// only where all three hold x in t and t is the smallest table none of the
// three misses counts every element stored in all three once, as the scan's
// witness rule does; elements failed in any of them come from their F lists.
// One warp per routed candidate; lanes take the narrowest BatMap's words.
__global__ void __launch_bounds__(256) k_witness_probe(View V, const uint32_t *__restrict__ cand,
                                                       const uint32_t *__restrict__ list,
                                                       const unsigned long long *__restrict__ count,
                                                       uint32_t *__restrict__ sup) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x / 32);
    const uint64_t np = *count;
    const uint32_t s = V.shift, r0m = (1u << s) - 1u;
    const uint8_t *bytes = reinterpret_cast<const uint8_t *>(V.bm);
    __shared__ uint32_t s_slots[8][512];  // per warp: the nonempty slots of 32 chunks
    uint32_t *slots = s_slots[threadIdx.x >> 5];
    for (uint64_t q = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) / 32; q < np; q += nwarps) {
        const uint32_t i = list[q];
        const uint32_t it[3] = {cand[3ull * i], cand[3ull * i + 1], cand[3ull * i + 2]};
        const uint32_t l0 = V.rlog[it[0]], l1 = V.rlog[it[1]], l2 = V.rlog[it[2]];
        // narrowest set n0 (log range ln) and the other two, o1 and o2
        const bool first = l0 <= l1 && l0 <= l2, second = !first && l1 <= l2;
        const uint32_t n0 = first ? it[0] : second ? it[1] : it[2];
        const uint32_t ln = first ? l0 : second ? l1 : l2;
        const uint32_t o1 = first ? it[1] : it[0], lo1 = first ? l1 : l0;
        const uint32_t o2 = (first || second) ? it[2] : it[1], lo2 = (first || second) ? l2 : l1;
        const uint32_t r1 = 1u << lo1, r2 = 1u << lo2;
        const uint32_t *w0 = V.bm + (V.base[n0] >> 2);
        const uint8_t *b1 = bytes + V.base[o1], *b2 = bytes + V.base[o2];
        const uint32_t words = 1u << ln;  // 4 r bytes of the narrowest BatMap
        // Lanes read 16-byte chunks of the narrowest BatMap; the warp packs its
        // nonempty slots (byte offset << 8 | byte) into shared memory by a
        // prefix sum, then every lane takes whole slots, so lanes stay busy
        // and each issues its two probes back to back.
        uint32_t cnt = 0;
        const uint4 *c0 = reinterpret_cast<const uint4 *>(w0);
        for (uint32_t base = 0; base < words / 4; base += 32) {
            const uint32_t q = base + lane;
            const uint4 v = q < words / 4 ? __ldg(&c0[q]) : make_uint4(0, 0, 0, 0);
            const uint32_t vw[4] = {v.x, v.y, v.z, v.w};
            uint32_t n = 0;
#pragma unroll
            for (int j = 0; j < 16; j++) n += ((vw[j >> 2] >> (8 * (j & 3))) & CODE_MASK) ? 1u : 0u;
            uint32_t incl = n;  // inclusive prefix sum over the warp
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t o = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= (uint32_t)d) incl += o;
            }
            const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
            uint32_t pos = incl - n;
#pragma unroll
            for (int j = 0; j < 16; j++) {
                const uint32_t byte = (vw[j >> 2] >> (8 * (j & 3))) & 0xFFu;
                if (byte & CODE_MASK) slots[pos++] = ((q * 16u + (uint32_t)j) << 8) | byte;
            }
            __syncwarp();
            for (uint32_t e = lane; e < total; e += 32) {
                const uint32_t ent = slots[e], h = ent >> 8, byte = ent & 0xFFu, code = byte & CODE_MASK;
                const uint32_t t = (h >> s) & 3u;
                const uint32_t pi = ((code - 1u) << s) | (h & r0m);
                const uint32_t y1 = __ldg(&b1[slot4(t, pi, r1, s)]);
                const uint32_t y2 = __ldg(&b2[slot4(t, pi, r2, s)]);
                // smallest table missed by none of the three (each misses one, never t)
                const uint32_t missed = (1u << (byte >> 6)) | (1u << (y1 >> 6)) | (1u << (y2 >> 6));
                cnt += (y1 & CODE_MASK) == code && (y2 & CODE_MASK) == code &&
                               (uint32_t)(__ffs(~missed) - 1) == t ? 1u : 0u;
            }
            __syncwarp();
        }
        cnt += failed_common<3, 4>(V, it, lane);
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, d);
        if (lane == 0) sup[i] = cnt;
    }
}

__global__ void k_unit_counts(const uint64_t *cand_off, uint64_t np, uint64_t *ucnt) {
    for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < np;
         p += (uint64_t)gridDim.x * blockDim.x)
        ucnt[p] = (cand_off[p + 1] - cand_off[p] + GROUP - 1) / GROUP;
}

__global__ void k_unit_fill(const uint64_t *cand_off, const uint64_t *uoff, uint64_t np, uint2 *units) {
    for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < np;
         p += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t nu = uoff[p + 1] - uoff[p];
        for (uint64_t q = 0; q < nu; q++) units[uoff[p] + q] = make_uint2((uint32_t)p, (uint32_t)(q * GROUP));
    }
}

// What a and b leave to c in one word, per lane, for a slot of table T: the
// tables u < T that neither a nor b misses.  None: c is free; exactly one,
// v: c must miss v; two or more: no c makes T the witness.  This becomes an
// expected byte pat (a's code; v in the top bits where constrained) under a
// mask msk (msk7 = msk without bit 7) and a validity flag val (bit 7) for
// lanes where a and b agree on a nonempty code and the rule can hold.
//
// A copy stored in table T never names T as its missing table, so each pass
// sees only three missing tables M (high bit h at bit 7, low bit l at bit 6):
//   T = 0: M in {1, 2, 3}; c is always free.
//   T = 1: M in {0, 2, 3}, M != 0 iff h; if h_a and h_b, c must miss 0,
//          which for c is h_c = 0.
//   T = 2: M in {0, 1, 3}, M in {0, 1} iff h = 0; h_a and h_b: both miss 3,
//          tables 0 and 1 stay open (invalid); h_a = h_b = 0 and l_a != l_b:
//          a and b miss 0 and 1 (free); otherwise c must miss v = 1 - l of
//          the set with h = 0 (l_a if h_a = 0, else l_b).
//   T = 3: M in {0, 1, 2}; valid iff M_a != M_b, and then c must miss the
//          third one, v = ~(M_a | M_b) (two bits).
template <int T>
__device__ __forceinline__ void pair_rule(uint32_t xa, uint32_t xb, uint32_t &pat, uint32_t &msk, uint32_t &msk7,
                                          uint32_t &val) {
    constexpr uint32_t C6 = 0x3F3F3F3Fu, B6 = 0x40404040u, H7 = 0x80808080u, L7 = 0x7E7E7E7Eu;
    const uint32_t x = xa ^ xb;
    const uint32_t za = xa & C6;
    // bit 7 of 2 e + 0x7E (e <= 0x3F per lane, no carry leaves a lane) is set iff e != 0
    const uint32_t ne = (x & C6) * 2u + L7;  // codes differ
    const uint32_t nz = za * 2u + L7;        // slot not empty
    if (T == 0) {
        pat = za;
        msk = msk7 = C6;
        val = nz & ~ne & H7;
    } else if (T == 1) {
        const uint32_t c7 = xa & xb & H7;  // constrained: c must have h = 0
        pat = za;
        msk7 = C6;
        msk = C6 | c7;
        val = nz & ~ne & H7;
    } else if (T == 2) {
        const uint32_t c7 = (xa | xb | ~(x << 1)) & H7;       // not free
        const uint32_t sel = xa >> 1;                          // h_a at bit 6
        const uint32_t l = (sel & xb) | (~sel & xa);           // bit 6: l of the set with h = 0 (a first)
        pat = za | (~l & B6);
        msk7 = C6 | (c7 >> 1);
        msk = msk7 | c7;
        val = nz & ~(ne | (xa & xb)) & H7;
    } else {
        pat = (xa & C6) | (~xa & ~xb & ~C6);  // a's code, v = ~(M_a | M_b)
        msk = 0xFFFFFFFFu;
        msk7 = 0x7F7F7F7Fu;
        val = nz & ~ne & (x | (x << 1)) & H7;  // M_a != M_b
    }
}

// One pass of a unit over the chunks of table T.
template <int T>
__device__ __forceinline__ void group_pass(const uint4 *__restrict__ bm4, uint32_t lane, uint32_t tq, uint32_t kmax,
                                           uint64_t ca, uint32_t ma, uint64_t cb, uint32_t mb,
                                           const uint64_t (&cc)[GROUP], const uint32_t (&mc)[GROUP],
                                           const uint32_t (&klim)[GROUP], uint32_t (&cnt)[GROUP]) {
    constexpr uint32_t C6 = 0x3F3F3F3Fu, K7 = 0x7F7F7F7Fu;
    const uint32_t low = (1u << tq) - 1u;
    for (uint32_t k = lane; k < kmax; k += 32) {
        const uint32_t q = ((k & ~low) << 2) | ((uint32_t)T << tq) | (k & low);
        const uint4 A = __ldg(&bm4[ca + (q & ma)]);
        const uint4 Bv = __ldg(&bm4[cb + (q & mb)]);
        // all of the unit's column chunks are requested before any is used
        uint4 Cs[GROUP];
#pragma unroll
        for (uint32_t j = 0; j < GROUP; j++)
            Cs[j] = k < klim[j] ? __ldg(&bm4[cc[j] + (q & mc[j])]) : make_uint4(0, 0, 0, 0);
        const uint32_t xa[4] = {A.x, A.y, A.z, A.w}, xb[4] = {Bv.x, Bv.y, Bv.z, Bv.w};
        uint32_t pat[4], msk[4], msk7[4], val[4];
#pragma unroll
        for (int w = 0; w < 4; w++) pair_rule<T>(xa[w], xb[w], pat[w], msk[w], msk7[w], val[w]);
#pragma unroll
        for (uint32_t j = 0; j < GROUP; j++) {
            if (k >= klim[j]) break;  // sorted: the rest of the unit has ended too (unused slots: klim = 0)
            const uint32_t xc[4] = {Cs[j].x, Cs[j].y, Cs[j].z, Cs[j].w};
            uint32_t hits = 0;
#pragma unroll
            for (int w = 0; w < 4; w++) {
                uint32_t ok;
                if (T == 0) {
                    // c is free: only the code has to agree
                    ok = val[w] & ~(((xc[w] ^ xa[w]) & C6) + K7);
                } else {
                    // lane of d is zero iff c matches the expected byte under the mask;
                    // bit 7 of d7 + 0x7F.. flags a nonzero lane of d7 (no carry leaves a lane)
                    const uint32_t d = (xc[w] ^ pat[w]) & msk[w];
                    const uint32_t d7 = (xc[w] ^ pat[w]) & msk7[w];
                    ok = val[w] & ~((d7 + K7) | d);
                }
                hits = __dp4a(ok, 0x01010101u, hits);  // 128 per counted slot
            }
            cnt[j] += hits >> 7;
        }
    }
}

__global__ void __launch_bounds__(WG_TPB) k_witness_group(View V, const uint32_t *__restrict__ pairs,
                                                       const uint64_t *__restrict__ cand_off,
                                                       const uint32_t *__restrict__ cand,
                                                       const uint2 *__restrict__ units, uint64_t nu,
                                                       uint32_t *__restrict__ sup) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint4 *bm4 = reinterpret_cast<const uint4 *>(V.bm);
    const uint32_t tq = V.shift - 4;  // 16-byte chunks per table block = r_0 / 16 = 2^(s-4)
    const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x / 32);
    for (uint64_t uid = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) / 32; uid < nu; uid += nwarps) {
        const uint2 u = units[uid];
        const uint64_t c0 = cand_off[u.x] + u.y;
        const uint64_t left = cand_off[u.x + 1] - c0;
        const uint32_t gn = left < GROUP ? (uint32_t)left : GROUP;
        const uint32_t a = pairs[3ull * u.x], b = pairs[3ull * u.x + 1];
        const uint32_t ra = 1u << V.rlog[a], rb = 1u << V.rlog[b];
        const uint64_t ca = V.base[a] >> 4, cb = V.base[b] >> 4;
        const uint32_t ma = ra / 4 - 1, mb = rb / 4 - 1;
        uint64_t cc[GROUP];
        uint32_t mc[GROUP], klim[GROUP], cnt[GROUP];
        uint32_t kmax = 0, probed = 0;  // probed: original slots routed to k_witness_probe
        const uint32_t la = V.rlog[a], lb = V.rlog[b];
#pragma unroll
        for (uint32_t j = 0; j < GROUP; j++) {
            cnt[j] = 0;
            const uint32_t c = j < gn ? cand[3 * (c0 + j) + 2] : 0u;
            const uint32_t lc = j < gn ? V.rlog[c] : 0u;
            if (j < gn && probe_route(la, lb, lc)) probed |= 1u << j;
            if (j < gn && !((probed >> j) & 1u)) {
                const uint32_t rc = 1u << lc;
                cc[j] = V.base[c] >> 4;
                mc[j] = rc / 4 - 1;
                klim[j] = max(max(ra, rb), rc) / 16;  // chunks of one table this triple runs over
            } else {
                cc[j] = 0;
                mc[j] = 0;
                klim[j] = 0;
            }
            kmax = max(kmax, klim[j]);
        }
        // Order the unit by decreasing klim (odd-even transposition sort), so
        // the candidates still running at chunk k are a prefix; pos holds the
        // original slot of each (four bits per slot).
        uint32_t pos = 0;
#pragma unroll
        for (uint32_t j = 0; j < GROUP; j++) pos |= j << (4 * j);
#pragma unroll
        for (uint32_t r = 0; r < GROUP; r++) {
#pragma unroll
            for (uint32_t j = r & 1u; j + 1 < GROUP; j += 2) {
                if (klim[j] < klim[j + 1]) {
                    const uint32_t tk = klim[j], tm = mc[j];
                    const uint64_t tc = cc[j];
                    klim[j] = klim[j + 1];
                    mc[j] = mc[j + 1];
                    cc[j] = cc[j + 1];
                    klim[j + 1] = tk;
                    mc[j + 1] = tm;
                    cc[j + 1] = tc;
                    const uint32_t f = ((pos >> (4 * j)) ^ (pos >> (4 * j + 4))) & 15u;
                    pos ^= (f << (4 * j)) | (f << (4 * j + 4));
                }
            }
        }
        group_pass<0>(bm4, lane, tq, kmax, ca, ma, cb, mb, cc, mc, klim, cnt);
        group_pass<1>(bm4, lane, tq, kmax, ca, ma, cb, mb, cc, mc, klim, cnt);
        group_pass<2>(bm4, lane, tq, kmax, ca, ma, cb, mb, cc, mc, klim, cnt);
        group_pass<3>(bm4, lane, tq, kmax, ca, ma, cb, mb, cc, mc, klim, cnt);
#pragma unroll
        for (uint32_t j = 0; j < GROUP; j++) {
            if (j >= gn) break;  // unused slots (klim = 0) sort last
            const uint32_t o = (pos >> (4 * j)) & 15u;
            if ((probed >> o) & 1u) continue;  // written by k_witness_probe
            const uint32_t it[3] = {a, b, cand[3 * (c0 + o) + 2]};
            uint32_t v = cnt[j] + failed_common<3, 4>(V, it, lane);
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
            if (lane == 0) sup[c0 + o] = v;
        }
    }
}

// ---- Apriori level 3 ------------------------------------------------------------

// Frequent pairs (i, j, support), i < j, lexicographic: err <- 1 unless the
// list is strictly increasing with ids < n.  row_off[i] = first pair of row i.
__global__ void k_check_pairs(const uint32_t *pairs, uint64_t np, uint32_t n, int *err) {
    for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < np;
         p += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t a = pairs[3 * p], b = pairs[3 * p + 1];
        bool bad = !(a < b) || b >= n;
        if (p + 1 < np) {
            const uint32_t a2 = pairs[3 * p + 3], b2 = pairs[3 * p + 4];
            bad |= !(a < a2 || (a == a2 && b < b2));
        }
        if (bad) atomicExch(err, 1);
    }
}

__global__ void k_pair_rows(const uint32_t *pairs, uint64_t np, uint32_t n, uint64_t *row_off) {
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i > n) return;
    uint64_t lo = 0, hi = np;
    while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        if (pairs[3 * mid] < i) lo = mid + 1; else hi = mid;
    }
    row_off[i] = lo;
}

// For the frequent pair p = (a, b): every c > b with (a, c) and (b, c)
// frequent -- the merge of the rest of row a after p with row b (both
// ascending).  COUNT writes the number into cnt[p]; otherwise the triples
// are written from offset cnt[p] (the exclusive scan of the counts).
template <bool WRITE>
__global__ void k_candidates(const uint32_t *__restrict__ pairs, uint64_t np, const uint64_t *__restrict__ row_off,
                             uint64_t *cnt, uint32_t *__restrict__ out) {
    for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < np;
         p += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t a = pairs[3 * p], b = pairs[3 * p + 1];
        uint64_t u = p + 1, ue = row_off[a + 1], v = row_off[b], ve = row_off[b + 1];
        uint64_t k = WRITE ? cnt[p] : 0;
        while (u < ue && v < ve) {
            const uint32_t cu = pairs[3 * u + 1], cv = pairs[3 * v + 1];
            if (cu < cv) {
                u++;
            } else if (cv < cu) {
                v++;
            } else {
                if (WRITE) {
                    out[3 * k] = a;
                    out[3 * k + 1] = b;
                    out[3 * k + 2] = cu;
                }
                k++;
                u++;
                v++;
            }
        }
        if (!WRITE) cnt[p] = k;
    }
}

// Ordered compaction of the K-item candidates with support >= s into
// (item_1, .., item_K, support).
constexpr int TH_PER = 8;
template <int K, bool WRITE>
__global__ void k_tuple_threshold(const uint32_t *__restrict__ cand, const uint32_t *__restrict__ sup, uint64_t nc,
                                  uint32_t s, uint64_t *blocksums, uint32_t *__restrict__ out, uint64_t cap) {
    const uint64_t b0 = (uint64_t)blockIdx.x * SCAN_TPB * TH_PER;
    uint64_t running = WRITE ? blocksums[blockIdx.x] : 0;
    for (int j = 0; j < TH_PER; j++) {
        const uint64_t c = b0 + (uint64_t)j * SCAN_TPB + threadIdx.x;
        const bool keep = c < nc && sup[c] >= s;
        uint64_t tot;
        const uint64_t rank = block_exclusive_scan(keep ? 1 : 0, &tot);
        if (WRITE && keep && running + rank < cap) {
            const uint64_t o = (K + 1) * (running + rank);
#pragma unroll
            for (int q = 0; q < K; q++) out[o + q] = cand[(uint64_t)K * c + q];
            out[o + K] = sup[c];
        }
        running += tot;
    }
    if (!WRITE && threadIdx.x == 0) blocksums[blockIdx.x] = running;
}

// ---- Apriori level 4 ------------------------------------------------------------

// Frequent triples (a, b, c, support), a < b < c < n, lexicographic: err <- 1
// unless the list is strictly increasing with ids < n.
__global__ void k_check_triples(const uint32_t *t3, uint64_t nt, uint32_t n, int *err) {
    for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < nt;
         p += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t a = t3[4 * p], b = t3[4 * p + 1], c = t3[4 * p + 2];
        bool bad = !(a < b && b < c) || c >= n;
        if (p + 1 < nt) {
            const uint32_t a2 = t3[4 * p + 4], b2 = t3[4 * p + 5], c2 = t3[4 * p + 6];
            bad |= !(a < a2 || (a == a2 && (b < b2 || (b == b2 && c < c2))));
        }
        if (bad) atomicExch(err, 1);
    }
}

// Is (a, b, c) one of the nt lexicographic triples?  (binary search)
__device__ __forceinline__ bool has_triple(const uint32_t *t3, uint64_t nt, uint32_t a, uint32_t b, uint32_t c) {
    uint64_t lo = 0, hi = nt;
    while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        const uint32_t x = t3[4 * mid], y = t3[4 * mid + 1], z = t3[4 * mid + 2];
        const bool less = x < a || (x == a && (y < b || (y == b && z < c)));
        if (less) lo = mid + 1; else hi = mid;
    }
    return lo < nt && t3[4 * lo] == a && t3[4 * lo + 1] == b && t3[4 * lo + 2] == c;
}

// For the frequent triple p = (a, b, c): every d > c with (a, b, d) frequent
// (the later triples of p's (a, b) run) whose other 3-subsets (a, c, d) and
// (b, c, d) are frequent too.  COUNT writes the number into cnt[p]; otherwise
// the quadruples are written from offset cnt[p].
template <bool WRITE>
__global__ void k_quad_candidates(const uint32_t *__restrict__ t3, uint64_t nt, uint64_t *cnt,
                                  uint32_t *__restrict__ out) {
    for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < nt;
         p += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t a = t3[4 * p], b = t3[4 * p + 1], c = t3[4 * p + 2];
        uint64_t k = WRITE ? cnt[p] : 0;
        for (uint64_t q = p + 1; q < nt && t3[4 * q] == a && t3[4 * q + 1] == b; q++) {
            const uint32_t d = t3[4 * q + 2];
            if (has_triple(t3, nt, a, c, d) && has_triple(t3, nt, b, c, d)) {
                if (WRITE) {
                    out[4 * k] = a;
                    out[4 * k + 1] = b;
                    out[4 * k + 2] = c;
                    out[4 * k + 3] = d;
                }
                k++;
            }
        }
        if (!WRITE) cnt[p] = k;
    }
}

}  // namespace wit

// One warp per query: k ids each, on a set of d + 1 tables.
static void launch_witness(const wit::View &V, uint32_t d, uint32_t k, const uint32_t *d_items, uint64_t nq,
                           uint32_t *d_support, cudaStream_t st, uint32_t skip_routed = 0) {
    using namespace wit;
    if (nq == 0) return;
    const unsigned grid = (unsigned)std::min<uint64_t>((nq + 7) / 8, 152ull * 64);
    if (d == 3) {
        if (k == 1) k_witness<1, 4><<<grid, 256, 0, st>>>(V, d_items, nq, d_support, skip_routed);
        if (k == 2) k_witness<2, 4><<<grid, 256, 0, st>>>(V, d_items, nq, d_support, skip_routed);
        if (k == 3) k_witness<3, 4><<<grid, 256, 0, st>>>(V, d_items, nq, d_support, skip_routed);
    } else {
        if (k == 1) k_witness<1, 5><<<grid, 256, 0, st>>>(V, d_items, nq, d_support, skip_routed);
        if (k == 2) k_witness<2, 5><<<grid, 256, 0, st>>>(V, d_items, nq, d_support, skip_routed);
        if (k == 3) k_witness<3, 5><<<grid, 256, 0, st>>>(V, d_items, nq, d_support, skip_routed);
        if (k == 4) k_witness<4, 5><<<grid, 256, 0, st>>>(V, d_items, nq, d_support, skip_routed);
    }
    BM_CHECK_LAUNCH();
}

// Candidate supports on a 4-of-5 set with both routes: the scan kernel skips
// the width-skewed candidates, the probe kernel takes them.  Records event 4
// of E between the two.
static void witness_routed5(const wit::View &V, uint32_t k, const uint32_t *d_items, uint64_t nq,
                            const uint32_t *d_rlog, uint32_t *d_support, PhaseEvents &E, cudaStream_t st) {
    using namespace wit;
    if (nq == 0) return;
    launch_witness(V, 4, k, d_items, nq, d_support, st, 1);
    E.record(4, st);
    DevBuf<uint32_t> plist(nq);
    DevBuf<unsigned long long> pcount(1);
    BM_CUDA(cudaMemsetAsync(pcount.p, 0, sizeof(unsigned long long), st));
    if (k == 3) k_route_probe_k<3, 5><<<grid_for(nq), 256, 0, st>>>(d_items, nq, d_rlog, plist.p, pcount.p);
    else k_route_probe_k<4, 5><<<grid_for(nq), 256, 0, st>>>(d_items, nq, d_rlog, plist.p, pcount.p);
    BM_CHECK_LAUNCH();
    if (k == 3) k_witness_probe_k<3, 5><<<152 * 16, 256, 0, st>>>(V, d_items, plist.p, pcount.p, d_support);
    else k_witness_probe_k<4, 5><<<152 * 16, 256, 0, st>>>(V, d_items, plist.p, pcount.p, d_support);
    BM_CHECK_LAUNCH();
}

// Supports of n_q queries of k item ids each (k in 1..d) on a d-of-(d+1) set.
void witness_support(batmap_set *S, uint32_t k, uint64_t nq, const uint32_t *d_items, uint32_t *d_support,
                     cudaStream_t st) {
    using namespace wit;
    BM_REQUIRE(S && (S->d == 3 || S->d == 4), BATMAP_ERR_ARG, "itemset supports need a set built with d = 3 or 4");
    BM_REQUIRE(k >= 1 && k <= S->d, BATMAP_ERR_ARG, "k must be in 1..d");
    if (nq == 0) return;
    BM_REQUIRE(d_items && d_support, BATMAP_ERR_ARG, "NULL argument");
    {
        DevBuf<int> err(1);
        BM_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), st));
        k_check_ids<<<grid_for(nq * k), 256, 0, st>>>(d_items, nq * k, S->n, err.p);
        BM_CHECK_LAUNCH();
        int h = 0;
        BM_CUDA(cudaMemcpyAsync(&h, err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        BM_CUDA(cudaStreamSynchronize(st));
        BM_REQUIRE(h == 0, BATMAP_ERR_ARG, "item id >= n in a query");
    }
    const View V{reinterpret_cast<const uint32_t *>(S->d_bm.p), S->d_base.p, S->d_rlog.p, S->perm,
                 S->d_fail_off.p, S->d_fail_tid.p, S->m, S->n, S->shift};
    launch_witness(V, S->d, k, d_items, nq, d_support, st);
}

// Frequent itemsets of size 3 from the frequent pairs (Apriori join and
// prune), supports by the witness rule, compaction in lexicographic order.
void frequent_triples(batmap_set *S, uint32_t s, const uint32_t *d_pairs, uint64_t np, uint32_t *d_out,
                      uint64_t cap, uint64_t *n_out, uint64_t *n_cand, cudaStream_t st) {
    using namespace wit;
    BM_REQUIRE(S && (S->d == 3 || S->d == 4), BATMAP_ERR_ARG, "frequent_triples needs a set built with d = 3 or 4");
    const bool grouped = S->d == 3;  // the grouped kernel reads the 3-of-4 format
    BM_REQUIRE(n_out, BATMAP_ERR_ARG, "n_out is NULL");
    BM_REQUIRE(np == 0 || d_pairs, BATMAP_ERR_ARG, "d_pairs is NULL");
    BM_REQUIRE(cap == 0 || d_out, BATMAP_ERR_ARG, "d_out is NULL with cap > 0");
    PhaseEvents &E = S->pairs_ev;
    E.create();
    E.record(0, st);
    const uint32_t n = S->n;
    uint64_t nc = 0, n_units = 0;
    DevBuf<uint32_t> cand, sup;
    DevBuf<uint2> units;
    DevBuf<uint64_t> cnt;  // candidate offsets per frequent pair, [np + 1]
    if (np) {
        DevBuf<int> err(1);
        BM_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), st));
        k_check_pairs<<<grid_for(np), 256, 0, st>>>(d_pairs, np, n, err.p);
        BM_CHECK_LAUNCH();
        DevBuf<uint64_t> row_off(n + 1), tot(1);
        cnt.alloc(np + 1);
        k_pair_rows<<<grid_for(n + 1), 256, 0, st>>>(d_pairs, np, n, row_off.p);
        BM_CHECK_LAUNCH();
        int h = 0;
        BM_CUDA(cudaMemcpyAsync(&h, err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        BM_CUDA(cudaStreamSynchronize(st));
        BM_REQUIRE(h == 0, BATMAP_ERR_ARG, "pairs must be (i, j, support) with i < j < n, lexicographic");
        k_candidates<false><<<grid_for(np), 256, 0, st>>>(d_pairs, np, row_off.p, cnt.p, nullptr);
        BM_CHECK_LAUNCH();
        k_scan_single_block<<<1, SCAN_TPB, 0, st>>>(cnt.p, np, tot.p, 1);  // cnt[np] = total
        BM_CHECK_LAUNCH();
        BM_CUDA(cudaMemcpyAsync(&nc, tot.p, 8, cudaMemcpyDeviceToHost, st));
        BM_CUDA(cudaStreamSynchronize(st));
        cand.alloc(3 * nc);
        sup.alloc(nc);
        if (nc) {
            k_candidates<true><<<grid_for(np), 256, 0, st>>>(d_pairs, np, row_off.p, cnt.p, cand.p);
            BM_CHECK_LAUNCH();
        }
        if (nc && grouped) {
            // work units of up to GROUP candidates sharing their frequent pair
            DevBuf<uint64_t> uoff(np + 1), utot(1);
            k_unit_counts<<<grid_for(np), 256, 0, st>>>(cnt.p, np, uoff.p);
            BM_CHECK_LAUNCH();
            k_scan_single_block<<<1, SCAN_TPB, 0, st>>>(uoff.p, np, utot.p, 1);
            BM_CHECK_LAUNCH();
            uint64_t nu = 0;
            BM_CUDA(cudaMemcpyAsync(&nu, utot.p, 8, cudaMemcpyDeviceToHost, st));
            BM_CUDA(cudaStreamSynchronize(st));
            units.alloc(nu);
            k_unit_fill<<<grid_for(np), 256, 0, st>>>(cnt.p, uoff.p, np, units.p);
            BM_CHECK_LAUNCH();
            n_units = nu;
        }
    }
    if (n_cand) *n_cand = nc;
    E.record(1, st);
    if (nc) {
        const View V{reinterpret_cast<const uint32_t *>(S->d_bm.p), S->d_base.p, S->d_rlog.p, S->perm,
                     S->d_fail_off.p, S->d_fail_tid.p, S->m, S->n, S->shift};
        if (grouped) {
            const uint64_t wpb = WG_TPB / 32;
            const unsigned grid = (unsigned)std::min<uint64_t>((n_units + wpb - 1) / wpb, 152ull * 64);
            k_witness_group<<<grid, WG_TPB, 0, st>>>(V, d_pairs, cnt.p, cand.p, units.p, n_units, sup.p);
            BM_CHECK_LAUNCH();
            E.record(4, st);
            DevBuf<uint32_t> plist(nc);
            DevBuf<unsigned long long> pcount(1);
            BM_CUDA(cudaMemsetAsync(pcount.p, 0, sizeof(unsigned long long), st));
            k_route_probe<<<grid_for(nc), 256, 0, st>>>(cand.p, nc, S->d_rlog.p, plist.p, pcount.p);
            BM_CHECK_LAUNCH();
            k_witness_probe<<<152 * 16, 256, 0, st>>>(V, cand.p, plist.p, pcount.p, sup.p);
            BM_CHECK_LAUNCH();
        } else {
            witness_routed5(V, 3, cand.p, nc, S->d_rlog.p, sup.p, E, st);  // one warp per candidate or probe
        }
    }
    E.record(2, st);
    uint64_t total = 0;
    if (nc) {
        const uint64_t per_block = (uint64_t)SCAN_TPB * TH_PER;
        const uint64_t nb = (nc + per_block - 1) / per_block;
        DevBuf<uint64_t> bs(nb + 1), tot(1);
        k_tuple_threshold<3, false><<<(unsigned)nb, SCAN_TPB, 0, st>>>(cand.p, sup.p, nc, s, bs.p, nullptr, 0);
        BM_CHECK_LAUNCH();
        k_scan_single_block<<<1, SCAN_TPB, 0, st>>>(bs.p, nb, tot.p, 1);
        BM_CHECK_LAUNCH();
        k_tuple_threshold<3, true><<<(unsigned)nb, SCAN_TPB, 0, st>>>(cand.p, sup.p, nc, s, bs.p, d_out, cap);
        BM_CHECK_LAUNCH();
        BM_CUDA(cudaMemcpyAsync(&total, tot.p, 8, cudaMemcpyDeviceToHost, st));
    }
    E.record(3, st);
    BM_CUDA(cudaStreamSynchronize(st));
    S->timing.compare_ms = E.ms(1, 2);
    S->timing.compact_ms = E.ms(0, 1) + E.ms(2, 3);
    S->timing.pairs_ms = E.ms(0, 3);
    const bool split = nc > 0;  // event 4 sits between the scan and the probe kernels (both routes)
    S->timing.scan_ms = split ? E.ms(1, 4) : S->timing.compare_ms;
    S->timing.probe_ms = split ? E.ms(4, 2) : 0.f;
    *n_out = total;
    if (total > cap)
        throw Error{BATMAP_ERR_CAPACITY, "d_out too small: " + std::to_string(total) + " triples qualify"};
}

// Frequent itemsets of size 4 from the frequent triples (Apriori join of the
// triples sharing (a, b), pruned by the other two 3-subsets), supports by the
// five-table witness rule, compaction in lexicographic order.
void frequent_quadruples(batmap_set *S, uint32_t s, const uint32_t *d_triples, uint64_t nt, uint32_t *d_out,
                         uint64_t cap, uint64_t *n_out, uint64_t *n_cand, cudaStream_t st) {
    using namespace wit;
    BM_REQUIRE(S && S->d == 4, BATMAP_ERR_ARG, "frequent_quadruples needs a set built with d = 4");
    BM_REQUIRE(n_out, BATMAP_ERR_ARG, "n_out is NULL");
    BM_REQUIRE(nt == 0 || d_triples, BATMAP_ERR_ARG, "d_triples is NULL");
    BM_REQUIRE(cap == 0 || d_out, BATMAP_ERR_ARG, "d_out is NULL with cap > 0");
    PhaseEvents &E = S->pairs_ev;
    E.create();
    E.record(0, st);
    uint64_t nc = 0;
    DevBuf<uint32_t> cand, sup;
    if (nt) {
        DevBuf<int> err(1);
        DevBuf<uint64_t> cnt(nt + 1), tot(1);
        BM_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), st));
        k_check_triples<<<grid_for(nt), 256, 0, st>>>(d_triples, nt, S->n, err.p);
        BM_CHECK_LAUNCH();
        int h = 0;
        BM_CUDA(cudaMemcpyAsync(&h, err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        BM_CUDA(cudaStreamSynchronize(st));
        BM_REQUIRE(h == 0, BATMAP_ERR_ARG, "triples must be (a, b, c, support) with a < b < c < n, lexicographic");
        k_quad_candidates<false><<<grid_for(nt), 256, 0, st>>>(d_triples, nt, cnt.p, nullptr);
        BM_CHECK_LAUNCH();
        k_scan_single_block<<<1, SCAN_TPB, 0, st>>>(cnt.p, nt, tot.p, 1);
        BM_CHECK_LAUNCH();
        BM_CUDA(cudaMemcpyAsync(&nc, tot.p, 8, cudaMemcpyDeviceToHost, st));
        BM_CUDA(cudaStreamSynchronize(st));
        cand.alloc(4 * nc);
        sup.alloc(nc);
        if (nc) {
            k_quad_candidates<true><<<grid_for(nt), 256, 0, st>>>(d_triples, nt, cnt.p, cand.p);
            BM_CHECK_LAUNCH();
        }
    }
    if (n_cand) *n_cand = nc;
    E.record(1, st);
    if (nc) {
        const View V{reinterpret_cast<const uint32_t *>(S->d_bm.p), S->d_base.p, S->d_rlog.p, S->perm,
                     S->d_fail_off.p, S->d_fail_tid.p, S->m, S->n, S->shift};
        witness_routed5(V, 4, cand.p, nc, S->d_rlog.p, sup.p, E, st);
    }
    E.record(2, st);
    uint64_t total = 0;
    if (nc) {
        const uint64_t per_block = (uint64_t)SCAN_TPB * TH_PER;
        const uint64_t nb = (nc + per_block - 1) / per_block;
        DevBuf<uint64_t> bs(nb + 1), tot(1);
        k_tuple_threshold<4, false><<<(unsigned)nb, SCAN_TPB, 0, st>>>(cand.p, sup.p, nc, s, bs.p, nullptr, 0);
        BM_CHECK_LAUNCH();
        k_scan_single_block<<<1, SCAN_TPB, 0, st>>>(bs.p, nb, tot.p, 1);
        BM_CHECK_LAUNCH();
        k_tuple_threshold<4, true><<<(unsigned)nb, SCAN_TPB, 0, st>>>(cand.p, sup.p, nc, s, bs.p, d_out, cap);
        BM_CHECK_LAUNCH();
        BM_CUDA(cudaMemcpyAsync(&total, tot.p, 8, cudaMemcpyDeviceToHost, st));
    }
    E.record(3, st);
    BM_CUDA(cudaStreamSynchronize(st));
    S->timing.compare_ms = E.ms(1, 2);
    S->timing.scan_ms = nc ? E.ms(1, 4) : 0.f;  // event 4 sits between the scan and the probe kernels
    S->timing.probe_ms = nc ? E.ms(4, 2) : 0.f;
    S->timing.compact_ms = E.ms(0, 1) + E.ms(2, 3);
    S->timing.pairs_ms = E.ms(0, 3);
    *n_out = total;
    if (total > cap)
        throw Error{BATMAP_ERR_CAPACITY, "d_out too small: " + std::to_string(total) + " quadruples qualify"};
}

}  // namespace bm
