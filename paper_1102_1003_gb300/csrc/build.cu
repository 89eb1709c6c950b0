// BatMap construction on the GPU (Sec. II and Sec. III-A/C).
//
//   validate  : tids strictly increasing and < m per item; each permutation
//               row a bijection of [0, m)
//   size      : s, r_0, r_i, widths 3 r_i, width-sorted order (host)
//   place     : parallel generalised cuckoo INSERT into uint32 tables
//   finalize  : every element with exactly two copies gets its two bytes
//               (indicator << 7 | code); the rest are failed insertions
//   failures  : F_i in (item, tid) order, then the correction entries: one
//               (min, max) item pair per failed common transaction
//   schedule  : compare work units (host, compare.cu)
#include <algorithm>
#include <cstring>
#include <mutex>
#include <numeric>

#include "common.cuh"
#include "items.cuh"
#include "perm.cuh"
#include "scan.cuh"

namespace bm {

void build_schedule(batmap_set *S);  // compare.cu

// ---- validation ---------------------------------------------------------------

__global__ void k_validate_tids(ItemView v, uint32_t m, int *err) {
    uint32_t item;
    uint64_t e0, e1;
    chunk_range(v, blockIdx.x, &item, &e0, &e1);
    for (uint64_t e = e0 + threadIdx.x; e < e1; e += TPB) {
        uint32_t x = v.tids[e];
        bool bad = x >= m;
        if (e + 1 < v.off[item + 1]) bad |= !(x < v.tids[e + 1]);
        if (bad) atomicExch(err, 1);
    }
}

__global__ void k_validate_perm(const uint32_t *perm, uint32_t m, uint32_t rows, uint32_t *bits, int *err) {
    uint64_t total = (uint64_t)rows * m;
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < total;
         q += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t t = (uint32_t)(q / m);
        uint32_t val = perm[q];
        if (val >= m) {
            atomicExch(err, 2);
            continue;
        }
        uint64_t w = (uint64_t)t * ((m + 31) / 32) + val / 32;
        uint32_t bit = 1u << (val % 32);
        uint32_t old = atomicOr(&bits[w], bit);
        if (old & bit) atomicExch(err, 2);
    }
}

// ---- placement: parallel 2-of-3 cuckoo insertion (Sec. II-A) --------------------
//
// Each thread carries one copy of one element.  Copy c starts in table c; a
// copy is swapped into its slot of table t; the evicted occupant (if any)
// continues in table t+1 (cyclic order 1,2,3,1,...).  Swapping a copy with
// the other copy of the same element leaves the table unchanged and the
// element continues in the next table, so the two copies always end in two
// distinct tables.  Atomic exchanges conserve copies; a chain that exceeds
// 3*MaxLoop moves drops the copy it holds, and finalize then reports that
// element as a failed insertion.
__global__ void k_place(ItemView v, const PermView P, uint32_t shift, uint32_t max_moves,
                        uint32_t *__restrict__ table) {
    const uint32_t m = P.m;
    uint32_t item;
    uint64_t e0, e1;
    chunk_range(v, blockIdx.x >> 1, &item, &e0, &e1);
    const uint32_t copy = blockIdx.x & 1u;
    const uint64_t base = v.base[item];
    const uint32_t r = 1u << v.rlog[item];
    for (uint64_t e = e0 + threadIdx.x; e < e1; e += TPB) {
        uint32_t x = v.tids[e];
        if (x >= m) continue;  // rejected by validation; never index past perm
        uint32_t t = copy;
        for (uint32_t mv = 0; mv < max_moves; mv++) {
            uint32_t pi = P(t, x);
            uint64_t pos = base + slot_of(t, pi, r, shift);
            uint32_t old = atomicExch(&table[pos], x);
            if (old == EMPTY) break;
            x = old;  // old == x: same element, continue in the next table
            t = (t == 2) ? 0 : t + 1;
        }
    }
}

struct Copies {
    uint32_t pi[3];
    uint64_t pos[3];
    uint32_t has;  // bit t set: a copy sits in table t
};

__device__ __forceinline__ Copies find_copies(uint32_t x, uint64_t base, uint32_t r, uint32_t shift,
                                              const PermView &P, const uint32_t *__restrict__ table) {
    Copies c;
    c.has = 0;
#pragma unroll
    for (uint32_t t = 0; t < 3; t++) {
        c.pi[t] = P(t, x);
        c.pos[t] = base + slot_of(t, c.pi[t], r, shift);
        if (table[c.pos[t]] == x) c.has |= 1u << t;
    }
    return c;
}

__device__ __forceinline__ bool two_copies(uint32_t has) { return __popc(has) == 2; }

// Writes the two bytes of every element stored twice.  The indicator is 1 on
// the copy whose twin sits in the cyclic predecessor table (Fig. 3).
// Also counts the block's failed insertions into blocksums[block] (the count
// pass of the ordered compaction that lists them).
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
        uint32_t x = v.tids[e];
        if (x >= m) continue;
        Copies c = find_copies(x, base, r, shift, P, table);
        if (!two_copies(c.has)) {
            fails++;
            continue;
        }
#pragma unroll
        for (uint32_t t = 0; t < 3; t++) {
            if (c.has & (1u << t)) {
                uint32_t pred = (t + 2) % 3;
                uint32_t ind = (c.has >> pred) & 1u;
                out[c.pos[t]] = (uint8_t)element_byte(c.pi[t], shift, ind);
            }
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) fails += __shfl_xor_sync(0xffffffffu, fails, d);
    if ((threadIdx.x & 31) == 0 && fails) atomicAdd(&s_fail, fails);
    __syncthreads();
    if (threadIdx.x == 0) blocksums[blockIdx.x] = s_fail;
}

// ---- failed insertions, in (item, tid) order --------------------------------------

// Rank of each failing element inside its block, in element order.
template <bool WRITE>
__global__ void k_failures(ItemView v, const PermView P, uint32_t shift, const uint32_t *__restrict__ table,
                           uint64_t *blocksums, uint32_t *f_item, uint32_t *f_tid) {
    const uint32_t m = P.m;
    uint32_t item;
    uint64_t e0, e1;
    chunk_range(v, blockIdx.x, &item, &e0, &e1);
    const uint64_t base = v.base[item];
    const uint32_t r = 1u << v.rlog[item];
    uint64_t running = WRITE ? blocksums[blockIdx.x] : 0;
    if (WRITE && blocksums[blockIdx.x + 1] == running) return;  // no failure in this block
    for (int j = 0; j < PER_THREAD; j++) {
        uint64_t e = e0 + (uint64_t)j * TPB + threadIdx.x;
        bool fail = false;
        uint32_t x = 0;
        if (e < e1) {
            x = v.tids[e];
            fail = x < m && !two_copies(find_copies(x, base, r, shift, P, table).has);
        }
        uint64_t tot;
        uint64_t rank = block_exclusive_scan(fail ? 1 : 0, &tot);
        if (WRITE && fail) {
            f_item[running + rank] = item;
            f_tid[running + rank] = x;
        }
        running += tot;
    }
    if (!WRITE && threadIdx.x == 0) blocksums[blockIdx.x] = running;
}

// f_off[i] = first failure of item i (lower bound in the sorted f_item list).
__global__ void k_fail_offsets(const uint32_t *f_item, uint64_t nfail, uint32_t n, uint64_t *f_off) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n) return;
    uint64_t lo = 0, hi = nfail;
    while (lo < hi) {
        uint64_t mid = (lo + hi) >> 1;
        if (f_item[mid] < i) lo = mid + 1; else hi = mid;
    }
    f_off[i] = lo;
}

// ---- correction entries (Sec. III-C "Failed insertions") --------------------------
//
// For a failed (a, x) and every item c != a containing x, the pair {a, c}
// misses x in the BatMap comparison.  When x failed in c as well, the pair
// is generated from the smaller id only, so each (x, pair) is added once.

__global__ void k_mark_failed(const uint32_t *f_tid, uint64_t nfail, uint32_t *bits) {
    for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < nfail;
         k += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t x = f_tid[k];
        atomicOr(&bits[x >> 5], 1u << (x & 31));
    }
}

__global__ void k_popc_words(const uint32_t *bits, uint64_t nwords, uint64_t *out) {
    for (uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; w < nwords;
         w += (uint64_t)gridDim.x * blockDim.x)
        out[w] = __popc(bits[w]);
}

__device__ __forceinline__ bool failed_bit(const uint32_t *bits, uint32_t x) {
    return (bits[x >> 5] >> (x & 31)) & 1u;
}

__device__ __forceinline__ uint32_t bit_rank(const uint32_t *bits, const uint64_t *wrank, uint32_t x) {
    return (uint32_t)(wrank[x >> 5] + __popc(bits[x >> 5] & ((1u << (x & 31)) - 1u)));
}

__global__ void k_count_per_tid(const uint32_t *f_tid, uint64_t nfail, const uint32_t *bits,
                                const uint64_t *wrank, uint64_t *cnt) {
    for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < nfail;
         k += (uint64_t)gridDim.x * blockDim.x)
        atomicAdd((unsigned long long *)&cnt[bit_rank(bits, wrank, f_tid[k])], 1ull);
}

__global__ void k_fill_per_tid(const uint32_t *f_item, const uint32_t *f_tid, uint64_t nfail,
                               const uint32_t *bits, const uint64_t *wrank, const uint64_t *fptr,
                               unsigned long long *cursor, uint32_t *fitems) {
    for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < nfail;
         k += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t u = bit_rank(bits, wrank, f_tid[k]);
        uint64_t p = fptr[u] + atomicAdd(&cursor[u], 1ull);
        fitems[p] = f_item[k];
    }
}

template <bool WRITE>
__global__ void k_corrections(ItemView v, uint32_t m, const uint32_t *bits, const uint64_t *wrank,
                              const uint64_t *fptr, const uint32_t *fitems,
                              unsigned long long *counter, uint32_t *corr) {
    uint32_t c;
    uint64_t e0, e1;
    chunk_range(v, blockIdx.x, &c, &e0, &e1);
    for (uint64_t e = e0 + threadIdx.x; e < e1; e += TPB) {
        uint32_t x = v.tids[e];
        if (x >= m || !failed_bit(bits, x)) continue;
        uint32_t u = bit_rank(bits, wrank, x);
        uint64_t b0 = fptr[u], b1 = fptr[u + 1];
        bool c_failed = false;
        for (uint64_t k = b0; k < b1; k++) c_failed |= (fitems[k] == c);
        for (uint64_t k = b0; k < b1; k++) {
            uint32_t a = fitems[k];
            if (a == c) continue;
            if (c_failed && c < a) continue;  // generated from c's side
            unsigned long long slot = atomicAdd(counter, 1ull);
            if (WRITE) {
                corr[2 * slot] = a < c ? a : c;
                corr[2 * slot + 1] = a < c ? c : a;
            }
        }
    }
}

// ---- host side -------------------------------------------------------------------

PermView make_perm_view(const uint32_t *table, uint32_t m, uint64_t seed) {
    PermView P{};
    P.table = table;
    P.m = m;
    uint32_t b = 0;
    while (b < 32 && (1ull << b) < (uint64_t)m) b++;  // ceil(log2 m)
    b = std::max<uint32_t>(b, 2);
    b += b & 1u;
    P.half = b / 2;
    P.mask = (1u << P.half) - 1u;
    // SplitMix64 from the seed: four round keys per table, low 32 bits each
    uint64_t state = seed;
    uint32_t k[4 * PERM_MAX_TABLES];
    for (int j = 0; j < 4 * PERM_MAX_TABLES; j++) {
        state += 0x9E3779B97F4A7C15ull;
        uint64_t z = state;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        k[j] = (uint32_t)(z ^ (z >> 31));
    }
    for (int t = 0; t < PERM_MAX_TABLES; t++) P.key[t] = make_uint4(k[4 * t], k[4 * t + 1], k[4 * t + 2], k[4 * t + 3]);
    return P;
}

static uint32_t shift_bits(uint32_t m, uint32_t min_shift) {
    uint32_t s = min_shift;
    while ((uint64_t)m > 127ull << s) s++;
    return s;
}

// The placement scratch (one uint32 per BatMap byte) is kept between builds
// so that repeated builds do not pay for allocating and freeing it; it is
// released when a build needs less than a quarter of it or on
// batmap_release_scratch().  Builds are serialised on it.
std::mutex g_scratch_mu;
static DevBuf<uint32_t> g_scratch;

DevBuf<uint32_t> &scratch_table(uint64_t slots) {
    if (g_scratch.n < slots || g_scratch.n > 4 * slots + (1u << 20)) g_scratch.alloc(slots);
    return g_scratch;
}

void release_scratch() {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    g_scratch.release();
    bm_buffer_release_all();
}

// ---- cache of BatMap arrays ----------------------------------------------------------

namespace {
struct CachedBuf {
    uint8_t *p;
    size_t cap;
};
std::mutex g_bm_cache_mu;
std::vector<CachedBuf> g_bm_cache;  // at most two, oldest first
}  // namespace

uint8_t *bm_buffer_take(size_t bytes, size_t *capacity) {
    {
        std::lock_guard<std::mutex> lock(g_bm_cache_mu);
        int best = -1;
        for (int i = 0; i < (int)g_bm_cache.size(); i++) {
            const size_t c = g_bm_cache[i].cap;
            if (c >= bytes && c <= 2 * bytes + (64ull << 20) && (best < 0 || c < g_bm_cache[best].cap)) best = i;
        }
        if (best >= 0) {
            const CachedBuf b = g_bm_cache[best];
            g_bm_cache.erase(g_bm_cache.begin() + best);
            *capacity = b.cap;
            return b.p;
        }
    }
    uint8_t *p = nullptr;
    BM_CUDA(cudaMalloc(&p, bytes));
    *capacity = bytes;
    return p;
}

void bm_buffer_give(uint8_t *p, size_t capacity) {
    // no queued work may still use the array when it is handed out again
    cudaDeviceSynchronize();
    std::lock_guard<std::mutex> lock(g_bm_cache_mu);
    g_bm_cache.push_back({p, capacity});
    if (g_bm_cache.size() > 2) {
        cudaFree(g_bm_cache.front().p);
        g_bm_cache.erase(g_bm_cache.begin());
    }
}

void bm_buffer_release_all() {
    std::lock_guard<std::mutex> lock(g_bm_cache_mu);
    for (auto &b : g_bm_cache) cudaFree(b.p);
    g_bm_cache.clear();
}

void build_set(batmap_set *S, const uint64_t *d_offsets, const uint32_t *d_tids,
               const uint32_t *d_perm) {
    std::lock_guard<std::mutex> scratch_lock(g_scratch_mu);
    const uint32_t m = S->m, n = S->n;
    cudaStream_t st = S->stream;
    const batmap_params &P = S->params;
    PhaseEvents &E = S->build_ev;
    E.create();
    E.record(0, st);

    // CSR offsets on the host: sizes drive the layout and the schedule.
    std::vector<uint64_t> off(n + 1, 0);
    if (n) {
        BM_REQUIRE(d_offsets != nullptr, BATMAP_ERR_ARG, "d_offsets is NULL");
        BM_CUDA(cudaMemcpyAsync(off.data(), d_offsets, (n + 1) * sizeof(uint64_t),
                                cudaMemcpyDeviceToHost, st));
        BM_CUDA(cudaStreamSynchronize(st));
    }
    BM_REQUIRE(off[0] == 0, BATMAP_ERR_ARG, "offsets[0] must be 0");
    for (uint32_t i = 0; i < n; i++)
        BM_REQUIRE(off[i + 1] >= off[i], BATMAP_ERR_ARG, "offsets must be non-decreasing");
    const uint64_t T = off[n];
    S->n_elements = T;
    BM_REQUIRE(T == 0 || d_tids != nullptr, BATMAP_ERR_ARG, "d_tids is NULL");
    const PermView PV = make_perm_view(d_perm, m, P.perm_seed);

    // ---- sizes (Sec. III-A) and width-sorted order (Sec. III-C) ----
    S->shift = shift_bits(m, P.min_shift);
    S->r0 = 1u << S->shift;
    std::vector<uint32_t> rlog(n);
    S->range.resize(n);
    for (uint32_t i = 0; i < n; i++) {
        rlog[i] = log2_range(off[i + 1] - off[i], P.load_num, P.load_den, S->shift);
        BM_REQUIRE(rlog[i] <= 31, BATMAP_ERR_ARG, "hash range exceeds 2^31");
        S->range[i] = 1u << rlog[i];
    }
    S->order.resize(n);
    std::iota(S->order.begin(), S->order.end(), 0u);
    // width-sorted (stable by id); in cross mode family A [0, n_a) first
    const uint32_t na = S->n_a;
    std::stable_sort(S->order.begin(), S->order.end(), [&](uint32_t a, uint32_t b) {
        const bool fa = na && a >= na, fb = na && b >= na;
        return fa != fb ? fb : rlog[a] < rlog[b];
    });
    S->rank.assign(n, 0);
    S->byte_off.assign(n, 0);
    S->wshift_sorted.assign(n, 0);
    std::vector<uint64_t> base(n, 0);
    std::vector<uint32_t> line_off(n, 0);
    uint64_t pos = 0;
    S->class_begin.clear();
    for (uint32_t q = 0; q < n; q++) {
        uint32_t i = S->order[q];
        S->rank[i] = q;
        S->byte_off[q] = pos;
        base[i] = pos;
        BM_REQUIRE(pos / 128 < (1ull << 32), BATMAP_ERR_ARG, "BatMap array exceeds 512 GB");
        line_off[q] = (uint32_t)(pos / 128);
        S->wshift_sorted[q] = rlog[i] - 2;
        if (q == 0 || rlog[S->order[q - 1]] != rlog[i] || (na && q == na)) S->class_begin.push_back(q);
        pos += 3ull << rlog[i];
    }
    S->class_begin.push_back(n);
    S->bytes = pos;
    // the compare kernel addresses BatMaps as 32-bit indices of 16-byte chunks
    BM_REQUIRE(pos <= (1ull << 36), BATMAP_ERR_ARG, "BatMaps of one set exceed 64 GB; split the instance");

    // algorithmic work of the compare: sum over pairs of the wider width / 4
    double wp = 0.0;
    if (!na) {
        for (uint32_t q = 0; q < n; q++) wp += (double)q * (double)((3ull << (S->wshift_sorted[q] + 2)) / 4);
    } else {
        // both families are width-sorted: A items no wider than b contribute b's width,
        // the wider ones their own (suffix sums over A)
        std::vector<double> suffix(na + 1, 0.0);
        for (uint32_t a = na; a-- > 0;) suffix[a] = suffix[a + 1] + (double)(3ull << S->wshift_sorted[a]);
        uint32_t a = 0;
        for (uint32_t b = na; b < n; b++) {
            while (a < na && S->wshift_sorted[a] <= S->wshift_sorted[b]) a++;
            wp += (double)a * (double)(3ull << S->wshift_sorted[b]) + suffix[a];
        }
    }
    S->word_pairs = wp;

    // ---- device metadata ----
    S->d_bm.alloc(S->bytes);
    S->d_line_off.alloc(n);
    S->d_wshift.alloc(n);
    S->d_order.alloc(n);
    if (n) {
        BM_CUDA(cudaMemcpyAsync(S->d_line_off.p, line_off.data(), n * 4, cudaMemcpyHostToDevice, st));
        BM_CUDA(cudaMemcpyAsync(S->d_wshift.p, S->wshift_sorted.data(), n * 4, cudaMemcpyHostToDevice, st));
        BM_CUDA(cudaMemcpyAsync(S->d_order.p, S->order.data(), n * 4, cudaMemcpyHostToDevice, st));
    }
    if (S->bytes) BM_CUDA(cudaMemsetAsync(S->d_bm.p, 0, S->bytes, st));

    // per-element chunks: block b handles elements [ch_start[b], +CHUNK) of item ch_item[b]
    std::vector<uint32_t> ch_item;
    std::vector<uint64_t> ch_start;
    for (uint32_t i = 0; i < n; i++)
        for (uint64_t s = off[i]; s < off[i + 1]; s += CHUNK) {
            ch_item.push_back(i);
            ch_start.push_back(s);
        }
    const uint32_t nch = (uint32_t)ch_item.size();

    S->d_fail_off.alloc(n + 1);
    if (T == 0) {
        BM_CUDA(cudaMemsetAsync(S->d_fail_off.p, 0, (n + 1) * sizeof(uint64_t), st));
        if (!S->skip_schedule) build_schedule(S);
        E.record(1, st);
        BM_CUDA(cudaStreamSynchronize(st));
        S->timing.build_ms = E.ms(0, 1);
        S->timing.place_ms = S->timing.finalize_ms = 0.f;
        return;
    }

    DevBuf<uint32_t> d_ch_item(nch), d_rlog(n);
    DevBuf<uint64_t> d_ch_start(nch), d_base(n);
    BM_CUDA(cudaMemcpyAsync(d_ch_item.p, ch_item.data(), nch * 4ull, cudaMemcpyHostToDevice, st));
    BM_CUDA(cudaMemcpyAsync(d_ch_start.p, ch_start.data(), nch * 8ull, cudaMemcpyHostToDevice, st));
    BM_CUDA(cudaMemcpyAsync(d_rlog.p, rlog.data(), n * 4ull, cudaMemcpyHostToDevice, st));
    BM_CUDA(cudaMemcpyAsync(d_base.p, base.data(), n * 8ull, cudaMemcpyHostToDevice, st));
    ItemView v{d_offsets, d_tids, d_base.p, d_rlog.p, d_ch_item.p, d_ch_start.p};

    // ---- validation ----
    if (P.validate) {
        DevBuf<int> d_err(1);
        DevBuf<uint32_t> d_bits(d_perm ? 3ull * ((m + 31) / 32) : 0);
        BM_CUDA(cudaMemsetAsync(d_err.p, 0, sizeof(int), st));
        if (d_perm) BM_CUDA(cudaMemsetAsync(d_bits.p, 0, d_bits.bytes(), st));
        k_validate_tids<<<nch, TPB, 0, st>>>(v, m, d_err.p);
        BM_CHECK_LAUNCH();
        if (d_perm) {  // computed permutations are bijections by construction
            k_validate_perm<<<grid_for(3ull * m), 256, 0, st>>>(d_perm, m, 3, d_bits.p, d_err.p);
            BM_CHECK_LAUNCH();
        }
        int err = 0;
        BM_CUDA(cudaMemcpyAsync(&err, d_err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        BM_CUDA(cudaStreamSynchronize(st));
        BM_REQUIRE(err != 1, BATMAP_ERR_ARG, "tids must be strictly increasing per item and < m");
        BM_REQUIRE(err != 2, BATMAP_ERR_ARG, "each permutation row must be a bijection of [0, m)");
    }

    // ---- place + finalize ----
    {
        DevBuf<uint32_t> &table = scratch_table(S->bytes);
        BM_CUDA(cudaMemsetAsync(table.p, 0xFF, S->bytes * sizeof(uint32_t), st));
        const uint32_t max_moves = 3u * std::max<uint32_t>(P.max_loop, 1u);
        E.record(2, st);
        k_place<<<2u * nch, TPB, 0, st>>>(v, PV, S->shift, max_moves, table.p);
        BM_CHECK_LAUNCH();
        E.record(3, st);
        // failed insertions, ordered by (item, tid): counted by finalize, listed below
        DevBuf<uint64_t> bs(nch + 1), d_tot(1);
        k_finalize<<<nch, TPB, 0, st>>>(v, PV, S->shift, table.p, S->d_bm.p, bs.p);
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
            k_failures<true><<<nch, TPB, 0, st>>>(v, PV, S->shift, table.p, bs.p, f_item.p,
                                                  S->d_fail_tid.p);
            BM_CHECK_LAUNCH();
        }
        k_fail_offsets<<<(n + 1 + 255) / 256, 256, 0, st>>>(f_item.p, nfail, n, S->d_fail_off.p);
        BM_CHECK_LAUNCH();

        // ---- correction entries ----
        S->n_corr = 0;
        if (nfail) {
            const uint64_t nwords = (m + 31) / 32;
            DevBuf<uint32_t> bits(nwords);
            DevBuf<uint64_t> wrank(nwords + 1), d_nu(1);
            BM_CUDA(cudaMemsetAsync(bits.p, 0, bits.bytes(), st));
            k_mark_failed<<<grid_for(nfail), 256, 0, st>>>(S->d_fail_tid.p, nfail, bits.p);
            BM_CHECK_LAUNCH();
            k_popc_words<<<grid_for(nwords), 256, 0, st>>>(bits.p, nwords, wrank.p);
            BM_CHECK_LAUNCH();
            scan_exclusive(wrank.p, nwords, d_nu.p, st);
            uint64_t nu = 0;
            BM_CUDA(cudaMemcpyAsync(&nu, d_nu.p, 8, cudaMemcpyDeviceToHost, st));
            BM_CUDA(cudaStreamSynchronize(st));
            DevBuf<uint64_t> fptr(nu + 1), cursor(nu + 1), d_sum(1);
            DevBuf<uint32_t> fitems(nfail);
            BM_CUDA(cudaMemsetAsync(fptr.p, 0, fptr.bytes(), st));
            BM_CUDA(cudaMemsetAsync(cursor.p, 0, cursor.bytes(), st));
            k_count_per_tid<<<grid_for(nfail), 256, 0, st>>>(S->d_fail_tid.p, nfail, bits.p, wrank.p, fptr.p);
            BM_CHECK_LAUNCH();
            k_scan_single_block<<<1, SCAN_TPB, 0, st>>>(fptr.p, nu, d_sum.p, 1);
            BM_CHECK_LAUNCH();
            k_fill_per_tid<<<grid_for(nfail), 256, 0, st>>>(f_item.p, S->d_fail_tid.p, nfail, bits.p,
                                                           wrank.p, fptr.p,
                                                           (unsigned long long *)cursor.p, fitems.p);
            BM_CHECK_LAUNCH();
            DevBuf<unsigned long long> counter(1);
            BM_CUDA(cudaMemsetAsync(counter.p, 0, 8, st));
            k_corrections<false><<<nch, TPB, 0, st>>>(v, m, bits.p, wrank.p, fptr.p, fitems.p, counter.p,
                                                       nullptr);
            BM_CHECK_LAUNCH();
            unsigned long long ncorr = 0;
            BM_CUDA(cudaMemcpyAsync(&ncorr, counter.p, 8, cudaMemcpyDeviceToHost, st));
            BM_CUDA(cudaStreamSynchronize(st));
            S->n_corr = ncorr;
            if (ncorr) {
                S->d_corr.alloc(2 * ncorr);
                BM_CUDA(cudaMemsetAsync(counter.p, 0, 8, st));
                k_corrections<true><<<nch, TPB, 0, st>>>(v, m, bits.p, wrank.p, fptr.p, fitems.p,
                                                          counter.p, S->d_corr.p);
                BM_CHECK_LAUNCH();
            }
        }
    }

    E.record(4, st);
    if (!S->skip_schedule) build_schedule(S);
    E.record(1, st);
    BM_CUDA(cudaStreamSynchronize(st));
    S->timing.build_ms = E.ms(0, 1);
    S->timing.place_ms = E.ms(2, 3);
    S->timing.finalize_ms = E.ms(3, 4);
}

}  // namespace bm
