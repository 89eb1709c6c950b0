// Serving: a device-resident pool of sets answering intersection-size and
// conjunctive queries (Sec. I: a conjunctive query is a set intersection),
// with a continuous-batching request loop.
//
// Pool storage.  Every set keeps its sorted tidlist.  Sets for which the 8-bit
// BatMap is compact (|S| >= r_0 / c, Sec. III-A: compression pays only when
// the set is dense enough) also get a BatMap, built by the same GPU build as
// pair mining.  A query |S_a1 cap ... cap S_ak| enumerates the smallest set
// and counts the elements present in every other set (the k-way counting idea
// of Sec. V): membership in a BatMap is two byte probes -- x is stored in two
// of the three tables, so tables 1 and 2 always hold at least one copy -- plus
// a binary search of the set's failed insertions; a set without a BatMap is
// searched in two levels: a sampled index of every IDX_STRIDE-th tid of each
// set (1/64 of the tidlists, small enough that its upper levels stay in L2)
// narrows the search to one block of IDX_STRIDE tids (256 contiguous bytes),
// so a membership test takes about two dependent DRAM reads instead of one per
// level of a binary search over the whole tidlist.
//
// Work is cut into tasks of up to 1024 elements of the smallest set; one warp
// runs a task and adds its count with one atomic.
#include <algorithm>
#include <chrono>
#include <memory>
#include <cstring>
#include <thread>

#include "common.cuh"
#include "perm.cuh"
#include "scan.cuh"

namespace bm {

void build_set(batmap_set *S, const uint64_t *d_offsets, const uint32_t *d_tids, const uint32_t *d_perm);

constexpr uint32_t TASK_ELEMS = 1024;
constexpr uint32_t MAX_K = 8;
constexpr uint32_t IDX_STRIDE = 64;  // tids per block of the sampled index

struct QueryDesc {
    uint32_t k;
    uint32_t ids[MAX_K];  // smallest set first
};
struct ProbeTask {
    uint32_t q;      // query index within the batch
    uint32_t begin;  // element range of the smallest set
    uint32_t end;
};

struct PoolView {
    const uint64_t *off;      // [n+1] CSR of all sets
    const uint32_t *tids;
    PermView perm;            // pi_0 .. pi_2 (the caller's table or computed)
    const int32_t *bm_index;  // [n] index among BatMap-backed sets or -1
    const uint64_t *bm_base;  // [nb] byte offset of the BatMap
    const uint32_t *bm_rlog;  // [nb] log2 r
    const uint64_t *f_off;    // [nb+1] failed insertions per BatMap-backed set
    const uint32_t *f_tid;
    const uint8_t *bm;        // BatMap bytes
    uint32_t m, shift;
    const uint64_t *idx_off;  // [n+1] sampled index: ceil(|S_c| / IDX_STRIDE) entries per set
    const uint32_t *idx;      // entry j of set c = tid IDX_STRIDE * j of set c
};

__device__ __forceinline__ bool bsearch_u32(const uint32_t *a, uint64_t lo, uint64_t hi, uint32_t x) {
    while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        const uint32_t v = a[mid];
        if (v == x) return true;
        if (v < x) lo = mid + 1; else hi = mid;
    }
    return false;
}

// x in set c's sorted tidlist: the last index entry <= x names the block of
// IDX_STRIDE tids that can hold x; that block is binary-searched.
__device__ __forceinline__ bool tidlist_member(const PoolView &P, uint32_t c, uint32_t x) {
    const uint64_t i0 = P.idx_off[c];
    uint64_t lo = i0, hi = P.idx_off[c + 1];
    while (lo < hi) {  // first entry > x
        const uint64_t mid = (lo + hi) >> 1;
        const uint32_t v = P.idx[mid];
        if (v == x) return true;
        if (v < x) lo = mid + 1; else hi = mid;
    }
    if (lo == i0) return false;  // x below the set's first tid
    const uint64_t s0 = P.off[c], first = s0 + (uint64_t)IDX_STRIDE * (lo - 1 - i0);
    const uint64_t end = min(P.off[c + 1], first + IDX_STRIDE);
    return bsearch_u32(P.tids, first + 1, end, x);  // the block's first tid is the entry, != x
}

__device__ __forceinline__ bool member(const PoolView &P, uint32_t c, uint32_t x) {
    const int32_t b = P.bm_index[c];
    if (b < 0) return tidlist_member(P, c, x);
    const uint64_t base = P.bm_base[b];
    const uint32_t r = 1u << P.bm_rlog[b];
#pragma unroll
    for (uint32_t t = 0; t < 2; t++) {
        const uint32_t pi = P.perm(t, x);
        const uint8_t byte = P.bm[base + slot_of(t, pi, r, P.shift)];
        if ((uint32_t)(byte & 0x7F) == (pi >> P.shift) + 1u) return true;
    }
    return bsearch_u32(P.f_tid, P.f_off[b], P.f_off[b + 1], x);
}

__global__ void k_probe(PoolView P, const QueryDesc *__restrict__ qs, const ProbeTask *__restrict__ tasks,
                        uint32_t ntasks, unsigned long long *__restrict__ counts) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < ntasks; w += warps) {
        const ProbeTask tk = tasks[w];
        const QueryDesc &Q = qs[tk.q];
        const uint32_t a = Q.ids[0];
        const uint64_t a0 = P.off[a];
        uint32_t cnt = 0;
        for (uint32_t i = tk.begin + lane; i < tk.end; i += 32) {
            const uint32_t x = P.tids[a0 + i];
            bool in_all = true;
            for (uint32_t t = 1; t < Q.k && in_all; t++) in_all = member(P, Q.ids[t], x);
            cnt += in_all ? 1u : 0u;
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, d);
        if (lane == 0 && cnt) atomicAdd(&counts[tk.q], (unsigned long long)cnt);
    }
}

// Materialised answers: the count pass stores one count per task; after an
// exclusive scan over tasks the write pass lists each task's matches in
// element order (a warp ballot ranks them), so every answer is ascending.
__global__ void k_probe_count(PoolView P, const QueryDesc *__restrict__ qs, const ProbeTask *__restrict__ tasks,
                              uint32_t ntasks, uint64_t *__restrict__ task_counts) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < ntasks; w += warps) {
        const ProbeTask tk = tasks[w];
        const QueryDesc &Q = qs[tk.q];
        const uint64_t a0 = P.off[Q.ids[0]];
        uint32_t cnt = 0;
        for (uint32_t i = tk.begin + lane; i < tk.end; i += 32) {
            const uint32_t x = P.tids[a0 + i];
            bool in_all = true;
            for (uint32_t t = 1; t < Q.k && in_all; t++) in_all = member(P, Q.ids[t], x);
            cnt += in_all ? 1u : 0u;
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, d);
        if (lane == 0) task_counts[w] = cnt;
    }
}

__global__ void k_probe_write(PoolView P, const QueryDesc *__restrict__ qs, const ProbeTask *__restrict__ tasks,
                              uint32_t ntasks, const uint64_t *__restrict__ task_off, uint32_t *__restrict__ out,
                              uint64_t cap) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < ntasks; w += warps) {
        const ProbeTask tk = tasks[w];
        const QueryDesc &Q = qs[tk.q];
        const uint64_t a0 = P.off[Q.ids[0]];
        uint64_t running = task_off[w];
        for (uint32_t base = tk.begin; base < tk.end; base += 32) {
            const uint32_t i = base + lane;
            bool in_all = false;
            uint32_t x = 0;
            if (i < tk.end) {
                x = P.tids[a0 + i];
                in_all = true;
                for (uint32_t t = 1; t < Q.k && in_all; t++) in_all = member(P, Q.ids[t], x);
            }
            const uint32_t mask = __ballot_sync(0xffffffffu, in_all);
            const uint64_t pos = running + __popc(mask & ((1u << lane) - 1u));
            if (in_all && pos < cap) out[pos] = x;
            running += __popc(mask);
        }
    }
}

__global__ void k_query_offsets(const uint64_t *__restrict__ task_off, const uint32_t *__restrict__ first_task,
                                uint32_t nq, uint64_t *__restrict__ out_off) {
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q <= nq) out_off[q] = task_off[first_task[q]];
}

// The sampled index: entry j of set c is tid IDX_STRIDE * j of set c.
__global__ void k_sample_index(const uint64_t *__restrict__ off, const uint32_t *__restrict__ tids, uint32_t n,
                               const uint64_t *__restrict__ idx_off, uint32_t *__restrict__ idx) {
    for (uint32_t c = blockIdx.x; c < n; c += gridDim.x) {
        const uint64_t b = off[c], k0 = idx_off[c], nk = idx_off[c + 1] - k0;
        for (uint64_t j = threadIdx.x; j < nk; j += blockDim.x) idx[k0 + j] = tids[b + (uint64_t)IDX_STRIDE * j];
    }
}

// One warp per set: every tid < m and strictly increasing within its set.
__global__ void k_validate_sets(const uint64_t *__restrict__ off, const uint32_t *__restrict__ tids, uint32_t n,
                                uint32_t m, int *err) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < n; c += warps) {
        const uint64_t b = off[c], e = off[c + 1];
        bool bad = e < b;
        for (uint64_t i = b + lane; i < e && !bad; i += 32) {
            const uint32_t x = tids[i];
            bad = x >= m || (i + 1 < e && !(x < tids[i + 1]));
        }
        if (bad) atomicExch(err, 1);
    }
}

}  // namespace bm

using namespace bm;

struct batmap_pool {
    uint32_t m = 0, n = 0;
    std::vector<uint64_t> h_off;
    DevBuf<uint64_t> d_off;
    DevBuf<uint32_t> d_tids, d_perm;
    DevBuf<int32_t> d_bm_index;
    DevBuf<uint64_t> d_bm_base, d_fail_off;
    DevBuf<uint32_t> d_bm_rlog, d_fail_tid;
    DevBuf<uint8_t> d_bm;
    DevBuf<uint64_t> d_idx_off;  // sampled index of the tidlists
    DevBuf<uint32_t> d_idx;
    uint32_t n_big = 0, shift = 0;
    uint64_t bm_bytes = 0, n_failed = 0;
    PoolView view{};
};

namespace bm {

static void pool_create(const batmap_params *p, uint32_t m, uint32_t n, const uint64_t *d_offsets,
                        const uint32_t *d_tids, const uint32_t *d_perm, cudaStream_t st, batmap_pool **out) {
    BM_REQUIRE(out, BATMAP_ERR_ARG, "out is NULL");
    BM_REQUIRE(m >= 1 && m <= (1u << 30), BATMAP_ERR_ARG, "m must be in [1, 2^30]");
    batmap_params P;
    batmap_default_params(&P);
    if (p) P = *p;
    auto pool = std::make_unique<batmap_pool>();
    pool->m = m;
    pool->n = n;
    pool->h_off.assign(n + 1, 0);
    if (n) {
        BM_REQUIRE(d_offsets, BATMAP_ERR_ARG, "d_offsets is NULL");
        BM_CUDA(cudaMemcpyAsync(pool->h_off.data(), d_offsets, (n + 1) * 8ull, cudaMemcpyDeviceToHost, st));
        BM_CUDA(cudaStreamSynchronize(st));
    }
    const uint64_t T = pool->h_off[n];
    pool->d_off.alloc(n + 1);
    pool->d_tids.alloc(T);
    if (d_perm) pool->d_perm.alloc(3ull * m);  // computed permutations need no table
    if (n) BM_CUDA(cudaMemcpyAsync(pool->d_off.p, d_offsets, (n + 1) * 8ull, cudaMemcpyDeviceToDevice, st));
    if (T) BM_CUDA(cudaMemcpyAsync(pool->d_tids.p, d_tids, T * 4ull, cudaMemcpyDeviceToDevice, st));
    if (d_perm) BM_CUDA(cudaMemcpyAsync(pool->d_perm.p, d_perm, 3ull * m * 4, cudaMemcpyDeviceToDevice, st));
    if (n) {
        DevBuf<int> err(1);
        BM_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), st));
        k_validate_sets<<<(unsigned)std::min<uint64_t>((n + 7) / 8, 65535), 256, 0, st>>>(pool->d_off.p,
                                                                                          pool->d_tids.p, n, m, err.p);
        BM_CHECK_LAUNCH();
        int h = 0;
        BM_CUDA(cudaMemcpyAsync(&h, err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        BM_CUDA(cudaStreamSynchronize(st));
        BM_REQUIRE(h == 0, BATMAP_ERR_ARG, "tids must be strictly increasing per set and < m");
    }

    // the sampled index of every tidlist (all sets: BatMap-backed ones keep it too)
    {
        std::vector<uint64_t> ioff(n + 1, 0);
        for (uint32_t i = 0; i < n; i++)
            ioff[i + 1] = ioff[i] + (pool->h_off[i + 1] - pool->h_off[i] + IDX_STRIDE - 1) / IDX_STRIDE;
        pool->d_idx_off.alloc(n + 1);
        pool->d_idx.alloc(std::max<uint64_t>(ioff[n], 1));
        BM_CUDA(cudaMemcpyAsync(pool->d_idx_off.p, ioff.data(), (n + 1) * 8ull, cudaMemcpyHostToDevice, st));
        if (ioff[n]) {
            k_sample_index<<<(unsigned)std::min<uint32_t>(std::max<uint32_t>(n, 1), 65535), 256, 0, st>>>(
                pool->d_off.p, pool->d_tids.p, n, pool->d_idx_off.p, pool->d_idx.p);
            BM_CHECK_LAUNCH();
        }
    }

    // sets whose 8-bit BatMap is compact: c |S| >= r_0
    uint32_t shift = P.min_shift;
    while ((uint64_t)m > 127ull << shift) shift++;
    const uint64_t r0 = 1ull << shift;
    std::vector<int32_t> bm_index(n, -1);
    std::vector<uint32_t> big_ids;
    std::vector<uint64_t> sub_off(1, 0);
    for (uint32_t i = 0; i < n; i++) {
        const uint64_t sz = pool->h_off[i + 1] - pool->h_off[i];
        if (sz && (uint64_t)P.load_num * sz >= r0 * P.load_den) {
            bm_index[i] = (int32_t)big_ids.size();
            big_ids.push_back(i);
            sub_off.push_back(sub_off.back() + sz);
        }
    }
    const uint32_t nb = (uint32_t)big_ids.size();
    pool->n_big = nb;
    pool->d_bm_index.alloc(std::max<uint32_t>(n, 1));
    if (n) BM_CUDA(cudaMemcpyAsync(pool->d_bm_index.p, bm_index.data(), n * 4ull, cudaMemcpyHostToDevice, st));
    std::vector<uint64_t> base(nb);
    std::vector<uint32_t> rlog(nb);
    std::vector<uint64_t> f_off(nb + 1, 0);
    if (nb) {
        // BatMap bytes of every big set (same sizing rule as the build)
        uint64_t total_bytes = 0;
        std::vector<uint64_t> bytes_of(nb);
        for (uint32_t b = 0; b < nb; b++) {
            const uint64_t sz = sub_off[b + 1] - sub_off[b];
            const uint64_t need = (P.load_num * sz + P.load_den - 1) / P.load_den;
            uint64_t r = 1;
            while (r < need) r <<= 1;
            bytes_of[b] = 3 * std::max<uint64_t>(r, r0);
            total_bytes += bytes_of[b];
        }
        pool->d_bm.alloc(total_bytes);
        std::vector<uint32_t> f_chunks_tid;
        uint64_t bm_pos = 0, f_pos = 0;
        // build in chunks of at most ~4 GB of BatMaps so the placement scratch
        // (4 bytes per slot) stays bounded
        for (uint32_t c0 = 0; c0 < nb;) {
            uint32_t c1 = c0;
            uint64_t cb = 0;
            while (c1 < nb && (c1 == c0 || cb + bytes_of[c1] <= (4ull << 30))) cb += bytes_of[c1++];
            const uint32_t cn = c1 - c0;
            std::vector<uint64_t> coff(cn + 1, 0);
            for (uint32_t j = 0; j < cn; j++) coff[j + 1] = coff[j] + (sub_off[c0 + j + 1] - sub_off[c0 + j]);
            DevBuf<uint64_t> s_off(cn + 1);
            DevBuf<uint32_t> s_tids(coff[cn]);
            BM_CUDA(cudaMemcpyAsync(s_off.p, coff.data(), (cn + 1) * 8ull, cudaMemcpyHostToDevice, st));
            for (uint32_t j = 0; j < cn; j++) {
                const uint32_t i = big_ids[c0 + j];
                BM_CUDA(cudaMemcpyAsync(s_tids.p + coff[j], d_tids + pool->h_off[i], (coff[j + 1] - coff[j]) * 4ull,
                                        cudaMemcpyDeviceToDevice, st));
            }
            batmap_set S;
            S.params = P;
            S.params.tile = 0;
            S.m = m;
            S.n = cn;
            S.stream = st;
            S.skip_schedule = true;
            build_set(&S, s_off.p, s_tids.p, d_perm ? pool->d_perm.p : nullptr);
            pool->shift = S.shift;
            BM_CUDA(cudaMemcpyAsync(pool->d_bm.p + bm_pos, S.d_bm.p, S.bytes, cudaMemcpyDeviceToDevice, st));
            std::vector<uint64_t> cf(cn + 1, 0);
            BM_CUDA(cudaMemcpyAsync(cf.data(), S.d_fail_off.p, (cn + 1) * 8ull, cudaMemcpyDeviceToHost, st));
            BM_CUDA(cudaStreamSynchronize(st));
            if (S.n_failed) {
                std::vector<uint32_t> ft(S.n_failed);
                BM_CUDA(cudaMemcpy(ft.data(), S.d_fail_tid.p, S.n_failed * 4ull, cudaMemcpyDeviceToHost));
                f_chunks_tid.insert(f_chunks_tid.end(), ft.begin(), ft.end());
            }
            for (uint32_t j = 0; j < cn; j++) {
                base[c0 + j] = bm_pos + S.byte_off[S.rank[j]];
                uint32_t lg = 0;
                while ((1u << lg) < S.range[j]) lg++;
                rlog[c0 + j] = lg;
                f_off[c0 + j + 1] = f_pos + cf[j + 1];
            }
            f_pos += S.n_failed;
            bm_pos += S.bytes;
            pool->n_failed += S.n_failed;
            c0 = c1;
        }
        pool->bm_bytes = bm_pos;
        pool->d_fail_tid.alloc(std::max<uint64_t>(f_chunks_tid.size(), 1));
        if (!f_chunks_tid.empty())
            BM_CUDA(cudaMemcpyAsync(pool->d_fail_tid.p, f_chunks_tid.data(), f_chunks_tid.size() * 4ull,
                                    cudaMemcpyHostToDevice, st));
        BM_CUDA(cudaStreamSynchronize(st));
    }
    pool->d_fail_off.alloc(nb + 1);
    BM_CUDA(cudaMemcpyAsync(pool->d_fail_off.p, f_off.data(), (nb + 1) * 8ull, cudaMemcpyHostToDevice, st));
    pool->d_bm_base.alloc(std::max<uint32_t>(nb, 1));
    pool->d_bm_rlog.alloc(std::max<uint32_t>(nb, 1));
    if (nb) {
        BM_CUDA(cudaMemcpyAsync(pool->d_bm_base.p, base.data(), nb * 8ull, cudaMemcpyHostToDevice, st));
        BM_CUDA(cudaMemcpyAsync(pool->d_bm_rlog.p, rlog.data(), nb * 4ull, cudaMemcpyHostToDevice, st));
    }
    pool->view = PoolView{pool->d_off.p,     pool->d_tids.p,     make_perm_view(d_perm ? pool->d_perm.p : nullptr, m, P.perm_seed),
                          pool->d_bm_index.p, pool->d_bm_base.p, pool->d_bm_rlog.p,
                          pool->d_fail_off.p, pool->d_fail_tid.p, pool->d_bm.p,
                          m,                  nb ? pool->shift : shift,
                          pool->d_idx_off.p,  pool->d_idx.p};
    BM_CUDA(cudaStreamSynchronize(st));
    *out = pool.release();
}

// Host-side preparation of one batch: descriptors with the smallest set first,
// and the element tasks.  Returns the number of tasks.
static uint64_t prepare_batch(const batmap_pool *pool, const uint32_t *qoff, const uint32_t *ids, uint64_t q0,
                              uint64_t q1, std::vector<QueryDesc> *qs, std::vector<ProbeTask> *tasks) {
    qs->resize(q1 - q0);
    tasks->clear();
    for (uint64_t q = q0; q < q1; q++) {
        const uint32_t k = qoff[q + 1] - qoff[q];
        BM_REQUIRE(k >= 1 && k <= MAX_K, BATMAP_ERR_ARG, "each query names 1..8 sets");
        QueryDesc &d = (*qs)[q - q0];
        d.k = k;
        for (uint32_t t = 0; t < k; t++) {
            const uint32_t c = ids[qoff[q] + t];
            BM_REQUIRE(c < pool->n, BATMAP_ERR_ARG, "query names a set id >= n");
            d.ids[t] = c;
        }
        std::sort(d.ids, d.ids + k, [&](uint32_t a, uint32_t b) {
            const uint64_t sa = pool->h_off[a + 1] - pool->h_off[a], sb = pool->h_off[b + 1] - pool->h_off[b];
            return sa < sb || (sa == sb && a < b);
        });
        const uint32_t small = (uint32_t)(pool->h_off[d.ids[0] + 1] - pool->h_off[d.ids[0]]);
        for (uint32_t b = 0; b < small; b += TASK_ELEMS)
            tasks->push_back({(uint32_t)(q - q0), b, std::min(small, b + TASK_ELEMS)});
    }
    return tasks->size();
}

static uint64_t query_work(const batmap_pool *pool, const uint32_t *qoff, const uint32_t *ids, uint64_t q) {
    uint64_t small = UINT64_MAX;
    for (uint32_t t = qoff[q]; t < qoff[q + 1]; t++) {
        const uint32_t c = ids[t];
        if (c < pool->n) small = std::min<uint64_t>(small, pool->h_off[c + 1] - pool->h_off[c]);
    }
    return (small == UINT64_MAX ? 0 : small) * (qoff[q + 1] - qoff[q]) + 1;
}

// Answers as element lists: out_off[q] .. out_off[q+1] in out (ascending).
static void intersect_list(const batmap_pool *pool, const uint32_t *qoff, const uint32_t *ids, uint32_t nq,
                           uint64_t *d_out_off, uint32_t *d_out, uint64_t cap, uint64_t *n_total, cudaStream_t st) {
    BM_REQUIRE(pool && qoff && n_total && d_out_off, BATMAP_ERR_ARG, "NULL argument");
    BM_REQUIRE(cap == 0 || d_out, BATMAP_ERR_ARG, "d_out is NULL with cap > 0");
    std::vector<QueryDesc> qs;
    std::vector<ProbeTask> tasks;
    if (nq) prepare_batch(pool, qoff, ids, 0, nq, &qs, &tasks);
    const uint64_t nt = tasks.size();
    std::vector<uint32_t> first(nq + 1, (uint32_t)nt);
    for (uint64_t t = nt; t-- > 0;) first[tasks[t].q] = (uint32_t)t;
    for (uint32_t q = nq; q-- > 0;) first[q] = std::min(first[q], first[q + 1]);
    DevBuf<QueryDesc> d_q(std::max<uint64_t>(qs.size(), 1));
    DevBuf<ProbeTask> d_t(std::max<uint64_t>(nt, 1));
    DevBuf<uint64_t> d_toff(nt + 1), d_total(1);
    DevBuf<uint32_t> d_first(nq + 1);
    if (nq) BM_CUDA(cudaMemcpyAsync(d_q.p, qs.data(), qs.size() * sizeof(QueryDesc), cudaMemcpyHostToDevice, st));
    if (nt) BM_CUDA(cudaMemcpyAsync(d_t.p, tasks.data(), nt * sizeof(ProbeTask), cudaMemcpyHostToDevice, st));
    BM_CUDA(cudaMemcpyAsync(d_first.p, first.data(), (nq + 1) * 4ull, cudaMemcpyHostToDevice, st));
    const unsigned blocks = (unsigned)std::min<uint64_t>((nt + 7) / 8, 4096);
    if (nt) {
        k_probe_count<<<blocks, 256, 0, st>>>(pool->view, d_q.p, d_t.p, (uint32_t)nt, d_toff.p);
        BM_CHECK_LAUNCH();
    }
    k_scan_single_block<<<1, SCAN_TPB, 0, st>>>(d_toff.p, nt, d_total.p, 1);
    BM_CHECK_LAUNCH();
    k_query_offsets<<<(nq + 1 + 255) / 256, 256, 0, st>>>(d_toff.p, d_first.p, nq, d_out_off);
    BM_CHECK_LAUNCH();
    if (nt && cap) {
        k_probe_write<<<blocks, 256, 0, st>>>(pool->view, d_q.p, d_t.p, (uint32_t)nt, d_toff.p, d_out, cap);
        BM_CHECK_LAUNCH();
    }
    uint64_t total = 0;
    BM_CUDA(cudaMemcpyAsync(&total, d_total.p, 8, cudaMemcpyDeviceToHost, st));
    BM_CUDA(cudaStreamSynchronize(st));
    *n_total = total;
    if (total > cap)
        throw Error{BATMAP_ERR_CAPACITY, "d_out too small: " + std::to_string(total) + " elements in the answers"};
}

// Staging for one in-flight batch (pinned host + device, fixed capacity).
struct Slot {
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr;
    QueryDesc *h_q = nullptr;
    ProbeTask *h_t = nullptr;
    DevBuf<QueryDesc> d_q;
    DevBuf<ProbeTask> d_t;
    uint64_t qcap = 0, tcap = 0;
    uint64_t q0 = 0, q1 = 0, work = 0;
    bool busy = false;
    void init(uint64_t qc, uint64_t tc, bool own_stream, cudaStream_t shared) {
        qcap = qc;
        tcap = tc;
        if (own_stream) {
            BM_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        } else {
            st = shared;
        }
        BM_CUDA(cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
        BM_CUDA(cudaMallocHost(&h_q, qc * sizeof(QueryDesc)));
        BM_CUDA(cudaMallocHost(&h_t, tc * sizeof(ProbeTask)));
        d_q.alloc(qc);
        d_t.alloc(tc);
    }
    void destroy(bool own_stream) {
        if (done) cudaEventDestroy(done);
        if (own_stream && st) cudaStreamDestroy(st);
        if (h_q) cudaFreeHost(h_q);
        if (h_t) cudaFreeHost(h_t);
        done = nullptr;
        st = nullptr;
        h_q = nullptr;
        h_t = nullptr;
    }
};

static void launch_batch(const batmap_pool *pool, Slot &S, const std::vector<QueryDesc> &qs,
                         const std::vector<ProbeTask> &tasks, unsigned long long *d_counts) {
    std::memcpy(S.h_q, qs.data(), qs.size() * sizeof(QueryDesc));
    if (!tasks.empty()) std::memcpy(S.h_t, tasks.data(), tasks.size() * sizeof(ProbeTask));
    BM_CUDA(cudaMemcpyAsync(S.d_q.p, S.h_q, qs.size() * sizeof(QueryDesc), cudaMemcpyHostToDevice, S.st));
    if (!tasks.empty())
        BM_CUDA(cudaMemcpyAsync(S.d_t.p, S.h_t, tasks.size() * sizeof(ProbeTask), cudaMemcpyHostToDevice, S.st));
    BM_CUDA(cudaMemsetAsync(d_counts + S.q0, 0, (S.q1 - S.q0) * sizeof(unsigned long long), S.st));
    if (!tasks.empty()) {
        const uint32_t warps_per_block = 8;
        const uint64_t blocks = std::min<uint64_t>((tasks.size() + warps_per_block - 1) / warps_per_block, 4096);
        k_probe<<<(unsigned)blocks, 32 * warps_per_block, 0, S.st>>>(pool->view, S.d_q.p, S.d_t.p,
                                                                      (uint32_t)tasks.size(), d_counts + S.q0);
        BM_CHECK_LAUNCH();
    }
    BM_CUDA(cudaEventRecord(S.done, S.st));
}

static void intersect(const batmap_pool *pool, const uint32_t *qoff, const uint32_t *ids, uint32_t nq,
                      unsigned long long *d_counts, cudaStream_t st) {
    BM_REQUIRE(pool && qoff && (nq == 0 || ids) && (nq == 0 || d_counts), BATMAP_ERR_ARG, "NULL argument");
    if (!nq) return;
    std::vector<QueryDesc> qs;
    std::vector<ProbeTask> tasks;
    prepare_batch(pool, qoff, ids, 0, nq, &qs, &tasks);
    Slot S;
    S.init(nq, std::max<uint64_t>(tasks.size(), 1), false, st);
    S.q0 = 0;
    S.q1 = nq;
    try {
        launch_batch(pool, S, qs, tasks, d_counts);
        BM_CUDA(cudaStreamSynchronize(st));
    } catch (...) {
        cudaStreamSynchronize(st);
        S.destroy(false);
        throw;
    }
    S.destroy(false);
}

// The continuous-batching request loop.  Queries arrive at h_arrival[q]
// seconds after the start (non-decreasing).  Whenever a slot is free, the
// loop gathers the queries that have arrived and not been submitted, up to
// max_batch queries and while the work in flight stays within the budget
// (work = elements of the smallest set x sets named), copies their
// descriptors to the slot's device buffers and launches them on the slot's
// stream; batches on different slots overlap on the device.  A query's
// latency is the host time at which its batch's completion event was
// observed minus its arrival time.
static void serve(const batmap_pool *pool, const uint32_t *qoff, const uint32_t *ids, const double *arrival,
                  uint32_t nq, const batmap_serve_opts *o, uint64_t *h_counts, double *h_latency,
                  batmap_serve_stats *stats, cudaStream_t st) {
    BM_REQUIRE(pool && qoff && arrival && h_counts && h_latency, BATMAP_ERR_ARG, "NULL argument");
    batmap_serve_opts opt{64, 4, 1ull << 26, 0};
    if (o) opt = *o;
    BM_REQUIRE(opt.max_batch >= 1 && opt.slots >= 1 && opt.slots <= 64, BATMAP_ERR_ARG, "bad serve options");
    for (uint32_t q = 1; q < nq; q++)
        BM_REQUIRE(arrival[q] >= arrival[q - 1], BATMAP_ERR_ARG, "arrival times must be non-decreasing");
    std::vector<uint64_t> work(nq);
    uint64_t max_tasks = 1, max_work = 1;
    for (uint32_t q = 0; q < nq; q++) {
        work[q] = query_work(pool, qoff, ids, q);
        max_work = std::max(max_work, work[q]);
    }
    // task capacity of a slot: the largest batch the budget admits
    for (uint32_t q = 0; q < nq; q++) {
        uint64_t small = work[q] / std::max<uint32_t>(1, qoff[q + 1] - qoff[q]);
        max_tasks = std::max<uint64_t>(max_tasks, small / TASK_ELEMS + 1);
    }
    const uint64_t budget = std::max<uint64_t>(opt.work_budget, max_work);
    const uint64_t tcap = std::max<uint64_t>(max_tasks * 2, budget / TASK_ELEMS + (uint64_t)opt.max_batch);
    DevBuf<unsigned long long> d_counts(std::max<uint32_t>(nq, 1));
    std::vector<Slot> slots(opt.slots);
    for (auto &s : slots) s.init(opt.max_batch, tcap, true, st);
    std::vector<QueryDesc> qs;
    std::vector<ProbeTask> tasks;
    using clk = std::chrono::steady_clock;
    const auto t0 = clk::now();
    auto now_s = [&] { return std::chrono::duration<double>(clk::now() - t0).count(); };
    uint64_t next = 0, done = 0, inflight_work = 0, batches = 0, max_inflight = 0, inflight = 0;
    try {
        while (done < nq) {
            const double t = now_s();
            bool progressed = false;
            for (auto &s : slots) {
                if (!s.busy) continue;
                cudaError_t e = cudaEventQuery(s.done);
                if (e == cudaErrorNotReady) continue;
                BM_CUDA(e);
                const double tc = now_s();
                for (uint64_t q = s.q0; q < s.q1; q++) h_latency[q] = tc - arrival[q];
                done += s.q1 - s.q0;
                inflight_work -= s.work;
                inflight--;
                s.busy = false;
                progressed = true;
            }
            for (auto &s : slots) {
                if (s.busy || next >= nq || arrival[next] > t) continue;
                uint64_t q1 = next, w = 0;
                while (q1 < nq && arrival[q1] <= t && q1 - next < opt.max_batch &&
                       (q1 == next ? inflight_work + work[q1] <= budget || inflight == 0
                                   : inflight_work + w + work[q1] <= budget))
                    w += work[q1++];
                if (q1 == next) break;  // budget full: wait for completions
                prepare_batch(pool, qoff, ids, next, q1, &qs, &tasks);
                if (tasks.size() > s.tcap) {  // admit fewer queries
                    q1 = next + 1;
                    prepare_batch(pool, qoff, ids, next, q1, &qs, &tasks);
                    BM_REQUIRE(tasks.size() <= s.tcap, BATMAP_ERR_INTERNAL, "task capacity");
                    w = work[next];
                }
                s.q0 = next;
                s.q1 = q1;
                s.work = w;
                launch_batch(pool, s, qs, tasks, d_counts.p);
                s.busy = true;
                inflight++;
                inflight_work += w;
                max_inflight = std::max(max_inflight, inflight);
                batches++;
                next = q1;
                progressed = true;
            }
            if (!progressed) {
                const double wait = next < nq ? arrival[next] - now_s() : 0.0;
                if (wait > 200e-6) std::this_thread::sleep_for(std::chrono::microseconds(50));
            }
        }
        const double makespan = now_s();
        if (nq) BM_CUDA(cudaMemcpy(h_counts, d_counts.p, nq * sizeof(uint64_t), cudaMemcpyDeviceToHost));
        if (stats) {
            std::memset(stats, 0, sizeof(*stats));
            stats->makespan_s = makespan;
            stats->batches = batches;
            stats->max_inflight = max_inflight;
            std::vector<double> lat(h_latency, h_latency + nq);
            std::sort(lat.begin(), lat.end());
            if (nq) {
                stats->p50_s = lat[(size_t)(0.50 * (nq - 1))];
                stats->p99_s = lat[(size_t)(0.99 * (nq - 1))];
                stats->max_s = lat.back();
                stats->queries_per_s = nq / std::max(makespan, 1e-9);
            }
        }
    } catch (...) {
        for (auto &s : slots) {
            if (s.st) cudaStreamSynchronize(s.st);
            s.destroy(true);
        }
        throw;
    }
    for (auto &s : slots) {
        cudaStreamSynchronize(s.st);
        s.destroy(true);
    }
}

}  // namespace bm

extern "C" {

#define BM_GUARD(body)                              \
    try {                                           \
        body;                                       \
        return BATMAP_OK;                           \
    } catch (const bm::Error &e) {                  \
        bm::set_error(e.msg);                       \
        return e.code;                              \
    } catch (...) {                                 \
        bm::set_error("unexpected internal error"); \
        return BATMAP_ERR_INTERNAL;                 \
    }

batmap_status batmap_pool_create(const batmap_params *p, uint32_t m, uint32_t n, const uint64_t *d_offsets,
                                 const uint32_t *d_tids, const uint32_t *d_perm, cudaStream_t stream,
                                 batmap_pool **out) {
    BM_GUARD(bm::pool_create(p, m, n, d_offsets, d_tids, d_perm, stream, out));
}

void batmap_pool_free(batmap_pool *pool) { delete pool; }

batmap_status batmap_pool_info(const batmap_pool *pool, uint32_t *n_batmaps, uint64_t *batmap_bytes,
                               uint64_t *n_elements) {
    BM_GUARD({
        BM_REQUIRE(pool, BATMAP_ERR_ARG, "NULL pool");
        if (n_batmaps) *n_batmaps = pool->n_big;
        if (batmap_bytes) *batmap_bytes = pool->bm_bytes;
        if (n_elements) *n_elements = pool->h_off[pool->n];
    });
}

batmap_status intersect_query(const batmap_pool *pool, const uint32_t *h_qoff, const uint32_t *h_ids,
                              uint32_t n_queries, uint64_t *d_counts, cudaStream_t stream) {
    BM_GUARD(bm::intersect(pool, h_qoff, h_ids, n_queries, reinterpret_cast<unsigned long long *>(d_counts),
                           stream));
}

batmap_status intersect_query_list(const batmap_pool *pool, const uint32_t *h_qoff, const uint32_t *h_ids,
                                   uint32_t n_queries, uint64_t *d_out_off, uint32_t *d_out, uint64_t cap,
                                   uint64_t *n_total, cudaStream_t stream) {
    BM_GUARD(bm::intersect_list(pool, h_qoff, h_ids, n_queries, d_out_off, d_out, cap, n_total, stream));
}

batmap_status batmap_serve(const batmap_pool *pool, const uint32_t *h_qoff, const uint32_t *h_ids,
                           const double *h_arrival_s, uint32_t n_queries, const batmap_serve_opts *opts,
                           uint64_t *h_counts, double *h_latency_s, batmap_serve_stats *stats, cudaStream_t stream) {
    BM_GUARD(bm::serve(pool, h_qoff, h_ids, h_arrival_s, n_queries, opts, h_counts, h_latency_s, stats, stream));
}

}  // extern "C"
