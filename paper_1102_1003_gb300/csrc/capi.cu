// The extern "C" boundary: argument checks, error translation, and the
// orchestration of build -> compare -> correct -> compact on one stream.
#include <atomic>
#include <mutex>
#include <cstring>
#include <new>
#include <string>

#include "common.cuh"
#include "compare.cuh"

namespace bm {

static thread_local std::string g_last_error;
static std::atomic<uint64_t> g_launches{0};

void set_error(const std::string &msg) { g_last_error = msg; }
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void build_set(batmap_set *S, const uint64_t *d_offsets, const uint32_t *d_tids, const uint32_t *d_perm);
void build_witness_set(batmap_set *S, const uint64_t *d_offsets, const uint32_t *d_tids, const uint32_t *d_perm);
void witness_support(batmap_set *S, uint32_t k, uint64_t nq, const uint32_t *d_items, uint32_t *d_support,
                     cudaStream_t st);
void frequent_triples(batmap_set *S, uint32_t s, const uint32_t *d_pairs, uint64_t np, uint32_t *d_out,
                      uint64_t cap, uint64_t *n_out, uint64_t *n_cand, cudaStream_t st);
void frequent_quadruples(batmap_set *S, uint32_t s, const uint32_t *d_triples, uint64_t nt, uint32_t *d_out,
                         uint64_t cap, uint64_t *n_out, uint64_t *n_cand, cudaStream_t st);
void enqueue_correct_compact(batmap_set *S, uint32_t *C, uint32_t s, uint32_t *d_pairs, uint64_t cap,
                             uint64_t *d_total, cudaStream_t st);
void run_batch(batmap_set *const *sets, const uint32_t *s, uint32_t k, batmap_out *outs, cudaStream_t st);
void autotune(batmap_set *const *sets, uint32_t k, double *eff_out, cudaStream_t st);
void release_scratch();
void release_dense_workspace();
void release_batch_plan();

static std::atomic<uint64_t> g_gen{1};

// Workspace of pair_support_host: device copies of the caller's host inputs and the pair
// output, grown as needed and released by batmap_release_scratch.
struct HostPathWork {
    DevBuf<uint64_t> off;
    DevBuf<uint32_t> tids, perm, pairs;
};
static std::mutex g_host_mu;
static HostPathWork g_host_work;

void release_host_workspace() {
    std::lock_guard<std::mutex> lock(g_host_mu);
    g_host_work.off.release();
    g_host_work.tids.release();
    g_host_work.perm.release();
    g_host_work.pairs.release();
}

template <typename F>
static batmap_status guarded(F &&f) {
    try {
        f();
        return BATMAP_OK;
    } catch (const Error &e) {
        set_error(e.msg);
        return e.code;
    } catch (const std::bad_alloc &) {
        set_error("host allocation failed");
        return BATMAP_ERR_NOMEM;
    } catch (...) {
        set_error("unexpected internal error");
        return BATMAP_ERR_INTERNAL;
    }
}

// Zero C, run every shape's persistent compare launch over the set's units.
void enqueue_compare(batmap_set *S, uint32_t *C, const InstView *d_view, cudaStream_t st) {
    const uint64_t npairs = S->npairs();
    if (npairs) BM_CUDA(cudaMemsetAsync(C, 0, npairs * sizeof(uint32_t), st));
    S->d_counters.ensure(COMPARE_COUNTERS);
    BM_CUDA(cudaMemsetAsync(S->d_counters.p, 0, COMPARE_COUNTERS * sizeof(uint32_t), st));
    S->pairs_ev.record(1, st);
    launch_compare(d_view, S->d_units.p, unit_parts(S->units), S->d_counters.p, st, nullptr, S->pairs_ev.ev[4]);
    S->pairs_ev.record(2, st);
}

}  // namespace bm

using namespace bm;

extern "C" {

void batmap_default_params(batmap_params *p) {
    if (!p) return;
    p->load_num = 2;
    p->load_den = 1;
    p->max_loop = 32;
    p->min_shift = 7;
    p->tile = 0;
    p->validate = 1;
    p->shape_mask = 0;
    p->probe_log = 0;
    p->perm_seed = 1;
}

const char *batmap_last_error(void) { return g_last_error.c_str(); }

static batmap_status build_any(const batmap_params *p, uint32_t m, uint32_t n, uint32_t n_a,
                               const uint64_t *d_offsets, const uint32_t *d_tids, const uint32_t *d_perm,
                               cudaStream_t stream, batmap_set **out, uint32_t d = 2) {
    return guarded([&] {
        BM_REQUIRE(out != nullptr, BATMAP_ERR_ARG, "out is NULL");
        *out = nullptr;
        batmap_params P;
        batmap_default_params(&P);
        if (p) P = *p;
        BM_REQUIRE(m >= 1 && m <= (1u << 30), BATMAP_ERR_ARG, "m must be in [1, 2^30]");
        BM_REQUIRE(P.load_num >= 1 && P.load_den >= 1 && P.load_num <= 16 * P.load_den,
                   BATMAP_ERR_ARG, "load factor must be in [1/load_den, 16]");
        BM_REQUIRE(P.min_shift >= 7 && P.min_shift <= 24, BATMAP_ERR_ARG, "min_shift must be in [7, 24]");
        BM_REQUIRE(P.tile <= NUM_SHAPES, BATMAP_ERR_ARG, "tile must be 0..BATMAP_NUM_SHAPES (18)");
        BM_REQUIRE(P.max_loop >= 1 && P.max_loop <= (1u << 20), BATMAP_ERR_ARG, "max_loop out of range");
        batmap_set *S = new batmap_set();
        S->params = P;
        S->m = m;
        S->n = n;
        S->stream = stream;
        S->n_a = n_a;
        S->d = d;
        S->gen = g_gen.fetch_add(1);
        try {
            if (d == 3 || d == 4) build_witness_set(S, d_offsets, d_tids, d_perm);
            else build_set(S, d_offsets, d_tids, d_perm);
        } catch (...) {
            delete S;
            throw;
        }
        *out = S;
    });
}

batmap_status batmap_build(const batmap_params *p, uint32_t m, uint32_t n, const uint64_t *d_offsets,
                           const uint32_t *d_tids, const uint32_t *d_perm, cudaStream_t stream,
                           batmap_set **out) {
    return build_any(p, m, n, 0, d_offsets, d_tids, d_perm, stream, out);
}

batmap_status batmap_build_cross(const batmap_params *p, uint32_t m, uint32_t n_a, uint32_t n_b,
                                 const uint64_t *d_offsets, const uint32_t *d_tids, const uint32_t *d_perm,
                                 cudaStream_t stream, batmap_set **out) {
    if (n_a == 0 || n_b == 0) {
        set_error("batmap_build_cross needs two non-empty families");
        return BATMAP_ERR_ARG;
    }
    if ((uint64_t)n_a + n_b > 0xFFFFFFFFull) {
        set_error("n_a + n_b exceeds 2^32 - 1");
        return BATMAP_ERR_ARG;
    }
    return build_any(p, m, n_a + n_b, n_a, d_offsets, d_tids, d_perm, stream, out);
}

batmap_status batmap_build_d(const batmap_params *p, uint32_t d, uint32_t m, uint32_t n,
                             const uint64_t *d_offsets, const uint32_t *d_tids, const uint32_t *d_perm,
                             cudaStream_t stream, batmap_set **out) {
    if (d < 2 || d > 4) {
        set_error("d must be 2, 3 or 4");
        return BATMAP_ERR_ARG;
    }
    return build_any(p, m, n, 0, d_offsets, d_tids, d_perm, stream, out, d);
}

batmap_status itemset_support(batmap_set *S, uint32_t k, uint64_t n_q, const uint32_t *d_items,
                              uint32_t *d_support, cudaStream_t st) {
    return guarded([&] { witness_support(S, k, n_q, d_items, d_support, st); });
}

batmap_status frequent_triples(batmap_set *S, uint32_t s, const uint32_t *d_pairs, uint64_t n_pairs,
                               uint32_t *d_out, uint64_t cap, uint64_t *n_out, uint64_t *n_candidates,
                               cudaStream_t st) {
    return guarded([&] { bm::frequent_triples(S, s, d_pairs, n_pairs, d_out, cap, n_out, n_candidates, st); });
}

batmap_status frequent_quadruples(batmap_set *S, uint32_t s, const uint32_t *d_triples, uint64_t n_triples,
                                  uint32_t *d_out, uint64_t cap, uint64_t *n_out, uint64_t *n_candidates,
                                  cudaStream_t st) {
    return guarded(
        [&] { bm::frequent_quadruples(S, s, d_triples, n_triples, d_out, cap, n_out, n_candidates, st); });
}

void batmap_free(batmap_set *set) {
    if (!set) return;
    cudaStreamSynchronize(set->stream);
    release_batch_plan();  // a cached batch graph may point into this set
    delete set;
}

batmap_status batmap_get_info(const batmap_set *S, batmap_info *info) {
    return guarded([&] {
        BM_REQUIRE(S && info, BATMAP_ERR_ARG, "NULL argument");
        std::memset(info, 0, sizeof(*info));
        info->m = S->m;
        info->n = S->n;
        info->shift = S->shift;
        info->r0 = S->r0;
        info->bytes = S->bytes;
        info->n_elements = S->n_elements;
        info->n_failed = S->n_failed;
        info->n_corrections = S->n_corr;
        info->n_work_units = S->units.size();
        info->n_classes = S->class_begin.empty() ? 0 : (uint32_t)S->class_begin.size() - 1;
        info->n_a = S->n_a;
        info->word_pairs = S->word_pairs;
        info->probe_word_pairs = S->probe_word_pairs;
        info->probe_words = S->probe_words;
        info->d = S->d;
    });
}

batmap_status batmap_export_layout(const batmap_set *S, uint8_t *h_bytes, uint64_t *h_byte_offset,
                                   uint32_t *h_range, uint64_t *h_fail_offsets, uint32_t *h_fail_tids) {
    return guarded([&] {
        BM_REQUIRE(S, BATMAP_ERR_ARG, "NULL set");
        cudaStream_t st = S->stream;
        if (h_bytes && S->bytes)
            BM_CUDA(cudaMemcpyAsync(h_bytes, S->d_bm.p, S->bytes, cudaMemcpyDeviceToHost, st));
        if (h_byte_offset)
            for (uint32_t i = 0; i < S->n; i++) h_byte_offset[i] = S->byte_off[S->rank[i]];
        if (h_range)
            for (uint32_t i = 0; i < S->n; i++) h_range[i] = S->range[i];
        if (h_fail_offsets)
            BM_CUDA(cudaMemcpyAsync(h_fail_offsets, S->d_fail_off.p, (S->n + 1) * sizeof(uint64_t),
                                    cudaMemcpyDeviceToHost, st));
        if (h_fail_tids && S->n_failed)
            BM_CUDA(cudaMemcpyAsync(h_fail_tids, S->d_fail_tid.p, S->n_failed * sizeof(uint32_t),
                                    cudaMemcpyDeviceToHost, st));
        BM_CUDA(cudaStreamSynchronize(st));
    });
}

static void pair_support_impl(batmap_set *S, uint32_t s, uint32_t *d_pairs, uint64_t cap,
                              uint64_t *n_out, uint32_t *d_full, cudaStream_t st) {
    BM_REQUIRE(S, BATMAP_ERR_ARG, "NULL set");
    BM_REQUIRE(S->d == 2, BATMAP_ERR_ARG, "pair calls need a 2-of-3 set (built with d = 2)");
    BM_REQUIRE(n_out, BATMAP_ERR_ARG, "n_out is NULL");
    BM_REQUIRE(cap == 0 || d_pairs, BATMAP_ERR_ARG, "d_pairs is NULL with cap > 0");
    const uint64_t npairs = S->npairs();
    uint32_t *C = d_full;
    if (!C) {
        S->d_C.ensure(npairs);
        C = S->d_C.p;
    }
    static thread_local InstView h_view;
    h_view = InstView{reinterpret_cast<const uint4 *>(S->d_bm.p), S->d_line_off.p, S->d_wshift.p,
                      S->d_order.p, C, S->n, S->n_a, S->shift};
    S->d_total.ensure(1);
    S->d_view.ensure(1);
    S->pairs_ev.create();
    S->pairs_ev.record(0, st);
    BM_CUDA(cudaMemcpyAsync(S->d_view.p, &h_view, sizeof(InstView), cudaMemcpyHostToDevice, st));
    enqueue_compare(S, C, S->d_view.p, st);  // records events 1, 2 around the launch
    enqueue_correct_compact(S, C, s, d_pairs, cap, S->d_total.p, st);
    S->pairs_ev.record(3, st);
    uint64_t total = 0;
    BM_CUDA(cudaMemcpyAsync(&total, S->d_total.p, 8, cudaMemcpyDeviceToHost, st));
    BM_CUDA(cudaStreamSynchronize(st));
    S->timing.compare_ms = S->pairs_ev.ms(1, 2);
    S->timing.scan_ms = S->pairs_ev.ms(1, 4);
    S->timing.probe_ms = S->pairs_ev.ms(4, 2);
    S->timing.compact_ms = S->pairs_ev.ms(2, 3);
    S->timing.pairs_ms = S->pairs_ev.ms(0, 3);
    *n_out = total;
    if (total > cap)
        throw Error{BATMAP_ERR_CAPACITY, "d_pairs too small: " + std::to_string(total) + " pairs qualify"};
}

batmap_status pair_support_all(batmap_set *S, uint32_t s, uint32_t *d_pairs, uint64_t cap, uint64_t *n_out,
                               uint32_t *d_full, cudaStream_t st) {
    return guarded([&] { pair_support_impl(S, s, d_pairs, cap, n_out, d_full, st); });
}

batmap_status pair_support_host(const batmap_params *p, uint32_t m, uint32_t n, const uint64_t *h_offsets,
                                const uint32_t *h_tids, const uint32_t *h_perm, uint32_t s, uint32_t *h_pairs,
                                uint64_t cap, uint64_t *n_out, cudaStream_t st) {
    return guarded([&] {
        BM_REQUIRE(h_offsets && n_out, BATMAP_ERR_ARG, "NULL argument");
        BM_REQUIRE(cap == 0 || h_pairs, BATMAP_ERR_ARG, "h_pairs is NULL with cap > 0");
        const uint64_t T = h_offsets[n];
        // device copies of the inputs and the output, kept for the next call (each call ends
        // with a stream synchronisation; calls are serialised on the workspace)
        std::lock_guard<std::mutex> lock(g_host_mu);
        HostPathWork &W = g_host_work;
        W.off.ensure(n + 1);
        W.tids.ensure(T);
        if (h_perm) W.perm.ensure(3ull * m);
        W.pairs.ensure(3 * cap);
        BM_CUDA(cudaMemcpyAsync(W.off.p, h_offsets, (n + 1) * 8ull, cudaMemcpyHostToDevice, st));
        if (T) BM_CUDA(cudaMemcpyAsync(W.tids.p, h_tids, T * 4ull, cudaMemcpyHostToDevice, st));
        if (h_perm) BM_CUDA(cudaMemcpyAsync(W.perm.p, h_perm, 3ull * m * 4, cudaMemcpyHostToDevice, st));
        batmap_set *S = nullptr;
        batmap_status rc = batmap_build(p, m, n, W.off.p, W.tids.p, h_perm ? W.perm.p : nullptr, st, &S);
        if (rc != BATMAP_OK) throw Error{rc, g_last_error};
        uint32_t *d_pairs = W.pairs.p;
        std::string msg;
        try {
            uint64_t total = 0;
            rc = pair_support_all(S, s, d_pairs, cap, &total, nullptr, st);
            msg = g_last_error;
            *n_out = total;
            if (rc != BATMAP_OK && rc != BATMAP_ERR_CAPACITY) throw Error{rc, msg};
            uint64_t ncopy = std::min<uint64_t>(total, cap);
            if (ncopy)
                BM_CUDA(cudaMemcpyAsync(h_pairs, d_pairs, ncopy * 12ull, cudaMemcpyDeviceToHost, st));
            BM_CUDA(cudaStreamSynchronize(st));
        } catch (...) {
            batmap_free(S);
            throw;
        }
        batmap_free(S);
        if (rc == BATMAP_ERR_CAPACITY) throw Error{rc, msg};
    });
}

batmap_status batmap_get_timing(const batmap_set *S, batmap_timing *t) {
    return guarded([&] {
        BM_REQUIRE(S && t, BATMAP_ERR_ARG, "NULL argument");
        *t = S->timing;
    });
}

uint64_t batmap_kernel_launches(void) { return g_launches.load(); }

void batmap_release_scratch(void) {
    release_scratch();
    release_dense_workspace();
    release_host_workspace();
}

static void require_pair_sets(batmap_set *const *sets, uint32_t k) {
    BM_REQUIRE(k == 0 || sets, BATMAP_ERR_ARG, "sets is NULL");
    for (uint32_t i = 0; i < k; i++)
        BM_REQUIRE(sets[i] && sets[i]->d == 2, BATMAP_ERR_ARG, "pair calls need 2-of-3 sets (built with d = 2)");
}

batmap_status batmap_autotune(batmap_set *const *sets, uint32_t k, double *shape_eff, cudaStream_t st) {
    return guarded([&] {
        require_pair_sets(sets, k);
        autotune(sets, k, shape_eff, st);
    });
}

batmap_status pair_support_batch(batmap_set *const *sets, const uint32_t *s, uint32_t k, batmap_out *outs,
                                 cudaStream_t st) {
    return guarded([&] {
        require_pair_sets(sets, k);
        run_batch(sets, s, k, outs, st);
    });
}

}  // extern "C"
