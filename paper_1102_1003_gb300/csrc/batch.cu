// Batched form: many independent mining instances in ONE persistent compare
// launch, captured with the per-instance correction and compaction into a
// CUDA graph that is replayed while the same sets and outputs are used.
//
// The work units of all instances are merged into one queue ordered longest
// first, so small instances fill the SMs left idle by large ones and the
// tail of one instance overlaps the work of the others.
#include <algorithm>
#include <memory>
#include <mutex>
#include <string>

#include "common.cuh"
#include "compare.cuh"

namespace bm {

void enqueue_correct_compact(batmap_set *S, uint32_t *C, uint32_t s, uint32_t *d_pairs, uint64_t cap,
                             uint64_t *d_total, cudaStream_t st);
void prepare_compaction(batmap_set *S);

struct BatchPlan {
    std::vector<uint64_t> key;
    std::vector<uint32_t *> C;
    DevBuf<InstView> d_views;
    DevBuf<WorkUnit> d_units;
    DevBuf<uint32_t> d_counter;
    DevBuf<uint64_t> d_totals;
    UnitParts parts;
    cudaStream_t stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    DevBuf<unsigned long long> d_stamps;  // the compare's span: earliest CTA start, latest CTA end (ns)
    PhaseEvents ev;                       // 0 / 1 around the graph launch (on the stream, not captured)
    ~BatchPlan() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
    }
};

static std::mutex g_batch_mu;
static std::unique_ptr<BatchPlan> g_plan;

static std::vector<uint64_t> plan_key(batmap_set *const *sets, const uint32_t *s, uint32_t k,
                                      const batmap_out *outs, cudaStream_t st) {
    std::vector<uint64_t> key;
    key.push_back((uint64_t)(uintptr_t)st);
    key.push_back(k);
    for (uint32_t q = 0; q < k; q++) {
        key.push_back(sets[q]->gen);
        key.push_back(s[q]);
        key.push_back((uint64_t)(uintptr_t)outs[q].d_pairs);
        key.push_back(outs[q].cap);
        key.push_back((uint64_t)(uintptr_t)outs[q].d_full);
    }
    return key;
}

static void enqueue_batch(BatchPlan *P, batmap_set *const *sets, const uint32_t *s, uint32_t k,
                          const batmap_out *outs, cudaStream_t st) {
    for (uint32_t q = 0; q < k; q++) {
        const uint64_t np = sets[q]->npairs();
        if (np) BM_CUDA(cudaMemsetAsync(P->C[q], 0, np * sizeof(uint32_t), st));
    }
    BM_CUDA(cudaMemsetAsync(P->d_counter.p, 0, COMPARE_COUNTERS * sizeof(uint32_t), st));
    BM_CUDA(cudaMemsetAsync(P->d_stamps.p, 0xFF, sizeof(unsigned long long), st));
    BM_CUDA(cudaMemsetAsync(P->d_stamps.p + 1, 0, sizeof(unsigned long long), st));
    launch_compare(P->d_views.p, P->d_units.p, P->parts, P->d_counter.p, st, P->d_stamps.p);
    for (uint32_t q = 0; q < k; q++)
        enqueue_correct_compact(sets[q], P->C[q], s[q], outs[q].d_pairs, outs[q].cap, P->d_totals.p + q, st);
}

static BatchPlan *make_plan(batmap_set *const *sets, const uint32_t *s, uint32_t k, const batmap_out *outs,
                            cudaStream_t st, std::vector<uint64_t> key) {
    auto P = std::make_unique<BatchPlan>();
    P->key = std::move(key);
    P->stream = st;
    std::vector<InstView> views(k);
    std::vector<WorkUnit> units;
    P->C.resize(k);
    for (uint32_t q = 0; q < k; q++) {
        batmap_set *S = sets[q];
        uint32_t *C = outs[q].d_full;
        if (!C) {
            S->d_C.ensure(S->npairs());
            C = S->d_C.p;
        }
        P->C[q] = C;
        views[q] = InstView{reinterpret_cast<const uint4 *>(S->d_bm.p), S->d_line_off.p, S->d_wshift.p,
                            S->d_order.p, C, S->n, S->n_a, S->shift};
        for (WorkUnit u : S->units) {
            u.inst = q;
            units.push_back(u);
        }
        prepare_compaction(S);
    }
    sort_units(&units);
    P->parts = unit_parts(units);
    P->d_views.alloc(k);
    P->d_units.alloc(units.size());
    P->d_counter.alloc(COMPARE_COUNTERS);
    P->d_totals.alloc(k);
    P->d_stamps.alloc(2);
    BM_CUDA(cudaMemcpyAsync(P->d_views.p, views.data(), k * sizeof(InstView), cudaMemcpyHostToDevice, st));
    if (!units.empty())
        BM_CUDA(cudaMemcpyAsync(P->d_units.p, units.data(), units.size() * sizeof(WorkUnit),
                                cudaMemcpyHostToDevice, st));
    BM_CUDA(cudaStreamSynchronize(st));
    prepare_compare();
    P->ev.create();

    // capture the whole batch (zeroing, one compare launch, k compactions)
    cudaStream_t cap_st = st;
    bool own_stream = false;
    if (cap_st == nullptr) {  // the legacy default stream cannot be captured
        BM_CUDA(cudaStreamCreateWithFlags(&cap_st, cudaStreamNonBlocking));
        own_stream = true;
    }
    try {
        BM_CUDA(cudaStreamBeginCapture(cap_st, cudaStreamCaptureModeThreadLocal));
        try {
            enqueue_batch(P.get(), sets, s, k, outs, cap_st);
        } catch (...) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(cap_st, &g);
            if (g) cudaGraphDestroy(g);
            throw;
        }
        BM_CUDA(cudaStreamEndCapture(cap_st, &P->graph));
        BM_CUDA(cudaGraphInstantiate(&P->exec, P->graph, 0));
    } catch (...) {
        if (own_stream) cudaStreamDestroy(cap_st);
        throw;
    }
    if (own_stream) cudaStreamDestroy(cap_st);
    return P.release();
}

void run_batch(batmap_set *const *sets, const uint32_t *s, uint32_t k, batmap_out *outs, cudaStream_t st) {
    BM_REQUIRE(sets && s && outs, BATMAP_ERR_ARG, "NULL argument");
    for (uint32_t q = 0; q < k; q++) {
        BM_REQUIRE(sets[q], BATMAP_ERR_ARG, "NULL set in batch");
        BM_REQUIRE(outs[q].cap == 0 || outs[q].d_pairs, BATMAP_ERR_ARG, "d_pairs is NULL with cap > 0");
    }
    if (k == 0) return;
    std::lock_guard<std::mutex> lock(g_batch_mu);
    auto key = plan_key(sets, s, k, outs, st);
    if (!g_plan || g_plan->key != key) {
        g_plan.reset();
        g_plan.reset(make_plan(sets, s, k, outs, st, std::move(key)));
    }
    BatchPlan *P = g_plan.get();
    P->ev.record(0, st);
    BM_CUDA(cudaGraphLaunch(P->exec, st));
    P->ev.record(1, st);
    std::vector<uint64_t> totals(k);
    unsigned long long stamps[2] = {0, 0};
    BM_CUDA(cudaMemcpyAsync(totals.data(), P->d_totals.p, k * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    BM_CUDA(cudaMemcpyAsync(stamps, P->d_stamps.p, sizeof(stamps), cudaMemcpyDeviceToHost, st));
    BM_CUDA(cudaStreamSynchronize(st));
    // every set of the batch reports the batched pass: the one compare launch
    // over all instances (its CTAs' globaltimer span) and the rest of the pass
    // (zeroing, corrections, compactions)
    const float all = P->ev.ms(0, 1);
    const float cmp = stamps[1] > stamps[0] ? (float)((double)(stamps[1] - stamps[0]) * 1e-6) : 0.f;
    const float cc = all > cmp ? all - cmp : 0.f;
    bool overflow = false;
    for (uint32_t q = 0; q < k; q++) {
        outs[q].n_out = totals[q];
        overflow |= totals[q] > outs[q].cap;
        sets[q]->timing.compare_ms = cmp;
        sets[q]->timing.compact_ms = cc;
        sets[q]->timing.pairs_ms = all;
    }
    if (overflow) throw Error{BATMAP_ERR_CAPACITY, "an instance's d_pairs is too small (see n_out)"};
}

// ---- autotuner ----------------------------------------------------------------
//
// Measures the throughput (padded word pairs per second) of every tile shape
// on the caller's own sets: for each shape, the sampled sets are scheduled
// with that shape alone and compared once, timed with events.  The relative
// throughputs replace the built-in efficiency prior of the scheduler, and
// every given set is rescheduled with them.

static std::mutex g_tune_mu;
static bool g_tuned = false;
static double g_tuned_eff[NUM_SHAPES];

bool tuned_shape_eff(double *eff) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    if (!g_tuned) return false;
    for (int s = 0; s < NUM_SHAPES; s++) eff[s] = g_tuned_eff[s];
    return true;
}

void autotune(batmap_set *const *sets, uint32_t k, double *eff_out, cudaStream_t st) {
    BM_REQUIRE(sets && k, BATMAP_ERR_ARG, "no sets to tune on");
    std::vector<uint32_t> idx;
    for (uint32_t q = 0; q < k; q++) {
        BM_REQUIRE(sets[q], BATMAP_ERR_ARG, "NULL set");
        if (sets[q]->npairs()) idx.push_back(q);
    }
    BM_REQUIRE(!idx.empty(), BATMAP_ERR_ARG, "no set with a pair to tune on");
    std::sort(idx.begin(), idx.end(), [&](uint32_t a, uint32_t b) { return sets[a]->word_pairs > sets[b]->word_pairs; });
    if (idx.size() > 4) idx.resize(4);
    std::vector<InstView> views;
    for (uint32_t q : idx) {
        batmap_set *S = sets[q];
        S->d_C.ensure(S->npairs());
        views.push_back(InstView{reinterpret_cast<const uint4 *>(S->d_bm.p), S->d_line_off.p, S->d_wshift.p,
                                 S->d_order.p, S->d_C.p, S->n, S->n_a, S->shift});
    }
    DevBuf<InstView> d_views(views.size());
    DevBuf<uint32_t> d_counter(COMPARE_COUNTERS);
    BM_CUDA(cudaMemcpyAsync(d_views.p, views.data(), views.size() * sizeof(InstView), cudaMemcpyHostToDevice, st));
    PhaseEvents ev;
    ev.create();
    double rate[NUM_SHAPES];
    double best = 0.0;
    for (int s = 0; s < NUM_SHAPES; s++) {
        std::vector<WorkUnit> units;
        for (uint32_t v = 0; v < idx.size(); v++) {
            std::vector<WorkUnit> u;
            schedule_units(sets[idx[v]], (uint32_t)s + 1, nullptr, 0.0, &u);
            for (auto &w : u) w.inst = v;
            units.insert(units.end(), u.begin(), u.end());
        }
        sort_units(&units);
        double padded = 0.0;
        for (const auto &w : units) {
            const ShapeDesc &sh = SHAPES[w.shape & UNIT_SHAPE_MASK];
            padded += (double)sh.TR * sh.TC * w.klen;
        }
        DevBuf<WorkUnit> d_units(units.size());
        if (!units.empty())
            BM_CUDA(cudaMemcpyAsync(d_units.p, units.data(), units.size() * sizeof(WorkUnit), cudaMemcpyHostToDevice, st));
        BM_CUDA(cudaMemsetAsync(d_counter.p, 0, COMPARE_COUNTERS * sizeof(uint32_t), st));
        ev.record(0, st);
        launch_compare(d_views.p, d_units.p, unit_parts(units), d_counter.p, st);
        ev.record(1, st);
        BM_CUDA(cudaStreamSynchronize(st));
        const double ms = ev.ms(0, 1);
        rate[s] = ms > 0 ? padded / ms : 0.0;
        best = std::max(best, rate[s]);
    }
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        for (int s = 0; s < NUM_SHAPES; s++) g_tuned_eff[s] = best > 0 ? std::max(rate[s] / best, 1e-3) : 1.0;
        g_tuned = true;
        if (eff_out)
            for (int s = 0; s < NUM_SHAPES; s++) eff_out[s] = g_tuned_eff[s];
    }
    {
        std::lock_guard<std::mutex> lock(g_batch_mu);
        g_plan.reset();  // units change: cached batch graphs are stale
    }
    for (uint32_t q = 0; q < k; q++) build_schedule(sets[q]);
    BM_CUDA(cudaStreamSynchronize(st));
}

void release_batch_plan() {
    std::lock_guard<std::mutex> lock(g_batch_mu);
    g_plan.reset();
}

}  // namespace bm
