/*
 * batmap.h -- C ABI of the GB300 BatMap library (all-pairs support counting).
 *
 * Problem (Sec. I of Amossen & Pagh, "A New Data Layout For Set Intersection
 * on GPUs"): given transactions T_1..T_m over items 1..n, the support of an
 * item pair {i, j} is |S_i intersect S_j|, where the tidlist S_i holds the
 * transactions that contain item i.  Frequent pair mining reports every pair
 * whose support is at least s; the paper's GPU experiment outputs the support
 * of every pair (Sec. IV-A).
 *
 * Conventions for every call:
 *   - Transaction ids are 0-based uint32 in [0, m) (the paper numbers 1..m).
 *   - Tidlists come in CSR form: offsets[n+1] (uint64, offsets[0] = 0,
 *     non-decreasing) and tids[offsets[n]] (uint32); the tids of item i are
 *     tids[offsets[i] .. offsets[i+1]), strictly increasing, each < m.
 *   - Pointers named d_* are DEVICE pointers owned by the caller; h_* are host
 *     pointers owned by the caller.  The library never frees caller memory.
 *   - Calls are ordered on the given CUDA stream.  Unless stated otherwise a
 *     call returns after its work is enqueued; calls that report a count on
 *     the host synchronise the stream.
 *   - Every call returns BATMAP_OK (0) or a negative error code; the message
 *     of the last error on the calling thread is batmap_last_error().  No C++
 *     exception crosses this interface.  On error, outputs are unspecified
 *     except where a call documents otherwise.
 *   - One GPU per process.  The library's one-time setup (kernel shared-memory
 *     limits, the SM count, cached placement scratch and BatMap arrays) is
 *     made on the device current at the first call; every later call must
 *     run with that device current.  Drive several GPUs with one process per
 *     GPU (bench.py under torchrun does).  A handle (set or pool) is used by
 *     one host thread at a time; batmap_serve runs its own request loop.
 */
#ifndef BATMAP_H
#define BATMAP_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int batmap_status;

#define BATMAP_OK 0
#define BATMAP_ERR_ARG (-1)      /* invalid argument or malformed input data        */
#define BATMAP_ERR_NOMEM (-2)    /* device or host allocation failed                */
#define BATMAP_ERR_CAPACITY (-3) /* caller buffer too small; required size reported */
#define BATMAP_ERR_CUDA (-4)     /* a CUDA runtime call or kernel failed            */
#define BATMAP_ERR_TIMEOUT (-5)  /* a bounded device-side wait gave up              */
#define BATMAP_ERR_INTERNAL (-6) /* internal invariant violated                     */

/*
 * Build parameters.
 *   load_num / load_den : load factor c of the hash range, r_i = the smallest
 *       power of two >= c |S_i|, never below r_0 (Sec. III-A; the paper uses
 *       c = 2, giving width 3 * 2^ceil(log 2|S|) bytes, Sec. IV-A).  Any c
 *       keeps counts exact (failed insertions are corrected).  Default 2/1.
 *   max_loop : MaxLoop of the INSERT procedure (Sec. II-A): a placement chain
 *       gives up after 3 * max_loop moves and its element becomes a failed
 *       insertion.  Default 32.
 *   min_shift : r_0 = 2^s with s the smallest shift >= min_shift such that
 *       m <= 127 * 2^s (7-bit codes 1..127, 0x00 = empty slot; Sec. III-A).
 *       Must be >= 7 so that every BatMap is a multiple of 384 bytes.
 *       Default 7.
 *   tile : 0 lets the scheduler choose compare tile shapes per width class;
 *       1..BATMAP_NUM_SHAPES forces one shape for every class (testing and
 *       autotuning).
 *   validate : nonzero checks that tids are strictly increasing and < m per
 *       item and that each permutation row is a bijection of [0, m); a
 *       violation returns BATMAP_ERR_ARG.  Default 1.
 *   shape_mask : bit s-1 allows compare tile shape s (1..BATMAP_NUM_SHAPES)
 *       when tile is 0;
 *       0 allows every shape.  Default 0.
 *   probe_log : width-skewed pairs may be counted by probing instead of the
 *       cyclic scan (Sec. V's second k-way idea: look up the elements of the
 *       smaller set in the larger one).  A pair whose wider BatMap is at least
 *       2^probe_log times as wide as the narrower is eligible; the probe
 *       visits every nonempty slot of the narrower BatMap and reads the one
 *       slot of the wider BatMap that can hold the same element: a slot in
 *       table t at byte h with code c holds pi_t(x) = ((c - 1) << s) |
 *       (h mod r_0).  Per width class the scheduler probes the eligible rows
 *       where its cost model (the measured rates of both routes) makes the
 *       probe cheaper.  Both routes count the same slot pairs, so supports
 *       are identical.  0 selects the default, 2 (ratio 4); 32 or more turns
 *       the route off.  Ignored when `tile` forces a shape.  Default 0.
 *   perm_seed : seed of the permutations pi_t that the library computes when
 *       a build is given no permutation table (d_perm = NULL).  Sec. III-A
 *       draws pi_1..pi_3 at random without fixing a generator; the library's
 *       pi_t (t = 0, 1, 2; up to 4 for 3-of-4 and 4-of-5 sets) is defined as
 *       follows.
 *       Round keys: SplitMix64 (Steele, Lea, Flood 2014) started from the
 *       seed; table t takes outputs 4t .. 4t+3, low 32 bits each.  One pass
 *       E_t: a four-round balanced Feistel network on b bits, b the smallest
 *       even number >= max(2, ceil(log2 m)), halves of b/2 bits, each round
 *       (L, R) -> (R, L xor (fmix32(R xor k) mod 2^(b/2))) with fmix32 the
 *       32-bit finalizer of MurmurHash3.  pi_t(x): E_t applied to x until the
 *       value is below m (cycle walking).  Computed in the kernels; no table
 *       is stored.  Default 1.
 */
/* Number of compare tile shapes (batmap_params.tile, shape_mask, autotune). */
#define BATMAP_NUM_SHAPES 18

typedef struct batmap_params {
    uint32_t load_num;
    uint32_t load_den;
    uint32_t max_loop;
    uint32_t min_shift;
    uint32_t tile;
    uint32_t validate;
    uint32_t shape_mask;
    uint32_t probe_log;
    uint64_t perm_seed;
} batmap_params;

/* Opaque handle to n BatMaps built from one instance (owned by the library). */
typedef struct batmap_set batmap_set;

/* Summary of a built set (host struct filled by batmap_get_info). */
typedef struct batmap_info {
    uint32_t m;              /* transactions                                   */
    uint32_t n;              /* items                                          */
    uint32_t shift;          /* s: codes are (pi >> s) + 1                     */
    uint32_t r0;             /* 2^s, the smallest hash range                   */
    uint64_t bytes;          /* total BatMap bytes, sum of 3 r_i               */
    uint64_t n_elements;     /* total tids, offsets[n]                         */
    uint64_t n_failed;       /* failed insertions, sum of |F_i|                */
    uint64_t n_corrections;  /* correction entries (one per failed common tid) */
    uint64_t n_work_units;   /* compare work units scheduled                   */
    uint32_t n_classes;      /* distinct BatMap widths                         */
    uint32_t n_a;            /* cross mode: size of family A (0 = all pairs)    */
    double word_pairs;       /* sum over reported pairs of max(|B_i|,|B_j|)/4  */
    uint32_t d;              /* copies per element: 2 (2-of-3) or 3 (3-of-4)   */
    uint32_t reserved;
    double probe_word_pairs; /* part of word_pairs counted by the probe route  */
    double probe_words;      /* words the probe route reads: sum over probe-
                                routed pairs of min(|B_i|,|B_j|)/4             */
} batmap_info;

/* Fills *p with the defaults documented above. */
void batmap_default_params(batmap_params *p);

/* Message of the last error raised on the calling thread ("" if none). */
const char *batmap_last_error(void);

/*
 * Build the BatMaps of all n items (Sec. II and Sec. III-A):
 *   - sizes r_i, widths |B_i| = 3 r_i bytes, and the width-sorted order of
 *     the items (Sec. III-C);
 *   - places every tid of S_i in two of its three hash tables with a
 *     parallel generalisation of the cuckoo INSERT procedure (Sec. II-A);
 *   - writes the 8-bit elements: indicator bit << 7 | ((pi_t(x) >> s) + 1),
 *     0x00 for empty slots, at h_t^(i)(x) = |B_0| floor((pi_t(x) mod r_i)/r_0)
 *     + (pi_t(x) mod r_0) + (t-1) r_0 (Sec. III-A);
 *   - records failed insertions F_i and precomputes their correction entries
 *     (Sec. III-C, "Failed insertions").
 * Arguments:
 *   p         : parameters, or NULL for the defaults.
 *   m, n      : transactions (1 <= m <= 2^30) and items (n >= 0).
 *   d_offsets : device uint64[n+1], CSR offsets.
 *   d_tids    : device uint32[offsets[n]], CSR tids (may be NULL when empty).
 *   d_perm    : device uint32[3*m]; row t (t = 0, 1, 2) is the permutation
 *               pi_{t+1} of [0, m) used by the layout hash; or NULL for the
 *               permutations the library computes from p->perm_seed.
 *   stream    : CUDA stream for all work of this call.
 *   out       : receives the new handle; release it with batmap_free.
 * The call synchronises the stream (sizes are needed on the host).  The
 * caller may free its input buffers once the call returns.
 */
batmap_status batmap_build(const batmap_params *p, uint32_t m, uint32_t n,
                           const uint64_t *d_offsets, const uint32_t *d_tids,
                           const uint32_t *d_perm, cudaStream_t stream, batmap_set **out);

/*
 * Cross mode: the supports |A_i cap B_j| between two families of sets over
 * the same transactions (Sec. I: sparse boolean matrix multiplication and
 * join-project reduce to these intersections; pairs with support >= 1 are
 * the non-zeros of the boolean product).  The CSR holds n_a sets of family A
 * followed by n_b sets of family B; otherwise as batmap_build.  On a set
 * built this way, pair_support_all reports the n_a x n_b supports: d_full is
 * uint32[n_a * n_b] row-major (A item, B item), and the triples are
 * (a, b, support) with a in [0, n_a) and b in [0, n_b), lexicographic.
 */
batmap_status batmap_build_cross(const batmap_params *p, uint32_t m, uint32_t n_a, uint32_t n_b,
                                 const uint64_t *d_offsets, const uint32_t *d_tids, const uint32_t *d_perm,
                                 cudaStream_t stream, batmap_set **out);

/*
 * d-of-(d+1) BatMaps, the generalisation that closes Sec. V: every element is
 * kept in d of d+1 hashed tables, so the sets of any itemset of size up to d
 * share a table that witnesses each common element.  d = 2 is batmap_build
 * (the paper's 2-of-3 format; all pair calls apply).  d = 3 and d = 4 build
 * 3-of-4 and 4-of-5 BatMaps for k-way supports (itemset_support,
 * frequent_triples, frequent_quadruples only):
 *   width (d+1) r_i bytes (d+1 tables interleaved in blocks of r_0), slot
 *   h_t(x) = (d+1) r_0 floor((pi_t(x) mod r_i)/r_0) + (pi_t(x) mod r_0)
 *   + t r_0; the byte holds the element's missing table in its top bits and
 *   the code (pi_t(x) >> s) + 1 in the rest, 0x00 empty: d = 3: two missing
 *   bits, six code bits, s the smallest shift >= min_shift with
 *   m <= 63 * 2^s; d = 4: three missing bits, five code bits, m <= 31 * 2^s;
 *   elements left with fewer than d copies are failed insertions (F_i),
 *   corrected exactly.
 *   d_perm : device uint32[(d+1) * m], rows pi_0 .. pi_d (the library keeps a
 *            copy for d >= 3), or NULL for the computed permutations of
 *            p->perm_seed (rows t = 0 .. d).  Other arguments as batmap_build.
 * Items keep their original order (no width sort); h_bytes of
 * batmap_export_layout follow it.  Errors: BATMAP_ERR_ARG for d outside
 * {2, 3, 4} or invalid input.
 */
batmap_status batmap_build_d(const batmap_params *p, uint32_t d, uint32_t m, uint32_t n,
                             const uint64_t *d_offsets, const uint32_t *d_tids, const uint32_t *d_perm,
                             cudaStream_t stream, batmap_set **out);

/*
 * |S_a1 ∩ ... ∩ S_ak| for n_q queries of k item ids (1 <= k <= d) on a set
 * built with d = 3 or d = 4, by the witness rule: the slot of table t counts
 * iff the code bits of the k bytes agree and are nonzero and t is the
 * smallest table missed by none of the k sets (read from the bytes' missing-
 * table fields); failed common elements are added from the F lists.
 *   d_items   : device uint32[k * n_q], query q = d_items[k q .. k q + k),
 *               ids < n (checked; repeats allowed).
 *   d_support : device uint32[n_q] (written).
 * Asynchronous apart from the id check (one stream synchronisation).
 * Errors: BATMAP_ERR_ARG (d not 3 or 4, k out of range, id >= n, NULL pointer).
 */
batmap_status itemset_support(batmap_set *set, uint32_t k, uint64_t n_q, const uint32_t *d_items,
                              uint32_t *d_support, cudaStream_t stream);

/*
 * Frequent itemsets of size 3 (the problem of Sec. I beyond pairs): the
 * Apriori join-and-prune step turns the frequent pairs into the candidates
 * {a < b < c} whose three 2-subsets are all frequent, itemset_support counts
 * them on the 3-of-4 set, and those with support >= s are written.
 *   d_pairs : device uint32[3 * n_pairs], (i, j, support) with i < j < n in
 *             lexicographic order: the output of pair_support_all for the
 *             same tidlists and threshold s (checked: order and ids).
 *   d_out   : device uint32[4 * cap], (a, b, c, support), lexicographic.
 *   n_out   : host, number of frequent triples (all of them, even > cap).
 *   n_candidates : host, may be NULL; number of candidates counted.
 * The set may be built with d = 3 or d = 4.  Candidates whose widest BatMap
 * is at least 8x (d = 3) or 2x (d = 4) the narrowest are counted by probing
 * the narrowest set's slots in the others (Sec. V: look up the elements of
 * the smallest set); the rest by the witness scan (grouped by pair for d = 3,
 * one warp per candidate for d = 4).  Both count the same elements.
 * Synchronises `stream`.  Timing: compare_ms = the support kernels (scan_ms
 * the scan, probe_ms the probe), compact_ms = candidate generation +
 * compaction, pairs_ms = the call.  Errors: BATMAP_ERR_ARG,
 * BATMAP_ERR_CAPACITY (cap < *n_out; the first cap triples are written).
 */
batmap_status frequent_triples(batmap_set *set, uint32_t s, const uint32_t *d_pairs, uint64_t n_pairs,
                               uint32_t *d_out, uint64_t cap, uint64_t *n_out, uint64_t *n_candidates,
                               cudaStream_t stream);

/*
 * Frequent itemsets of size 4 (the problem of Sec. I, Apriori level 4): the
 * frequent triples sharing their first two items are joined into candidates
 * {a < b < c < d}, those whose other two 3-subsets are not frequent are
 * pruned, itemset_support counts the rest on a 4-of-5 set, and those with
 * support >= s are written.
 *   d_triples : device uint32[4 * n_triples], (a, b, c, support) with
 *               a < b < c < n in lexicographic order: the output of
 *               frequent_triples for the same tidlists and threshold s
 *               (checked: order and ids).
 *   d_out     : device uint32[5 * cap], (a, b, c, d, support), lexicographic.
 *   n_out     : host, number of frequent quadruples (all of them, even > cap).
 *   n_candidates : host, may be NULL; number of candidates counted.
 * Needs a set built with d = 4; candidates are routed between the probe and
 * the scan as in frequent_triples on a d = 4 set.  Synchronises `stream`;
 * timing as frequent_triples.  Errors: BATMAP_ERR_ARG, BATMAP_ERR_CAPACITY
 * (the first cap quadruples are written).
 */
batmap_status frequent_quadruples(batmap_set *set, uint32_t s, const uint32_t *d_triples, uint64_t n_triples,
                                  uint32_t *d_out, uint64_t cap, uint64_t *n_out, uint64_t *n_candidates,
                                  cudaStream_t stream);

/* Release a handle and all device memory it owns (NULL is ignored). */
void batmap_free(batmap_set *set);

/* Copy the summary of a built set into *info. */
batmap_status batmap_get_info(const batmap_set *set, batmap_info *info);

/*
 * Copy the built layout to host buffers (used to check layouts against the
 * definition).  Any pointer may be NULL to skip that output.
 *   h_bytes        : uint8[info.bytes], all BatMaps, width-sorted order.
 *   h_byte_offset  : uint64[n], byte offset of item i's BatMap (original id).
 *   h_range        : uint32[n], r_i of item i.
 *   h_fail_offsets : uint64[n+1], CSR offsets of the failed tids per item.
 *   h_fail_tids    : uint32[info.n_failed], F_i sorted ascending per item.
 * Synchronises the set's stream.
 */
batmap_status batmap_export_layout(const batmap_set *set, uint8_t *h_bytes,
                                   uint64_t *h_byte_offset, uint32_t *h_range,
                                   uint64_t *h_fail_offsets, uint32_t *h_fail_tids);

/*
 * Support of every item pair and the frequent pairs (Sec. I problem
 * statement; Sec. III-B/C all-pairs comparison, failure correction).  Pairs
 * of similar width run the cyclic scan; pairs whose widths differ by
 * 2^probe_log or more run the probe route (batmap_params.probe_log); both
 * count the same slot pairs.
 *   s       : support threshold; pairs with support >= s are reported.
 *   d_pairs : device uint32[3*cap]: triples (i, j, support) with original
 *             item ids i < j, in lexicographic (i, j) order.  May be NULL
 *             when cap == 0.
 *   cap     : capacity of d_pairs in triples.
 *   n_out   : host; receives the number of qualifying pairs.  If it exceeds
 *             cap, the first cap triples are written and BATMAP_ERR_CAPACITY
 *             is returned.
 *   d_full  : optional device uint32[n(n-1)/2]: support of every pair i < j,
 *             packed row-major upper triangle, index i*n - i(i+1)/2 + j-i-1.
 *             NULL to skip.
 * Synchronises the stream (to report n_out).
 */
batmap_status pair_support_all(batmap_set *set, uint32_t s, uint32_t *d_pairs, uint64_t cap,
                               uint64_t *n_out, uint32_t *d_full, cudaStream_t stream);

/*
 * End-to-end convenience for callers holding their data on the HOST: copies
 * the CSR tidlists and permutations to the device, builds the BatMaps, counts
 * all pairs, and copies the frequent pairs back.
 *   h_offsets, h_tids, h_perm : host inputs as in batmap_build (pinned
 *       memory gives the fastest copies); h_perm may be NULL (computed
 *       permutations, nothing to copy).
 *   h_pairs, cap, n_out : host output triples as in pair_support_all.
 * Synchronises the stream.  The device copies of the inputs and of the output
 * are kept by the library for the next call (grown when a call needs more)
 * until batmap_release_scratch; calls from several threads are serialised.
 */
batmap_status pair_support_host(const batmap_params *p, uint32_t m, uint32_t n,
                                const uint64_t *h_offsets, const uint32_t *h_tids,
                                const uint32_t *h_perm, uint32_t s, uint32_t *h_pairs,
                                uint64_t cap, uint64_t *n_out, cudaStream_t stream);

/*
 * Autotuner of the compare schedule.  Runs the all-pairs compare of (up to
 * four of the largest of) the given sets once per tile shape, each shape
 * alone, and measures its throughput in padded word pairs per second.  The
 * relative throughputs become the scheduler's shape costs for every later
 * batmap_build in the process, and all k sets are rescheduled with them (the
 * width class -> tile shape choice and the split of column words into work
 * units).
 *   shape_eff : optional host double[BATMAP_NUM_SHAPES], receives the
 *               relative throughputs.
 * Synchronises the stream.
 */
batmap_status batmap_autotune(batmap_set *const *sets, uint32_t k, double *shape_eff, cudaStream_t stream);

/*
 * Device-side durations of the most recent batmap_build / pair_support_all
 * on a set, measured with CUDA events recorded on the call's stream around
 * each phase (milliseconds; 0 for a phase that did not run).
 */
typedef struct batmap_timing {
    float build_ms;     /* whole batmap_build, first to last enqueued operation */
    float place_ms;     /* 2-of-3 placement kernel                              */
    float finalize_ms;  /* byte writing + failure lists + correction entries    */
    float compare_ms;   /* the all-pairs compare: scan and probe kernels        */
    float compact_ms;   /* failure correction + threshold compaction            */
    float pairs_ms;     /* whole pair_support_all                               */
    float scan_ms;      /* frequent_triples / _quadruples: the witness scan;
                           pair_support_all: the cyclic-scan compare kernels    */
    float probe_ms;     /* frequent_triples / _quadruples and pair_support_all:
                           the probe kernel of width-skewed tuples              */
} batmap_timing;

/* Copy the phase durations of the set's most recent calls into *t. */
batmap_status batmap_get_timing(const batmap_set *set, batmap_timing *t);

/* Release the scratch the library caches between calls (the placement table
 * of batmap_build, one uint32 per BatMap byte; the dense path's bitmap and
 * workspace; pair_support_host's device copies of its inputs and output).
 * Call when no other call of the library is running. */
void batmap_release_scratch(void);

/* Number of kernels this library has launched in the process so far (a
 * diagnostic counter; differences around a region count its launches). */
uint64_t batmap_kernel_launches(void);

/* Per-instance outputs of pair_support_batch (host struct). */
typedef struct batmap_out {
    uint32_t *d_pairs; /* device uint32[3*cap] triples, as in pair_support_all */
    uint64_t cap;      /* capacity in triples                                 */
    uint64_t n_out;    /* filled in: qualifying pairs of this instance        */
    uint32_t *d_full;  /* optional packed upper triangle, or NULL             */
} batmap_out;

/*
 * Many independent mining instances in one pass: the compare work of all k
 * sets runs in ONE persistent launch that pulls (instance, tile, k-range)
 * units from a shared queue, followed by the per-instance correction and
 * compaction.  Results equal k separate pair_support_all calls.
 *   sets : k built handles.   s : host uint32[k] thresholds.
 *   outs : host batmap_out[k]; n_out is filled in for each instance.
 * Returns BATMAP_ERR_CAPACITY if any instance overflowed its buffer (that
 * instance's first cap triples are written).  Synchronises the stream.
 * Afterwards batmap_get_timing of every set of the batch reports the batched
 * pass: compare_ms = the one compare launch over all instances (the span of
 * its CTAs on the GPU's global timer), pairs_ms = the whole pass (events
 * around it), compact_ms = the rest (zeroing, corrections, compactions).
 */
batmap_status pair_support_batch(batmap_set *const *sets, const uint32_t *s, uint32_t k,
                                 batmap_out *outs, cudaStream_t stream);

/* ---- serving: a resident pool of sets and conjunctive queries ----------- */

/* Opaque handle to a device-resident pool of sets (owned by the library). */
typedef struct batmap_pool batmap_pool;

/*
 * Build a pool from n sets over the universe [0, m) given as CSR tidlists (as
 * in batmap_build).  Every set keeps a device copy of its sorted tidlist; sets
 * for which the 8-bit BatMap is compact (c |S| >= r_0, Sec. III-A) also get a
 * BatMap built with the same GPU build as batmap_build.  d_perm is the
 * caller's device uint32[3*m] permutation table (copied) or NULL for the
 * permutations the library computes from p->perm_seed (no table is kept).
 * The caller may free its buffers after the call.  Synchronises the stream.
 */
batmap_status batmap_pool_create(const batmap_params *p, uint32_t m, uint32_t n, const uint64_t *d_offsets,
                                 const uint32_t *d_tids, const uint32_t *d_perm, cudaStream_t stream,
                                 batmap_pool **out);
void batmap_pool_free(batmap_pool *pool);
/* Pool summary: BatMap-backed sets, their bytes, total elements (any may be NULL). */
batmap_status batmap_pool_info(const batmap_pool *pool, uint32_t *n_batmaps, uint64_t *batmap_bytes,
                               uint64_t *n_elements);

/*
 * Conjunctive queries |S_a1 cap ... cap S_ak| (Sec. I conjunctive queries;
 * Sec. V: count, for each element of the smallest set, its occurrences in the
 * others).  Query q names the sets h_ids[h_qoff[q] .. h_qoff[q+1]) (1..8 ids,
 * host arrays); d_counts is a device uint64[n_queries].  Synchronises.
 */
batmap_status intersect_query(const batmap_pool *pool, const uint32_t *h_qoff, const uint32_t *h_ids,
                              uint32_t n_queries, uint64_t *d_counts, cudaStream_t stream);

/*
 * Materialised answers of conjunctive queries: the elements of
 * S_a1 cap ... cap S_ak, ascending.  Queries as in intersect_query.
 *   d_out_off : device uint64[n_queries + 1]; query q's elements are
 *               d_out[d_out_off[q] .. d_out_off[q+1]).
 *   d_out     : device uint32[cap].
 *   n_total   : host; receives the total number of elements.  If it exceeds
 *               cap, d_out_off is complete, elements beyond cap are not
 *               written and BATMAP_ERR_CAPACITY is returned.
 * Synchronises the stream.
 */
batmap_status intersect_query_list(const batmap_pool *pool, const uint32_t *h_qoff, const uint32_t *h_ids,
                                   uint32_t n_queries, uint64_t *d_out_off, uint32_t *d_out, uint64_t cap,
                                   uint64_t *n_total, cudaStream_t stream);

/* Options of the serving loop. */
typedef struct batmap_serve_opts {
    uint32_t max_batch;   /* queries per micro-batch (default 64)                        */
    uint32_t slots;       /* micro-batches in flight, one CUDA stream each (default 4)    */
    uint64_t work_budget; /* admission bound on in-flight work: sum over queries of
                             |smallest set| x sets named (default 2^26); it also sizes
                             each slot's fixed task buffers                              */
    uint64_t reserved;
} batmap_serve_opts;

/* Statistics of one serving run (seconds). */
typedef struct batmap_serve_stats {
    double makespan_s, queries_per_s, p50_s, p99_s, max_s;
    uint64_t batches, max_inflight;
} batmap_serve_stats;

/*
 * Continuous-batching request loop over a pool.  Query q (as in
 * intersect_query) arrives h_arrival_s[q] seconds after the call starts
 * (non-decreasing).  Arrived queries are admitted into a free slot while the
 * in-flight work stays within the budget, launched as one micro-batch on the
 * slot's stream, and overlap on the device with batches in other slots.
 * Outputs (host): h_counts[q], h_latency_s[q] = completion - arrival, stats.
 * opts may be NULL for the defaults.
 */
batmap_status batmap_serve(const batmap_pool *pool, const uint32_t *h_qoff, const uint32_t *h_ids,
                           const double *h_arrival_s, uint32_t n_queries, const batmap_serve_opts *opts,
                           uint64_t *h_counts, double *h_latency_s, batmap_serve_stats *stats,
                           cudaStream_t stream);

/*
 * Dense-bitmap comparison path (Sec. I-B: the bitmap vertical representation,
 * m*n bits, where a support is AND + popcount).  Builds the item x transaction
 * bit matrix (packed, one bit per pair) and computes all supports as the dense
 * contraction M M^T on the tensor cores: each K step's bits are expanded to
 * e4m3 {0, 1} bytes in shared memory and multiplied with tcgen05
 * kind::f8f6f4 (FP32 accumulation in tensor memory, exact because every
 * product is 0 or 1 and every partial sum an integer below 2^24), then the
 * same threshold compaction as pair_support_all.
 *   m, n, d_offsets, d_tids : CSR tidlists as in batmap_build (1 <= m <= 2^24).
 *   s, d_pairs, cap, n_out, d_full : as in pair_support_all.
 *   timing  : optional host struct; build_ms = bitmap build, compare_ms = the
 *             tensor-core kernel, compact_ms = compaction.
 * The bit matrix (n rows of ceil(m/128)*128 bits) and scratch are cached
 * inside the library between calls.  Synchronises the stream.
 */
batmap_status pair_support_dense(uint32_t m, uint32_t n, const uint64_t *d_offsets, const uint32_t *d_tids,
                                 uint32_t s, uint32_t *d_pairs, uint64_t cap, uint64_t *n_out,
                                 uint32_t *d_full, batmap_timing *timing, cudaStream_t stream);

/*
 * Test hook for the error path of the dense kernel's bounded pipeline waits
 * (no GPU fault is involved).  The next pair_support_dense call in this
 * process launches its tensor-core kernel with the TMA producer issuing no
 * loads and every mbarrier wait limited to spin_limit polls: every consumer
 * wait gives up while no copy and no MMA is in flight, the kernel frees its
 * tensor memory and returns, and the call returns BATMAP_ERR_TIMEOUT (its
 * outputs are unspecified).  The hook applies to one call; spin_limit 0
 * cancels it.  Later calls run normally.
 */
void batmap_test_dense_timeout(uint32_t spin_limit);

/*
 * Frequent pairs from already counted supports, for callers that cannot
 * allocate device memory.  The paper has no counterpart: this is an
 * interface convenience.
 *
 * Callers such as a serving loop confined to a fixed, pre-partitioned memory
 * budget, or latency-critical code that must not pay for the implicit device
 * synchronisation cudaMalloc / cudaFree may perform, cannot let the library
 * allocate.  This call performs the same support-threshold compaction as
 * pair_support_all and allocates nothing: its scratch is a fixed device array
 * of 512 KiB + 8 bytes inside the library, which every GPU that loads the
 * library holds until the process exits.
 *   d_full  : device uint32[n(n-1)/2], supports of all pairs i < j as the
 *             packed upper triangle written by pair_support_all's d_full.
 *   n       : items; at most 23,170 (n(n-1)/2 <= 2^28).  Larger n returns
 *             BATMAP_ERR_CAPACITY without touching the GPU.
 *   s       : support threshold.
 *   d_pairs, cap, n_out : as in pair_support_all (lexicographic triples;
 *             BATMAP_ERR_CAPACITY with the first cap triples if cap is short).
 * The first call on a device looks up the device address of the fixed array
 * (once per device, with that device current); make that first call before
 * any stream capture.  With lazy module loading (the CUDA default) that
 * first lookup is also when the array's memory is reserved on the device, so
 * a caller that must not see any reservation during its critical section
 * makes one call beforehand.  All calls share the one array: calls whose
 * work overlaps on the GPU (different streams or threads without ordering)
 * race and must not be issued.  Synchronises the stream.
 */
batmap_status pair_threshold_noalloc(const uint32_t *d_full, uint32_t n, uint32_t s, uint32_t *d_pairs,
                                     uint64_t cap, uint64_t *n_out, cudaStream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* BATMAP_H */
