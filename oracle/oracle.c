/*
 * Oracle for all-pairs support counting -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, single-threaded C.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference arm of bench.py may load this library.  It shares
 * no code with the CUDA path.
 *
 * What it computes is the plain definition of the problem (Sec. I): the
 * support of the item pair {i, j} is |S_i intersect S_j|, the number of
 * transactions holding both items, where S_i is the sorted tidlist of item i.
 * Each intersection is the folklore two-pointer merge of two sorted lists
 * (Sec. I "Set representations", Sec. II first paragraph, Sec. IV-B).
 *
 * Tidlists arrive in CSR form: offsets[n+1] (uint64) and tids (uint32), the
 * tids of item i being tids[offsets[i] .. offsets[i+1]), strictly increasing.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* |A intersect B| by merging two sorted lists (Sec. IV-B, "Comparison with merging"). */
uint64_t oracle_intersect_count(const uint32_t *a, uint64_t na,
                                const uint32_t *b, uint64_t nb)
{
    uint64_t i = 0, j = 0, c = 0;
    while (i < na && j < nb) {
        if (a[i] < b[j]) {
            i++;
        } else if (a[i] > b[j]) {
            j++;
        } else {
            c++;
            i++;
            j++;
        }
    }
    return c;
}

static uint64_t support(const uint64_t *off, const uint32_t *tids, uint32_t i, uint32_t j)
{
    return oracle_intersect_count(tids + off[i], off[i + 1] - off[i],
                                  tids + off[j], off[j + 1] - off[j]);
}

/*
 * Supports of all pairs i < j, packed row-major upper triangle:
 * out[idx(i, j)] with idx(i, j) = i*n - i*(i+1)/2 + (j - i - 1).
 * Rows [row_begin, row_end) only, so callers may split the work.
 */
void oracle_pairs_rows(uint32_t n, const uint64_t *off, const uint32_t *tids,
                       uint32_t row_begin, uint32_t row_end, uint32_t *out)
{
    for (uint32_t i = row_begin; i < row_end && i < n; i++) {
        uint64_t base = (uint64_t)i * n - (uint64_t)i * (i + 1) / 2;
        for (uint32_t j = i + 1; j < n; j++)
            out[base + (j - i - 1)] = (uint32_t)support(off, tids, i, j);
    }
}

/* Supports of an explicit list of pairs (ii[k], jj[k]). */
void oracle_pairs_list(uint64_t k, const uint32_t *ii, const uint32_t *jj,
                       const uint64_t *off, const uint32_t *tids, uint32_t *out)
{
    for (uint64_t q = 0; q < k; q++)
        out[q] = (uint32_t)support(off, tids, ii[q], jj[q]);
}

/*
 * Frequent pairs (Sec. I, problem statement): every (i, j, support) with
 * i < j and support >= s, in lexicographic (i, j) order.  Writes at most cap
 * triples; returns the total number of qualifying pairs.
 */
uint64_t oracle_pairs_threshold(uint32_t n, const uint64_t *off, const uint32_t *tids,
                                uint32_t s, uint32_t *triples, uint64_t cap)
{
    uint64_t cnt = 0;
    for (uint32_t i = 0; i < n; i++) {
        for (uint32_t j = i + 1; j < n; j++) {
            uint64_t v = support(off, tids, i, j);
            if (v >= s) {
                if (cnt < cap) {
                    triples[3 * cnt + 0] = i;
                    triples[3 * cnt + 1] = j;
                    triples[3 * cnt + 2] = (uint32_t)v;
                }
                cnt++;
            }
        }
    }
    return cnt;
}

/*
 * |S_a1 intersect ... intersect S_ak| by iterated merging (the conjunctive
 * query of Sec. I reduced to repeated two-list intersection).  `scratch`
 * needs room for the first list, S_a1.
 */
uint64_t oracle_kway_count(uint32_t k, const uint32_t *ids, const uint64_t *off,
                           const uint32_t *tids, uint32_t *scratch)
{
    if (k == 0)
        return 0;
    uint64_t len = off[ids[0] + 1] - off[ids[0]];
    memcpy(scratch, tids + off[ids[0]], len * sizeof(uint32_t));
    for (uint32_t q = 1; q < k && len > 0; q++) {
        const uint32_t *b = tids + off[ids[q]];
        uint64_t nb = off[ids[q] + 1] - off[ids[q]];
        uint64_t i = 0, j = 0, w = 0;
        while (i < len && j < nb) {
            if (scratch[i] < b[j]) {
                i++;
            } else if (scratch[i] > b[j]) {
                j++;
            } else {
                scratch[w++] = scratch[i];
                i++;
                j++;
            }
        }
        len = w;
    }
    return len;
}

/*
 * The elements of S_a1 intersect ... intersect S_ak (the answer of a
 * conjunctive query, Sec. I), ascending, into out (room for the first
 * list, S_a1); returns their number.
 */
uint64_t oracle_kway_elems(uint32_t k, const uint32_t *ids, const uint64_t *off,
                           const uint32_t *tids, uint32_t *out)
{
    return oracle_kway_count(k, ids, off, tids, out);
}

/* Batched k-way queries: query q uses ids[qoff[q] .. qoff[q+1]). */
void oracle_kway_list(uint64_t nq, const uint32_t *qoff, const uint32_t *ids,
                      const uint64_t *off, const uint32_t *tids, uint32_t *scratch,
                      uint64_t *out)
{
    for (uint64_t q = 0; q < nq; q++)
        out[q] = oracle_kway_count(qoff[q + 1] - qoff[q], ids + qoff[q], off, tids, scratch);
}
