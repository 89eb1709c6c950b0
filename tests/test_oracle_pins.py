"""Pins of the merge oracle against things other than itself (CPU only).

* brute force over a dense boolean transaction x item matrix on tiny inputs;
* Python's built-in set intersection;
* the naive horizontal pair scan (Sec. I, "Set representations": count the
  pairs inside every transaction);
* invariants: support(i, i) = |S_i|, symmetry, support <= min(|S_i|, |S_j|),
  and sum_{j != i} support(i, j) = sum_{x in S_i} (|T_x| - 1);
* the threshold output is exactly the pairs with support >= s, lexicographic;
* k-way counts against set intersection of Python sets.
"""
import numpy as np
import pytest

import datagen
import oracle


def _random_instance(rng, m, n, p=None):
    lists = []
    for _ in range(n):
        q = rng.uniform(0, 1) if p is None else p
        lists.append(np.flatnonzero(rng.random(m) < q).astype(np.uint32))
    return datagen.from_lists(lists, m)


def _dense(inst):
    M = np.zeros((inst.n, inst.m), dtype=np.int64)
    for i in range(inst.n):
        M[i, inst.tidlist(i)] = 1
    return M


@pytest.mark.parametrize("seed", range(40))
def test_merge_matches_bruteforce_tiny(seed):
    rng = np.random.default_rng(seed)
    m = int(rng.integers(1, 65))
    n = int(rng.integers(2, 9))
    inst = _random_instance(rng, m, n)
    M = _dense(inst)
    brute = np.zeros((n, n), dtype=np.int64)
    for i in range(n):
        for j in range(n):
            brute[i, j] = sum(1 for x in range(m) if M[i, x] and M[j, x])
    full = oracle.pairs_full(inst.offsets, inst.tids)
    ii, jj = np.triu_indices(n, 1)
    assert np.array_equal(full.astype(np.int64), brute[ii, jj])


def test_merge_edge_cases():
    cases = [
        ([], []), ([], [1, 2]), ([5], [5]), ([5], [6]), ([0, 1, 2, 3], [0, 1, 2, 3]),
        ([0, 2, 4, 6], [1, 3, 5, 7]), ([0, 2, 4, 6], [6]), ([2**32 - 2, 2**32 - 1], [2**32 - 1]),
    ]
    for a, b in cases:
        assert oracle.intersect_count(a, b) == len(set(a) & set(b))
        assert oracle.intersect_count(b, a) == len(set(a) & set(b))


def test_merge_matches_python_sets():
    rng = np.random.default_rng(7)
    for _ in range(200):
        m = int(rng.integers(1, 100000))
        a = np.unique(rng.integers(0, m, int(rng.integers(0, 3000)))).astype(np.uint32)
        b = np.unique(rng.integers(0, m, int(rng.integers(0, 3000)))).astype(np.uint32)
        assert oracle.intersect_count(a, b) == len(set(a.tolist()) & set(b.tolist()))


def test_merge_matches_transaction_scan():
    # configuration-1 sized instance: m = 10,000, n = 200, p = 0.05
    inst = datagen.workload_instance("bern_m10k_n200")
    n = inst.n
    # horizontal form: transaction x -> items containing it
    trans = [[] for _ in range(inst.m)]
    for i in range(n):
        for x in inst.tidlist(i).tolist():
            trans[x].append(i)
    scan = np.zeros((n, n), dtype=np.int64)
    for items in trans:
        if len(items) > 1:
            a = np.array(items)
            ii, jj = np.meshgrid(a, a, indexing="ij")
            keep = ii < jj
            np.add.at(scan, (ii[keep], jj[keep]), 1)
    ii, jj = np.triu_indices(n, 1)
    full = oracle.pairs_full(inst.offsets, inst.tids, threads=4)
    assert np.array_equal(full.astype(np.int64), scan[ii, jj])


def test_invariants():
    inst = datagen.zipf_tidlists(20000, 60, 0.05, seed=3)
    n = inst.n
    full = oracle.pairs_full(inst.offsets, inst.tids)
    sizes = inst.sizes
    S = np.zeros((n, n), dtype=np.int64)
    ii, jj = np.triu_indices(n, 1)
    S[ii, jj] = full
    # symmetry through the explicit-pair entry point
    sym = oracle.pairs_list(inst.offsets, inst.tids, jj, ii)
    assert np.array_equal(sym, full)
    S[jj, ii] = full
    for i in range(n):
        assert oracle.intersect_count(inst.tidlist(i), inst.tidlist(i)) == sizes[i]
    assert (full <= np.minimum(sizes[ii], sizes[jj])).all()
    # sum over partners = sum over transactions of (length - 1)
    tlen = np.zeros(inst.m, dtype=np.int64)
    np.add.at(tlen, inst.tids.astype(np.int64), 1)
    for i in range(n):
        assert S[i].sum() == (tlen[inst.tidlist(i)] - 1).sum()


def test_threshold_is_filtered_full_matrix():
    inst = datagen.workload_instance("bern_m10k_n200")
    full = oracle.pairs_full(inst.offsets, inst.tids)
    for s in (0, 1, 25, 30, 10**9):
        trip = oracle.pairs_threshold(inst.offsets, inst.tids, s)
        ref = oracle.threshold_from_full(full, inst.n, s)
        assert np.array_equal(trip, ref)
        if trip.shape[0] > 1:
            key = trip[:, 0].astype(np.int64) * inst.n + trip[:, 1]
            assert (np.diff(key) > 0).all()
            assert (trip[:, 0] < trip[:, 1]).all()


def test_threads_do_not_change_results():
    inst = datagen.zipf_tidlists(50000, 120, 0.03, seed=9)
    a = oracle.pairs_full(inst.offsets, inst.tids, threads=1)
    b = oracle.pairs_full(inst.offsets, inst.tids, threads=6)
    assert np.array_equal(a, b)
    rng = np.random.default_rng(1)
    ii = rng.integers(0, inst.n, 500)
    jj = rng.integers(0, inst.n, 500)
    c = oracle.pairs_list(inst.offsets, inst.tids, ii, jj, threads=5)
    d = np.array([len(set(inst.tidlist(i).tolist()) & set(inst.tidlist(j).tolist()))
                  for i, j in zip(ii, jj)])
    assert np.array_equal(c, d)


def test_kway_matches_python_sets():
    rng = np.random.default_rng(11)
    inst = _random_instance(rng, 3000, 30)
    queries = []
    for _ in range(300):
        k = int(rng.integers(1, 9))
        queries.append(rng.choice(inst.n, k, replace=bool(rng.integers(0, 2))).tolist())
    got = oracle.kway_counts(inst.offsets, inst.tids, queries)
    for q, g in zip(queries, got):
        ref = set(inst.tidlist(q[0]).tolist())
        for a in q[1:]:
            ref &= set(inst.tidlist(a).tolist())
        assert g == len(ref)


def test_generators_are_valid_csr():
    for inst in (datagen.workload_instance("bern_m10k_n200"), datagen.zipf_tidlists(100000, 300, 0.02, 5),
                 datagen.pool_tidlists(200, 2**20, 10, 10**5, 3)):
        assert inst.offsets[0] == 0 and (np.diff(inst.offsets.astype(np.int64)) >= 0).all()
        for i in range(inst.n):
            t = inst.tidlist(i).astype(np.int64)
            assert (np.diff(t) > 0).all() and (t < inst.m).all()
    # seeded: the same call gives the same data
    a = datagen.zipf_tidlists(20000, 50, 0.02, 4)
    b = datagen.zipf_tidlists(20000, 50, 0.02, 4)
    assert np.array_equal(a.tids, b.tids) and np.array_equal(a.offsets, b.offsets)
    p = datagen.permutations(1000, 3)
    for t in range(3):
        assert np.array_equal(np.sort(p[t]), np.arange(1000))


def test_kway_elems_matches_python_sets():
    rng = np.random.default_rng(13)
    inst = _random_instance(rng, 2000, 20)
    for _ in range(100):
        q = rng.choice(inst.n, int(rng.integers(1, 6)), replace=False).tolist()
        ref = set(inst.tidlist(q[0]).tolist())
        for a in q[1:]:
            ref &= set(inst.tidlist(a).tolist())
        got = oracle.kway_elems(inst.offsets, inst.tids, q)
        assert got.tolist() == sorted(ref)
