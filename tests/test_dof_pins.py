"""Pins of the d-of-(d+1) BatMap rules (Sec. V generalisation) against things
other than themselves (CPU only), for d = 3 (3-of-4) and d = 4 (4-of-5, a
three-bit missing-table field): the pigeonhole witness property checked
exhaustively, the serial layout's counts against Python set intersections and
the merge oracle, layout validity, planted mistakes, and the Apriori
candidate steps (levels 3 and 4) against brute force."""
import itertools

import numpy as np
import pytest

import datagen
import oracle
from oracle import dof_rules as R


@pytest.mark.parametrize("d", [2, 3, 4])
def test_exactly_one_witness_for_up_to_d_sets(d):
    # every assignment of missing tables to k <= d sets leaves >= 1 common table
    # (pigeonhole), and the rule selects exactly one of them
    for k in range(1, d + 1):
        for missing in itertools.product(range(d + 1), repeat=k):
            common = [t for t in range(d + 1) if t not in missing]
            assert common, (d, missing)
            chosen = [t for t in common if R.witness_table(missing, d) == t]
            assert len(chosen) == 1
    # d + 1 sets can miss every table: no witness, hence k <= d
    assert R.witness_table(list(range(d + 1)), d) is None


def test_slot_rule_needs_equal_nonempty_codes():
    b = R.element_byte(1, 5 << 7, 7)            # missing table 1, code 6
    assert R.slot_counts(0, [b, b, b])
    assert not R.slot_counts(2, [b, b, b])     # table 2 is not the smallest common one
    other = R.element_byte(1, 6 << 7, 7)
    assert not R.slot_counts(0, [b, other, b])
    assert not R.slot_counts(0, [0, 0, 0])     # empty slots never count
    # missing tables {0, 1, 2} leave table 3 as the only witness
    bs = [R.element_byte(u, 9 << 7, 7) for u in (0, 1, 2)]
    assert [R.slot_counts(t, bs) for t in range(4)] == [False, False, False, True]


def test_slot_rule_five_tables():
    # d = 4: three missing-table bits, five code bits
    assert R.missing_bits(4) == 3 and R.code_bits(4) == 5 and R.code_max(4) == 31
    assert R.missing_bits(3) == 2 and R.code_bits(3) == 6
    b = R.element_byte(4, 5 << 7, 7, d=4)        # missing table 4, code 6
    assert b == (4 << 5) | 6
    assert R.slot_counts(0, [b] * 4, d=4) and not R.slot_counts(1, [b] * 4, d=4)
    # four sets missing tables 0..3 leave only table 4
    bs = [R.element_byte(u, 9 << 7, 7, d=4) for u in (0, 1, 2, 3)]
    assert [R.slot_counts(t, bs, d=4) for t in range(5)] == [False] * 4 + [True]
    assert R.shift_bits(31 * 128, d=4) == 7 and R.shift_bits(31 * 128 + 1, d=4) == 8


def test_sizing_boundaries():
    assert R.shift_bits(63 * 128) == 7 and R.shift_bits(63 * 128 + 1) == 8
    assert R.shift_bits(1) == 7 and R.shift_bits(10**6) == 14   # 63 * 2^14 = 1,032,192
    assert R.width_bytes(R.hash_range(2500, 128)) == 4 * 8192
    # codes stay in [1, 63] for every pi in [0, m)
    for m in (100, 8064, 8065, 10**6):
        s = R.shift_bits(m)
        assert int(R.code6(m - 1, s)) <= 63


def _instance(rng, m, n, pmax=0.4):
    lists = [np.flatnonzero(rng.random(m) < rng.uniform(0.02, pmax)).astype(np.uint32) for _ in range(n)]
    return datagen.from_lists(lists, m)


def _layouts(inst, perms, c=2, max_loop=32, d=3):
    s = R.shift_bits(inst.m, d=d)
    r0 = 1 << s
    out = []
    for i in range(inst.n):
        r = R.hash_range(inst.tidlist(i).size, r0, c, 1)
        bm, f = R.serial_layout(inst.tidlist(i), perms, r, r0, s, d, max_loop)
        assert R.check_layout(bm, inst.tidlist(i), f, perms, r, r0, s, d) == []
        out.append((bm, f))
    return out, r0


@pytest.mark.parametrize("d", [3, 4])
@pytest.mark.parametrize("seed", range(6))
def test_serial_layout_counts_match_set_intersections(seed, d):
    rng = np.random.default_rng(seed)
    inst = _instance(rng, int(rng.integers(200, 3000)), 6)
    perms = datagen.permutations(inst.m, seed, count=d + 1)
    lay, r0 = _layouts(inst, perms, d=d)
    sets = [set(inst.tidlist(i).tolist()) for i in range(inst.n)]
    for k in range(1, d + 1):
        for q in itertools.combinations(range(inst.n), k):
            exact = len(set.intersection(*[sets[i] for i in q]))
            got = R.kway_count([lay[i][0] for i in q], r0, d) + \
                R.correction([inst.tidlist(i) for i in q], [lay[i][1] for i in q])
            assert got == exact
    # and the merge oracle agrees on the same queries
    qs = [list(q) for q in itertools.combinations(range(inst.n), d)]
    ref = oracle.kway_counts(inst.offsets, inst.tids, qs)
    for q, v in zip(qs, ref):
        assert v == len(set.intersection(*[sets[i] for i in q]))


@pytest.mark.parametrize("d", [3, 4])
def test_forced_failures_are_corrected(d):
    rng = np.random.default_rng(7)
    inst = _instance(rng, 2000, 5, pmax=0.6)
    perms = datagen.permutations(inst.m, 3, count=d + 1)
    lay, r0 = _layouts(inst, perms, c=1, max_loop=1, d=d)     # load d/(d+1) per table, one round
    assert sum(f.size for _, f in lay) > 0
    sets = [set(inst.tidlist(i).tolist()) for i in range(inst.n)]
    for q in itertools.combinations(range(inst.n), d):
        got = R.kway_count([lay[i][0] for i in q], r0, d) + \
            R.correction([inst.tidlist(i) for i in q], [lay[i][1] for i in q])
        assert got == len(set.intersection(*[sets[i] for i in q]))


def test_planted_mistakes_are_caught():
    rng = np.random.default_rng(3)
    inst = _instance(rng, 1500, 4)
    perms = datagen.permutations(inst.m, 1, count=4)
    lay, r0 = _layouts(inst, perms)
    sets = [set(inst.tidlist(i).tolist()) for i in range(inst.n)]
    q = (0, 1, 2)
    exact = len(set.intersection(*[sets[i] for i in q]))
    corr = R.correction([inst.tidlist(i) for i in q], [lay[i][1] for i in q])
    # a wrong missing-table field in one set changes the count or the layout check
    bad = lay[1][0].copy()
    nz = np.flatnonzero(bad)
    bad[nz] = (bad[nz] & R.CODE_MAX) | (((bad[nz] >> R.CODE_BITS) + 1) % 4 << R.CODE_BITS)
    assert R.kway_count([lay[0][0], bad, lay[2][0]], r0) + corr != exact
    # counting every common table (no witness rule) over-counts
    W = max(lay[i][0].size for i in q)
    cols = [np.tile(lay[i][0], W // lay[i][0].size) & R.CODE_MAX for i in q]
    every = int(((cols[0] == cols[1]) & (cols[1] == cols[2]) & (cols[0] != 0)).sum())
    assert exact > 0 and every + corr > exact


@pytest.mark.parametrize("seed", range(5))
def test_triple_candidates_match_bruteforce(seed):
    rng = np.random.default_rng(seed)
    n = 14
    allp = [(i, j) for i in range(n) for j in range(i + 1, n)]
    keep = [p for p in allp if rng.random() < 0.5]
    a = R.triple_candidates(keep)
    b = R.triple_candidates_bruteforce(n, keep)
    assert np.array_equal(a, b)
    if a.shape[0] > 1:
        key = (a[:, 0].astype(np.int64) * n + a[:, 1]) * n + a[:, 2]
        assert (np.diff(key) > 0).all()


def test_frequent_triples_by_brute_force():
    # Apriori level 3 on a tiny instance equals scanning every triple
    rng = np.random.default_rng(5)
    inst = _instance(rng, 400, 10, pmax=0.5)
    s = 12
    sets = [set(inst.tidlist(i).tolist()) for i in range(inst.n)]
    pairs = oracle.pairs_threshold(inst.offsets, inst.tids, s)[:, :2]
    cand = R.triple_candidates(pairs)
    sup = oracle.kway_counts(inst.offsets, inst.tids, cand.tolist())
    got = {tuple(c) for c, v in zip(cand.tolist(), sup) if v >= s}
    want = {q for q in itertools.combinations(range(inst.n), 3)
            if len(set.intersection(*[sets[i] for i in q])) >= s}
    assert got == want


def test_planted_mistakes_are_caught_five_tables():
    rng = np.random.default_rng(4)
    inst = _instance(rng, 3000, 5, pmax=0.7)
    perms = datagen.permutations(inst.m, 2, count=5)
    lay, r0 = _layouts(inst, perms, d=4)
    sets = [set(inst.tidlist(i).tolist()) for i in range(inst.n)]
    q = (0, 1, 2, 3)
    exact = len(set.intersection(*[sets[i] for i in q]))
    corr = R.correction([inst.tidlist(i) for i in q], [lay[i][1] for i in q])
    assert R.kway_count([lay[i][0] for i in q], r0, 4) + corr == exact
    cm, cb = R.code_max(4), R.code_bits(4)
    # one set claiming to miss table 0 everywhere moves witnesses off their tables
    bad = lay[2][0].copy()
    nz = np.flatnonzero(bad)
    bad[nz] = bad[nz] & cm
    assert R.kway_count([lay[0][0], lay[1][0], bad, lay[3][0]], r0, 4) + corr != exact
    # reading a five-table layout with the four-table fields (d = 3) miscounts
    assert R.kway_count([lay[i][0] for i in q], r0, 3) + corr != exact
    W = max(lay[i][0].size for i in q)
    cols = [np.tile(lay[i][0], W // lay[i][0].size) & cm for i in q]
    every = int(((cols[0] == cols[1]) & (cols[1] == cols[2]) & (cols[2] == cols[3]) & (cols[0] != 0)).sum())
    assert exact > 0 and every + corr > exact


@pytest.mark.parametrize("seed", range(5))
def test_quadruple_candidates_match_bruteforce(seed):
    rng = np.random.default_rng(seed)
    n = 11
    allt = list(itertools.combinations(range(n), 3))
    keep = [t for t in allt if rng.random() < 0.6]
    a = R.quadruple_candidates(keep)
    b = R.quadruple_candidates_bruteforce(n, keep)
    assert np.array_equal(a, b)
    if a.shape[0] > 1:
        key = ((a[:, 0].astype(np.int64) * n + a[:, 1]) * n + a[:, 2]) * n + a[:, 3]
        assert (np.diff(key) > 0).all()


def test_frequent_quadruples_by_brute_force():
    # Apriori level 4 on a tiny instance equals scanning every 4-subset
    rng = np.random.default_rng(6)
    inst = _instance(rng, 300, 9, pmax=0.7)
    s = 20
    sets = [set(inst.tidlist(i).tolist()) for i in range(inst.n)]
    pairs = oracle.pairs_threshold(inst.offsets, inst.tids, s)[:, :2]
    cand3 = R.triple_candidates(pairs)
    sup3 = oracle.kway_counts(inst.offsets, inst.tids, cand3.tolist())
    trip = cand3[sup3 >= s]
    cand4 = R.quadruple_candidates(trip)
    sup4 = oracle.kway_counts(inst.offsets, inst.tids, cand4.tolist())
    got = {tuple(c) for c, v in zip(cand4.tolist(), sup4) if v >= s}
    want = {q for q in itertools.combinations(range(inst.n), 4)
            if len(set.intersection(*[sets[i] for i in q])) >= s}
    assert got == want and len(want) > 0
