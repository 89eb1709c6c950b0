"""The k-way probe route on d-of-(d+1) BatMaps, restated on the CPU and checked
against the oracle (CPU only).

For K <= d sets of different widths the support kernels may visit only the
nonempty slots of the narrowest BatMap: a slot in table t at byte h holding code
c carries pi_t(x) = ((c - 1) << s) | (h mod r_0), every other set is read at its
own slot for pi_t(x) in table t, and the copy counts where all K codes agree and
t is the smallest table that none of the K missing-table fields names (the
witness, Sec. V).  The claim is that this counts what the cyclic witness scan
counts.  The rule is restated here independently of the CUDA code and compared,
on serial 3-of-4 and 4-of-5 BatMaps built by the oracle's INSERT (also with
forced failures), with the oracle's scan rule (`kway_count`) and, after the
failure correction, with the exact intersection sizes; planted mistakes (no
witness test, the wrong missing-field width, the narrowest set's range for the
others) must fail.
"""
import itertools

import numpy as np
import pytest

import datagen
from oracle import dof_rules as R


def probe_count(bms, r0, s, d, mistake=None):
    """Restatement of the probe route over the K BatMaps `bms` (uint8 arrays of
    widths (d + 1) r_j)."""
    k = len(bms)
    j0 = int(np.argmin([b.size for b in bms]))
    nar = bms[j0].astype(np.int64)
    cm, cb = R.code_max(d), R.code_bits(d)
    if mistake == "field":
        cb -= 1
    h = np.flatnonzero(nar & cm)
    byte = nar[h]
    code = byte & cm
    t = (h // r0) % (d + 1)
    pi = ((code - 1) << s) | (h % r0)
    all_eq = np.ones(h.size, dtype=bool)
    missed = [byte >> cb]
    for j in range(k):
        if j == j0:
            continue
        r = bms[j].size // (d + 1) if mistake != "range" else nar.size // (d + 1)
        y = bms[j].astype(np.int64)[R.slot(t, pi, r, r0, d) % bms[j].size]
        all_eq &= (y & cm) == code
        missed.append(y >> cb)
    if mistake == "witness":
        return int(all_eq.sum())
    wit = np.full(h.size, -1, dtype=np.int64)
    for u in range(d, -1, -1):  # smallest table missed by none
        free = np.ones(h.size, dtype=bool)
        for mf in missed:
            free &= mf != u
        wit[free] = u
    return int((all_eq & (wit == t)).sum())


def _sets(rng, m, dens):
    return [np.flatnonzero(rng.random(m) < p).astype(np.uint32) for p in dens]


@pytest.mark.parametrize("d", [3, 4])
@pytest.mark.parametrize("seed,m,max_loop,c_den", [(0, 4000, 32, 1), (1, 9000, 32, 1), (2, 6000, 1, 2)])
def test_probe_equals_witness_scan_and_intersections(d, seed, m, max_loop, c_den):
    rng = np.random.default_rng(seed)
    dens = [0.6, 0.55, 0.12, 0.1, 0.03, 0.02]  # the first two share a width
    lists = _sets(rng, m, dens)
    base = lists[4]
    lists = [np.union1d(l, base[: base.size // 2]).astype(np.uint32) for l in lists]  # many common elements
    perms = datagen.permutations(m, seed, count=d + 1)
    s = R.shift_bits(m, d=d)
    r0 = 1 << s
    lay = []
    for l in lists:
        r = R.hash_range(l.size, r0, 2, c_den)
        bm, f = R.serial_layout(l, perms, r, r0, s, d, max_loop)
        assert R.check_layout(bm, l, f, perms, r, r0, s, d) == []
        lay.append((bm, f))
    if max_loop == 1:
        assert sum(f.size for _, f in lay) > 0
    sets = [set(l.tolist()) for l in lists]
    widths = set()
    for k in range(2, d + 1):
        for q in itertools.combinations(range(len(lists)), k):
            bms = [lay[i][0] for i in q]
            widths.add(max(b.size for b in bms) // min(b.size for b in bms))
            scan = R.kway_count(bms, r0, d)
            assert probe_count(bms, r0, s, d) == scan, q
            corr = R.correction([lists[i] for i in q], [lay[i][1] for i in q])
            assert scan + corr == len(set.intersection(*[sets[i] for i in q]))
    assert 1 in widths and max(widths) >= 8  # equal widths and skewed ones


@pytest.mark.parametrize("mistake", ["witness", "field", "range"])
def test_planted_mistakes_fail(mistake):
    rng = np.random.default_rng(5)
    m, d = 6000, 4
    lists = _sets(rng, m, [0.5, 0.4, 0.05, 0.03])
    lists = [np.union1d(l, lists[3][:100]).astype(np.uint32) for l in lists]
    perms = datagen.permutations(m, 5, count=d + 1)
    s = R.shift_bits(m, d=d)
    r0 = 1 << s
    bms = [R.serial_layout(l, perms, R.hash_range(l.size, r0), r0, s, d)[0] for l in lists]
    bad = 0
    for k in (3, 4):
        for q in itertools.combinations(range(4), k):
            sub = [bms[i] for i in q]
            bad += probe_count(sub, r0, s, d, mistake) != R.kway_count(sub, r0, d)
    assert bad > 0
