"""The probe route's slot arithmetic, restated on the CPU and checked against
the oracle (CPU only).

For a pair whose BatMaps differ in width, the compare kernels may visit only
the nonempty slots of the narrower BatMap: a slot in table t at byte h holding
code c carries pi_t(x) = ((c - 1) << s) | (h mod r_0) (Sec. III-A: the code is
the bits of pi_t(x) above s, the slot the bits below), and the wider BatMap is
read at its own slot for pi_t(x) in the same table.  The counting rule of
Sec. II / Fig. 3 is then applied to that byte pair.  The kernel's claim is that
this adds exactly what the cyclic scan of Fig. 1 adds.  Here the rule is
restated independently of the CUDA code and compared with the oracle's scan
(batmap_pair_count) and, after the failure correction, with the merge oracle,
on serial BatMaps built by the oracle's INSERT; planted mistakes in the
restatement (the wrong table, no indicator test, the narrow set's range in
place of the wide one's) must fail.
"""
import numpy as np
import pytest

import datagen
import oracle
from oracle import batmap_rules as R


def probe_count(b_narrow, b_wide, r_wide, r0, s, mistake=None):
    """Restatement of the probe route: one byte read in the wide BatMap per
    nonempty slot of the narrow one."""
    h = np.flatnonzero(b_narrow & 0x7F).astype(np.int64)
    byte = b_narrow[h].astype(np.int64)
    t = (h // r0) % 3
    pi = (((byte & 0x7F) - 1) << s) | (h % r0)
    if mistake == "table":
        t = (t + 1) % 3
    r = r_wide if mistake != "range" else (b_narrow.size // 3)
    hj = 3 * r0 * ((pi % r) // r0) + t * r0 + (pi % r0)
    y = b_wide[hj % b_wide.size].astype(np.int64)
    if mistake == "indicator":
        return int(((byte & 0x7F) == (y & 0x7F)).sum())
    return int(R.count_rule(byte, y).sum())


def _pair(rng, m, p_narrow, p_wide, perms, max_loop=32, c_den=1):
    s = R.shift_bits(m)
    r0 = 1 << s
    a = np.flatnonzero(rng.random(m) < p_narrow).astype(np.uint32)
    b = np.flatnonzero(rng.random(m) < p_wide).astype(np.uint32)
    # force a large common part so that every table and both indicators occur
    b = np.union1d(b, a[: a.size // 2]).astype(np.uint32)
    ra, rb = R.hash_range(a.size, r0, 2, c_den), R.hash_range(b.size, r0, 2, c_den)
    ba, fa = R.serial_layout(a, perms, ra, r0, s, max_loop)
    bb, fb = R.serial_layout(b, perms, rb, r0, s, max_loop)
    return a, b, ba, bb, fa, fb, ra, rb, r0, s


@pytest.mark.parametrize("seed,m,pn,pw,max_loop,c_den", [
    (0, 3000, 0.02, 0.6, 32, 1), (1, 20000, 0.01, 0.5, 32, 1), (2, 5000, 0.05, 0.9, 32, 1),
    (3, 8000, 0.01, 0.3, 1, 2), (4, 40000, 0.003, 0.4, 32, 1), (5, 2000, 0.3, 0.3, 32, 1)])
def test_probe_equals_scan_and_merge(seed, m, pn, pw, max_loop, c_den):
    rng = np.random.default_rng(seed)
    perms = datagen.permutations(m, seed)
    a, b, ba, bb, fa, fb, ra, rb, r0, s = _pair(rng, m, pn, pw, perms, max_loop, c_den)
    assert rb >= ra
    scan = R.batmap_pair_count(ba, bb)
    assert probe_count(ba, bb, rb, r0, s) == scan
    merge = int(oracle.pairs_list(datagen.from_lists([a, b], m).offsets,
                                  datagen.from_lists([a, b], m).tids,
                                  np.array([0]), np.array([1]))[0])
    assert scan + R.correction(a, b, fa, fb) == merge
    if max_loop == 1:
        assert fa.size + fb.size > 0  # the forced-failure case really fails insertions


def test_width_ratios_cover_the_route():
    # the same identity at every width ratio 1 .. 2^6 (the route's threshold range)
    rng = np.random.default_rng(11)
    m = 60000
    perms = datagen.permutations(m, 11)
    ratios = set()
    for pw in (0.002, 0.004, 0.01, 0.03, 0.06, 0.12, 0.25):
        a, b, ba, bb, fa, fb, ra, rb, r0, s = _pair(rng, m, 0.002, pw, perms)
        ratios.add(rb // ra)
        assert probe_count(ba, bb, rb, r0, s) == R.batmap_pair_count(ba, bb)
    assert {1, 8, 32, 64} <= ratios


@pytest.mark.parametrize("mistake", ["table", "indicator", "range"])
def test_planted_mistakes_fail(mistake):
    rng = np.random.default_rng(7)
    m = 20000
    perms = datagen.permutations(m, 7)
    bad = 0
    for _ in range(4):
        a, b, ba, bb, fa, fb, ra, rb, r0, s = _pair(rng, m, 0.01, 0.5, perms)
        bad += probe_count(ba, bb, rb, r0, s, mistake) != R.batmap_pair_count(ba, bb)
    assert bad > 0
