"""Pins of the CPU restatement of the BatMap rules (oracle/batmap_rules.py).

Each rule is checked against what the paper prints or what mathematics fixes:
* sizing against the worked example of Sec. IV-A (|S| = 2500 -> 3 * 2^13 B);
* the indicator rule against Fig. 3 and the claim that every combination of
  assignments counts the common element exactly once (Sec. II);
* the 2-of-3 property of Fig. 2;
* the counting rule against the paper's SWAR formula (Sec. III-A), exhaustively
  over all byte pairs in every lane;
* the serial INSERT build + counting + failure correction against the merge
  oracle (exact), including builds forced to fail often;
* the layout checker accepts valid layouts and rejects mutated ones;
* planted mistakes in the rules (a flipped indicator, a wrong wrap, a dropped
  +1 in the code) are caught by these pins.
"""
import os

import numpy as np
import pytest

import datagen
import oracle
from oracle import batmap_rules as R

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kv(name):
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            out[k] = float(v)
    return out


def _rows(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append(line.split())
    return rows


# ---- sizing ---------------------------------------------------------------

def test_width_of_worked_example():
    g = _kv("throughput_example.txt")
    # 10^7 total items over n = 4000 items at p = 5%: m = 10^7 / (0.05 * 4000) = 50,000
    m = 50_000
    s = R.shift_bits(m)
    r0 = 1 << s
    r = R.hash_range(int(g["set_size"]), r0)
    assert R.width_bytes(r) == int(g["width_bytes"]) == 3 * 2**13
    # logical bytes / time reproduces the printed 36.2 Gbyte/s (Gbyte = 10^9 B)
    gbs = g["n"] ** 2 * R.width_bytes(r) / g["seconds"] / 1e9
    assert abs(gbs - g["gbyte_per_s"]) < 0.1
    eps = g["n"] ** 2 * g["set_size"] / g["seconds"]
    assert abs(eps - g["elements_per_s"]) / g["elements_per_s"] < 0.01


def test_shift_bits_compression_floor():
    # Sec. III-A: after shifting s bits, 7 bits remain: 2^s >= (m+1)/128.  With
    # 0-based values and code 0 reserved for the empty slot: m <= 127 * 2^s.
    for m in [1, 127 * 128, 127 * 128 + 1, 10_000, 1_000_000, 4_194_304, 2**26]:
        s = R.shift_bits(m, min_shift=0)
        assert m <= 127 * 2**s
        assert s == 0 or m > 127 * 2 ** (s - 1)
        assert 2**s >= (m + 1) / 128 - 1e-9 or m <= 127 * 2**s
        codes = R.code7(np.arange(m)[-1:], s)
        assert 1 <= int(codes[0]) <= 127
    assert R.shift_bits(10_000) == 7 and R.shift_bits(1_000_000) == 13
    assert R.shift_bits(4_194_304) == 16


def test_hash_range_rule():
    r0 = 128
    assert R.hash_range(0, r0) == r0
    assert R.hash_range(64, r0) == 128
    assert R.hash_range(65, r0) == 256
    assert R.hash_range(500, r0) == 1024 and R.hash_range(513, r0) == 2048
    for size in range(1, 5000, 37):
        r = R.hash_range(size, 1)
        assert r >= 2 * size and r < 4 * size and r & (r - 1) == 0


# ---- layout hash and wrap -------------------------------------------------

def test_slot_is_bijective_and_wraps():
    r0, s = 128, 7
    for r in (128, 256, 1024):
        seen = set()
        for t in range(3):
            for pi in range(r):
                p = int(R.slot(t, pi, r, r0))
                assert 0 <= p < 3 * r
                seen.add(p)
                assert R.table_of_slot(p, r0) == t
        assert len(seen) == 3 * r
    # for r_i | r_j the slot in B_i is the slot in B_j modulo |B_i| (Fig. 1 bottom)
    rng = np.random.default_rng(0)
    pis = rng.integers(0, 127 * 2**s, 2000)
    for ri, rj in ((128, 256), (128, 1024), (256, 2048)):
        for t in range(3):
            assert (R.slot(t, pis, ri, r0) == R.slot(t, pis, rj, r0) % (3 * ri)).all()


def test_decode_inverts_slot_and_code():
    r0, s = 256, 8
    rng = np.random.default_rng(1)
    pis = rng.integers(0, 127 * 2**s, 5000)
    for r in (256, 4096):
        for t in range(3):
            pos = R.slot(t, pis, r, r0)
            byte = R.code7(pis, s)
            assert (R.decode_pi(pos, byte, r0, s) == pis).all()


# ---- indicator rule (Fig. 3) ----------------------------------------------

def _fig3():
    rows = _rows("fig3_indicator.txt")
    out = {}
    for a, t, p, b in rows:
        out.setdefault(a, []).append((int(t) - 1, int(p), int(b)))
    return out


def test_indicator_direction_matches_fig3():
    # the bit is 1 on the copy in the cyclic successor of its twin's table
    for occ in _fig3().values():
        (t1, _, b1), (t2, _, b2) = occ
        succ = t1 if (t2 + 1) % 3 == t1 else t2
        for t, _, b in occ:
            assert b == (1 if t == succ else 0)


def _single_element_batmap(tables, r, r0, s, pi):
    bm = np.zeros(3 * r, dtype=np.uint8)
    ta, tb = tables
    succ = ta if (tb + 1) % 3 == ta else tb
    for t in tables:
        bm[int(R.slot(t, pi[t], r, r0))] = ((1 if t == succ else 0) << 7) | int(R.code7(pi[t], s))
    return bm


@pytest.mark.parametrize("ri,rj", [(128, 128), (128, 256), (256, 1024)])
def test_every_assignment_pair_counts_once(ri, rj):
    # Sec. II: whether x sits in the same two tables in both BatMaps or overlaps
    # in one table only, it is counted exactly once.
    r0, s = 128, 7
    rng = np.random.default_rng(ri + rj)
    assignments = [(0, 1), (1, 2), (2, 0)]
    for _ in range(30):
        pi = rng.integers(0, 127 * 2**s, 3)
        for a in assignments:
            for b in assignments:
                bi = _single_element_batmap(a, ri, r0, s, pi)
                bj = _single_element_batmap(b, rj, r0, s, pi)
                assert R.batmap_pair_count(bi, bj) == 1


def test_empty_slots_never_count():
    # the bottom byte 0x00 never matches an element (code >= 1) nor another bottom
    elems = np.array([b for b in range(256) if b & 0x7F != 0])
    assert R.count_rule(np.zeros(elems.size, np.int64), elems).sum() == 0
    assert R.count_rule(0, 0) == 0


# ---- Fig. 2 ---------------------------------------------------------------

def test_fig2_is_a_2_of_3_assignment():
    rows = _rows("fig2_assignment.txt")
    per = {}
    slots = {}
    for e, t, p, st in rows:
        per.setdefault(e, []).append((int(t), int(p), int(st)))
        if int(st):
            key = (int(t), int(p))
            assert key not in slots, "two elements stored in one slot"
            slots[key] = e
    for e, occ in per.items():
        assert len(occ) == 3 and sum(st for _, _, st in occ) == 2
        assert sorted(t for t, _, _ in occ) == [1, 2, 3]


# ---- SWAR formula vs counting rule (Sec. III-A) ---------------------------

def test_swar_exhaustive_byte_pairs_every_lane():
    xb, yb = np.meshgrid(np.arange(256), np.arange(256), indexing="ij")
    xb, yb = xb.ravel(), yb.ravel()
    ref = R.count_rule(xb, yb)
    rng = np.random.default_rng(2)
    for lane in range(4):
        # other lanes random, so borrows across lanes would show
        fx = rng.integers(0, 2**32, xb.size, dtype=np.uint64)
        fy = rng.integers(0, 2**32, xb.size, dtype=np.uint64)
        mask = np.uint64(0xFF << (8 * lane))
        x = (fx & ~mask) | (xb.astype(np.uint64) << np.uint64(8 * lane))
        y = (fy & ~mask) | (yb.astype(np.uint64) << np.uint64(8 * lane))
        others = np.zeros(xb.size, dtype=np.int64)
        for l2 in range(4):
            if l2 != lane:
                others += R.count_rule((x >> np.uint64(8 * l2)) & np.uint64(0xFF),
                                       (y >> np.uint64(8 * l2)) & np.uint64(0xFF))
        assert np.array_equal(R.swar_count(x, y), ref + others)


def test_swar_random_words():
    rng = np.random.default_rng(3)
    x = rng.integers(0, 2**32, 200000, dtype=np.uint64)
    y = x.copy()
    flip = rng.random(x.size) < 0.5
    y[flip] = rng.integers(0, 2**32, int(flip.sum()), dtype=np.uint64)
    # force many equal-code lanes
    y ^= rng.integers(0, 2, x.size, dtype=np.uint64) * np.uint64(0x80008000)
    ref = sum(R.count_rule((x >> np.uint64(8 * l)) & np.uint64(0xFF),
                           (y >> np.uint64(8 * l)) & np.uint64(0xFF)) for l in range(4))
    assert np.array_equal(R.swar_count(x, y), ref)


# ---- the whole method on the CPU vs the merge oracle ----------------------

def _serial_instance(inst, perms, c_num=2, c_den=1, max_loop=32, min_shift=7):
    s = R.shift_bits(inst.m, min_shift)
    r0 = 1 << s
    bms, fs, rs = [], [], []
    for i in range(inst.n):
        r = R.hash_range(len(inst.tidlist(i)), r0, c_num, c_den)
        bm, f = R.serial_layout(inst.tidlist(i), perms, r, r0, s, max_loop)
        bms.append(bm)
        fs.append(f)
        rs.append(r)
    return bms, fs, rs, r0, s


def _serial_counts(inst, bms, fs):
    n = inst.n
    out = []
    for i in range(n):
        for j in range(i + 1, n):
            c = R.batmap_pair_count(bms[i], bms[j])
            c += R.correction(inst.tidlist(i), inst.tidlist(j), fs[i], fs[j])
            out.append(c)
    return np.array(out, dtype=np.int64)


@pytest.mark.parametrize("seed,c_num,c_den,max_loop", [
    (0, 2, 1, 32), (1, 2, 1, 32), (2, 1, 1, 32), (3, 2, 1, 1), (4, 1, 2, 2), (5, 1, 4, 1)])
def test_serial_method_matches_oracle(seed, c_num, c_den, max_loop):
    rng = np.random.default_rng(seed)
    m = int(rng.integers(200, 3000))
    n = int(rng.integers(3, 9))
    lists = [np.flatnonzero(rng.random(m) < rng.uniform(0.0, 0.4)).astype(np.uint32)
             for _ in range(n)]
    inst = datagen.from_lists(lists, m)
    perms = datagen.permutations(m, seed)
    bms, fs, rs, r0, s = _serial_instance(inst, perms, c_num, c_den, max_loop)
    for i in range(n):
        assert R.check_layout(bms[i], inst.tidlist(i), fs[i], perms, rs[i], r0, s) == []
    ref = oracle.pairs_full(inst.offsets, inst.tids).astype(np.int64)
    assert np.array_equal(_serial_counts(inst, bms, fs), ref)
    if c_num * 4 <= c_den * 1 or max_loop == 1:
        # the forced-failure settings really exercise the correction
        assert sum(f.size for f in fs) > 0


def test_failure_rate_small_at_load_one_third():
    # Sec. II-B: with r >= (2 + eps) |S| failures are rare.
    m = 20000
    perms = datagen.permutations(m, 5)
    rng = np.random.default_rng(5)
    total = failed = 0
    for _ in range(6):
        tids = np.flatnonzero(rng.random(m) < 0.05).astype(np.uint32)
        r = R.hash_range(tids.size, 128)
        _, f = R.serial_layout(tids, perms, r, 128, R.shift_bits(m), 32)
        total += tids.size
        failed += f.size
    assert failed <= 0.01 * total


# ---- the layout checker ---------------------------------------------------

def test_checker_rejects_mutations():
    m = 3000
    rng = np.random.default_rng(9)
    tids = np.flatnonzero(rng.random(m) < 0.1).astype(np.uint32)
    perms = datagen.permutations(m, 9)
    s = R.shift_bits(m)
    r0 = 1 << s
    r = R.hash_range(tids.size, r0)
    bm, f = R.serial_layout(tids, perms, r, r0, s)
    assert R.check_layout(bm, tids, f, perms, r, r0, s) == []
    occupied = np.flatnonzero(bm)
    k = int(occupied[len(occupied) // 2])
    bad = bm.copy(); bad[k] ^= 0x80                      # flipped indicator
    assert R.check_layout(bad, tids, f, perms, r, r0, s)
    bad = bm.copy(); bad[k] = (bad[k] & 0x80) | ((bad[k] & 0x7F) % 127 + 1)  # wrong code
    assert R.check_layout(bad, tids, f, perms, r, r0, s)
    bad = bm.copy(); bad[k] = 0                          # lost copy
    assert R.check_layout(bad, tids, f, perms, r, r0, s)
    empty = np.flatnonzero(bm == 0)
    bad = bm.copy(); bad[int(empty[0])] = 0x05           # stray byte
    assert R.check_layout(bad, tids, f, perms, r, r0, s)
    x = int(tids[0])                                     # claims failure but stored
    assert R.check_layout(bm, tids, np.array([x], np.uint32), perms, r, r0, s)


# ---- planted mistakes are caught ------------------------------------------

def test_planted_mistakes_are_caught(monkeypatch):
    m = 1500
    rng = np.random.default_rng(12)
    lists = [np.flatnonzero(rng.random(m) < 0.2).astype(np.uint32) for _ in range(4)]
    inst = datagen.from_lists(lists, m)
    perms = datagen.permutations(m, 12)
    ref = oracle.pairs_full(inst.offsets, inst.tids).astype(np.int64)

    def run():
        bms, fs, rs, r0, s = _serial_instance(inst, perms)
        return np.array_equal(_serial_counts(inst, bms, fs), ref)

    assert run()
    orig_rule = R.count_rule
    # 1) indicator ignored: same-two-table overlaps count twice
    monkeypatch.setattr(R, "count_rule",
                        lambda a, b: ((np.asarray(a) & 0x7F) == (np.asarray(b) & 0x7F))
                        & ((np.asarray(a) | np.asarray(b)) != 0))
    assert not run()
    monkeypatch.setattr(R, "count_rule", orig_rule)
    # 2) code without the +1: empty slots collide with code 0
    orig_code = R.code7
    monkeypatch.setattr(R, "code7", lambda pi, s: np.asarray(pi, dtype=np.int64) >> s)
    assert not run()
    monkeypatch.setattr(R, "code7", orig_code)
    # 3) wrap by the wrong block size in the different-size comparison
    orig_cnt = R.batmap_pair_count

    def bad_count(bi, bj):
        big, small = (bi, bj) if bi.size >= bj.size else (bj, bi)
        rep = np.resize(small[::-1], big.size)
        return int(R.count_rule(big, rep).sum())
    monkeypatch.setattr(R, "batmap_pair_count", bad_count)
    assert not run()
    monkeypatch.setattr(R, "batmap_pair_count", orig_cnt)
    assert run()
