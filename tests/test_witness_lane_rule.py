"""The lane arithmetic of the grouped triple-support kernel, restated in
Python, against the oracle's witness rule (CPU only).

`k_witness_group` reduces the BatMaps of a frequent pair (a, b) to an
expected byte, a mask and a validity flag per lane of a 32-bit word, then tests
each candidate c with two masked XORs, an add and an and-not (Sec. V
generalisation, 3-of-4 tables).  Here the same steps run on Python integers
with four independent lanes per word, and every combination of codes (empty,
equal, different) and missing tables (any table but the slot's own) of three
sets is compared with `oracle.dof_rules.slot_counts` in each table."""
import itertools

import numpy as np

from oracle import dof_rules as R

M32 = 0xFFFFFFFF
C6, B6, H7, L7, K7 = 0x3F3F3F3F, 0x40404040, 0x80808080, 0x7E7E7E7E, 0x7F7F7F7F


def pair_rule(T, xa, xb):
    """(pat, msk, msk7, val) of a pair's word for a slot of table T.  A copy
    in table T never names T as its missing table, so each table sees three
    missing tables and the kernel specialises the reduction per table."""
    x = xa ^ xb
    za = xa & C6
    ne = ((x & C6) * 2 + L7) & M32   # bit 7: codes differ
    nz = (za * 2 + L7) & M32         # bit 7: not empty
    if T == 0:
        return za, C6, C6, nz & ~ne & H7 & M32
    if T == 1:
        c7 = xa & xb & H7            # both miss 2 or 3: c must miss 0 (high bit 0)
        return za, C6 | c7, C6, nz & ~ne & H7 & M32
    if T == 2:
        c7 = (xa | xb | (~(x << 1) & M32)) & H7       # not free
        sel = xa >> 1
        low = (sel & xb) | (~sel & M32 & xa)
        msk7 = C6 | (c7 >> 1)
        return (za | (~low & M32 & B6), msk7 | c7, msk7,
                nz & ~(ne | (xa & xb)) & H7 & M32)
    pat = (xa & C6) | (~xa & ~xb & ~C6 & M32)
    return pat, M32, 0x7F7F7F7F, nz & ~ne & (x | ((x << 1) & M32)) & H7 & M32


def candidate_ok(T, xa, xb, xc):
    """Bit 7 of each lane set iff c completes a counted slot."""
    pat, msk, msk7, val = pair_rule(T, xa, xb)
    if T == 0:
        return val & ~((((xc ^ xa) & C6) + K7) & M32) & M32
    d = (xc ^ pat) & msk
    d7 = (xc ^ pat) & msk7
    return val & ~(((d7 + K7) & M32) | d) & M32


def lane_bytes(T):
    """Every byte a slot of table T can hold, with two codes (and empty)."""
    out = [0]
    for code in (1, 2):
        out += [(u << 6) | code for u in range(4) if u != T]
    return out


def pack(bs):
    return sum(int(b) << (8 * i) for i, b in enumerate(bs))


def test_lane_rule_matches_witness_rule_exhaustively():
    rng = np.random.default_rng(3)
    for T in range(4):
        combos = list(itertools.product(lane_bytes(T), repeat=3))
        want = np.array([R.slot_counts(T, c) for c in combos])
        assert want.any() and not want.all()
        # four independent combinations per word, in shuffled lane positions
        order = np.concatenate([rng.permutation(len(combos)) for _ in range(4)])
        order = np.concatenate([order, order[: (-order.size) % 4]])
        for w in range(0, order.size, 4):
            idx = order[w:w + 4]
            xa, xb, xc = (pack([combos[i][s] for i in idx]) for s in range(3))
            ok = candidate_ok(T, xa, xb, xc)
            assert ok & ~H7 == 0
            got = [(ok >> (8 * lane + 7)) & 1 for lane in range(4)]
            assert got == [int(want[i]) for i in idx], (T, [combos[i] for i in idx])


def test_lane_rule_detects_a_dropped_constraint():
    # with table 2's constraint dropped, a and b missing tables 0 and 1 leave
    # table 3 to c only if c misses table 2; the rule above must reject c
    # missing table 0 (then table 2 is the witness)
    a, b = (0 << 6) | 1, (1 << 6) | 1
    c_ok, c_bad = (2 << 6) | 1, (0 << 6) | 1
    assert R.slot_counts(3, [a, b, c_ok]) and not R.slot_counts(3, [a, b, c_bad])
    assert candidate_ok(3, a, b, c_ok) == 0x80
    assert candidate_ok(3, a, b, c_bad) == 0
