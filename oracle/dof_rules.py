"""d-of-(d+1) BatMaps restated on the CPU -- TEST INFRASTRUCTURE ONLY.

Plain Python / numpy, sharing no code with the CUDA path.  Only tests/,
__graft_entry__.smoke() and bench.py's CPU legs may use it.

The paper closes (Sec. V) with a generalisation of BatMaps that keeps every
element in d of d+1 hashed tables, so that the sets of any itemset of size up
to d share at least one table in which all of them hold the element: d+1
tables, each set missing the element in at most one of them, k <= d sets
miss at most k of the d+1 tables (pigeonhole).  The paper gives no format and
no rule for counting every common element exactly once.  The readings used
here (each also listed in the design notes of the repository):

  * layout as in Sec. III-A with d+1 tables instead of 3: block size
    (d+1) r_0, slot h_t(x) = (d+1) r_0 floor((pi_t(x) mod r) / r_0)
    + (pi_t(x) mod r_0) + t r_0, width (d+1) r bytes, r chosen as for d = 2;
  * an 8-bit slot holds the MISSING table of the element (the one table
    without a copy) in its top bits and the code (pi_t(x) >> s) + 1 in the
    low bits, 0x00 = empty: two missing-table bits and six code bits for
    d = 3 (s the smallest shift with m <= 63 * 2^s), three and five for
    d = 4 (m <= 31 * 2^s);
  * witness rule: for an intersection of k <= d sets, the copies in table t
    count iff the codes agree, the slot is not empty, and t is the SMALLEST
    table not missed by any of the k sets -- a function of t and the k
    stored missing-table fields only, true for exactly one table;
  * placement: the paper's INSERT (Sec. II-A) with d insertions per element,
    pushing through tables 0, 1, .., d cyclically; an element left with
    fewer than d copies is deleted and reported failed (F_i);
  * correction of a k-set intersection: the common elements that failed in
    at least one of the k sets.
"""
from __future__ import annotations

import itertools

import numpy as np

EMPTY = -1
D = 3              # the default: 3-of-4 BatMaps
CODE_BITS = 6      # code bits of the d = 3 format
CODE_MAX = (1 << CODE_BITS) - 1   # 63


def missing_bits(d: int) -> int:
    """Bits of the missing-table field: tables 0..d (2 for d = 3, 3 for d = 4)."""
    return max(2, int(d).bit_length())


def code_bits(d: int) -> int:
    return 8 - missing_bits(d)


def code_max(d: int) -> int:
    return (1 << code_bits(d)) - 1


# ---- sizing ----------------------------------------------------------------

def shift_bits(m: int, min_shift: int = 7, d: int = D) -> int:
    """Smallest s >= min_shift with m <= code_max(d) * 2^s (codes 1..code_max, 0 = empty)."""
    s = min_shift
    while m > code_max(d) * (1 << s):
        s += 1
    return s


def hash_range(size: int, r0: int, c_num: int = 2, c_den: int = 1) -> int:
    """Smallest power of two >= c |S_i|, at least r_0 (the d = 2 rule)."""
    need = -(-c_num * max(int(size), 1) // c_den)
    r = 1
    while r < need:
        r <<= 1
    return max(r, r0)


def width_bytes(r: int, d: int = D) -> int:
    return (d + 1) * r


def slot(t: int, pi, r: int, r0: int, d: int = D):
    pi = np.asarray(pi, dtype=np.int64)
    return (d + 1) * r0 * ((pi % r) // r0) + (pi % r0) + t * r0


def table_of_slot(pos, r0: int, d: int = D):
    return (np.asarray(pos, dtype=np.int64) % ((d + 1) * r0)) // r0


def code6(pi, s: int):
    return (np.asarray(pi, dtype=np.int64) >> s) + 1


def element_byte(missing: int, pi: int, s: int, d: int = D) -> int:
    return (int(missing) << code_bits(d)) | int(code6(pi, s))


# ---- the witness rule -----------------------------------------------------

def witness_table(missing, d: int = D):
    """The smallest table index not missed by any of the sets (None if all are)."""
    free = sorted(set(range(d + 1)) - set(int(x) for x in missing))
    return free[0] if free else None


def slot_counts(t: int, bytes_k, d: int = D) -> bool:
    """Does table t's slot holding bytes b_1..b_k count one common element?"""
    cm, cb = code_max(d), code_bits(d)
    codes = [int(b) & cm for b in bytes_k]
    if codes[0] == 0 or any(c != codes[0] for c in codes):
        return False
    return witness_table([int(b) >> cb for b in bytes_k], d) == t


def kway_count(bms, r0: int, d: int = D) -> int:
    """Witness count over k BatMaps (uint8 arrays of widths (d+1) r_i); the
    narrower ones are read cyclically against the widest (Fig. 1 rule)."""
    W = max(b.size for b in bms)
    if any(b.size == 0 for b in bms):
        return 0
    cols = [np.tile(b, W // b.size) for b in bms]
    tab = table_of_slot(np.arange(W), r0, d)
    stacked = np.stack([c.astype(np.int64) for c in cols])
    codes = stacked & code_max(d)
    equal = (codes == codes[0]).all(axis=0) & (codes[0] != 0)
    total = 0
    for w in np.flatnonzero(equal):
        if witness_table(stacked[:, w] >> code_bits(d), d) == tab[w]:
            total += 1
    return total


# ---- serial INSERT with d copies (Sec. II-A generalised) -------------------

class SerialBatMapD:
    """One set's d-of-(d+1) tables; A[t][h] holds a tid or EMPTY, h = pi_t(x) mod r."""

    def __init__(self, r: int, perms: np.ndarray, d: int = D, max_loop: int = 32):
        self.r, self.perms, self.d, self.max_loop = r, perms, d, max_loop
        self.A = np.full((d + 1, r), EMPTY, dtype=np.int64)

    def h(self, t: int, x: int) -> int:
        return int(self.perms[t][x]) % self.r

    def insert(self, tau: int) -> int:
        for _ in range(self.max_loop):
            for t in range(self.d + 1):
                p = self.h(t, tau)
                tau, self.A[t][p] = int(self.A[t][p]), tau
                if tau == EMPTY:
                    return EMPTY
        return tau

    def copies(self, x: int):
        return [t for t in range(self.d + 1) if self.A[t][self.h(t, x)] == x]

    def delete(self, x: int):
        for t in self.copies(x):
            self.A[t][self.h(t, x)] = EMPTY

    def build(self, elements) -> list:
        for x in elements:
            for _ in range(self.d):
                tau = self.insert(int(x))
                if tau != EMPTY:
                    self.delete(int(x))
                    if tau != int(x):
                        self.insert(tau)
                    break
        failed = []
        for x in elements:
            if len(self.copies(int(x))) != self.d:
                self.delete(int(x))
                failed.append(int(x))
        return failed


def serial_layout(tids, perms, r: int, r0: int, s: int, d: int = D, max_loop: int = 32):
    """(bytes uint8[(d+1) r], F_i) built with the serial procedure."""
    bm = SerialBatMapD(r, perms, d, max_loop)
    failed = bm.build(np.asarray(tids).tolist())
    out = np.zeros((d + 1) * r, dtype=np.uint8)
    for t in range(d + 1):
        for h in range(r):
            x = int(bm.A[t][h])
            if x == EMPTY:
                continue
            missing = [u for u in range(d + 1) if bm.A[u][bm.h(u, x)] != x]
            assert len(missing) == 1
            pi = int(perms[t][x])
            out[int(slot(t, pi, r, r0, d))] = element_byte(missing[0], pi, s, d)
    return out, np.array(sorted(failed), dtype=np.uint32)


def check_layout(bm, tids, failed, perms, r: int, r0: int, s: int, d: int = D) -> list:
    """Violations of the d-of-(d+1) layout (empty list when valid): every
    non-failed x is stored with its code in exactly d tables and each copy
    names the remaining table; failed elements are not stored; F_i is a
    subset of S_i; nothing else is stored."""
    errs = []
    bm = np.asarray(bm, dtype=np.uint8)
    if bm.size != (d + 1) * r:
        return [f"width {bm.size} != (d+1) r = {(d + 1) * r}"]
    tids = np.asarray(tids, dtype=np.int64)
    failed = np.asarray(failed, dtype=np.int64)
    if failed.size and not np.isin(failed, tids).all():
        errs.append("F_i not a subset of S_i")
    is_ok = ~np.isin(tids, failed)
    stored = np.zeros((d + 1, tids.size), dtype=bool)
    pos = np.zeros((d + 1, tids.size), dtype=np.int64)
    for t in range(d + 1):
        pi = perms[t][tids].astype(np.int64)
        pos[t] = slot(t, pi, r, r0, d)
        stored[t] = (bm[pos[t]].astype(np.int64) & code_max(d)) == code6(pi, s)
    ncopies = stored.sum(axis=0)
    if (ncopies[is_ok] != d).any():
        errs.append(f"{int((ncopies[is_ok] != d).sum())} elements without exactly {d} copies")
    if (ncopies[~is_ok] != 0).any():
        errs.append(f"{int((ncopies[~is_ok] != 0).sum())} failed elements still stored")
    missing = np.argmin(stored, axis=0)
    for t in range(d + 1):
        sel = stored[t] & is_ok
        if ((bm[pos[t][sel]] >> code_bits(d)) != missing[sel]).any():
            errs.append(f"missing-table field wrong in table {t}")
    nonzero = int(np.count_nonzero(bm))
    if nonzero != d * int(is_ok.sum()):
        errs.append(f"{nonzero} occupied slots, expected {d * int(is_ok.sum())}")
    return errs


def correction(tid_lists, fail_lists) -> int:
    """Common elements of the k sets that failed in at least one of them."""
    common = tid_lists[0]
    for t in tid_lists[1:]:
        common = np.intersect1d(common, t)
    if common.size == 0:
        return 0
    anyfail = np.unique(np.concatenate([np.asarray(f) for f in fail_lists]))
    return int(np.isin(common, anyfail).sum())


# ---- Apriori level 3 (Sec. I problem statement, beyond pairs) --------------

def triple_candidates(frequent_pairs) -> np.ndarray:
    """Every a < b < c whose three 2-subsets are all frequent, lexicographic
    (the Apriori join-and-prune step for itemsets of size 3)."""
    pairs = {(int(i), int(j)) for i, j in frequent_pairs}
    nbr = {}
    for i, j in sorted(pairs):
        nbr.setdefault(i, []).append(j)
    out = []
    for a in sorted(nbr):
        ja = nbr[a]
        for x, b in enumerate(ja):
            for c in ja[x + 1:]:
                if (b, c) in pairs:
                    out.append((a, b, c))
    return np.array(out, dtype=np.uint32).reshape(-1, 3)


def triple_candidates_bruteforce(n: int, frequent_pairs) -> np.ndarray:
    pairs = {(int(i), int(j)) for i, j in frequent_pairs}
    out = [(a, b, c) for a, b, c in itertools.combinations(range(n), 3)
           if (a, b) in pairs and (a, c) in pairs and (b, c) in pairs]
    return np.array(out, dtype=np.uint32).reshape(-1, 3)


# ---- Apriori level 4 --------------------------------------------------------

def quadruple_candidates(frequent_triples) -> np.ndarray:
    """Every a < b < c < d whose four 3-subsets are all frequent, lexicographic
    (the Apriori join of triples sharing (a, b), pruned by the other subsets)."""
    trip = {tuple(int(v) for v in t) for t in frequent_triples}
    by_prefix = {}
    for a, b, c in sorted(trip):
        by_prefix.setdefault((a, b), []).append(c)
    out = []
    for (a, b), cs in sorted(by_prefix.items()):
        for x, c in enumerate(cs):
            for dd in cs[x + 1:]:
                if (a, c, dd) in trip and (b, c, dd) in trip:
                    out.append((a, b, c, dd))
    return np.array(out, dtype=np.uint32).reshape(-1, 4)


def quadruple_candidates_bruteforce(n: int, frequent_triples) -> np.ndarray:
    trip = {tuple(int(v) for v in t) for t in frequent_triples}
    out = [q for q in itertools.combinations(range(n), 4)
           if all(tuple(x for x in q if x != y) in trip for y in q)]
    return np.array(out, dtype=np.uint32).reshape(-1, 4)
