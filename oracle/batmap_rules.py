"""The paper's BatMap rules restated on the CPU -- TEST INFRASTRUCTURE ONLY.

Plain Python / numpy, written from the paper, sharing no code with the CUDA
path.  Used for pins (the rules checked against the paper's figures and
formulas) and to check that a layout built on the GPU is a valid BatMap.

Notation (Sec. II and Sec. III-A): tables t = 0, 1, 2 (the paper's 1, 2, 3),
pi_t the three permutations of the transaction ids, r_i the power-of-two hash
range of item i, r_0 = 2^s the smallest range, |B_0| = 3 r_0.

Readings where the paper is silent or ambiguous (each also listed in the design
notes of the repository):
  * transaction ids and pi values are 0-based, in [0, m);
  * the 7-bit code of an element is (pi_t(x) >> s) + 1, in [1, 127], and an
    empty slot (bottom) is the byte 0x00, so s is the smallest shift with
    m <= 127 * 2^s (never below `min_shift`);
  * r_i = max(r_0, 2^ceil(log2(c |S_i|))) with load factor c = 2 (Sec. III-A,
    Sec. IV-A "Throughput computation");
  * the indicator bit is 1 on the copy whose table is the cyclic successor of
    the table of its twin (Fig. 3);
  * correction(i, j) = |{x in S_i cap S_j : x in F_i or x in F_j}|, each pair
    generated once (Sec. III-C "Failed insertions").
"""
from __future__ import annotations

import numpy as np

EMPTY = -1


# ---- sizing (Sec. III-A "Layout of data structures", Sec. IV-A) ----------

def shift_bits(m: int, min_shift: int = 7) -> int:
    """Smallest s >= min_shift with m <= 127 * 2^s (7-bit codes 1..127, 0 = bottom)."""
    s = min_shift
    while m > 127 * (1 << s):
        s += 1
    return s


def hash_range(size: int, r0: int, c_num: int = 2, c_den: int = 1) -> int:
    """r_i: the smallest power of two >= c |S_i| (at least r_0)."""
    need = -(-c_num * max(int(size), 1) // c_den)
    r = 1
    while r < need:
        r <<= 1
    return max(r, r0)


def width_bytes(r: int) -> int:
    """|B_i| = 3 r_i bytes (three tables, one byte per slot)."""
    return 3 * r


# ---- layout hash and element codes (Sec. III-A) ---------------------------

def slot(t: int, pi, r: int, r0: int):
    """Byte position h_t^(i)(x) = |B_0| floor((pi mod r_i) / r_0) + (pi mod r_0) + t r_0."""
    pi = np.asarray(pi, dtype=np.int64)
    return 3 * r0 * ((pi % r) // r0) + (pi % r0) + t * r0


def code7(pi, s: int):
    """The stored 7 most significant bits of pi_t(x), shifted up by one (0 = bottom)."""
    return (np.asarray(pi, dtype=np.int64) >> s) + 1


def table_of_slot(pos, r0: int):
    return (np.asarray(pos, dtype=np.int64) % (3 * r0)) // r0


def decode_pi(pos, byte, r0: int, s: int):
    """pi_t(x) from a slot position and its stored byte (inverse of slot/code7)."""
    pos = np.asarray(pos, dtype=np.int64)
    code = (np.asarray(byte, dtype=np.int64) & 0x7F) - 1
    return (code << s) | (pos % r0)


# ---- counting rule (Sec. II, Fig. 3; Sec. III-A SWAR form) ----------------

def count_rule(bx, by):
    """A position counts iff the element bits agree and either indicator is set."""
    bx = np.asarray(bx, dtype=np.int64)
    by = np.asarray(by, dtype=np.int64)
    return (((bx & 0x7F) == (by & 0x7F)) & (((bx | by) & 0x80) != 0)).astype(np.int64)


def swar_count(x, y):
    """The paper's branch-free count of matches among the 2 x 4 bytes of two words."""
    x = np.asarray(x, dtype=np.uint64) & 0xFFFFFFFF
    y = np.asarray(y, dtype=np.uint64) & 0xFFFFFFFF
    p = (((x ^ y) | 0x80808080) - 0x01010101) & 0xFFFFFFFF
    pp = (p ^ 0xFFFFFFFF) & ((x | y) & 0x80808080)
    return (((pp >> 7) + (pp >> 15) + (pp >> 23) + (pp >> 31)) & 7).astype(np.int64)


def batmap_pair_count(bi: np.ndarray, bj: np.ndarray) -> int:
    """Count over two BatMaps (uint8 arrays); the smaller one wraps (Fig. 1, Sec. II)."""
    big, small = (bi, bj) if bi.size >= bj.size else (bj, bi)
    if small.size == 0:
        return 0
    assert big.size % small.size == 0
    rep = np.tile(small, big.size // small.size)
    return int(count_rule(big, rep).sum())


# ---- the serial INSERT procedure (Sec. II-A) ------------------------------

class SerialBatMap:
    """One set's 2-of-3 tables built with the paper's generalized cuckoo INSERT.

    A[t][h] holds an element (tid) or EMPTY, with h = pi_t(x) mod r."""

    def __init__(self, r: int, perms: np.ndarray, max_loop: int = 32):
        self.r = r
        self.perms = perms
        self.max_loop = max_loop
        self.A = np.full((3, r), EMPTY, dtype=np.int64)

    def h(self, t: int, x: int) -> int:
        return int(self.perms[t][x]) % self.r

    def insert(self, tau: int) -> int:
        """Push tau through tables 1,2,3,1,... swapping with the occupant; return
        EMPTY on success or the element left nestless after MaxLoop rounds."""
        for _ in range(self.max_loop):
            for t in range(3):
                p = self.h(t, tau)
                tau, self.A[t][p] = int(self.A[t][p]), tau
                if tau == EMPTY:
                    return EMPTY
        return tau

    def copies(self, x: int):
        return [t for t in range(3) if self.A[t][self.h(t, x)] == x]

    def delete(self, x: int):
        for t in self.copies(x):
            self.A[t][self.h(t, x)] = EMPTY

    def build(self, elements) -> list:
        """Two insertions per element; on failure delete x and re-insert the
        nestless element once; finally every element with fewer than two copies
        is deleted and reported failed (F_i)."""
        for x in elements:
            for _ in range(2):
                tau = self.insert(int(x))
                if tau != EMPTY:
                    self.delete(int(x))
                    if tau != int(x):
                        self.insert(tau)
                    break
        failed = []
        for x in elements:
            if len(self.copies(int(x))) != 2:
                self.delete(int(x))
                failed.append(int(x))
        return failed


def serial_layout(tids: np.ndarray, perms: np.ndarray, r: int, r0: int, s: int,
                  max_loop: int = 32):
    """Build one BatMap with the serial procedure; returns (bytes uint8[3r], F_i)."""
    bm = SerialBatMap(r, perms, max_loop)
    failed = bm.build(tids)
    out = np.zeros(3 * r, dtype=np.uint8)
    for t in range(3):
        for h in range(r):
            x = int(bm.A[t][h])
            if x == EMPTY:
                continue
            pi = int(perms[t][x])
            twin = (t - 1) % 3
            ind = 1 if bm.A[twin][int(perms[twin][x]) % r] == x else 0
            out[int(slot(t, pi, r, r0))] = (ind << 7) | int(code7(pi, s))
    return out, np.array(sorted(failed), dtype=np.uint32)


# ---- layout validity (what a GPU-built BatMap must satisfy) ---------------

def check_layout(bm: np.ndarray, tids: np.ndarray, failed: np.ndarray, perms: np.ndarray,
                 r: int, r0: int, s: int) -> list:
    """Return a list of violations (empty when the BatMap is valid):
    every x in S_i minus F_i is stored in exactly two cyclically adjacent tables
    at its hash positions with its code, the indicator set on the successor
    copy; no x in F_i is stored; F_i is a subset of S_i; nothing else is stored."""
    errs = []
    bm = np.asarray(bm, dtype=np.uint8)
    if bm.size != 3 * r:
        return [f"width {bm.size} != 3r = {3 * r}"]
    tids = np.asarray(tids, dtype=np.int64)
    failed = np.asarray(failed, dtype=np.int64)
    if failed.size and not np.isin(failed, tids).all():
        errs.append("F_i not a subset of S_i")
    ok = tids[~np.isin(tids, failed)]
    stored = np.zeros((3, tids.size), dtype=bool)
    pos = np.zeros((3, tids.size), dtype=np.int64)
    for t in range(3):
        pi = perms[t][tids].astype(np.int64)
        pos[t] = slot(t, pi, r, r0)
        stored[t] = (bm[pos[t]].astype(np.int64) & 0x7F) == code7(pi, s)
    ncopies = stored.sum(axis=0)
    is_ok = ~np.isin(tids, failed)
    if (ncopies[is_ok] != 2).any():
        errs.append(f"{int((ncopies[is_ok] != 2).sum())} elements without exactly two copies")
    if (ncopies[~is_ok] != 0).any():
        errs.append(f"{int((ncopies[~is_ok] != 0).sum())} failed elements still stored")
    for t in range(3):
        succ = (t + 1) % 3
        both = stored[t] & stored[succ] & is_ok
        ind_succ = bm[pos[succ][both]] >> 7
        ind_here = bm[pos[t][both]] >> 7
        if (ind_succ != 1).any() or (ind_here != 0).any():
            errs.append(f"indicator wrong for copies in tables {t},{succ}")
    nonzero = int(np.count_nonzero(bm))
    if nonzero != 2 * ok.size:
        errs.append(f"{nonzero} occupied slots, expected {2 * ok.size}")
    return errs


def correction(tids_i, tids_j, f_i, f_j) -> int:
    """Common elements that at least one side failed to store (Sec. III-C)."""
    common = np.intersect1d(tids_i, tids_j)
    if common.size == 0:
        return 0
    return int(np.isin(common, np.union1d(f_i, f_j)).sum())
