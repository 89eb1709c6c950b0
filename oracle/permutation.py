"""The layout hash's permutations pi_t, restated on the CPU -- TEST INFRASTRUCTURE ONLY.

Plain Python / numpy, sharing no code with the CUDA path.  Sec. III-A builds
the layout hash from random permutations pi_1, pi_2, pi_3 of the transaction
ids and leaves open how they are drawn.  The library draws them itself from
a 64-bit seed; this module writes that definition out so that every layout
the GPU builds can be checked against it:

  * round keys: the SplitMix64 generator (Steele, Lea and Flood, "Fast
    splittable pseudorandom number generators", OOPSLA 2014) started from the
    seed; table t (0-based) takes outputs 4t .. 4t+3, each truncated to its
    low 32 bits;
  * round function: the 32-bit finalizer fmix32 of MurmurHash3 (Appleby),
    of the right half XOR the round key, truncated to a half;
  * one pass E_t: a balanced four-round Feistel network on b bits, b the
    smallest EVEN number >= max(2, ceil(log2 m)), halves of b/2 bits, each
    round (L, R) -> (R, L xor f(R xor k));
  * pi_t(x): cycle walking -- apply E_t to x until the value is below m.

Every Feistel network is a bijection of [0, 2^b) whatever its round function,
and cycle walking restricts a bijection of a superset to one of [0, m); the
counts are exact for any bijection (only the failure rate of the insertion
depends on the permutations).
"""
from __future__ import annotations

import numpy as np

_M64 = (1 << 64) - 1
GOLDEN_GAMMA = 0x9E3779B97F4A7C15


def splitmix64(seed: int, count: int) -> list[int]:
    """The first `count` outputs of SplitMix64 started from `seed`."""
    out = []
    state = seed & _M64
    for _ in range(count):
        state = (state + GOLDEN_GAMMA) & _M64
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        out.append(z ^ (z >> 31))
    return out


def round_keys(seed: int, tables: int) -> np.ndarray:
    """uint32[tables, 4]: the four round keys of each table's Feistel network."""
    raw = splitmix64(seed, 4 * tables)
    return np.array([x & 0xFFFFFFFF for x in raw], dtype=np.uint32).reshape(tables, 4)


def fmix32(z):
    """MurmurHash3's 32-bit finalizer, on numpy uint32 arrays (arithmetic mod 2^32)."""
    z = np.asarray(z, dtype=np.uint32).copy()
    z ^= z >> np.uint32(16)
    z *= np.uint32(0x85EBCA6B)
    z ^= z >> np.uint32(13)
    z *= np.uint32(0xC2B2AE35)
    z ^= z >> np.uint32(16)
    return z


def domain_bits(m: int) -> int:
    """b: the smallest even number >= max(2, ceil(log2 m))."""
    b = max(2, int(m - 1).bit_length() if m > 1 else 0)
    return b + (b & 1)


def feistel(v, keys, b: int):
    """One pass E of the four-round Feistel network on b-bit values."""
    h = b // 2
    mask = np.uint32((1 << h) - 1)
    v = np.asarray(v, dtype=np.uint32)
    left, right = v >> np.uint32(h), v & mask
    for k in keys:
        left, right = right, left ^ (fmix32(right ^ np.uint32(k)) & mask)
    return (left << np.uint32(h)) | right


def feistel_inverse(v, keys, b: int):
    """E^-1: the rounds run backwards, (L, R) -> (R xor f(L xor k), L)."""
    h = b // 2
    mask = np.uint32((1 << h) - 1)
    v = np.asarray(v, dtype=np.uint32)
    left, right = v >> np.uint32(h), v & mask
    for k in reversed(list(keys)):
        left, right = right ^ (fmix32(left ^ np.uint32(k)) & mask), left
    return (left << np.uint32(h)) | right


def permutation(m: int, seed: int, t: int) -> np.ndarray:
    """pi_t as uint32[m]: pi_t[x] for every transaction id x in [0, m)."""
    if m <= 0:
        return np.zeros(0, dtype=np.uint32)
    b = domain_bits(m)
    keys = round_keys(seed, t + 1)[t]
    y = feistel(np.arange(m, dtype=np.uint32), keys, b)
    walk = np.flatnonzero(y >= m)
    while walk.size:
        y[walk] = feistel(y[walk], keys, b)
        walk = walk[y[walk] >= m]
    return y


def permutations(m: int, seed: int, count: int = 3) -> np.ndarray:
    """uint32[count, m]: pi_0 .. pi_{count-1} (row t does not depend on count)."""
    out = np.empty((count, max(m, 0)), dtype=np.uint32)
    for t in range(count):
        out[t] = permutation(m, seed, t)
    return out
