"""Pins of the oracle's layout-hash permutations (oracle/permutation.py), CPU only.

The paper draws pi_1..pi_3 at random (Sec. III-A) and fixes no generator; the
library's generator is a seeded Feistel network with cycle walking, written
from published definitions.  Its pins are values published for those
building blocks and properties that any correct construction has:
  * SplitMix64's first outputs from seed 0 (the generator's published test
    values) pin the key schedule;
  * MurmurHash3_x86_32 of the empty input with seeds 1 and 0xFFFFFFFF (its
    published test values) equal fmix32(seed), which pins the round function;
  * the Feistel pass has an inverse with the rounds run backwards, exhaustively
    on small domains (a transposed half or a missing mask breaks it);
  * every pi_t is a bijection of [0, m) (exhaustive for many m), its rows do
    not depend on how many are drawn, and different tables and seeds differ.
Planted mistakes in the oracle fail these pins.
"""
import numpy as np
import pytest

from oracle import permutation as P


def test_splitmix64_published_values():
    assert P.splitmix64(0, 3) == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_fmix32_published_murmur3_values():
    # MurmurHash3_x86_32 of zero bytes is fmix32(seed ^ 0)
    assert int(P.fmix32(1)) == 0x514E28B7
    assert int(P.fmix32(0xFFFFFFFF)) == 0x81F16F39
    assert int(P.fmix32(0)) == 0


def test_fmix32_is_a_bijection_of_32_bit_words():
    # each step is invertible: xor-shift by >= 16 bits undoes itself after one
    # more application when the shift is >= 16, the multiplications by odd
    # constants have inverses mod 2^32
    rng = np.random.default_rng(1)
    z = rng.integers(0, 2**32, 100_000, dtype=np.uint64).astype(np.uint32)
    y = P.fmix32(z)
    inv1, inv2 = pow(0xC2B2AE35, -1, 2**32), pow(0x85EBCA6B, -1, 2**32)
    x = y.astype(np.uint64)
    x ^= x >> np.uint64(16)
    x = (x * np.uint64(inv1)) & np.uint64(0xFFFFFFFF)
    x ^= (x >> np.uint64(13)) ^ (x >> np.uint64(26))
    x = (x * np.uint64(inv2)) & np.uint64(0xFFFFFFFF)
    x ^= x >> np.uint64(16)
    assert np.array_equal(x.astype(np.uint32), z)


@pytest.mark.parametrize("b", [2, 4, 6, 8, 10, 12, 16])
def test_feistel_pass_is_a_bijection_with_its_inverse(b):
    keys = P.round_keys(12345, 2)[1]
    v = np.arange(1 << b, dtype=np.uint32)
    y = P.feistel(v, keys, b)
    assert np.unique(y).size == v.size and int(y.max()) < (1 << b)
    assert np.array_equal(P.feistel_inverse(y, keys, b), v)


def test_domain_bits():
    assert [P.domain_bits(m) for m in (1, 2, 3, 4, 5, 16, 17, 64, 65, 10**6, 1 << 22, (1 << 22) + 1, 1 << 26)] == \
        [2, 2, 2, 2, 4, 4, 6, 6, 8, 20, 22, 24, 26]


@pytest.mark.parametrize("seed", [0, 1, 0xDEADBEEF12345678])
def test_every_row_is_a_bijection(seed):
    for m in list(range(1, 300)) + [1000, 4097, 65_537, 100_000]:
        perms = P.permutations(m, seed, 4)
        for t in range(4):
            assert np.array_equal(np.sort(perms[t]), np.arange(m, dtype=np.uint32)), (m, t)


def test_rows_seeds_and_counts():
    m = 10_000
    a = P.permutations(m, 7, 3)
    b = P.permutations(m, 7, 4)
    assert np.array_equal(a, b[:3])
    assert not np.array_equal(a[0], a[1]) and not np.array_equal(a[1], a[2])
    assert not np.array_equal(a[0], P.permutation(m, 8, 0))
    # a permutation that moves nearly every element (identity-like rows would break hashing)
    assert (a[0] != np.arange(m)).mean() > 0.99


def test_cycle_walking_stays_on_the_cycle():
    # pi_t(x) is the first value below m on x's cycle under the Feistel pass
    m, seed, t = 1000, 3, 2
    b = P.domain_bits(m)
    keys = P.round_keys(seed, t + 1)[t]
    pi = P.permutation(m, seed, t)
    for x in range(0, m, 37):
        y = int(P.feistel(np.uint32(x), keys, b))
        while y >= m:
            y = int(P.feistel(np.uint32(y), keys, b))
        assert y == pi[x]


def test_planted_mistakes_are_caught(monkeypatch):
    # a round function that is not truncated to a half breaks the bijection
    def unmasked(v, keys, b):
        h = b // 2
        v = np.asarray(v, dtype=np.uint32)
        left, right = v >> np.uint32(h), v & np.uint32((1 << h) - 1)
        for k in keys:
            left, right = right, left ^ P.fmix32(right ^ np.uint32(k))
        return ((left << np.uint32(h)) | right) & np.uint32((1 << b) - 1)
    keys = P.round_keys(5, 1)[0]
    v = np.arange(1 << 8, dtype=np.uint32)
    assert np.unique(unmasked(v, keys, 8)).size < v.size
    # a wrong multiplier in the round function misses the published vector
    monkeypatch.setattr(P, "fmix32", lambda z: np.asarray(z, dtype=np.uint32) * np.uint32(0x85EBCA6B))
    assert int(P.fmix32(1)) != 0x514E28B7
