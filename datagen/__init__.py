"""Seeded synthetic transaction data shaped like the paper's pair-mining workloads.

This module only produces inputs: vertical tidlists in CSR form and the three
random permutations pi_1..pi_3 that the layout hash of Sec. III-A draws.  It
holds none of the method's arithmetic and is shared by the CUDA path, the
oracle, the tests and the benchmark.

CSR convention (used everywhere in this repository):
  offsets : uint64[n + 1], offsets[0] = 0, non-decreasing
  tids    : uint32[offsets[n]], tids[offsets[i]:offsets[i+1]] is the tidlist
            S_i of item i, strictly increasing, every value < m.
Transaction ids are 0-based (the paper numbers them 1..m).

Recipes (each a seeded numpy Generator, one independent stream per item):
  * bernoulli: item i contains transaction x independently with probability p
    (the instance generator of Sec. IV-A and the density sweep of Fig. 7).
  * zipf: item of rank k (1..n) is included with probability
    p_k = min(1, c / k**a); c is solved so that mean_k p_k equals the target
    density, and ranks are shuffled onto item ids.  Transaction lengths are then
    Poisson-binomial with mean density*n (close to Poisson for small p_k).
  * pool: serving sets over a universe U with sizes drawn from a discrete
    Zipf(1) law on [lo, hi]; members uniform (Bernoulli with p = size/U).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "Instance", "bernoulli_item", "bernoulli_tidlists", "zipf_probabilities",
    "zipf_tidlists", "permutations", "workload_instance", "batch_specs",
    "pool_sizes", "pool_tidlists", "from_lists", "transactions_to_tidlists",
    "WORKLOADS", "concat", "cross_instance", "triples_instance",
]


@dataclass
class Instance:
    """One mining instance: m transactions, n items, tidlists in CSR form."""
    m: int
    n: int
    offsets: np.ndarray  # uint64[n+1]
    tids: np.ndarray     # uint32[T]
    s: int = 0           # support threshold
    name: str = ""

    @property
    def sizes(self) -> np.ndarray:
        return np.diff(self.offsets).astype(np.int64)

    def tidlist(self, i: int) -> np.ndarray:
        return self.tids[int(self.offsets[i]):int(self.offsets[i + 1])]


def _item_rng(seed: int, item: int) -> np.random.Generator:
    return np.random.default_rng([int(seed), int(item)])


def bernoulli_item(rng: np.random.Generator, m: int, p: float) -> np.ndarray:
    """Sorted uint32 tids of one Bernoulli(p) subset of [0, m)."""
    if m <= 0 or p <= 0.0:
        return np.zeros(0, dtype=np.uint32)
    if p >= 1.0:
        return np.arange(m, dtype=np.uint32)
    if p > 0.25:
        return np.flatnonzero(rng.random(m) < p).astype(np.uint32)
    # geometric gap sampling: O(|S|) work for sparse items
    mean = m * p
    out = []
    pos = -1
    while True:
        cnt = int(mean + 6.0 * math.sqrt(mean) + 16)
        gaps = rng.geometric(p, size=cnt).astype(np.int64)
        pts = pos + np.cumsum(gaps)
        if pts[-1] >= m:
            out.append(pts[pts < m])
            break
        out.append(pts)
        pos = int(pts[-1])
    return np.concatenate(out).astype(np.uint32)


def from_lists(lists, m: int, s: int = 0, name: str = "") -> Instance:
    """Build an Instance from Python/numpy tidlists (sorted, unique, < m)."""
    n = len(lists)
    sizes = np.array([len(l) for l in lists], dtype=np.uint64)
    offsets = np.zeros(n + 1, dtype=np.uint64)
    np.cumsum(sizes, out=offsets[1:])
    tids = (np.concatenate([np.asarray(l, dtype=np.uint32) for l in lists])
            if n and int(offsets[-1]) else np.zeros(0, dtype=np.uint32))
    return Instance(m=m, n=n, offsets=offsets, tids=tids.astype(np.uint32), s=s, name=name)


def _bernoulli_block(args):
    """Worker: items [a, b) of a Bernoulli instance written into a new
    shared-memory block; returns (block name, sizes)."""
    from multiprocessing import shared_memory
    m, p, seed, a, b = args
    parts = [bernoulli_item(_item_rng(seed, i), m, p) for i in range(a, b)]
    total = sum(x.size for x in parts)
    shm = shared_memory.SharedMemory(create=True, size=max(4 * total, 4))
    out = np.ndarray((total,), dtype=np.uint32, buffer=shm.buf)
    pos = 0
    for x in parts:
        out[pos:pos + x.size] = x
        pos += x.size
    name = shm.name
    shm.close()
    return name, np.array([x.size for x in parts], dtype=np.int64)


def bernoulli_tidlists(m: int, n: int, p: float, seed: int, s: int = 0, name: str = "",
                       workers: int = 1) -> Instance:
    """Uniform density p for every item (the Bernoulli workloads).  With
    workers > 1 the items are generated in spawned processes (safe after CUDA
    is initialised); every item has its own stream, so the result is the same."""
    if workers <= 1 or n < 2 * workers:
        return from_lists([bernoulli_item(_item_rng(seed, i), m, p) for i in range(n)], m, s, name)
    import multiprocessing as mp
    from multiprocessing import shared_memory
    step = max(1, -(-n // (4 * workers)))
    jobs = [(m, p, seed, a, min(n, a + step)) for a in range(0, n, step)]
    sizes = np.zeros(n, dtype=np.int64)
    blocks = []
    with mp.get_context("spawn").Pool(workers) as pool:
        for (_, _, _, a, b), (shm_name, got) in zip(jobs, pool.imap(_bernoulli_block, jobs)):
            sizes[a:b] = got
            blocks.append(shm_name)
    offsets = np.zeros(n + 1, dtype=np.uint64)
    np.cumsum(sizes, out=offsets[1:])
    tids = np.empty(int(offsets[-1]), dtype=np.uint32)
    for (_, _, _, a, b), shm_name in zip(jobs, blocks):
        shm = shared_memory.SharedMemory(name=shm_name)
        try:
            cnt = int(offsets[b] - offsets[a])
            tids[int(offsets[a]):int(offsets[b])] = np.ndarray((cnt,), dtype=np.uint32, buffer=shm.buf)
        finally:
            shm.close()
            shm.unlink()
    return Instance(m=m, n=n, offsets=offsets, tids=tids, s=s, name=name)


def zipf_probabilities(n: int, density: float, exponent: float = 1.0) -> np.ndarray:
    """Per-rank inclusion probabilities p_k = min(1, c/k^a), mean = density."""
    if n == 0:
        return np.zeros(0)
    k = np.arange(1, n + 1, dtype=np.float64)
    base = k ** (-exponent)
    target = density * n
    lo, hi = 0.0, float(n) / base.min()
    for _ in range(200):
        c = 0.5 * (lo + hi)
        if np.minimum(1.0, c * base).sum() < target:
            lo = c
        else:
            hi = c
    return np.minimum(1.0, 0.5 * (lo + hi) * base)


def zipf_tidlists(m: int, n: int, density: float, seed: int, exponent: float = 1.0,
                  s: int = 0, name: str = "") -> Instance:
    """Zipf-skewed item frequencies with mean density `density` (the Zipf and batched workloads)."""
    probs = zipf_probabilities(n, density, exponent)
    rank_of_item = np.random.default_rng([int(seed), 0x5A1F]).permutation(n)
    lists = [bernoulli_item(_item_rng(seed, i), m, float(probs[rank_of_item[i]]))
             for i in range(n)]
    return from_lists(lists, m, s, name)


def transactions_to_tidlists(transactions, m: int, n: int) -> Instance:
    """Horizontal format (list of item lists per transaction) -> vertical CSR."""
    lists = [[] for _ in range(n)]
    for x, items in enumerate(transactions):
        for i in items:
            lists[i].append(x)
    return from_lists([sorted(set(l)) for l in lists], m)


def permutations(m: int, seed: int, count: int = 3) -> np.ndarray:
    """The random permutations pi_1..pi_count of [0, m) (Sec. III-A: three; a
    d-of-(d+1) BatMap uses d+1), uint32[count, m]; row t does not depend on count."""
    out = np.empty((count, max(m, 0)), dtype=np.uint32)
    for t in range(count):
        out[t] = np.random.default_rng([int(seed), 0xB47, t]).permutation(m).astype(np.uint32)
    return out


# ---- the five workload configurations -------------------------------------

WORKLOADS = {
    "bern_m10k_n200": dict(kind="bernoulli", m=10_000, n=200, p=0.05, s=25, seed=1),
    "zipf_m1m_n2000": dict(kind="zipf", m=1_000_000, n=2_000, density=0.02, s=1_000, seed=2),
    "bern_m4m_n8192_p0.1": dict(kind="bernoulli", m=4_194_304, n=8_192, p=0.001, s=4_195, seed=41),
    "bern_m4m_n8192_p1": dict(kind="bernoulli", m=4_194_304, n=8_192, p=0.01, s=4_195, seed=42),
    "bern_m4m_n8192_p5": dict(kind="bernoulli", m=4_194_304, n=8_192, p=0.05, s=4_195, seed=43),
}


def sorted_u32(count: int, seed: int, max_gap: int = 255) -> np.ndarray:
    """Strictly increasing uint32 values with independent gaps uniform in
    [1, max_gap] (two such arrays interleave at random)."""
    g = np.random.default_rng([seed, 0x5E7])
    vals = np.cumsum(g.integers(1, max_gap + 1, size=count, dtype=np.uint64))
    assert vals[-1] < 2 ** 32
    return vals.astype(np.uint32)


def workload_instance(name: str, scale_n: int | None = None, workers: int = 1) -> Instance:
    """Instance of a named workload; `scale_n` truncates the item count;
    `workers` > 1 generates Bernoulli workloads in parallel (same result)."""
    c = WORKLOADS[name]
    n = c["n"] if scale_n is None else min(c["n"], scale_n)
    if c["kind"] == "bernoulli":
        return bernoulli_tidlists(c["m"], n, c["p"], c["seed"], c["s"], name, workers=workers)
    return zipf_tidlists(c["m"], n, c["density"], c["seed"], 1.0, c["s"], name)


def nsweep_instance(n: int, total: int = 10_000_000, density: float = 0.05, seed: int = 7) -> Instance:
    """The experiment shape of Sec. IV-A / Fig. 5: a fixed total instance size
    (`total` items over all transactions) at item density `density`, so
    m = total / (density * n) transactions and |S_i| ~ total / n."""
    m = max(1, int(round(total / (density * n))))
    return bernoulli_tidlists(m, n, density, seed + n, s=1, name=f"nsweep{n}")


def concat(a: Instance, b: Instance, name: str = "") -> Instance:
    """Family A's tidlists followed by family B's, over the same m (cross mode input)."""
    assert a.m == b.m
    offsets = np.concatenate([a.offsets, a.offsets[-1] + b.offsets[1:]]).astype(np.uint64)
    return Instance(m=a.m, n=a.n + b.n, offsets=offsets, tids=np.concatenate([a.tids, b.tids]),
                    s=1, name=name)


CROSS = dict(m=1_000_000, n_a=2_000, density_a=0.01, n_b=4_000, p_b=0.002, seed=61)


def cross_instance(m: int = CROSS["m"], n_a: int = CROSS["n_a"], n_b: int = CROSS["n_b"],
                   density_a: float = CROSS["density_a"], p_b: float = CROSS["p_b"],
                   seed: int = CROSS["seed"]) -> tuple[Instance, int]:
    """Sparse boolean matrix multiplication / join-project shape (Sec. I): rows
    A_i of one matrix (Zipf(1) sizes at mean density `density_a`) against
    columns B_j of another (Bernoulli `p_b`); returns (A then B, n_a)."""
    a = zipf_tidlists(m, n_a, density_a, seed)
    b = bernoulli_tidlists(m, n_b, p_b, seed + 1)
    return concat(a, b, name="cross"), n_a


TRIPLES = dict(m=100_000, n=1_000, density=0.02, s=100, seed=71)


def triples_instance() -> Instance:
    """Frequent-itemset workload beyond pairs: m = 100,000 transactions, n = 1,000
    items with Zipf(1) inclusion probabilities at mean density 2%, s = 100 (0.1%)."""
    c = TRIPLES
    return zipf_tidlists(c["m"], c["n"], c["density"], c["seed"], 1.0, c["s"], "triples")


def batch_specs(k: int = 64, seed0: int = 1000, m_range=(1e4, 1e6), n_range=(100, 4000),
                d_range=(0.01, 0.10)):
    """Instance shapes of the batched workload: m log-uniform, n and density uniform."""
    specs = []
    for i in range(k):
        g = np.random.default_rng([seed0 + i, 0xBA7C])
        m = int(round(10 ** g.uniform(math.log10(m_range[0]), math.log10(m_range[1]))))
        n = int(g.integers(n_range[0], n_range[1] + 1))
        d = float(g.uniform(d_range[0], d_range[1]))
        specs.append(dict(m=m, n=n, density=d, seed=seed0 + i, s=int(math.ceil(0.001 * m))))
    return specs


def batch_instance(spec: dict) -> Instance:
    """One instance of the batched workload from its spec (see batch_specs)."""
    return zipf_tidlists(spec["m"], spec["n"], spec["density"], spec["seed"], 1.0, spec["s"],
                         f"batch{spec['seed']}")


def batch_instances(specs, workers: int = 8):
    """All instances of the batched workload, generated in spawned worker processes."""
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.map(batch_instance, specs)


def pool_sizes(count: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Discrete Zipf(1) set sizes on [lo, hi]: P(k) proportional to 1/k."""
    g = np.random.default_rng([int(seed), 0x9001])
    u = g.random(count)
    # inverse CDF of the continuous 1/k law, floored: k = lo * (hi/lo)^u
    return np.minimum(hi, np.floor(lo * np.exp(u * math.log((hi + 1) / lo)))).astype(np.int64)


def pool_set(universe: int, size: int, seed: int, i: int) -> np.ndarray:
    """Members of pool set i (Bernoulli with p = size / universe)."""
    return bernoulli_item(_item_rng(seed, i), universe, float(size) / universe)


def _pool_block(args):
    """Worker: generate sets [a, b) into a new shared-memory block; returns
    (name, sizes) and leaves the block for the parent to attach and unlink."""
    from multiprocessing import shared_memory
    universe, sizes, seed, a = args
    parts = [pool_set(universe, int(k), seed, a + j) for j, k in enumerate(sizes)]
    total = sum(p.size for p in parts)
    shm = shared_memory.SharedMemory(create=True, size=max(4 * total, 4))
    out = np.ndarray((total,), dtype=np.uint32, buffer=shm.buf)
    pos = 0
    for p in parts:
        out[pos:pos + p.size] = p
        pos += p.size
    name = shm.name
    shm.close()
    return name, np.array([p.size for p in parts], dtype=np.int64)


def pool_blocks(count: int, universe: int, lo: int, hi: int, seed: int, workers: int = 8, block: int = 2000):
    """The serving pool generated in parallel worker processes (spawned, so it
    is safe to call after CUDA is initialised).  Yields (first_set, sizes,
    tids) per block of sets, tids a uint32 array in shared memory that is
    released when the generator advances.  Same sets as pool_tidlists."""
    import multiprocessing as mp
    from multiprocessing import shared_memory
    sizes = pool_sizes(count, lo, hi, seed)
    jobs = [(universe, sizes[a:a + block], seed, a) for a in range(0, count, block)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        for (a, (name, got)) in zip(range(0, count, block), pool.imap(_pool_block, jobs)):
            shm = shared_memory.SharedMemory(name=name)
            try:
                arr = np.ndarray((int(got.sum()),), dtype=np.uint32, buffer=shm.buf)
                yield a, got, arr
                del arr
            finally:
                shm.close()
                shm.unlink()


def _pool_sets_job(args):
    universe, seed, pairs = args
    return [pool_set(universe, int(k), seed, int(i)) for i, k in pairs]


def pool_subset(universe: int, lo: int, hi: int, seed: int, count: int, ids, workers: int = 8) -> Instance:
    """The pool sets `ids` (in that order) of the pool pool_blocks / pool_tidlists
    generate, regenerated in spawned worker processes: the same sets, without
    generating the rest of the pool."""
    import multiprocessing as mp
    sizes = pool_sizes(count, lo, hi, seed)
    ids = [int(i) for i in ids]
    pairs = [(i, int(sizes[i])) for i in ids]
    step = max(1, -(-len(pairs) // (4 * max(workers, 1))))
    jobs = [(universe, seed, pairs[a:a + step]) for a in range(0, len(pairs), step)]
    with mp.get_context("spawn").Pool(max(workers, 1)) as pool:
        lists = [x for part in pool.map(_pool_sets_job, jobs) for x in part]
    return from_lists(lists, universe, 0, "pool_subset")


def pool_tidlists(count: int, universe: int, lo: int, hi: int, seed: int) -> Instance:
    """Serving pool: `count` sets over [0, universe) with Zipf sizes, uniform members."""
    sizes = pool_sizes(count, lo, hi, seed)
    lists = [pool_set(universe, int(sizes[i]), seed, i) for i in range(count)]
    return from_lists(lists, universe, 0, "pool")
