"""The seeded input generators give the same instances whether they run in one
process or in spawned worker processes (the full-size workloads are generated
in parallel on the GPU machine), and the same instance for the same seed (CPU only)."""
import numpy as np

import datagen


def _same(a, b):
    return a.m == b.m and a.n == b.n and np.array_equal(a.offsets, b.offsets) and np.array_equal(a.tids, b.tids)


def test_bernoulli_parallel_equals_serial():
    serial = datagen.bernoulli_tidlists(20_000, 37, 0.03, seed=5, workers=1)
    parallel = datagen.bernoulli_tidlists(20_000, 37, 0.03, seed=5, workers=3)
    assert _same(serial, parallel)
    assert not _same(serial, datagen.bernoulli_tidlists(20_000, 37, 0.03, seed=6, workers=1))


def test_pool_blocks_equal_the_serial_pool():
    count, universe, lo, hi, seed = 300, 1 << 16, 10, 5_000, 3
    ref = datagen.pool_tidlists(count, universe, lo, hi, seed)
    for a, sizes, arr in datagen.pool_blocks(count, universe, lo, hi, seed, workers=2, block=70):
        b = a + sizes.size
        assert np.array_equal(sizes, np.diff(ref.offsets[a:b + 1]).astype(sizes.dtype))
        assert np.array_equal(arr, ref.tids[int(ref.offsets[a]):int(ref.offsets[b])])


def test_batch_instances_parallel_equal_serial():
    specs = datagen.batch_specs(4, 77, m_range=(1e3, 2e4), n_range=(20, 60))
    par = datagen.batch_instances(specs, workers=2)
    for spec, inst in zip(specs, par):
        assert _same(datagen.batch_instance(spec), inst)


def test_workload_instances_deterministic():
    a = datagen.workload_instance("bern_m10k_n200")
    b = datagen.workload_instance("bern_m10k_n200", workers=2)
    assert _same(a, b) and a.s == b.s == 25
    assert a.tids.size > 0 and np.all(np.diff(a.offsets.astype(np.int64)) >= 0)
