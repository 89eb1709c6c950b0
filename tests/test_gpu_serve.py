"""Serving: conjunctive queries over a device-resident pool, alone and in the
continuous-batching loop, against the merge oracle (counts are exact, so the
tolerance is 0)."""
import numpy as np
import pytest

import datagen
import oracle
from tests.gpu_util import device_inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    torch.cuda.set_device(0)


def _pool_inst():
    # universe 2^20 (r_0 = 2^14: sets of >= 8192 elements get BatMaps), Zipf sizes on [10, 2e5]
    return datagen.pool_tidlists(1500, 1 << 20, 10, 200_000, seed=5)


def _queries(n, count, seed, big=None):
    rng = np.random.default_rng(seed)
    qs = []
    for _ in range(count):
        k = 2 if rng.random() < 0.8 else int(rng.integers(3, 9))
        qs.append(rng.integers(0, n, k).tolist())
    if big is not None and len(big) >= 3:
        qs += [[int(big[0]), int(big[1])], [int(big[2]), int(big[0]), int(big[1])], [int(big[0]), int(big[0])],
               [int(big[1])], [0, int(big[0])]]
    return qs


def _make_pool(inst, seed=1, params=None, table=False):
    import paper_1102_1003_gb300 as pkg
    off, tids, perm = device_inputs(inst, seed, table)
    return pkg.batmap_pool_create(inst.m, off, tids, perm, params=params)


@pytest.mark.parametrize("params,table", [(None, False), (None, True),
                                          (dict(load_num=1, load_den=2, max_loop=1), False)])
def test_intersect_query_exact(params, table):
    import paper_1102_1003_gb300 as pkg
    inst = _pool_inst()
    pool = _make_pool(inst, params=pkg.batmap_default_params(**params) if params else None, table=table)
    info = pool.info
    assert 0 < info["n_batmaps"] < inst.n
    big = np.flatnonzero(inst.sizes >= 8192)
    qs = _queries(inst.n, 600, 7, big)
    got = pkg.intersect_query(pool, qs).cpu().numpy()
    ref = oracle.kway_counts(inst.offsets, inst.tids, qs)
    assert np.array_equal(got.astype(np.uint64), ref)


def test_serve_results_same_alone_and_in_mix():
    import paper_1102_1003_gb300 as pkg
    inst = _pool_inst()
    pool = _make_pool(inst)
    qs = _queries(inst.n, 3000, 11, np.flatnonzero(inst.sizes >= 8192))
    ref = oracle.kway_counts(inst.offsets, inst.tids, qs)
    # Poisson arrivals at a high rate so that batches overlap on the device
    rng = np.random.default_rng(3)
    arrival = np.cumsum(rng.exponential(1.0 / 200_000.0, len(qs)))
    opts = pkg.batmap_serve_opts(max_batch=32, slots=4, work_budget=1 << 22, reserved=0)
    counts, lat, stats = pkg.batmap_serve(pool, qs, arrival, opts)
    assert np.array_equal(counts, ref)
    assert (lat >= 0).all() and stats["batches"] > 1 and stats["max_inflight"] >= 1
    assert stats["p50_s"] <= stats["p99_s"] <= stats["max_s"]
    # each query alone gives the same count as in the mix
    sample = list(range(0, len(qs), 37))
    for q in sample:
        alone = pkg.intersect_query(pool, [qs[q]]).cpu().numpy()[0]
        assert int(alone) == int(counts[q]), q
    # all arriving at once (closed loop) gives the same counts again
    counts2, _, stats2 = pkg.batmap_serve(pool, qs, np.zeros(len(qs)), opts)
    assert np.array_equal(counts2, ref) and stats2["max_inflight"] >= 2


def test_pool_rejects_bad_input():
    import paper_1102_1003_gb300 as pkg
    m = 1000
    inst = datagen.Instance(m, 2, np.array([0, 3, 5], np.uint64), np.array([1, 9, 5, 2, 3], np.uint32))
    with pytest.raises(pkg.BatmapError) as e:
        _make_pool(inst)
    assert e.value.code == pkg.BATMAP_ERR_ARG


@pytest.mark.parametrize("params", [None, dict(load_num=1, load_den=2, max_loop=1)])
def test_intersect_query_list_exact(params):
    import paper_1102_1003_gb300 as pkg
    inst = _pool_inst()
    pool = _make_pool(inst, params=pkg.batmap_default_params(**params) if params else None)
    qs = _queries(inst.n, 400, 19, np.flatnonzero(inst.sizes >= 8192))
    off, elems = pkg.intersect_query_list(pool, qs)
    off = off.cpu().numpy()
    elems = elems.cpu().numpy().astype(np.uint32)
    assert off[0] == 0 and off[-1] == elems.size and (np.diff(off) >= 0).all()
    counts = pkg.intersect_query(pool, qs).cpu().numpy()
    for q, query in enumerate(qs):
        ref = oracle.kway_elems(inst.offsets, inst.tids, query)
        assert np.array_equal(elems[off[q]:off[q + 1]], ref), q
        assert counts[q] == ref.size
