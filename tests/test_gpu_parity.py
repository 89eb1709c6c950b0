"""GPU parity: the CUDA path (through the C ABI) against the merge oracle.

Counts are exact integers, so every comparison is bit-exact (tolerance 0).
Layout placement is not unique (any valid 2-of-3 assignment is correct), so
built BatMaps are checked for validity against the definition instead of
byte-compared.
"""
import os

import numpy as np
import pytest

import datagen
import oracle
from tests.gpu_util import device_inputs, layout_errors, run_all_pairs

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 4


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    torch.cuda.set_device(0)


def _check_exact(inst, full, n_out, pairs, s=None):
    s = inst.s if s is None else s
    ref = oracle.pairs_full(inst.offsets, inst.tids, threads=THREADS)
    assert full is None or np.array_equal(full, ref), \
        f"{int((full != ref).sum())} of {ref.size} supports differ"
    ref_pairs = oracle.threshold_from_full(ref, inst.n, s)
    assert n_out == ref_pairs.shape[0]
    assert np.array_equal(pairs, ref_pairs)


def test_bernoulli_m10k_all_pairs_exact():
    inst = datagen.workload_instance("bern_m10k_n200")
    full, n_out, pairs, bset = run_all_pairs(inst, perm_seed=1)
    assert inst.n * (inst.n - 1) // 2 == 19_900
    _check_exact(inst, full, n_out, pairs)
    # the pair list of the oracle's own threshold routine agrees too
    assert np.array_equal(pairs, oracle.pairs_threshold(inst.offsets, inst.tids, inst.s))


@pytest.mark.parametrize("table", [False, True])
def test_bernoulli_m10k_layout_valid(table):
    """Every BatMap valid by the definition, with the library's computed
    permutations (checked against the oracle's restatement of the generator)
    and with a caller-made permutation table."""
    inst = datagen.workload_instance("bern_m10k_n200")
    _, _, _, bset = run_all_pairs(inst, perm_seed=1, want_full=False, table=table)
    assert layout_errors(inst, bset, 1, table=table) == []
    info = bset.info
    assert info["n_classes"] == 2  # widths 3 KiB and 6 KiB mixed (|S| straddles 512)


@pytest.mark.parametrize("seed", range(3))
def test_zipf_mixed_widths_exact_and_valid(seed):
    inst = datagen.zipf_tidlists(60_000, 300 + 37 * seed, 0.03, seed=100 + seed, s=50)
    full, n_out, pairs, bset = run_all_pairs(inst, perm_seed=seed)
    _check_exact(inst, full, n_out, pairs)
    assert bset.info["n_classes"] >= 3
    assert layout_errors(inst, bset, seed) == []


@pytest.mark.parametrize("tile", list(range(1, 19)))
def test_every_tile_shape_exact(tile):
    import paper_1102_1003_gb300 as pkg
    inst = datagen.zipf_tidlists(40_000, 333, 0.04, seed=7, s=30)
    full, n_out, pairs, _ = run_all_pairs(inst, params=pkg.batmap_default_params(tile=tile))
    _check_exact(inst, full, n_out, pairs)


@pytest.mark.parametrize("params", [dict(max_loop=1), dict(load_num=1, load_den=1),
                                    dict(load_num=1, load_den=2, max_loop=2),
                                    dict(load_num=1, load_den=4, max_loop=1)])
def test_forced_failures_stay_exact(params):
    import paper_1102_1003_gb300 as pkg
    inst = datagen.zipf_tidlists(20_000, 120, 0.08, seed=11, s=20)
    full, n_out, pairs, bset = run_all_pairs(inst, perm_seed=3, params=pkg.batmap_default_params(**params))
    info = bset.info
    assert info["n_failed"] > 0 and info["n_corrections"] > 0
    _check_exact(inst, full, n_out, pairs)
    assert layout_errors(inst, bset, 3, params.get("load_num", 2), params.get("load_den", 1)) == []


def test_all_elements_of_an_item_fail():
    import paper_1102_1003_gb300 as pkg
    # one dense item at load factor 1/8: nearly every insertion of it fails
    rng = np.random.default_rng(5)
    m = 5000
    lists = [np.arange(m, dtype=np.uint32)] + [np.flatnonzero(rng.random(m) < 0.3).astype(np.uint32)
                                                for _ in range(9)]
    inst = datagen.from_lists(lists, m, s=1)
    full, n_out, pairs, bset = run_all_pairs(inst, perm_seed=2,
                                             params=pkg.batmap_default_params(load_num=1, load_den=8,
                                                                              max_loop=1))
    assert bset.info["n_failed"] > m // 2
    _check_exact(inst, full, n_out, pairs)


@pytest.mark.parametrize("case", ["n0", "n1", "n2", "empty_items", "identical", "m1", "singletons",
                                  "full_items", "ragged_129", "ragged_257"])
def test_edge_cases(case):
    rng = np.random.default_rng(3)
    m = 3000
    if case == "n0":
        inst = datagen.from_lists([], m)
    elif case == "n1":
        inst = datagen.from_lists([np.arange(0, m, 3, dtype=np.uint32)], m)
    elif case == "n2":
        inst = datagen.from_lists([np.arange(0, m, 3, dtype=np.uint32), np.arange(0, m, 2, dtype=np.uint32)], m)
    elif case == "empty_items":
        inst = datagen.from_lists([[], np.arange(5, dtype=np.uint32), [], [], np.arange(3, 9, dtype=np.uint32), []], m)
    elif case == "identical":
        a = np.flatnonzero(rng.random(m) < 0.2).astype(np.uint32)
        inst = datagen.from_lists([a] * 12, m)
    elif case == "m1":
        inst = datagen.from_lists([[0], [], [0], [0]], 1)
    elif case == "singletons":
        inst = datagen.from_lists([[int(x)] for x in rng.integers(0, 40, 60)], m)
    elif case == "full_items":
        inst = datagen.from_lists([np.arange(m, dtype=np.uint32)] * 5 + [np.arange(0, m, 7, dtype=np.uint32)], m)
    else:
        n = int(case.split("_")[1])
        inst = datagen.bernoulli_tidlists(m, n, 0.05, seed=n)
    for s in (0, 1, 2):
        full, n_out, pairs, _ = run_all_pairs(inst, s=s, perm_seed=4)
        _check_exact(inst, full, n_out, pairs, s=s)


def test_threshold_extremes_and_capacity():
    import torch
    import paper_1102_1003_gb300 as pkg
    inst = datagen.workload_instance("bern_m10k_n200")
    off, tids, perm = device_inputs(inst, 0)
    bset = pkg.batmap_build(inst.m, off, tids, perm)
    ref = oracle.pairs_full(inst.offsets, inst.tids, threads=THREADS)
    for s in (0, 1, 25, int(ref.max()), int(ref.max()) + 1, 2**32 - 1):
        n_out, pairs = pkg.pair_support_all(bset, s)
        want = oracle.threshold_from_full(ref, inst.n, s)
        assert n_out == want.shape[0]
        assert np.array_equal(pairs.cpu().numpy().astype(np.uint32).reshape(-1, 3)[:n_out], want)
    # too small an output buffer: the first cap triples and the true count
    small = torch.empty((100, 3), dtype=torch.int32, device="cuda")
    n_out, got = pkg.pair_support_all(bset, 0, pairs=small)
    assert n_out == 19_900 and got.shape[0] == 100
    assert np.array_equal(got.cpu().numpy().astype(np.uint32), oracle.threshold_from_full(ref, inst.n, 0)[:100])
    # repeated calls reuse scratch and give the same answer
    a = pkg.pair_support_all(bset, 25)[1].cpu().numpy()
    b = pkg.pair_support_all(bset, 25)[1].cpu().numpy()
    assert np.array_equal(a, b)


def test_invalid_inputs_rejected():
    import torch
    import paper_1102_1003_gb300 as pkg
    m = 100
    good = datagen.from_lists([[1, 5, 9], [2, 5]], m)
    cases = {
        "unsorted": datagen.Instance(m, 2, good.offsets, np.array([5, 1, 9, 2, 5], np.uint32)),
        "duplicate": datagen.Instance(m, 2, good.offsets, np.array([1, 5, 5, 2, 5], np.uint32)),
        "out_of_range": datagen.Instance(m, 2, good.offsets, np.array([1, 5, 100, 2, 5], np.uint32)),
    }
    for name, inst in cases.items():
        off, tids, perm = device_inputs(inst, 0, table=True)
        with pytest.raises(pkg.BatmapError) as e:
            pkg.batmap_build(m, off, tids, perm)
        assert e.value.code == pkg.BATMAP_ERR_ARG, name
    off, tids, perm = device_inputs(good, 0, table=True)
    bad = perm.clone()
    bad[1, 3] = bad[1, 4]
    with pytest.raises(pkg.BatmapError) as e:
        pkg.batmap_build(m, off, tids, bad)
    assert e.value.code == pkg.BATMAP_ERR_ARG
    with pytest.raises(pkg.BatmapError):
        pkg.batmap_build(0, off, tids, perm)
    torch.cuda.synchronize()


def test_host_entry_point_matches_device_path():
    import torch
    import paper_1102_1003_gb300 as pkg
    inst = datagen.zipf_tidlists(50_000, 257, 0.03, seed=21, s=40)
    perm = datagen.permutations(inst.m, 5)
    ref = oracle.pairs_threshold(inst.offsets, inst.tids, inst.s)
    pinned = torch.empty((ref.shape[0] + 10) * 3, dtype=torch.int32, pin_memory=True).numpy()
    for p in (perm, None):  # a caller-made table, and the library's computed permutations
        pinned[:] = -1
        n_out = pkg.pair_support_host(inst.m, inst.offsets, inst.tids, p, inst.s, pinned)
        assert n_out == ref.shape[0]
        assert np.array_equal(pinned[:3 * n_out].reshape(-1, 3).astype(np.uint32), ref)


def test_batch_equals_separate_calls():
    import torch
    import paper_1102_1003_gb300 as pkg
    insts = [datagen.zipf_tidlists(m, n, d, seed=300 + q, s=max(1, m // 1000))
             for q, (m, n, d) in enumerate([(10_000, 150, 0.05), (30_000, 400, 0.02), (5_000, 97, 0.1),
                                            (60_000, 220, 0.03), (12_000, 2, 0.2), (8_000, 1, 0.1)])]
    sets, bufs, fulls, refs = [], [], [], []
    for q, inst in enumerate(insts):
        off, tids, perm = device_inputs(inst, q)
        sets.append(pkg.batmap_build(inst.m, off, tids, perm))
        ref = oracle.pairs_full(inst.offsets, inst.tids, threads=THREADS)
        refs.append(ref)
        want = oracle.threshold_from_full(ref, inst.n, inst.s).shape[0]
        bufs.append(torch.empty((max(want, 1), 3), dtype=torch.int32, device="cuda"))
        fulls.append(torch.empty(max(ref.size, 1), dtype=torch.int32, device="cuda"))
    for rep in range(2):  # second call replays the captured graph
        n_outs = pkg.pair_support_batch(sets, [i.s for i in insts], bufs, fulls)
        torch.cuda.synchronize()
        for q, inst in enumerate(insts):
            want = oracle.threshold_from_full(refs[q], inst.n, inst.s)
            assert n_outs[q] == want.shape[0]
            got = bufs[q].cpu().numpy().astype(np.uint32).reshape(-1, 3)[:n_outs[q]]
            assert np.array_equal(got, want), (rep, q)
            assert np.array_equal(fulls[q][:refs[q].size].cpu().numpy().astype(np.uint32), refs[q])


def test_zipf_full_scale_exact():
    """The Zipf workload at full size (m = 10^6, n = 2000, Zipf, 2% density):
    every one of the 1,999,000 supports against the merge oracle."""
    inst = datagen.workload_instance("zipf_m1m_n2000")
    full, n_out, pairs, bset = run_all_pairs(inst, perm_seed=2)
    _check_exact(inst, full, n_out, pairs)
    info = bset.info
    assert info["n_classes"] >= 6


def _skewed_instance(seed, n_wide=40, n_narrow=200, m=50_000):
    """Two width groups far apart (wide items at 50%, narrow at 0.2% .. 2%):
    every wide x narrow pair is width-skewed, the wide class has more columns
    than one probe unit takes (PROBE_COLS = 16), and the narrow items span
    several classes."""
    rng = np.random.default_rng(seed)
    lists = [np.flatnonzero(rng.random(m) < 0.5).astype(np.uint32) for _ in range(n_wide)]
    lists += [np.flatnonzero(rng.random(m) < rng.uniform(0.002, 0.02)).astype(np.uint32)
              for _ in range(n_narrow)]
    order = rng.permutation(len(lists))  # original ids mixed across widths
    return datagen.from_lists([lists[k] for k in order], m, s=20)


@pytest.mark.parametrize("probe_log", [1, 2, 3, 5, 32])
@pytest.mark.parametrize("params", [None, dict(max_loop=1, load_num=1, load_den=2)])
def test_probe_route_exact(probe_log, params):
    """The probe route (width-skewed pairs) and the cyclic scan give the same
    supports at every threshold ratio, with and without failed insertions;
    32 turns the route off."""
    import paper_1102_1003_gb300 as pkg
    for inst in (_skewed_instance(probe_log), datagen.zipf_tidlists(60_000, 300, 0.03, seed=probe_log, s=50)):
        p = pkg.batmap_default_params(probe_log=probe_log, **(params or {}))
        full, n_out, pairs, bset = run_all_pairs(inst, perm_seed=probe_log, params=p)
        _check_exact(inst, full, n_out, pairs)
        info = bset.info
        if probe_log >= 32:
            assert info["probe_word_pairs"] == 0
        else:
            assert info["probe_word_pairs"] > 0 and info["probe_words"] > 0
            assert info["probe_word_pairs"] <= info["word_pairs"]
        if params:
            assert info["n_failed"] > 0


def test_probe_route_cross_and_batch_exact():
    """The probe route inside cross mode (family A rows against wide family B
    columns and the reverse) and inside the batched form."""
    import torch
    import paper_1102_1003_gb300 as pkg
    m = 40_000
    rng = np.random.default_rng(8)
    fam_a = [np.flatnonzero(rng.random(m) < p).astype(np.uint32) for p in rng.uniform(0.002, 0.6, 90)]
    fam_b = [np.flatnonzero(rng.random(m) < p).astype(np.uint32) for p in rng.uniform(0.002, 0.6, 70)]
    union = datagen.from_lists(fam_a + fam_b, m)
    full_ref = oracle.pairs_full(union.offsets, union.tids, threads=THREADS)
    a, b = np.meshgrid(np.arange(90), np.arange(70), indexing="ij")
    ref_c = full_ref[oracle.packed_index(union.n, a.ravel(), 90 + b.ravel())].reshape(90, 70)
    skew = _skewed_instance(9)
    ref_s = oracle.pairs_full(skew.offsets, skew.tids, threads=THREADS)
    p = pkg.batmap_default_params(probe_log=2)
    o1, t1, _ = device_inputs(union, 1)
    o2, t2, _ = device_inputs(skew, 2)
    sets = [pkg.batmap_build_cross(m, 90, o1, t1, None, params=p), pkg.batmap_build(skew.m, o2, t2, None, params=p)]
    assert sets[0].info["probe_word_pairs"] > 0 and sets[1].info["probe_word_pairs"] > 0
    fulls = [torch.empty(90 * 70, dtype=torch.int32, device="cuda"),
             torch.empty(ref_s.size, dtype=torch.int32, device="cuda")]
    n_out, _ = pkg.pair_support_all(sets[0], 1, full=fulls[0])
    assert np.array_equal(fulls[0].cpu().numpy().astype(np.uint32).reshape(90, 70), ref_c)
    bufs = [torch.empty((int((ref_c >= 1).sum()), 3), dtype=torch.int32, device="cuda"),
            torch.empty((max(1, int((ref_s >= skew.s).sum())), 3), dtype=torch.int32, device="cuda")]
    for rep in range(2):
        fulls[0].fill_(-1)
        fulls[1].fill_(-1)
        pkg.pair_support_batch(sets, [1, skew.s], bufs, fulls)
        assert np.array_equal(fulls[0].cpu().numpy().astype(np.uint32).reshape(90, 70), ref_c), rep
        assert np.array_equal(fulls[1].cpu().numpy().astype(np.uint32), ref_s), rep
