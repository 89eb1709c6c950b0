"""3-of-4 BatMaps (the d-of-(d+1) generalisation of Sec. V): layouts valid by
the definition, k-way supports (k = 1, 2, 3) and frequent triples bit-exact
against the merge oracle and the Apriori candidate step."""
import os

import numpy as np
import pytest

import datagen
import oracle
from oracle import dof_rules as R

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


def _dev(inst, seed, table=False):
    """Device tidlists and, with `table`, a caller-made table of the four
    permutations (else None: the library computes them from perm_seed)."""
    import torch
    off = torch.from_numpy(inst.offsets.view(np.int64)).cuda()
    tids = torch.from_numpy(inst.tids.view(np.int32)).cuda()
    perm = (torch.from_numpy(datagen.permutations(inst.m, seed, count=4).view(np.int32)).cuda() if table
            else None)
    return off, tids, perm


def _build(inst, seed=1, table=False, **params):
    import paper_1102_1003_gb300 as pkg
    off, tids, perm = _dev(inst, seed, table)
    p = pkg.batmap_default_params(perm_seed=seed, **params)
    return pkg.batmap_build_d(3, inst.m, off, tids, perm, params=p)


def _layout_errors(inst, bset, seed, c_num=2, c_den=1, table=False):
    import paper_1102_1003_gb300 as pkg
    from oracle import permutation as OP
    lay = pkg.batmap_export_layout(bset)
    info = lay["info"]
    s, r0 = info["shift"], info["r0"]
    assert s == R.shift_bits(inst.m)
    perms = datagen.permutations(inst.m, seed, count=4) if table else OP.permutations(inst.m, seed, 4)
    errs = []
    for i in range(inst.n):
        r = int(lay["range"][i])
        assert r == R.hash_range(inst.tidlist(i).size, r0, c_num, c_den)
        b0 = int(lay["byte_offset"][i])
        bm = lay["bytes"][b0:b0 + 4 * r]
        f = lay["fail_tids"][int(lay["fail_offsets"][i]):int(lay["fail_offsets"][i + 1])]
        e = R.check_layout(bm, inst.tidlist(i), f, perms, r, r0, s)
        errs += [f"item {i}: {x}" for x in e]
    return errs, info


def _queries(rng, n, k, q):
    return rng.integers(0, n, size=(q, k)).astype(np.int32)


@pytest.mark.parametrize("params,table", [(None, False), (None, True),
                                          (dict(load_num=1, load_den=1, max_loop=1), False)])
def test_layout_and_kway_supports_exact(params, table):
    import torch
    import paper_1102_1003_gb300 as pkg
    inst = datagen.zipf_tidlists(60_000, 80, 0.04, seed=11)
    b = _build(inst, 1, table, **(params or {}))
    lf = (params["load_num"], params["load_den"]) if params else (2, 1)
    errs, info = _layout_errors(inst, b, 1, *lf, table=table)
    assert errs == []
    assert info["d"] == 3
    if params:
        assert info["n_failed"] > 0
    rng = np.random.default_rng(0)
    for k in (1, 2, 3):
        qs = _queries(rng, inst.n, k, 3000)
        got = pkg.itemset_support(b, torch.from_numpy(qs).cuda()).cpu().numpy().astype(np.uint64)
        ref = oracle.kway_counts(inst.offsets, inst.tids, qs.tolist())
        assert np.array_equal(got, ref), k


def test_item_failing_almost_entirely():
    import torch
    import paper_1102_1003_gb300 as pkg
    # one very large item at load 1/4 per slot and MaxLoop 1 fails often
    m = 20_000
    lists = [np.arange(0, m, 2, dtype=np.uint32), np.arange(0, m, 3, dtype=np.uint32),
             np.arange(0, m, 5, dtype=np.uint32), np.arange(1, m, 7, dtype=np.uint32)]
    inst = datagen.from_lists(lists, m)
    b = _build(inst, 2, load_num=1, load_den=4, max_loop=1)
    errs, info = _layout_errors(inst, b, 2, 1, 4)
    assert errs == [] and info["n_failed"] > 1000
    qs = np.array([(0, 1, 2), (0, 1, 3), (1, 2, 3), (0, 0, 1), (3, 3, 3), (2, 0, 1)], dtype=np.int32)
    got = pkg.itemset_support(b, torch.from_numpy(qs).cuda()).cpu().numpy().astype(np.uint64)
    assert np.array_equal(got, oracle.kway_counts(inst.offsets, inst.tids, qs.tolist()))


def test_edge_cases_and_rejections():
    import torch
    import paper_1102_1003_gb300 as pkg
    lists = [[], [0], [5, 9, 100], list(range(0, 400, 3)), [], list(range(400))]
    inst = datagen.from_lists([np.asarray(l, np.uint32) for l in lists], 400)
    b = _build(inst, 3)
    qs = np.array([(a, b_, c) for a in range(6) for b_ in range(6) for c in range(6)], dtype=np.int32)
    got = pkg.itemset_support(b, torch.from_numpy(qs).cuda()).cpu().numpy().astype(np.uint64)
    assert np.array_equal(got, oracle.kway_counts(inst.offsets, inst.tids, qs.tolist()))
    # empty query list, out-of-range ids, pair calls on a 3-of-4 set, bad d
    assert pkg.itemset_support(b, torch.zeros((0, 3), dtype=torch.int32, device="cuda")).numel() == 0
    with pytest.raises(pkg.BatmapError):
        pkg.itemset_support(b, torch.tensor([[0, 1, 6]], dtype=torch.int32, device="cuda"))
    with pytest.raises(pkg.BatmapError):
        pkg.pair_support_all(b, 1)
    off, tids, perm = _dev(inst, 3, table=True)
    with pytest.raises(pkg.BatmapError):
        pkg.batmap_build_d(4, inst.m, off, tids, torch.zeros(5 * inst.m, dtype=torch.int32, device="cuda"))
    # a 2-of-3 set does not answer k-way witness queries
    b2 = pkg.batmap_build_d(2, inst.m, off, tids, perm[:3].contiguous())
    with pytest.raises(pkg.BatmapError):
        pkg.itemset_support(b2, torch.tensor([[0, 1, 2]], dtype=torch.int32, device="cuda"))


def _oracle_triples(inst, s):
    pairs = oracle.pairs_threshold(inst.offsets, inst.tids, s)
    cand = R.triple_candidates(pairs[:, :2])
    sup = oracle.kway_counts(inst.offsets, inst.tids, cand.tolist()) if cand.size else np.zeros(0, np.uint64)
    keep = sup >= s
    return pairs, cand, np.concatenate([cand[keep], sup[keep, None].astype(np.uint32)], axis=1)


@pytest.mark.parametrize("name,s", [("bern_m10k_n200", 25), ("dense", 40), ("zipf", 60)])
def test_frequent_triples_exact(name, s):
    import torch
    import paper_1102_1003_gb300 as pkg
    inst = {"bern_m10k_n200": lambda: datagen.workload_instance("bern_m10k_n200"),           # no frequent triple at s = 25
            "dense": lambda: datagen.bernoulli_tidlists(2_000, 60, 0.3, seed=6),
            "zipf": lambda: datagen.zipf_tidlists(50_000, 300, 0.03, seed=5)}[name]()
    pairs_ref, cand, want = _oracle_triples(inst, s)
    table = name == "dense"  # one case with caller-made permutations, the rest computed
    off, tids, perm4 = _dev(inst, 4, table)
    p = pkg.batmap_default_params(perm_seed=4)
    b2 = pkg.batmap_build(inst.m, off, tids, perm4[:3].contiguous() if table else None, params=p)
    n_pairs, pairs = pkg.pair_support_all(b2, s)
    assert np.array_equal(pairs.cpu().numpy().astype(np.uint32), pairs_ref)
    b3 = pkg.batmap_build_d(3, inst.m, off, tids, perm4, params=p)
    n_out, trip, n_cand = pkg.frequent_triples(b3, s, pairs)
    assert n_cand == cand.shape[0]
    assert n_out == want.shape[0]
    assert np.array_equal(trip.cpu().numpy().astype(np.uint32), want)
    # capacity path: the first cap triples and the full count
    if n_out > 2:
        small = torch.empty((2, 4), dtype=torch.int32, device="cuda")
        k, head, _ = pkg.frequent_triples(b3, s, pairs, out=small)
        assert k == n_out and np.array_equal(head.cpu().numpy().astype(np.uint32), want[:2])
    # no frequent pairs -> no triples
    none = pkg.frequent_triples(b3, s, pairs[:0])
    assert none[0] == 0 and none[2] == 0


@pytest.mark.parametrize("params", [None, dict(load_num=1, load_den=1, max_loop=1)])
def test_frequent_triples_probe_and_scan_routes_exact(params):
    """Items of three densities (BatMap widths 2^15, 2^13 and 2^11 slots per
    table at m = 20,000), so the candidates split between the scan (widths
    within 8x) and the probe route (the widest at least 8x the narrowest);
    s = 1 keeps every candidate, and every triple support is compared with
    the merge oracle, also under forced failed insertions."""
    import paper_1102_1003_gb300 as pkg
    rng = np.random.default_rng(17)
    m = 20_000
    lists = [np.flatnonzero(rng.random(m) < p).astype(np.uint32) for p in [0.5] * 10 + [0.12] * 20 + [0.03] * 30]
    inst = datagen.from_lists(lists, m, s=1)
    pairs_ref, cand, want = _oracle_triples(inst, 1)
    off, tids, _ = _dev(inst, 7)
    p = pkg.batmap_default_params(perm_seed=7, **(params or {}))
    b2 = pkg.batmap_build(inst.m, off, tids, None, params=p)
    n_pairs, pairs = pkg.pair_support_all(b2, 1)
    assert np.array_equal(pairs.cpu().numpy().astype(np.uint32), pairs_ref)
    b3 = pkg.batmap_build_d(3, inst.m, off, tids, None, params=p)
    # both routes occur: log2 of the widest over the narrowest table range, >= 3 probes
    lg = np.log2(pkg.batmap_export_layout(b3)["range"].astype(np.float64)).astype(np.int64)
    spread = lg[cand].max(axis=1) - lg[cand].min(axis=1)
    assert (spread >= 3).sum() > 1000 and (spread < 3).sum() > 1000
    if params:
        assert b3.info["n_failed"] > 0
    n_out, trip, n_cand = pkg.frequent_triples(b3, 1, pairs)
    assert n_cand == cand.shape[0]
    assert n_out == want.shape[0]
    assert np.array_equal(trip.cpu().numpy().astype(np.uint32), want)


def test_unsorted_pairs_rejected():
    import torch
    import paper_1102_1003_gb300 as pkg
    inst = datagen.workload_instance("bern_m10k_n200")
    b3 = _build(inst, 1)
    bad = torch.tensor([[3, 4, 30], [1, 2, 30]], dtype=torch.int32, device="cuda")
    with pytest.raises(pkg.BatmapError):
        pkg.frequent_triples(b3, 25, bad)
