"""4-of-5 BatMaps (the d-of-(d+1) generalisation of Sec. V with d = 4: five
tables, a three-bit missing-table field, five-bit codes): layouts valid by
the definition, k-way supports (k = 1..4), frequent triples and frequent
quadruples (Apriori levels 3 and 4) bit-exact against the merge oracle and
the oracle's candidate steps."""
import numpy as np
import pytest

import datagen
import oracle
from oracle import dof_rules as R

pytestmark = pytest.mark.gpu
D = 4


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    torch.cuda.set_device(0)


def _dev(inst, seed, table=False):
    import torch
    off = torch.from_numpy(inst.offsets.view(np.int64)).cuda()
    tids = torch.from_numpy(inst.tids.view(np.int32)).cuda()
    perm = (torch.from_numpy(datagen.permutations(inst.m, seed, count=D + 1).view(np.int32)).cuda() if table
            else None)
    return off, tids, perm


def _build(inst, seed=1, table=False, **params):
    import paper_1102_1003_gb300 as pkg
    off, tids, perm = _dev(inst, seed, table)
    return pkg.batmap_build_d(D, inst.m, off, tids, perm, params=pkg.batmap_default_params(perm_seed=seed, **params))


def _layout_errors(inst, bset, seed, c_num=2, c_den=1, table=False):
    import paper_1102_1003_gb300 as pkg
    from oracle import permutation as OP
    lay = pkg.batmap_export_layout(bset)
    info = lay["info"]
    s, r0 = info["shift"], info["r0"]
    assert s == R.shift_bits(inst.m, d=D)
    perms = datagen.permutations(inst.m, seed, count=D + 1) if table else OP.permutations(inst.m, seed, D + 1)
    errs = []
    for i in range(inst.n):
        r = int(lay["range"][i])
        assert r == R.hash_range(inst.tidlist(i).size, r0, c_num, c_den)
        b0 = int(lay["byte_offset"][i])
        bm = lay["bytes"][b0:b0 + (D + 1) * r]
        f = lay["fail_tids"][int(lay["fail_offsets"][i]):int(lay["fail_offsets"][i + 1])]
        errs += [f"item {i}: {x}" for x in R.check_layout(bm, inst.tidlist(i), f, perms, r, r0, s, D)]
    return errs, info


@pytest.mark.parametrize("params,table", [(None, False), (None, True),
                                          (dict(load_num=1, load_den=1, max_loop=1), False)])
def test_layout_and_kway_supports_exact(params, table):
    import torch
    import paper_1102_1003_gb300 as pkg
    inst = datagen.zipf_tidlists(40_000, 70, 0.05, seed=13)
    b = _build(inst, 2, table, **(params or {}))
    lf = (params["load_num"], params["load_den"]) if params else (2, 1)
    errs, info = _layout_errors(inst, b, 2, *lf, table=table)
    assert errs == []
    assert info["d"] == D
    if params:
        assert info["n_failed"] > 0
    rng = np.random.default_rng(1)
    for k in (1, 2, 3, 4):
        qs = rng.integers(0, inst.n, size=(2500, k)).astype(np.int32)
        got = pkg.itemset_support(b, torch.from_numpy(qs).cuda()).cpu().numpy().astype(np.uint64)
        assert np.array_equal(got, oracle.kway_counts(inst.offsets, inst.tids, qs.tolist())), k


def test_item_failing_almost_entirely():
    import torch
    import paper_1102_1003_gb300 as pkg
    m = 20_000
    lists = [np.arange(0, m, 2, dtype=np.uint32), np.arange(0, m, 3, dtype=np.uint32),
             np.arange(0, m, 5, dtype=np.uint32), np.arange(1, m, 7, dtype=np.uint32),
             np.arange(0, m, 4, dtype=np.uint32)]
    inst = datagen.from_lists(lists, m)
    b = _build(inst, 3, load_num=1, load_den=4, max_loop=1)
    errs, info = _layout_errors(inst, b, 3, 1, 4)
    assert errs == [] and info["n_failed"] > 1000
    qs = np.array([(0, 1, 2, 3), (0, 1, 2, 4), (1, 2, 3, 4), (0, 0, 1, 4), (4, 4, 4, 4), (3, 0, 2, 1)],
                  dtype=np.int32)
    got = pkg.itemset_support(b, torch.from_numpy(qs).cuda()).cpu().numpy().astype(np.uint64)
    assert np.array_equal(got, oracle.kway_counts(inst.offsets, inst.tids, qs.tolist()))


def _oracle_levels(inst, s):
    """Frequent pairs, triples and quadruples by the oracle's candidate steps and merges."""
    pairs = oracle.pairs_threshold(inst.offsets, inst.tids, s)
    c3 = R.triple_candidates(pairs[:, :2])
    s3 = oracle.kway_counts(inst.offsets, inst.tids, c3.tolist()) if c3.size else np.zeros(0, np.uint64)
    trip = np.concatenate([c3[s3 >= s], s3[s3 >= s, None].astype(np.uint32)], axis=1).astype(np.uint32)
    c4 = R.quadruple_candidates(trip[:, :3])
    s4 = oracle.kway_counts(inst.offsets, inst.tids, c4.tolist()) if c4.size else np.zeros(0, np.uint64)
    quad = np.concatenate([c4[s4 >= s], s4[s4 >= s, None].astype(np.uint32)], axis=1).astype(np.uint32)
    return pairs, c3, trip, c4, quad


@pytest.mark.parametrize("name,s", [("dense", 60), ("zipf", 40)])
def test_frequent_triples_and_quadruples_exact(name, s):
    import torch
    import paper_1102_1003_gb300 as pkg
    inst = {"dense": lambda: datagen.bernoulli_tidlists(3_000, 50, 0.35, seed=8),
            "zipf": lambda: datagen.zipf_tidlists(30_000, 200, 0.04, seed=9)}[name]()
    pairs_ref, c3, trip_ref, c4, quad_ref = _oracle_levels(inst, s)
    assert quad_ref.shape[0] > 0
    off, tids, _ = _dev(inst, 5)
    p = pkg.batmap_default_params(perm_seed=5)
    b2 = pkg.batmap_build(inst.m, off, tids, None, params=p)
    _, pairs = pkg.pair_support_all(b2, s)
    assert np.array_equal(pairs.cpu().numpy().astype(np.uint32), pairs_ref)
    b4 = pkg.batmap_build_d(D, inst.m, off, tids, None, params=p)
    n3, trip, n3c = pkg.frequent_triples(b4, s, pairs)
    assert n3c == c3.shape[0] and n3 == trip_ref.shape[0]
    assert np.array_equal(trip.cpu().numpy().astype(np.uint32), trip_ref)
    n4, quad, n4c = pkg.frequent_quadruples(b4, s, trip)
    assert n4c == c4.shape[0] and n4 == quad_ref.shape[0]
    assert np.array_equal(quad.cpu().numpy().astype(np.uint32), quad_ref)
    # capacity path: the first cap quadruples and the full count
    if n4 > 2:
        small = torch.empty((2, 5), dtype=torch.int32, device="cuda")
        k, head, _ = pkg.frequent_quadruples(b4, s, trip, out=small)
        assert k == n4 and np.array_equal(head.cpu().numpy().astype(np.uint32), quad_ref[:2])
    # no frequent triples -> no quadruples
    none = pkg.frequent_quadruples(b4, s, trip[:0])
    assert none[0] == 0 and none[2] == 0


def test_rejections():
    import torch
    import paper_1102_1003_gb300 as pkg
    inst = datagen.bernoulli_tidlists(2_000, 12, 0.3, seed=4)
    b4 = _build(inst, 1)
    with pytest.raises(pkg.BatmapError):  # k > d
        pkg.itemset_support(b4, torch.zeros((3, 5), dtype=torch.int32, device="cuda"))
    bad = torch.tensor([[1, 2, 3, 40], [0, 1, 2, 40]], dtype=torch.int32, device="cuda")
    with pytest.raises(pkg.BatmapError):  # triples out of order
        pkg.frequent_quadruples(b4, 1, bad)
    off, tids, _ = _dev(inst, 1)
    b3 = pkg.batmap_build_d(3, inst.m, off, tids, None)
    good = torch.tensor([[0, 1, 2, 40]], dtype=torch.int32, device="cuda")
    with pytest.raises(pkg.BatmapError):  # a 3-of-4 set cannot witness four sets
        pkg.frequent_quadruples(b3, 1, good)
    with pytest.raises(pkg.BatmapError):
        pkg.batmap_build_d(5, inst.m, off, tids, None)


@pytest.mark.parametrize("params", [None, dict(max_loop=1, load_num=1, load_den=1)])
def test_quadruples_probe_and_scan_routes_exact(params):
    """Items of three densities on 4-of-5 BatMaps, so that the triple and
    quadruple candidates split between the scan (equal widths) and the probe
    route (the widest at least 2x the narrowest); s = 1 keeps every
    candidate, and every triple and quadruple support is compared with the
    merge oracle, also under forced failed insertions."""
    import paper_1102_1003_gb300 as pkg
    rng = np.random.default_rng(23)
    m = 12_000
    lists = [np.flatnonzero(rng.random(m) < p).astype(np.uint32) for p in [0.6] * 6 + [0.15] * 8 + [0.04] * 10]
    inst = datagen.from_lists(lists, m, s=1)
    pairs_ref, c3, trip_ref, c4, quad_ref = _oracle_levels(inst, 1)
    off, tids, _ = _dev(inst, 3)
    p = pkg.batmap_default_params(perm_seed=3, **(params or {}))
    b2 = pkg.batmap_build(inst.m, off, tids, None, params=p)
    _, pairs = pkg.pair_support_all(b2, 1)
    assert np.array_equal(pairs.cpu().numpy().astype(np.uint32), pairs_ref)
    b4 = pkg.batmap_build_d(D, inst.m, off, tids, None, params=p)
    lg = np.log2(pkg.batmap_export_layout(b4)["range"].astype(np.float64)).astype(np.int64)
    for cand in (c3, c4):
        spread = lg[cand].max(axis=1) - lg[cand].min(axis=1)
        assert (spread >= 1).sum() > 100 and (spread == 0).sum() >= 15
    if params:
        assert b4.info["n_failed"] > 0
    n3, trip, n3c = pkg.frequent_triples(b4, 1, pairs)
    assert n3c == c3.shape[0] and n3 == trip_ref.shape[0]
    assert np.array_equal(trip.cpu().numpy().astype(np.uint32), trip_ref)
    n4, quad, n4c = pkg.frequent_quadruples(b4, 1, trip)
    assert n4c == c4.shape[0] and n4 == quad_ref.shape[0]
    assert np.array_equal(quad.cpu().numpy().astype(np.uint32), quad_ref)
