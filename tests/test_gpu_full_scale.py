"""Full-size parity of the benchmark workloads against the merge oracle.

Counts are exact integers, so every comparison is bit-exact (tolerance 0).
  * density sweep (m = 4,194,304 transactions, n = 8,192 items, Bernoulli
    0.1% / 1% / 5%), BatMap path and dense tensor-core path: at 0.1% every
    one of the 33,550,336 supports; at 1% and 5% 256 whole rows (2.1M
    supports) plus 3,000 random pairs, and the row-sum invariant; the frequent
    pairs against the supports everywhere;
  * the batched form on the 64 uneven instances (m log-uniform in [1e4, 1e6],
    n in [100, 4000], density 1%..10%, Zipf items): full triangles for the
    instances with n <= 1,000, 20,000 random pairs and 16 whole rows for the
    rest, and every instance's frequent pairs against its supports;
  * serving over the full pool of 100,000 sets on 2^26 tids (Zipf sizes in
    [10, 10^6]): 5,000 queries (80% pairs, 20% 3..8-way) through the
    continuous-batching loop against the oracle on the regenerated sets;
  * the Sec. IV-A n-sweep shape at n = 16,000 and 64,000: sampled pairs and
    whole rows.
The oracle runs on all host cores (the same single-threaded merge on
disjoint blocks).
"""
import math
import os

import numpy as np
import pytest

import datagen
import oracle

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 4
ROWS = 256


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    torch.cuda.set_device(0)


_CACHE = {}


def _density_case(name):
    """Instance and oracle reference of one density, kept while its two paths run."""
    if _CACHE.get("name") != name:
        _CACHE.clear()
        inst = datagen.workload_instance(name, workers=THREADS)
        n = inst.n
        rng = np.random.default_rng(41)
        if name.endswith("p0.1"):
            ref = {"full": oracle.pairs_full(inst.offsets, inst.tids, threads=THREADS)}
        else:
            rows = np.sort(rng.choice(n, ROWS, replace=False))
            cols = np.arange(n)
            lo = np.concatenate([np.minimum(i, cols[cols != i]) for i in rows])
            hi = np.concatenate([np.maximum(i, cols[cols != i]) for i in rows])
            si = rng.integers(0, n - 1, 3000)
            sj = si + 1 + (rng.integers(0, n, 3000) % (n - 1 - si))
            ii, jj = np.concatenate([lo, si]), np.concatenate([hi, sj])
            ref = {"rows": rows, "ii": ii, "jj": jj,
                   "sup": oracle.pairs_list(inst.offsets, inst.tids, ii, jj, threads=THREADS)}
        _CACHE.update(name=name, inst=inst, ref=ref)
    return _CACHE["inst"], _CACHE["ref"]


def _run_path(inst, path):
    import torch
    import paper_1102_1003_gb300 as pkg
    off = torch.from_numpy(inst.offsets.view(np.int64)).cuda()
    tids = torch.from_numpy(inst.tids.view(np.int32)).cuda()
    npairs = inst.n * (inst.n - 1) // 2
    full = torch.full((npairs,), -1, dtype=torch.int32, device="cuda")
    if path == "batmap":
        bset = pkg.batmap_build(inst.m, off, tids, None, params=pkg.batmap_default_params(perm_seed=4))
        n_out, pairs = pkg.pair_support_all(bset, inst.s, full=full)
        bset.free()
    else:
        n_out, pairs, _ = pkg.pair_support_dense(inst.m, off, tids, inst.s, full=full)
    torch.cuda.synchronize()
    out = (full.cpu().numpy().astype(np.uint32), n_out, pairs.cpu().numpy().astype(np.uint32).reshape(-1, 3))
    del off, tids, full, pairs
    pkg.batmap_release_scratch()
    torch.cuda.empty_cache()
    return out


def _check_pairs_against_full(full, n, n_out, pairs, s):
    """The frequent pairs are exactly the supports >= s, lexicographic (i < j)."""
    assert n_out == int((full >= s).sum())
    assert pairs.shape[0] == n_out
    if n_out:
        key = pairs[:, 0].astype(np.int64) * n + pairs[:, 1]
        assert (np.diff(key) > 0).all() and (pairs[:, 0] < pairs[:, 1]).all()
        assert np.array_equal(full[oracle.packed_index(n, pairs[:, 0], pairs[:, 1])], pairs[:, 2])


@pytest.mark.parametrize("name,path", [(d, p) for d in ("bern_m4m_n8192_p0.1", "bern_m4m_n8192_p1",
                                                         "bern_m4m_n8192_p5") for p in ("batmap", "dense")])
def test_density_sweep_full_scale(name, path):
    inst, ref = _density_case(name)
    n = inst.n
    full, n_out, pairs = _run_path(inst, path)
    if "full" in ref:
        bad = int((full != ref["full"]).sum())
        assert bad == 0, f"{bad} of {full.size} supports differ"
        assert np.array_equal(pairs, oracle.threshold_from_full(ref["full"], n, inst.s))
        return
    got = full[oracle.packed_index(n, ref["ii"], ref["jj"])]
    bad = int((got != ref["sup"]).sum())
    assert bad == 0, f"{bad} of {got.size} row and sampled supports differ"
    # row sums: sum over partners of row i = sum over x in S_i of (|T_x| - 1)
    tlen = np.bincount(inst.tids, minlength=inst.m).astype(np.int64)
    per_row = ref["sup"][:ROWS * (n - 1)].astype(np.int64).reshape(ROWS, n - 1).sum(axis=1)
    for k, i in enumerate(ref["rows"]):
        assert per_row[k] == (tlen[inst.tidlist(int(i))] - 1).sum()
    _check_pairs_against_full(full, n, n_out, pairs, inst.s)


def test_batched_64_instances_full_scale():
    """The batched form (one graph-captured persistent pass over all 64
    instances) at full size against the merge oracle."""
    import torch
    import paper_1102_1003_gb300 as pkg
    _CACHE.clear()
    insts = datagen.batch_instances(datagen.batch_specs(64, 1000), workers=THREADS)
    sets, bufs, fulls, n_ref = [], [], [], []
    for q, inst in enumerate(insts):
        off = torch.from_numpy(inst.offsets.view(np.int64)).cuda()
        tids = torch.from_numpy(inst.tids.view(np.int32)).cuda()
        sets.append(pkg.batmap_build(inst.m, off, tids, None, params=pkg.batmap_default_params(perm_seed=100 + q)))
        del off, tids
        npairs = inst.n * (inst.n - 1) // 2
        fulls.append(torch.full((npairs,), -1, dtype=torch.int32, device="cuda"))
    counts = [pkg.pair_support_all(b, i.s)[0] for b, i in zip(sets, insts)]
    bufs = [torch.empty((max(k, 1), 3), dtype=torch.int32, device="cuda") for k in counts]
    n_outs = pkg.pair_support_batch(sets, [i.s for i in insts], bufs, fulls)
    torch.cuda.synchronize()
    assert n_outs == counts
    rng = np.random.default_rng(64)
    n_full = 0
    for q, inst in enumerate(insts):
        n = inst.n
        full = fulls[q].cpu().numpy().astype(np.uint32)
        pairs = bufs[q][:n_outs[q]].cpu().numpy().astype(np.uint32).reshape(-1, 3)
        if n <= 1000:
            ref = oracle.pairs_full(inst.offsets, inst.tids, threads=THREADS)
            assert np.array_equal(full, ref), q
            assert np.array_equal(pairs, oracle.threshold_from_full(ref, n, inst.s)), q
            n_full += 1
            continue
        rows = rng.choice(n, 16, replace=False)
        cols = np.arange(n)
        lo = np.concatenate([np.minimum(i, cols[cols != i]) for i in rows])
        hi = np.concatenate([np.maximum(i, cols[cols != i]) for i in rows])
        si = rng.integers(0, n - 1, 20_000)
        sj = si + 1 + (rng.integers(0, n, 20_000) % (n - 1 - si))
        ii, jj = np.concatenate([lo, si]), np.concatenate([hi, sj])
        ref = oracle.pairs_list(inst.offsets, inst.tids, ii, jj, threads=THREADS)
        assert np.array_equal(full[oracle.packed_index(n, ii, jj)], ref), q
        _check_pairs_against_full(full, n, n_outs[q], pairs, inst.s)
    assert n_full >= 8
    for b in sets:
        b.free()
    del fulls, bufs
    pkg.batmap_release_scratch()
    torch.cuda.empty_cache()


def test_serving_full_pool_exact():
    """Serving at full size: the pool of 100,000 sets over 2^26 tids with Zipf(1)
    sizes in [10, 10^6]; 5,000 queries through the continuous-batching loop,
    checked against the oracle on the named sets regenerated on the CPU; a
    sample of them alone gives the same counts as in the mix."""
    import torch
    import paper_1102_1003_gb300 as pkg
    _CACHE.clear()
    U, lo, hi, seed, count = 1 << 26, 10, 10**6, 5, 100_000
    sizes = datagen.pool_sizes(count, lo, hi, seed)
    ub = int(sum(int(k + 6 * math.sqrt(k) + 16) for k in sizes))
    d_tids = torch.empty(ub, dtype=torch.int32, device="cuda")
    real = np.zeros(count, dtype=np.int64)
    pos = 0
    for a, got, arr in datagen.pool_blocks(count, U, lo, hi, seed, workers=THREADS):
        d_tids[pos:pos + arr.size].copy_(torch.from_numpy(arr.view(np.int32)))
        real[a:a + got.size] = got
        pos += arr.size
    offsets = np.zeros(count + 1, dtype=np.uint64)
    offsets[1:] = np.cumsum(real)
    d_off = torch.from_numpy(offsets.view(np.int64)).cuda()
    pool = pkg.batmap_pool_create(U, d_off, d_tids[:pos], None)
    del d_tids
    torch.cuda.empty_cache()
    assert pool.info["n_elements"] == int(offsets[-1]) and pool.info["n_batmaps"] > 1000
    rng = np.random.default_rng(55)
    qs = [rng.integers(0, count, 2 if rng.random() < 0.8 else int(rng.integers(3, 9))).tolist()
          for _ in range(5000)]
    arrival = np.cumsum(rng.exponential(1.0 / 1e6, len(qs)))
    opts = pkg.batmap_serve_opts(max_batch=256, slots=4, work_budget=1 << 26, reserved=0)
    counts, lat, stats = pkg.batmap_serve(pool, qs, arrival, opts)
    ids = sorted({c for q in qs for c in q})
    remap = {c: j for j, c in enumerate(ids)}
    sub = datagen.pool_subset(U, lo, hi, seed, count, ids, workers=THREADS)
    assert np.array_equal(np.diff(sub.offsets).astype(np.int64), real[ids])
    ref = oracle.kway_counts(sub.offsets, sub.tids, [[remap[c] for c in q] for q in qs])
    assert np.array_equal(counts, ref)
    for q in range(0, len(qs), 50):
        assert int(pkg.intersect_query(pool, [qs[q]]).cpu().numpy()[0]) == int(counts[q]), q
    pool.free()
    torch.cuda.empty_cache()


@pytest.mark.parametrize("n", [16_000, 64_000])
def test_nsweep_shape_sampled(n):
    """The Sec. IV-A experiment shape (10^7 items at 5%, m = 10^7 / (0.05 n)) at
    n = 16,000 (128M pairs) and 64,000 (2.05e9 pairs, an 8.2 GB triangle):
    20,000 random pairs and 16 whole rows against the oracle, row sums by the
    invariant."""
    import torch
    import paper_1102_1003_gb300 as pkg
    _CACHE.clear()
    inst = datagen.nsweep_instance(n)
    off = torch.from_numpy(inst.offsets.view(np.int64)).cuda()
    tids = torch.from_numpy(inst.tids.view(np.int32)).cuda()
    npairs = n * (n - 1) // 2
    full = torch.full((npairs,), -1, dtype=torch.int32, device="cuda")
    b = pkg.batmap_build(inst.m, off, tids, None)
    none = torch.empty((1, 3), dtype=torch.int32, device="cuda")
    n_out, _ = pkg.pair_support_all(b, 2**32 - 1, pairs=none, full=full)
    torch.cuda.synchronize()
    assert n_out == 0
    rng = np.random.default_rng(n)
    rows = rng.choice(n, 16, replace=False)
    cols = np.arange(n)
    lo = np.concatenate([np.minimum(i, cols[cols != i]) for i in rows])
    hi = np.concatenate([np.maximum(i, cols[cols != i]) for i in rows])
    si = rng.integers(0, n - 1, 20_000)
    sj = si + 1 + (rng.integers(0, n, 20_000) % (n - 1 - si))
    ii, jj = np.concatenate([lo, si]), np.concatenate([hi, sj])
    idx = torch.from_numpy(oracle.packed_index(n, ii, jj)).cuda()
    got = full[idx].cpu().numpy().astype(np.uint32)
    ref = oracle.pairs_list(inst.offsets, inst.tids, ii, jj, threads=THREADS)
    assert np.array_equal(got, ref)
    tlen = np.bincount(inst.tids, minlength=inst.m).astype(np.int64)
    per_row = ref[:16 * (n - 1)].astype(np.int64).reshape(16, n - 1).sum(axis=1)
    for k, i in enumerate(rows):
        assert per_row[k] == (tlen[inst.tidlist(int(i))] - 1).sum()
    # no support is left unwritten (every entry was overwritten from -1)
    assert int((full == -1).sum().item()) == 0
    b.free()
    del full, off, tids
    pkg.batmap_release_scratch()
    torch.cuda.empty_cache()
