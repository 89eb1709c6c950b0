"""Cross mode (sparse boolean matrix multiplication / join-project, Sec. I):
supports |A_i cap B_j| between two families, bit-exact against the oracle."""
import os

import numpy as np
import pytest

import datagen
import oracle
from tests.gpu_util import device_inputs

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


def _families(m, na, nb, seed):
    a = datagen.zipf_tidlists(m, na, 0.03, seed=seed)
    b = datagen.bernoulli_tidlists(m, nb, 0.02, seed=seed + 1)
    return datagen.from_lists([a.tidlist(i) for i in range(na)] + [b.tidlist(j) for j in range(nb)], m)


def _expected(union, na):
    full = oracle.pairs_full(union.offsets, union.tids, threads=THREADS)
    nb = union.n - na
    a, b = np.meshgrid(np.arange(na), np.arange(nb), indexing="ij")
    return full[oracle.packed_index(union.n, a.ravel(), na + b.ravel())].reshape(na, nb)


@pytest.mark.parametrize("params", [None, dict(max_loop=1, load_num=1, load_den=2)])
@pytest.mark.parametrize("na,nb", [(150, 220), (1, 300), (257, 3)])
def test_cross_supports_exact(na, nb, params):
    import torch
    import paper_1102_1003_gb300 as pkg
    union = _families(40_000, na, nb, seed=na + nb)
    ref = _expected(union, na)
    off, tids, perm = device_inputs(union, 5)
    bset = pkg.batmap_build_cross(union.m, na, off, tids, perm,
                                  params=pkg.batmap_default_params(**params) if params else None)
    assert bset.info["n_a"] == na
    full = torch.empty(na * nb, dtype=torch.int32, device="cuda")
    for s in (1, 20):
        n_out, pairs = pkg.pair_support_all(bset, s, full=full)
        got = full.cpu().numpy().astype(np.uint32).reshape(na, nb)
        assert np.array_equal(got, ref)
        a, b = np.nonzero(ref >= s)
        want = np.stack([a, b, ref[a, b]], axis=1).astype(np.uint32)
        assert n_out == want.shape[0]
        assert np.array_equal(pairs.cpu().numpy().astype(np.uint32).reshape(-1, 3), want)


def test_cross_in_a_batch_with_an_all_pairs_set():
    import torch
    import paper_1102_1003_gb300 as pkg
    union = _families(30_000, 120, 90, seed=3)
    plain = datagen.zipf_tidlists(30_000, 200, 0.03, seed=4, s=30)
    ref_c = _expected(union, 120)
    ref_p = oracle.pairs_full(plain.offsets, plain.tids, threads=THREADS)
    o1, t1, p1 = device_inputs(union, 1)
    o2, t2, p2 = device_inputs(plain, 2)
    sets = [pkg.batmap_build_cross(union.m, 120, o1, t1, p1), pkg.batmap_build(plain.m, o2, t2, p2)]
    fulls = [torch.empty(120 * 90, dtype=torch.int32, device="cuda"),
             torch.empty(ref_p.size, dtype=torch.int32, device="cuda")]
    bufs = [torch.empty((int((ref_c >= 1).sum()), 3), dtype=torch.int32, device="cuda"),
            torch.empty((int((ref_p >= 30).sum()), 3), dtype=torch.int32, device="cuda")]
    pkg.pair_support_batch(sets, [1, 30], bufs, fulls)
    assert np.array_equal(fulls[0].cpu().numpy().astype(np.uint32).reshape(120, 90), ref_c)
    assert np.array_equal(fulls[1].cpu().numpy().astype(np.uint32), ref_p)
