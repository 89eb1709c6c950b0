"""The allocation-free compaction entry point (pair_threshold_noalloc).

It serves callers that cannot allocate device memory (a fixed memory budget,
or code that must not pay for the implicit synchronisation of cudaMalloc).
Its result must equal the compaction inside pair_support_all, exactly (the
counts are integers), on two calls in a row that share its fixed scratch
array.  This file is collected last so that a run stopping at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import datagen
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


def test_noalloc_matches_pair_support_all_twice():
    import torch
    import paper_1102_1003_gb300 as pkg
    from paper_1102_1003_gb300 import batmap as B
    inst = datagen.zipf_tidlists(40_000, 700, 0.03, seed=77, s=60)
    off, tids, perm = device_inputs(inst, 7)
    bset = pkg.batmap_build(inst.m, off, tids, perm)
    npairs = inst.n * (inst.n - 1) // 2
    full = torch.empty(npairs, dtype=torch.int32, device="cuda")
    for s in (inst.s, 1):
        n_ref, ref = pkg.pair_support_all(bset, s, full=full)
        ref = ref.cpu().numpy()
        for call in range(2):  # two calls in a row share the fixed scratch
            out = torch.full((n_ref + 5, 3), -1, dtype=torch.int32, device="cuda")
            n_out = pkg.pair_threshold_noalloc(full, inst.n, s, out)
            assert n_out == n_ref, (s, call)
            got = out.cpu().numpy()
            assert np.array_equal(got[:n_out], ref), (s, call)
            assert (got[n_out:] == -1).all()
    # capacity shortfall: first cap triples and the true count
    small = torch.empty((10, 3), dtype=torch.int32, device="cuda")
    assert pkg.pair_threshold_noalloc(full, inst.n, 1, small) == n_ref
    assert np.array_equal(small.cpu().numpy(), ref[:10])
    # beyond the fixed capacity: refused before any GPU work
    n_out = ctypes.c_uint64(0)
    rc = B.load_library().pair_threshold_noalloc(None, 30_000, 1, None, 0, ctypes.byref(n_out), None)
    assert rc == pkg.BATMAP_ERR_CAPACITY
    assert b"2^28" in B.load_library().batmap_last_error()


def _numpy_compaction(full: np.ndarray, n: int, s: int) -> np.ndarray:
    """(i, j, support) of the packed supports >= s, in array order (= lexicographic)."""
    idx = np.flatnonzero(full >= s).astype(np.int64)
    rows = np.arange(n, dtype=np.int64)
    starts = rows * n - rows * (rows + 1) // 2
    i = np.searchsorted(starts, idx, side="right") - 1
    j = idx - starts[i] + i + 1
    return np.stack([i, j, full[idx].astype(np.int64)], axis=1).astype(np.uint32)


@pytest.mark.parametrize("n", [5_000, 23_170])
def test_noalloc_random_supports_many_tiles_and_capacity_edge(n):
    """Random supports: n = 5,000 needs more than one tile of the single-block
    scan (3,052 block counts); n = 23,170 is the largest accepted size
    (n(n-1)/2 <= 2^28).  Two calls in a row, against a numpy compaction."""
    import torch
    import paper_1102_1003_gb300 as pkg
    npairs = n * (n - 1) // 2
    rng = np.random.default_rng(n)
    host = rng.integers(0, 1 << 20, npairs, dtype=np.uint32)
    s = (1 << 20) - 1500
    want = _numpy_compaction(host, n, s)
    full = torch.from_numpy(host.view(np.int32)).to("cuda")
    del host
    for call in range(2):
        out = torch.full((want.shape[0] + 3, 3), -1, dtype=torch.int32, device="cuda")
        n_out = pkg.pair_threshold_noalloc(full, n, s, out)
        assert n_out == want.shape[0], call
        got = out.cpu().numpy()
        assert np.array_equal(got[:n_out].astype(np.uint32), want), call
        assert (got[n_out:] == -1).all()


def test_noalloc_refuses_one_item_beyond_the_fixed_array():
    from paper_1102_1003_gb300 import batmap as B
    import paper_1102_1003_gb300 as pkg
    n_out = ctypes.c_uint64(0)
    rc = B.load_library().pair_threshold_noalloc(None, 23_171, 1, None, 0, ctypes.byref(n_out), None)
    assert rc == pkg.BATMAP_ERR_CAPACITY
