"""GPU parity of the dense-bitmap tensor-core path (M M^T on tcgen05) against
the merge oracle: bit-exact supports and frequent pairs."""
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


def _dense(inst, s=None):
    import torch
    import paper_1102_1003_gb300 as pkg
    off, tids, _ = device_inputs(inst, 0)
    npairs = inst.n * (inst.n - 1) // 2
    full = torch.full((max(npairs, 1),), -1, dtype=torch.int32, device="cuda")
    n_out, pairs, timing = pkg.pair_support_dense(inst.m, off, tids, inst.s if s is None else s, full=full)
    torch.cuda.synchronize()
    return (full[:npairs].cpu().numpy().astype(np.uint32), n_out,
            pairs.cpu().numpy().astype(np.uint32).reshape(-1, 3), timing)


def _check(inst, s=None):
    s = inst.s if s is None else s
    full, n_out, pairs, _ = _dense(inst, s)
    ref = oracle.pairs_full(inst.offsets, inst.tids, threads=THREADS)
    assert np.array_equal(full, ref), f"{int((full != ref).sum())} of {ref.size} supports differ"
    want = oracle.threshold_from_full(ref, inst.n, s)
    assert n_out == want.shape[0] and np.array_equal(pairs, want)


def test_dense_small_ragged():
    # n not a multiple of 128/256, m not a multiple of 64
    _check(datagen.bernoulli_tidlists(3001, 131, 0.07, seed=3, s=10))


def test_dense_bernoulli_m10k():
    _check(datagen.workload_instance("bern_m10k_n200"))


@pytest.mark.parametrize("n", [1, 2, 255, 257, 600])
def test_dense_sizes(n):
    _check(datagen.zipf_tidlists(70_001, n, 0.05, seed=n, s=40))


@pytest.mark.parametrize("m,n", [(20_000, 1500), (64, 600), (1000, 3000), (300_000, 520)])
def test_dense_k_splits_and_block_counts(m, n):
    """K ranges split over several CTAs with their partial sums added, a
    single K step, more blocks than SMs, diagonal blocks at every position."""
    _check(datagen.bernoulli_tidlists(m, n, 0.05, seed=m % 97 + n, s=3))


def test_dense_empty_and_full_items():
    m = 5000
    lists = [[], np.arange(m, dtype=np.uint32), [], np.arange(0, m, 3, dtype=np.uint32), [7]]
    _check(datagen.from_lists(lists, m, s=1))


def test_dense_zipf_full_scale_exact():
    """The m = 10^6, n = 2,000 Zipf workload: supports up to ~10^6, i.e. FP32 accumulation carries
    20-bit integers exactly."""
    inst = datagen.workload_instance("zipf_m1m_n2000")
    _check(inst)


def test_bounded_wait_timeout_path_then_exact():
    """The error path of the tensor-core kernel's bounded waits: with the test
    hook the TMA producer issues nothing and every wait gives up after a few
    thousand polls, with no copy or MMA in flight; the call reports
    BATMAP_ERR_TIMEOUT, and the next call on the same workspace is exact."""
    import paper_1102_1003_gb300 as pkg
    inst = datagen.bernoulli_tidlists(5_000, 300, 0.05, seed=9, s=12)
    pkg.batmap_test_dense_timeout(4096)
    with pytest.raises(pkg.BatmapError) as e:
        _dense(inst)
    assert e.value.code == pkg.BATMAP_ERR_TIMEOUT
    _check(inst)
    # the hook applies to one call only, and 0 cancels it
    pkg.batmap_test_dense_timeout(4096)
    pkg.batmap_test_dense_timeout(0)
    _check(inst)
