"""Autotuned schedules stay exact, and the batched form equals separate calls
after autotuning (CUDA graph rebuilt)."""
import os

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


def test_autotune_then_batch_exact():
    import torch
    import paper_1102_1003_gb300 as pkg
    specs = datagen.batch_specs(5, 2000, m_range=(1e4, 1e5), n_range=(100, 700))
    insts = [datagen.batch_instance(sp) for sp in specs]
    sets = []
    for q, inst in enumerate(insts):
        off, tids, perm = device_inputs(inst, q)
        sets.append(pkg.batmap_build(inst.m, off, tids, perm))
    eff = pkg.batmap_autotune(sets)
    assert len(eff) == pkg.NUM_SHAPES and max(eff) == pytest.approx(1.0) and min(eff) > 0
    fulls, bufs, refs = [], [], []
    for inst in insts:
        ref = oracle.pairs_full(inst.offsets, inst.tids, threads=os.cpu_count() or 4)
        refs.append(ref)
        fulls.append(torch.empty(ref.size, dtype=torch.int32, device="cuda"))
        bufs.append(torch.empty((max(int((ref >= inst.s).sum()), 1), 3), dtype=torch.int32, device="cuda"))
    n_outs = pkg.pair_support_batch(sets, [i.s for i in insts], bufs, fulls)
    for q, inst in enumerate(insts):
        assert np.array_equal(fulls[q].cpu().numpy().astype(np.uint32), refs[q])
        want = oracle.threshold_from_full(refs[q], inst.n, inst.s)
        assert n_outs[q] == want.shape[0]
        assert np.array_equal(bufs[q][:n_outs[q]].cpu().numpy().astype(np.uint32), want)
        # plain call after tuning agrees as well
        k, pairs = pkg.pair_support_all(sets[q], inst.s)
        assert k == want.shape[0] and np.array_equal(pairs.cpu().numpy().astype(np.uint32), want)
