"""Sets built and queried on different CUDA streams, freed and rebuilt in
mixed orders (the BatMap arrays of freed sets are recycled): every result
stays bit-exact against the oracle."""
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


def test_streams_and_recycled_arrays_stay_exact():
    import torch
    import paper_1102_1003_gb300 as pkg
    insts = [datagen.zipf_tidlists(80_000, 150, 0.03, seed=21),
             datagen.bernoulli_tidlists(20_000, 90, 0.05, seed=22),
             datagen.zipf_tidlists(200_000, 60, 0.02, seed=23)]
    refs = [oracle.pairs_full(i.offsets, i.tids, threads=THREADS) for i in insts]
    streams = [torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.current_stream()]
    for rep in range(3):
        order = [(rep + q) % 3 for q in range(3)]
        live = []
        for q in order:
            with torch.cuda.stream(streams[q]):
                off, tids, perm = device_inputs(insts[q], q)
                b = pkg.batmap_build(insts[q].m, off, tids, perm, stream=streams[q])
                full = torch.empty(refs[q].size, dtype=torch.int32, device="cuda")
                pkg.pair_support_all(b, 1, full=full, stream=streams[q])
                live.append((q, b, full))
        torch.cuda.synchronize()
        for q, b, full in live:
            assert np.array_equal(full.cpu().numpy().astype(np.uint32), refs[q]), (rep, q)
        # free in a different order than built, then release the caches every other round
        for q, b, _ in reversed(live):
            b.free()
        if rep % 2:
            pkg.batmap_release_scratch()
