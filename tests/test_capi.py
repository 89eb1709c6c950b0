"""The C-ABI library loads and exports every entry point include/batmap.h declares
(CPU only: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(",
                             text, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_1102_1003_gb300 import batmap
    return ctypes.CDLL(batmap.LIB_PATH)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("batmap_build", "pair_support_all", "pair_support_batch", "batmap_free",
                     "batmap_last_error", "pair_support_host"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_1102_1003_gb300 import batmap
    assert set(batmap.EXPORTED) <= set(_declared_functions())
    for name in batmap.EXPORTED:
        if name not in ("batmap_last_error",):
            assert hasattr(batmap, name) or name.startswith("batmap_"), name


def test_default_params_without_gpu(lib):
    from paper_1102_1003_gb300 import batmap
    p = batmap.batmap_default_params()
    assert (p.load_num, p.load_den, p.max_loop, p.min_shift, p.tile, p.validate, p.shape_mask) == \
        (2, 1, 32, 7, 0, 1, 0)
    assert batmap.load_library().batmap_last_error() == b""


def test_missing_library_fails_loudly(tmp_path):
    from paper_1102_1003_gb300 import batmap
    with pytest.raises(ImportError):
        batmap.load_library.__wrapped__(str(tmp_path / "nope.so")) if hasattr(
            batmap.load_library, "__wrapped__") else _load_missing(batmap, tmp_path)


def _load_missing(batmap, tmp_path):
    saved = batmap._lib
    batmap._lib = None
    try:
        batmap.load_library(str(tmp_path / "libbatmap_missing.so"))
    finally:
        batmap._lib = saved


def test_binding_refuses_malformed_tensors(lib):
    # checked before any device call, so this runs without a GPU
    import torch
    from paper_1102_1003_gb300 import batmap
    off = torch.tensor([0, 2], dtype=torch.int64)
    tids = torch.tensor([1, 3], dtype=torch.int32)
    perm = torch.arange(30, dtype=torch.int32).reshape(3, 10) % 10
    with pytest.raises(ValueError):
        batmap.batmap_build(10, off, tids.to(torch.int64), perm)          # 8-byte tids
    with pytest.raises(ValueError):
        batmap.batmap_build(10, off.to(torch.int32), tids, perm)          # 4-byte offsets
    with pytest.raises(ValueError):
        batmap.batmap_build(10, off, tids, perm[:2])                      # two permutation rows
    with pytest.raises(ValueError):
        batmap.batmap_build_d(3, 10, off, tids, perm)                     # d = 3 needs four rows
    with pytest.raises(ValueError):
        batmap.batmap_build(10, off, tids, perm)                          # host tensors


def test_binding_refuses_a_second_device(monkeypatch):
    # the library serves one GPU per process and works on the current device;
    # a stand-in tensor object exercises the check without a GPU
    from paper_1102_1003_gb300 import batmap

    class FakeCuda:
        is_cuda = True
        dtype = "int32"

        def __init__(self, index):
            self.device = type("D", (), {"index": index})()

        def is_contiguous(self):
            return True

        def element_size(self):
            return 4

        def data_ptr(self):
            return 4096

    current = {"dev": 0}
    monkeypatch.setattr(batmap, "_current_device", lambda: current["dev"])
    monkeypatch.setattr(batmap, "_device", None)
    assert batmap._ptr(FakeCuda(0)).value == 4096
    with pytest.raises(ValueError, match="is current"):
        batmap._ptr(FakeCuda(1))          # not the current device
    current["dev"] = 1
    with pytest.raises(ValueError, match="one GPU per process"):
        batmap._ptr(FakeCuda(1))          # a second GPU in the same process


def test_noalloc_wrapper_refuses_wrong_buffers():
    """The binding refuses supports or pair buffers of the wrong element size
    and a support array shorter than n(n-1)/2 before any call reaches the GPU."""
    torch = pytest.importorskip("torch")
    import paper_1102_1003_gb300 as pkg
    pairs = torch.zeros((4, 3), dtype=torch.int32)
    with pytest.raises(ValueError):
        pkg.pair_threshold_noalloc(torch.zeros(45, dtype=torch.int64), 10, 1, pairs)
    with pytest.raises(ValueError):
        pkg.pair_threshold_noalloc(torch.zeros(44, dtype=torch.int32), 10, 1, pairs)
    with pytest.raises(ValueError):
        pkg.pair_threshold_noalloc(torch.zeros(45, dtype=torch.int32), 10, 1, torch.zeros((4, 3), dtype=torch.int16))
    with pytest.raises(ValueError):
        pkg.pair_threshold_noalloc(None, 10, 1, pairs)
