"""Python binding of libbatmap.so (argument marshalling only).

Every function here has the name of the C entry point it calls (include/
batmap.h).  Device buffers are torch CUDA tensors, streams are torch CUDA
streams; all computation runs in the library's CUDA kernels.  There is no CPU
fallback: if the library is missing, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libbatmap.so")

BATMAP_OK = 0
BATMAP_ERR_ARG = -1
BATMAP_ERR_NOMEM = -2
BATMAP_ERR_CAPACITY = -3
BATMAP_ERR_CUDA = -4
BATMAP_ERR_TIMEOUT = -5
BATMAP_ERR_INTERNAL = -6
NUM_SHAPES = 18  # BATMAP_NUM_SHAPES: compare tile shapes

EXPORTED = [
    "batmap_default_params", "batmap_last_error", "batmap_build", "batmap_free",
    "batmap_get_info", "batmap_export_layout", "pair_support_all", "pair_support_host",
    "pair_support_batch", "batmap_get_timing", "batmap_kernel_launches", "pair_threshold_noalloc",
    "pair_support_dense", "batmap_pool_create", "batmap_pool_free", "batmap_pool_info", "intersect_query",
    "batmap_serve", "batmap_autotune", "batmap_release_scratch", "intersect_query_list", "batmap_build_cross",
    "batmap_build_d", "itemset_support", "frequent_triples", "batmap_test_dense_timeout",
    "frequent_quadruples",
]


class batmap_params(ctypes.Structure):
    _fields_ = [("load_num", ctypes.c_uint32), ("load_den", ctypes.c_uint32),
                ("max_loop", ctypes.c_uint32), ("min_shift", ctypes.c_uint32),
                ("tile", ctypes.c_uint32), ("validate", ctypes.c_uint32),
                ("shape_mask", ctypes.c_uint32), ("probe_log", ctypes.c_uint32),
                ("perm_seed", ctypes.c_uint64)]


class batmap_info(ctypes.Structure):
    _fields_ = [("m", ctypes.c_uint32), ("n", ctypes.c_uint32), ("shift", ctypes.c_uint32),
                ("r0", ctypes.c_uint32), ("bytes", ctypes.c_uint64),
                ("n_elements", ctypes.c_uint64), ("n_failed", ctypes.c_uint64),
                ("n_corrections", ctypes.c_uint64), ("n_work_units", ctypes.c_uint64),
                ("n_classes", ctypes.c_uint32), ("n_a", ctypes.c_uint32),
                ("word_pairs", ctypes.c_double), ("d", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("probe_word_pairs", ctypes.c_double), ("probe_words", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class batmap_timing(ctypes.Structure):
    _fields_ = [("build_ms", ctypes.c_float), ("place_ms", ctypes.c_float),
                ("finalize_ms", ctypes.c_float), ("compare_ms", ctypes.c_float),
                ("compact_ms", ctypes.c_float), ("pairs_ms", ctypes.c_float),
                ("scan_ms", ctypes.c_float), ("probe_ms", ctypes.c_float)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class batmap_out(ctypes.Structure):
    _fields_ = [("d_pairs", ctypes.c_void_p), ("cap", ctypes.c_uint64),
                ("n_out", ctypes.c_uint64), ("d_full", ctypes.c_void_p)]


class batmap_serve_opts(ctypes.Structure):
    _fields_ = [("max_batch", ctypes.c_uint32), ("slots", ctypes.c_uint32),
                ("work_budget", ctypes.c_uint64), ("reserved", ctypes.c_uint64)]


class batmap_serve_stats(ctypes.Structure):
    _fields_ = [("makespan_s", ctypes.c_double), ("queries_per_s", ctypes.c_double),
                ("p50_s", ctypes.c_double), ("p99_s", ctypes.c_double), ("max_s", ctypes.c_double),
                ("batches", ctypes.c_uint64), ("max_inflight", ctypes.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class BatmapError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"batmap error {code}: {msg}")
        self.code = code


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libbatmap.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(path)
    vp, u32, u64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
    L.batmap_default_params.argtypes = [ctypes.POINTER(batmap_params)]
    L.batmap_default_params.restype = None
    L.batmap_last_error.argtypes = []
    L.batmap_last_error.restype = ctypes.c_char_p
    L.batmap_build.argtypes = [ctypes.POINTER(batmap_params), u32, u32, vp, vp, vp, vp,
                               ctypes.POINTER(vp)]
    L.batmap_build.restype = ctypes.c_int
    L.batmap_build_cross.argtypes = [ctypes.POINTER(batmap_params), u32, u32, u32, vp, vp, vp, vp,
                                      ctypes.POINTER(vp)]
    L.batmap_build_cross.restype = ctypes.c_int
    L.batmap_free.argtypes = [vp]
    L.batmap_free.restype = None
    L.batmap_get_info.argtypes = [vp, ctypes.POINTER(batmap_info)]
    L.batmap_get_info.restype = ctypes.c_int
    L.batmap_export_layout.argtypes = [vp, vp, vp, vp, vp, vp]
    L.batmap_export_layout.restype = ctypes.c_int
    L.pair_support_all.argtypes = [vp, u32, vp, u64, ctypes.POINTER(u64), vp, vp]
    L.pair_support_all.restype = ctypes.c_int
    L.pair_support_host.argtypes = [ctypes.POINTER(batmap_params), u32, u32, vp, vp, vp, u32, vp,
                                    u64, ctypes.POINTER(u64), vp]
    L.pair_support_host.restype = ctypes.c_int
    L.pair_support_batch.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(u32), u32,
                                     ctypes.POINTER(batmap_out), vp]
    L.pair_support_batch.restype = ctypes.c_int
    L.batmap_get_timing.argtypes = [vp, ctypes.POINTER(batmap_timing)]
    L.batmap_get_timing.restype = ctypes.c_int
    L.batmap_kernel_launches.argtypes = []
    L.batmap_kernel_launches.restype = u64
    L.pair_support_dense.argtypes = [u32, u32, vp, vp, u32, vp, u64, ctypes.POINTER(u64), vp,
                                     ctypes.POINTER(batmap_timing), vp]
    L.pair_support_dense.restype = ctypes.c_int
    L.batmap_pool_create.argtypes = [ctypes.POINTER(batmap_params), u32, u32, vp, vp, vp, vp, ctypes.POINTER(vp)]
    L.batmap_pool_create.restype = ctypes.c_int
    L.batmap_pool_free.argtypes = [vp]
    L.batmap_pool_free.restype = None
    L.batmap_pool_info.argtypes = [vp, ctypes.POINTER(u32), ctypes.POINTER(u64), ctypes.POINTER(u64)]
    L.batmap_pool_info.restype = ctypes.c_int
    L.intersect_query.argtypes = [vp, vp, vp, u32, vp, vp]
    L.intersect_query.restype = ctypes.c_int
    L.intersect_query_list.argtypes = [vp, vp, vp, u32, vp, vp, u64, ctypes.POINTER(u64), vp]
    L.intersect_query_list.restype = ctypes.c_int
    L.batmap_serve.argtypes = [vp, vp, vp, vp, u32, ctypes.POINTER(batmap_serve_opts), vp, vp,
                               ctypes.POINTER(batmap_serve_stats), vp]
    L.batmap_serve.restype = ctypes.c_int
    L.batmap_release_scratch.argtypes = []
    L.batmap_release_scratch.restype = None
    L.batmap_autotune.argtypes = [ctypes.POINTER(vp), u32, ctypes.POINTER(ctypes.c_double), vp]
    L.batmap_autotune.restype = ctypes.c_int
    L.pair_threshold_noalloc.argtypes = [vp, u32, u32, vp, u64, ctypes.POINTER(u64), vp]
    L.pair_threshold_noalloc.restype = ctypes.c_int
    L.batmap_build_d.argtypes = [ctypes.POINTER(batmap_params), u32, u32, u32, vp, vp, vp, vp, ctypes.POINTER(vp)]
    L.batmap_build_d.restype = ctypes.c_int
    L.itemset_support.argtypes = [vp, u32, u64, vp, vp, vp]
    L.itemset_support.restype = ctypes.c_int
    L.frequent_triples.argtypes = [vp, u32, vp, u64, vp, u64, ctypes.POINTER(u64), ctypes.POINTER(u64), vp]
    L.frequent_triples.restype = ctypes.c_int
    L.frequent_quadruples.argtypes = [vp, u32, vp, u64, vp, u64, ctypes.POINTER(u64), ctypes.POINTER(u64), vp]
    L.frequent_quadruples.restype = ctypes.c_int
    L.batmap_test_dense_timeout.argtypes = [u32]
    L.batmap_test_dense_timeout.restype = None
    _lib = L
    return L


def _check(rc, allow=()):
    if rc != BATMAP_OK and rc not in allow:
        raise BatmapError(rc, load_library().batmap_last_error().decode())
    return rc


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


_device = None  # the one GPU this process's library works on (set at first use)


def _current_device() -> int:
    import torch
    return torch.cuda.current_device()


def _check_device(index: int) -> None:
    """The library works on the current device and on one GPU per process: a
    tensor on another device, or a second GPU, is refused here."""
    global _device
    cur = _current_device()
    if index != cur:
        raise ValueError(f"tensor on cuda:{index} but cuda:{cur} is current; the library works on the "
                         "current device")
    if _device is None:
        _device = index
    elif index != _device:
        raise ValueError(f"this process already uses cuda:{_device}; the library serves one GPU per process")


def _ptr(t):
    """Device pointer of a contiguous CUDA tensor of 4- or 8-byte elements (None -> NULL).
    The library reads raw memory, so a strided view or a host tensor is refused here."""
    if t is None:
        return ctypes.c_void_p(0)
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    if t.element_size() not in (4, 8):
        raise ValueError(f"expected 4- or 8-byte elements, got {t.dtype}")
    _check_device(t.device.index)
    return ctypes.c_void_p(t.data_ptr())


def _check_inputs(offsets, tids, perm=None):
    """CSR offsets are 8-byte, tids and permutations 4-byte elements (the ABI's uint64 / uint32).
    perm None selects the permutations the library computes (params.perm_seed)."""
    if offsets.element_size() != 8:
        raise ValueError(f"offsets must hold 8-byte integers, got {offsets.dtype}")
    if tids.element_size() != 4:
        raise ValueError(f"tids must hold 4-byte integers, got {tids.dtype}")
    if perm is not None and perm.element_size() != 4:
        raise ValueError(f"perm must hold 4-byte integers, got {perm.dtype}")


def batmap_default_params(**overrides) -> batmap_params:
    p = batmap_params()
    load_library().batmap_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        setattr(p, k, int(v))
    return p


class BatMapSet:
    """Owning wrapper of a built batmap_set handle."""

    def __init__(self, handle, m, n):
        self.handle = handle
        self.m = m
        self.n = n

    def __del__(self):
        self.free()

    def free(self):
        if getattr(self, "handle", None):
            load_library().batmap_free(self.handle)
            self.handle = None

    @property
    def info(self) -> dict:
        return batmap_get_info(self)


def batmap_build(m: int, offsets, tids, perm=None, params: batmap_params | None = None,
                 stream=None) -> BatMapSet:
    """Build the BatMaps of n = offsets.numel() - 1 items from device CSR tidlists.

    offsets: cuda uint64 (int64) tensor [n+1]; tids: cuda int32/uint32 [T];
    perm: cuda int32/uint32 [3, m] (three permutations of [0, m)), or None for the
    permutations the library computes from params.perm_seed."""
    _check_inputs(offsets, tids, perm)
    if perm is not None and int(m) >= 1 and int(perm.numel()) != 3 * int(m):
        raise ValueError(f"perm must hold 3 rows of m = {m} entries")
    L = load_library()
    n = int(offsets.numel()) - 1
    h = ctypes.c_void_p()
    pp = ctypes.byref(params) if params is not None else None
    _check(L.batmap_build(pp, int(m), n, _ptr(offsets), _ptr(tids) if tids.numel() else None,
                          _ptr(perm), _stream_handle(stream), ctypes.byref(h)))
    return BatMapSet(h, int(m), n)


def batmap_build_cross(m: int, n_a: int, offsets, tids, perm=None, params: batmap_params | None = None,
                       stream=None) -> BatMapSet:
    """Cross-mode set: the CSR holds n_a sets of family A then the sets of family B;
    pair_support_all then reports the n_a x n_b supports |A_i cap B_j|."""
    _check_inputs(offsets, tids, perm)
    if perm is not None and int(m) >= 1 and int(perm.numel()) != 3 * int(m):
        raise ValueError(f"perm must hold 3 rows of m = {m} entries")
    L = load_library()
    n = int(offsets.numel()) - 1
    h = ctypes.c_void_p()
    pp = ctypes.byref(params) if params is not None else None
    _check(L.batmap_build_cross(pp, int(m), int(n_a), n - int(n_a), _ptr(offsets),
                                _ptr(tids) if tids.numel() else None, _ptr(perm), _stream_handle(stream),
                                ctypes.byref(h)))
    b = BatMapSet(h, int(m), n)
    b.n_a = int(n_a)
    return b


def batmap_build_d(d: int, m: int, offsets, tids, perm=None, params: batmap_params | None = None,
                   stream=None) -> BatMapSet:
    """d-of-(d+1) BatMaps (Sec. V generalisation): d = 2 is batmap_build; d = 3 and 4 build
    3-of-4 and 4-of-5 BatMaps for itemset_support / frequent_triples / frequent_quadruples.
    perm: cuda [d+1, m] or None (computed from params.perm_seed)."""
    _check_inputs(offsets, tids, perm)
    L = load_library()
    n = int(offsets.numel()) - 1
    if perm is not None and d in (2, 3, 4) and int(m) >= 1 and int(perm.numel()) != (d + 1) * int(m):
        raise ValueError(f"perm must hold {d + 1} rows of m = {m} entries")
    h = ctypes.c_void_p()
    pp = ctypes.byref(params) if params is not None else None
    _check(L.batmap_build_d(pp, int(d), int(m), n, _ptr(offsets), _ptr(tids) if tids.numel() else None,
                            _ptr(perm), _stream_handle(stream), ctypes.byref(h)))
    b = BatMapSet(h, int(m), n)
    b.d = int(d)
    return b


def itemset_support(bset: BatMapSet, items, support=None, stream=None):
    """|S_a1 cap ... cap S_ak| for a cuda int32 tensor items [n_q, k] (k <= 3) on a
    3-of-4 set; returns the cuda int32 [n_q] supports."""
    import torch
    nq, k = int(items.shape[0]), int(items.shape[1])
    if support is None:
        support = torch.empty(max(nq, 1), dtype=torch.int32, device=items.device)
    _check(load_library().itemset_support(bset.handle, k, nq, _ptr(items) if nq else None,
                                          _ptr(support), _stream_handle(stream)))
    return support[:nq]


def frequent_triples(bset: BatMapSet, s: int, pairs, out=None, stream=None):
    """Frequent itemsets of size 3 from the frequent pairs (cuda int32 [k, 3], the
    output of pair_support_all with the same s); returns (n_out, triples view
    [min(n_out, cap), 4] of (a, b, c, support), n_candidates)."""
    import torch
    L = load_library()
    np_ = int(pairs.shape[0])
    n_out, n_cand = ctypes.c_uint64(0), ctypes.c_uint64(0)
    st = _stream_handle(stream)
    pp = _ptr(pairs) if np_ else None
    if out is None:
        rc = L.frequent_triples(bset.handle, int(s), pp, np_, None, 0, ctypes.byref(n_out),
                                ctypes.byref(n_cand), st)
        _check(rc, allow=(BATMAP_ERR_CAPACITY,))
        out = torch.empty((max(int(n_out.value), 1), 4), dtype=torch.int32, device="cuda")
    cap = out.numel() // 4
    rc = L.frequent_triples(bset.handle, int(s), pp, np_, _ptr(out), cap, ctypes.byref(n_out),
                            ctypes.byref(n_cand), st)
    _check(rc, allow=(BATMAP_ERR_CAPACITY,))
    k = min(int(n_out.value), cap)
    return int(n_out.value), out.view(-1, 4)[:k], int(n_cand.value)


def frequent_quadruples(bset: BatMapSet, s: int, triples, out=None, stream=None):
    """Frequent itemsets of size 4 from the frequent triples (cuda int32 [k, 4], the
    output of frequent_triples with the same s) on a 4-of-5 set; returns (n_out,
    quadruples view [min(n_out, cap), 5] of (a, b, c, d, support), n_candidates)."""
    import torch
    L = load_library()
    nt = int(triples.shape[0])
    n_out, n_cand = ctypes.c_uint64(0), ctypes.c_uint64(0)
    st = _stream_handle(stream)
    tp = _ptr(triples) if nt else None
    if out is None:
        rc = L.frequent_quadruples(bset.handle, int(s), tp, nt, None, 0, ctypes.byref(n_out),
                                   ctypes.byref(n_cand), st)
        _check(rc, allow=(BATMAP_ERR_CAPACITY,))
        out = torch.empty((max(int(n_out.value), 1), 5), dtype=torch.int32, device="cuda")
    cap = out.numel() // 5
    rc = L.frequent_quadruples(bset.handle, int(s), tp, nt, _ptr(out), cap, ctypes.byref(n_out),
                               ctypes.byref(n_cand), st)
    _check(rc, allow=(BATMAP_ERR_CAPACITY,))
    k = min(int(n_out.value), cap)
    return int(n_out.value), out.view(-1, 5)[:k], int(n_cand.value)


def batmap_free(bset: BatMapSet):
    bset.free()


def batmap_get_info(bset: BatMapSet) -> dict:
    info = batmap_info()
    _check(load_library().batmap_get_info(bset.handle, ctypes.byref(info)))
    return info.as_dict()


def batmap_get_timing(bset: BatMapSet) -> dict:
    """Device durations (ms) of the set's most recent build / pair_support_all phases."""
    t = batmap_timing()
    _check(load_library().batmap_get_timing(bset.handle, ctypes.byref(t)))
    return t.as_dict()


def batmap_release_scratch():
    """Free the scratch the library caches between calls."""
    load_library().batmap_release_scratch()


def batmap_kernel_launches() -> int:
    return int(load_library().batmap_kernel_launches())


def batmap_export_layout(bset: BatMapSet) -> dict:
    """Host copies of the built layout (for checking it against the definition)."""
    info = batmap_get_info(bset)
    n = bset.n
    out = dict(bytes=np.zeros(info["bytes"], np.uint8), byte_offset=np.zeros(n, np.uint64),
               range=np.zeros(n, np.uint32), fail_offsets=np.zeros(n + 1, np.uint64),
               fail_tids=np.zeros(max(info["n_failed"], 1), np.uint32), info=info)
    _check(load_library().batmap_export_layout(
        bset.handle, out["bytes"].ctypes.data, out["byte_offset"].ctypes.data, out["range"].ctypes.data,
        out["fail_offsets"].ctypes.data, out["fail_tids"].ctypes.data))
    out["fail_tids"] = out["fail_tids"][:info["n_failed"]]
    return out


def pair_support_all(bset: BatMapSet, s: int, pairs=None, full=None, stream=None):
    """Supports of all pairs; returns (n_out, pairs) with pairs a cuda int32 [k, 3] view
    (i, j, support) of the first min(n_out, cap) qualifying pairs.  If `pairs` is None a
    buffer is sized by a counting call first.  `full` (optional) receives the packed
    upper triangle."""
    import torch
    L = load_library()
    n_out = ctypes.c_uint64(0)
    st = _stream_handle(stream)
    if pairs is None:
        rc = L.pair_support_all(bset.handle, int(s), None, 0, ctypes.byref(n_out), _ptr(full), st)
        _check(rc, allow=(BATMAP_ERR_CAPACITY,))
        pairs = torch.empty((max(int(n_out.value), 1), 3), dtype=torch.int32, device="cuda")
    cap = pairs.numel() // 3
    rc = L.pair_support_all(bset.handle, int(s), _ptr(pairs), cap, ctypes.byref(n_out), _ptr(full), st)
    _check(rc, allow=(BATMAP_ERR_CAPACITY,))
    k = min(int(n_out.value), cap)
    return int(n_out.value), pairs.view(-1, 3)[:k]


def pair_support_dense(m: int, offsets, tids, s: int, pairs=None, full=None, stream=None):
    """Dense-bitmap tensor-core path; returns (n_out, pairs view, timing dict)."""
    import torch
    _check_inputs(offsets, tids)
    L = load_library()
    n = int(offsets.numel()) - 1
    n_out = ctypes.c_uint64(0)
    t = batmap_timing()
    st = _stream_handle(stream)
    if pairs is None:
        rc = L.pair_support_dense(int(m), n, _ptr(offsets), _ptr(tids), int(s), None, 0, ctypes.byref(n_out),
                                  _ptr(full), ctypes.byref(t), st)
        _check(rc, allow=(BATMAP_ERR_CAPACITY,))
        pairs = torch.empty((max(int(n_out.value), 1), 3), dtype=torch.int32, device="cuda")
    cap = pairs.numel() // 3
    rc = L.pair_support_dense(int(m), n, _ptr(offsets), _ptr(tids), int(s), _ptr(pairs), cap,
                              ctypes.byref(n_out), _ptr(full), ctypes.byref(t), st)
    _check(rc, allow=(BATMAP_ERR_CAPACITY,))
    k = min(int(n_out.value), cap)
    return int(n_out.value), pairs.view(-1, 3)[:k], t.as_dict()


def batmap_test_dense_timeout(spin_limit: int):
    """Make the next pair_support_dense call exercise its bounded-wait error path
    (producer issues nothing, waits give up after spin_limit polls); 0 cancels."""
    load_library().batmap_test_dense_timeout(int(spin_limit))


def batmap_autotune(sets, stream=None):
    """Measure every tile shape on these sets, adopt the result for scheduling and
    reschedule them; returns the relative throughput per shape (1..NUM_SHAPES)."""
    L = load_library()
    k = len(sets)
    handles = (ctypes.c_void_p * k)(*[b.handle for b in sets])
    eff = (ctypes.c_double * NUM_SHAPES)()
    _check(L.batmap_autotune(handles, k, eff, _stream_handle(stream)))
    return list(eff)


def pair_support_batch(sets, s_list, pairs_list, full_list=None, stream=None):
    """One batched call over several sets; returns the per-instance n_out list."""
    L = load_library()
    k = len(sets)
    handles = (ctypes.c_void_p * k)(*[b.handle for b in sets])
    svals = (ctypes.c_uint32 * k)(*[int(x) for x in s_list])
    outs = (batmap_out * k)()
    for q in range(k):
        outs[q].d_pairs = pairs_list[q].data_ptr() if pairs_list[q] is not None else None
        outs[q].cap = (pairs_list[q].numel() // 3) if pairs_list[q] is not None else 0
        outs[q].d_full = (full_list[q].data_ptr() if full_list is not None and full_list[q] is not None
                          else None)
    rc = L.pair_support_batch(handles, svals, k, outs, _stream_handle(stream))
    _check(rc, allow=(BATMAP_ERR_CAPACITY,))
    return [int(outs[q].n_out) for q in range(k)]


def pair_support_host(m: int, offsets: np.ndarray, tids: np.ndarray, perm, s: int,
                      pairs_out: np.ndarray, params: batmap_params | None = None, stream=None) -> int:
    """End to end from host (preferably pinned) numpy buffers; returns n_out.  perm None
    selects the computed permutations (nothing to copy)."""
    L = load_library()
    n = offsets.size - 1
    n_out = ctypes.c_uint64(0)
    pp = ctypes.byref(params) if params is not None else None
    rc = L.pair_support_host(pp, int(m), n, offsets.ctypes.data, tids.ctypes.data if tids.size else None,
                             perm.ctypes.data if perm is not None else None, int(s), pairs_out.ctypes.data,
                             pairs_out.size // 3,
                             ctypes.byref(n_out), _stream_handle(stream))
    _check(rc, allow=(BATMAP_ERR_CAPACITY,))
    return int(n_out.value)


def pair_threshold_noalloc(full, n: int, s: int, pairs, stream=None) -> int:
    """Frequent pairs from the packed supports `full` into the caller's `pairs`
    buffer (cuda int32 [cap, 3]) without any device allocation by the library;
    returns n_out.  For callers that cannot allocate device memory."""
    L = load_library()
    npairs = int(n) * (int(n) - 1) // 2 if int(n) > 1 else 0
    if full is not None and full.element_size() != 4:
        raise ValueError(f"full must hold 4-byte supports, got {full.dtype}")
    if pairs is not None and pairs.element_size() != 4:
        raise ValueError(f"pairs must hold 4-byte integers, got {pairs.dtype}")
    if npairs and (full is None or int(full.numel()) < npairs):
        raise ValueError(f"full must hold n(n-1)/2 = {npairs} supports for n = {n}")
    n_out = ctypes.c_uint64(0)
    cap = pairs.numel() // 3 if pairs is not None else 0
    rc = L.pair_threshold_noalloc(_ptr(full), int(n), int(s), _ptr(pairs), cap, ctypes.byref(n_out),
                                  _stream_handle(stream))
    _check(rc, allow=(BATMAP_ERR_CAPACITY,))
    return int(n_out.value)


class BatMapPool:
    """Owning wrapper of a batmap_pool handle."""

    def __init__(self, handle, m, n):
        self.handle, self.m, self.n = handle, m, n

    def __del__(self):
        self.free()

    def free(self):
        if getattr(self, "handle", None):
            load_library().batmap_pool_free(self.handle)
            self.handle = None

    @property
    def info(self) -> dict:
        nb, by, ne = ctypes.c_uint32(0), ctypes.c_uint64(0), ctypes.c_uint64(0)
        _check(load_library().batmap_pool_info(self.handle, ctypes.byref(nb), ctypes.byref(by), ctypes.byref(ne)))
        return {"n_batmaps": nb.value, "batmap_bytes": by.value, "n_elements": ne.value}


def batmap_pool_create(m: int, offsets, tids, perm=None, params: batmap_params | None = None,
                       stream=None) -> BatMapPool:
    """Resident pool of sets; perm None selects the computed permutations."""
    _check_inputs(offsets, tids, perm)
    if perm is not None and int(m) >= 1 and int(perm.numel()) != 3 * int(m):
        raise ValueError(f"perm must hold 3 rows of m = {m} entries")
    L = load_library()
    n = int(offsets.numel()) - 1
    h = ctypes.c_void_p()
    pp = ctypes.byref(params) if params is not None else None
    _check(L.batmap_pool_create(pp, int(m), n, _ptr(offsets), _ptr(tids) if tids.numel() else None, _ptr(perm),
                                _stream_handle(stream), ctypes.byref(h)))
    return BatMapPool(h, int(m), n)


def batmap_pool_free(pool: BatMapPool):
    pool.free()


def batmap_pool_info(pool: BatMapPool) -> dict:
    return pool.info


def _queries_csr(queries):
    qoff = np.zeros(len(queries) + 1, dtype=np.uint32)
    qoff[1:] = np.cumsum([len(q) for q in queries])
    ids = (np.concatenate([np.asarray(q, dtype=np.uint32) for q in queries]) if len(queries)
           else np.zeros(1, np.uint32))
    return qoff, np.ascontiguousarray(ids, dtype=np.uint32)


def intersect_query(pool: BatMapPool, queries, counts=None, stream=None):
    """|S_a1 cap ... cap S_ak| for each query (a list of set ids); returns a cuda int64 tensor."""
    import torch
    qoff, ids = _queries_csr(queries)
    if counts is None:
        counts = torch.zeros(max(len(queries), 1), dtype=torch.int64, device="cuda")
    _check(load_library().intersect_query(pool.handle, qoff.ctypes.data, ids.ctypes.data, len(queries),
                                          _ptr(counts), _stream_handle(stream)))
    return counts[:len(queries)]


def intersect_query_list(pool: BatMapPool, queries, stream=None):
    """Elements of each query's intersection; returns (offsets int64 [nq+1], elements int32),
    both cuda tensors.  Sizes the output with a first counting call."""
    import torch
    L = load_library()
    qoff, ids = _queries_csr(queries)
    nq = len(queries)
    off = torch.zeros(nq + 1, dtype=torch.int64, device="cuda")
    total = ctypes.c_uint64(0)
    st = _stream_handle(stream)
    rc = L.intersect_query_list(pool.handle, qoff.ctypes.data, ids.ctypes.data, nq, _ptr(off), None, 0,
                                ctypes.byref(total), st)
    _check(rc, allow=(BATMAP_ERR_CAPACITY,))
    out = torch.empty(max(int(total.value), 1), dtype=torch.int32, device="cuda")
    _check(L.intersect_query_list(pool.handle, qoff.ctypes.data, ids.ctypes.data, nq, _ptr(off), _ptr(out),
                                  out.numel(), ctypes.byref(total), st))
    return off, out[:int(total.value)]


def batmap_serve(pool: BatMapPool, queries, arrival_s, opts: batmap_serve_opts | None = None, stream=None):
    """Run the continuous-batching loop; returns (counts uint64, latency_s float64, stats dict)."""
    qoff, ids = _queries_csr(queries)
    arr = np.ascontiguousarray(arrival_s, dtype=np.float64)
    nq = len(queries)
    counts = np.zeros(max(nq, 1), dtype=np.uint64)
    lat = np.zeros(max(nq, 1), dtype=np.float64)
    st = batmap_serve_stats()
    _check(load_library().batmap_serve(pool.handle, qoff.ctypes.data, ids.ctypes.data, arr.ctypes.data, nq,
                                       ctypes.byref(opts) if opts is not None else None, counts.ctypes.data,
                                       lat.ctypes.data, ctypes.byref(st), _stream_handle(stream)))
    return counts[:nq], lat[:nq], st.as_dict()
