"""Oracle for all-pairs support counting -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
arm may import this package.  It shares no code with the CUDA path.

`oracle.c` holds the plain definition (|S_i intersect S_j| by sorted merge);
this module loads it with ctypes, compiling it with gcc on first use when no
built copy exists.  `batmap_rules` restates the paper's BatMap rules on the
CPU (sizing, layout hash, 8-bit codes, indicator bits, counting rule, the
serial INSERT procedure) for pins and for checking layouts built on the GPU;
`dof_rules` does the same for the d-of-(d+1) generalisation of Sec. V and holds
the Apriori candidate step for itemsets of size 3.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None
_lock = threading.Lock()

_u32p = ctypes.POINTER(ctypes.c_uint32)
_u64p = ctypes.POINTER(ctypes.c_uint64)


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library (plain -O2, single-threaded code)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            L.oracle_intersect_count.restype = ctypes.c_uint64
            L.oracle_intersect_count.argtypes = [_u32p, ctypes.c_uint64, _u32p, ctypes.c_uint64]
            L.oracle_pairs_rows.restype = None
            L.oracle_pairs_rows.argtypes = [ctypes.c_uint32, _u64p, _u32p, ctypes.c_uint32,
                                            ctypes.c_uint32, _u32p]
            L.oracle_pairs_list.restype = None
            L.oracle_pairs_list.argtypes = [ctypes.c_uint64, _u32p, _u32p, _u64p, _u32p, _u32p]
            L.oracle_pairs_threshold.restype = ctypes.c_uint64
            L.oracle_pairs_threshold.argtypes = [ctypes.c_uint32, _u64p, _u32p, ctypes.c_uint32,
                                                 _u32p, ctypes.c_uint64]
            L.oracle_kway_list.restype = None
            L.oracle_kway_elems.restype = ctypes.c_uint64
            L.oracle_kway_elems.argtypes = [ctypes.c_uint32, _u32p, _u64p, _u32p, _u32p]
            L.oracle_kway_list.argtypes = [ctypes.c_uint64, _u32p, _u32p, _u64p, _u32p, _u32p, _u64p]
            _lib = L
    return _lib


def _p32(a: np.ndarray):
    return a.ctypes.data_as(_u32p)


def _p64(a: np.ndarray):
    return a.ctypes.data_as(_u64p)


def _csr(offsets, tids):
    return (np.ascontiguousarray(offsets, dtype=np.uint64),
            np.ascontiguousarray(tids, dtype=np.uint32))


def intersect_count(a, b) -> int:
    a = np.ascontiguousarray(a, dtype=np.uint32)
    b = np.ascontiguousarray(b, dtype=np.uint32)
    return int(lib().oracle_intersect_count(_p32(a), a.size, _p32(b), b.size))


def packed_index(n: int, i, j):
    """Row-major packed upper-triangle index of the pair (i, j), i < j."""
    i = np.asarray(i, dtype=np.int64)
    j = np.asarray(j, dtype=np.int64)
    return i * n - i * (i + 1) // 2 + (j - i - 1)


def pairs_full(offsets, tids, threads: int = 1) -> np.ndarray:
    """Supports of all pairs i < j, packed row-major upper triangle (uint32).

    With threads > 1 the same single-threaded routine runs on disjoint row
    blocks (ctypes releases the GIL during the call)."""
    offsets, tids = _csr(offsets, tids)
    n = offsets.size - 1
    out = np.zeros(max(n * (n - 1) // 2, 0), dtype=np.uint32)
    if n < 2:
        return out
    L = lib()
    if threads <= 1:
        L.oracle_pairs_rows(n, _p64(offsets), _p32(tids), 0, n, _p32(out))
        return out
    # balance rows by pair count: row i has n-1-i pairs
    blocks = []
    per = (n * (n - 1) // 2) / (threads * 8)
    start, acc = 0, 0
    for i in range(n):
        acc += n - 1 - i
        if acc >= per:
            blocks.append((start, i + 1))
            start, acc = i + 1, 0
    if start < n:
        blocks.append((start, n))
    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(lambda b: L.oracle_pairs_rows(n, _p64(offsets), _p32(tids), b[0], b[1],
                                                  _p32(out)), blocks))
    return out


def pairs_list(offsets, tids, ii, jj, threads: int = 1) -> np.ndarray:
    """Supports of the explicit pairs (ii[k], jj[k])."""
    offsets, tids = _csr(offsets, tids)
    ii = np.ascontiguousarray(ii, dtype=np.uint32)
    jj = np.ascontiguousarray(jj, dtype=np.uint32)
    out = np.zeros(ii.size, dtype=np.uint32)
    L = lib()
    if threads <= 1 or ii.size < 2 * threads:
        L.oracle_pairs_list(ii.size, _p32(ii), _p32(jj), _p64(offsets), _p32(tids), _p32(out))
        return out
    bounds = np.linspace(0, ii.size, threads * 4 + 1).astype(np.int64)

    def run(k):
        a, b = int(bounds[k]), int(bounds[k + 1])
        if b > a:
            L.oracle_pairs_list(b - a, _p32(ii[a:b]), _p32(jj[a:b]), _p64(offsets), _p32(tids),
                                _p32(out[a:b]))
    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(run, range(bounds.size - 1)))
    return out


def pairs_threshold(offsets, tids, s: int) -> np.ndarray:
    """(i, j, support) for all i < j with support >= s, lexicographic; uint32[k, 3]."""
    offsets, tids = _csr(offsets, tids)
    n = offsets.size - 1
    if n < 2:
        return np.zeros((0, 3), dtype=np.uint32)
    L = lib()
    cnt = int(L.oracle_pairs_threshold(n, _p64(offsets), _p32(tids), s, _p32(np.zeros(3, np.uint32)), 0))
    out = np.zeros(3 * max(cnt, 1), dtype=np.uint32)
    L.oracle_pairs_threshold(n, _p64(offsets), _p32(tids), s, _p32(out), cnt)
    return out[:3 * cnt].reshape(cnt, 3)


def threshold_from_full(full: np.ndarray, n: int, s: int) -> np.ndarray:
    """Thresholded lexicographic triples from a packed upper triangle."""
    ii, jj = np.triu_indices(n, 1)
    keep = full >= s
    return np.stack([ii[keep], jj[keep], full[keep]], axis=1).astype(np.uint32)


def kway_counts(offsets, tids, queries) -> np.ndarray:
    """|S_a1 intersect ... intersect S_ak| for each query (a list of item ids)."""
    offsets, tids = _csr(offsets, tids)
    qoff = np.zeros(len(queries) + 1, dtype=np.uint32)
    qoff[1:] = np.cumsum([len(q) for q in queries])
    ids = (np.concatenate([np.asarray(q, dtype=np.uint32) for q in queries])
           if len(queries) else np.zeros(0, np.uint32))
    sizes = np.diff(offsets)
    scratch = np.zeros(int(sizes.max()) + 1 if sizes.size else 1, dtype=np.uint32)
    out = np.zeros(len(queries), dtype=np.uint64)
    lib().oracle_kway_list(len(queries), _p32(qoff), _p32(ids), _p64(offsets), _p32(tids),
                           _p32(scratch), _p64(out))
    return out


def kway_elems(offsets, tids, query) -> np.ndarray:
    """Sorted elements of S_a1 cap ... cap S_ak for one query (a list of item ids)."""
    offsets, tids = _csr(offsets, tids)
    ids = np.ascontiguousarray(query, dtype=np.uint32)
    sizes = np.diff(offsets)
    out = np.zeros(int(sizes[ids[0]]) + 1 if ids.size else 1, dtype=np.uint32)  # room for S_a1
    k = int(lib().oracle_kway_elems(ids.size, _p32(ids), _p64(offsets), _p32(tids), _p32(out)))
    return out[:k].copy()
