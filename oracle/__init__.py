"""CPU oracle for the record sort -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its binding) never loads it and shares no code with it.

The arithmetic lives in ``leysort_oracle.c`` (plain C, built with gcc); this
module only builds it and marshals numpy arrays.  Every function here is
pinned by ``tests/test_oracle_pins.py``; none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "leysort_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

u8p = ctypes.POINTER(ctypes.c_uint8)
u32p = ctypes.POINTER(ctypes.c_uint32)
u64p = ctypes.POINTER(ctypes.c_uint64)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP when available)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-pthread", _SRC,
            "-o", tmp]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True, text=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True, text=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_sort_records.restype = ctypes.c_int
            lib.oracle_sort_records.argtypes = [u8p, u8p, ctypes.c_uint64, ctypes.c_uint32,
                                                ctypes.c_uint32, u64p]
            lib.oracle_sort_records_threads.restype = ctypes.c_int
            lib.oracle_sort_records_threads.argtypes = [u8p, u8p, ctypes.c_uint64,
                                                        ctypes.c_uint32, ctypes.c_uint32,
                                                        ctypes.c_uint32]
            lib.oracle_sort_keys_index.restype = ctypes.c_int
            lib.oracle_sort_keys_index.argtypes = [u64p, u32p, u64p, u32p, ctypes.c_uint64]
            lib.oracle_digit_histogram.restype = None
            lib.oracle_digit_histogram.argtypes = [u8p, ctypes.c_uint64, ctypes.c_uint32,
                                                   ctypes.c_uint32, u64p]
            lib.oracle_msd_partition.restype = None
            lib.oracle_msd_partition.argtypes = [u8p, ctypes.c_uint64, ctypes.c_uint32,
                                                 ctypes.c_uint32, u64p]
            lib.oracle_kway_merge_records.restype = None
            lib.oracle_kway_merge_records.argtypes = [u8p, u64p, ctypes.c_uint32, ctypes.c_uint32,
                                                      ctypes.c_uint32, u8p]
            lib.oracle_rank_records.restype = None
            lib.oracle_rank_records.argtypes = [u8p, ctypes.c_uint64, ctypes.c_uint32,
                                                ctypes.c_uint32, u64p, ctypes.c_uint64, u64p]
            lib.oracle_rank_pairs.restype = None
            lib.oracle_rank_pairs.argtypes = [u64p, ctypes.c_uint64, u64p, ctypes.c_uint64, u64p]
            lib.oracle_check_sorted.restype = ctypes.c_int64
            lib.oracle_check_sorted.argtypes = [u8p, ctypes.c_uint64, ctypes.c_uint32,
                                                ctypes.c_uint32]
            lib.oracle_record_hash_sum.restype = ctypes.c_uint64
            lib.oracle_record_hash_sum.argtypes = [u8p, ctypes.c_uint64, ctypes.c_uint32]
            lib.oracle_check_tagged.restype = ctypes.c_int64
            lib.oracle_check_tagged.argtypes = [u8p, u8p, ctypes.c_uint64, ctypes.c_uint32,
                                                ctypes.c_uint32, ctypes.c_uint32]
            lib.oracle_check_tagged_threads.restype = ctypes.c_int64
            lib.oracle_check_tagged_threads.argtypes = [u8p, u8p, ctypes.c_uint64,
                                                        ctypes.c_uint32, ctypes.c_uint32,
                                                        ctypes.c_uint32, ctypes.c_uint32]
            lib.oracle_check_pairs_tagged.restype = ctypes.c_int64
            lib.oracle_check_pairs_tagged.argtypes = [u64p, u32p, u64p, ctypes.c_uint64]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray, t):
    assert a.flags["C_CONTIGUOUS"], "oracle inputs must be C-contiguous"
    return a.ctypes.data_as(t)


def _records(a) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a), dtype=np.uint8)
    if a.ndim != 2:
        raise ValueError("records must be a 2-D uint8 array [n, rec_bytes]")
    return a


def sort_records(records, key_bytes: int = 10, return_perm: bool = False):
    """Stable sort of records by their first key_bytes bytes (unsigned)."""
    a = _records(records)
    n, rec = a.shape
    out = np.empty_like(a)
    perm = np.empty(max(n, 1), dtype=np.uint64)
    rc = _load().oracle_sort_records(_ptr(a, u8p), _ptr(out, u8p), n, rec, key_bytes,
                                     _ptr(perm, u64p))
    if rc != 0:
        raise MemoryError("oracle_sort_records: out of memory")
    return (out, perm[:n]) if return_perm else out


def sort_records_threads(records, key_bytes: int = 10, threads: int | None = None):
    """The same sort on ``threads`` host threads (default: every core):
    contiguous chunks sorted in parallel, a T-way heap merge, a parallel
    record copy.  For the CPU baseline; equal to ``sort_records``."""
    a = _records(records)
    n, rec = a.shape
    T = threads if threads else (os.cpu_count() or 1)
    out = np.empty_like(a)
    rc = _load().oracle_sort_records_threads(_ptr(a, u8p), _ptr(out, u8p), n, rec, key_bytes, T)
    if rc != 0:
        raise MemoryError(f"oracle_sort_records_threads failed ({rc})")
    return out


def sort_keys_index(keys, idx):
    """Sort (u64 key, u32 payload) pairs by (key, input position)."""
    k = np.ascontiguousarray(np.asarray(keys).view(np.uint64))
    v = np.ascontiguousarray(np.asarray(idx).view(np.uint32))
    n = k.shape[0]
    ko = np.empty(max(n, 1), dtype=np.uint64)
    vo = np.empty(max(n, 1), dtype=np.uint32)
    rc = _load().oracle_sort_keys_index(_ptr(k, u64p), _ptr(v, u32p), _ptr(ko, u64p),
                                        _ptr(vo, u32p), n)
    if rc != 0:
        raise MemoryError("oracle_sort_keys_index: out of memory")
    return ko[:n], vo[:n]


def digit_histogram(records, digit: int) -> np.ndarray:
    a = _records(records)
    h = np.zeros(256, dtype=np.uint64)
    _load().oracle_digit_histogram(_ptr(a, u8p), a.shape[0], a.shape[1], digit, _ptr(h, u64p))
    return h


def msd_partition(records, digit: int) -> np.ndarray:
    a = _records(records)
    o = np.empty(max(a.shape[0], 1), dtype=np.uint64)
    _load().oracle_msd_partition(_ptr(a, u8p), a.shape[0], a.shape[1], digit, _ptr(o, u64p))
    return o[:a.shape[0]]


def kway_merge_records(runs, run_start, key_bytes: int = 10) -> np.ndarray:
    a = _records(runs)
    rs = np.ascontiguousarray(np.asarray(run_start, dtype=np.uint64))
    k = rs.shape[0] - 1
    out = np.empty((int(rs[-1] - rs[0]), a.shape[1]), dtype=np.uint8)
    _load().oracle_kway_merge_records(_ptr(a, u8p), _ptr(rs, u64p), k, a.shape[1], key_bytes,
                                      _ptr(out, u8p))
    return out


def rank_records(records, samples, key_bytes: int = 10) -> np.ndarray:
    a = _records(records)
    s = np.ascontiguousarray(np.asarray(samples, dtype=np.uint64))
    r = np.empty(max(s.shape[0], 1), dtype=np.uint64)
    _load().oracle_rank_records(_ptr(a, u8p), a.shape[0], a.shape[1], key_bytes, _ptr(s, u64p),
                                s.shape[0], _ptr(r, u64p))
    return r[:s.shape[0]]


def rank_pairs(keys, samples) -> np.ndarray:
    k = np.ascontiguousarray(np.asarray(keys).view(np.uint64))
    s = np.ascontiguousarray(np.asarray(samples, dtype=np.uint64))
    r = np.empty(max(s.shape[0], 1), dtype=np.uint64)
    _load().oracle_rank_pairs(_ptr(k, u64p), k.shape[0], _ptr(s, u64p), s.shape[0], _ptr(r, u64p))
    return r[:s.shape[0]]


def check_sorted(records, key_bytes: int = 10) -> int:
    a = _records(records)
    return int(_load().oracle_check_sorted(_ptr(a, u8p), a.shape[0], a.shape[1], key_bytes))


def record_hash_sum(records) -> int:
    a = _records(records)
    return int(_load().oracle_record_hash_sum(_ptr(a, u8p), a.shape[0], a.shape[1]))


def check_tagged(out, inp, key_bytes: int = 10, tag_offset: int = 10) -> int:
    o, i = _records(out), _records(inp)
    assert o.shape == i.shape
    return int(_load().oracle_check_tagged(_ptr(o, u8p), _ptr(i, u8p), o.shape[0], o.shape[1],
                                           key_bytes, tag_offset))


def check_tagged_threads(out, inp, key_bytes: int = 10, tag_offset: int = 10,
                         threads: int | None = None) -> int:
    """check_tagged on ``threads`` host threads (default: every core): -1 if
    exact, else a bad output position."""
    o, i = _records(out), _records(inp)
    assert o.shape == i.shape
    T = threads if threads else (os.cpu_count() or 1)
    return int(_load().oracle_check_tagged_threads(_ptr(o, u8p), _ptr(i, u8p), o.shape[0],
                                                   o.shape[1], key_bytes, tag_offset, T))


def check_pairs_tagged(keys_out, idx_out, keys_in) -> int:
    ko = np.ascontiguousarray(np.asarray(keys_out).view(np.uint64))
    io = np.ascontiguousarray(np.asarray(idx_out).view(np.uint32))
    ki = np.ascontiguousarray(np.asarray(keys_in).view(np.uint64))
    return int(_load().oracle_check_pairs_tagged(_ptr(ko, u64p), _ptr(io, u32p), _ptr(ki, u64p),
                                                 ko.shape[0]))
