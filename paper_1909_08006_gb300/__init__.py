"""leysort: GPU record sort for one GB300 (sm_103a), a re-design of the
data-parallel hot path of Leyenda (arXiv 1909.08006).

This module is a thin ctypes binding of the C ABI in ``include/leysort.h``
(``libleysort.so``): it marshals arguments and nothing else.  Every step of a
sort runs in the library's CUDA kernels; there is no CPU fallback, and the
import fails loudly when the library has not been built.

Functions keep the C names.  Buffers may be given as torch tensors (device or
pinned host memory; PyTorch is used for memory and streams only) or as raw
integer addresses.  A non-OK status raises :class:`LeyError`.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

__all__ = [
    "LeyError", "LEY_OK", "LEY_EINVAL", "LEY_ENOMEM", "LEY_EUNSUPPORTED", "LEY_ECUDA",
    "LEY_ETIMEOUT", "ley_sort_records", "ley_sort_records_async", "ley_plan_partitions",
    "ley_sort_keys_index",
    "ley_partition_records",
    "ley_workspace_bytes", "ley_host_scratch_bytes", "ley_status_string", "ley_last_device_status", "ley_launch_count",
    "ley_profile_enable", "ley_profile_read", "library_path", "exported_symbols",
    "ley_sort_records_noalloc", "LEY_NOALLOC_MAX_RECORDS", "ley_merge_records",
    "ley_release_cache", "ley_sort_records_batch", "ley_sort_keys_index_batch",
    "ley_server_create", "ley_server_submit_records", "ley_server_submit_pairs",
    "ley_server_wait", "ley_server_stats", "ley_server_destroy",
    "ley_get_tuning", "ley_set_tuning", "ley_autotune_records", "ley_autotune_records_on",
    "ley_selftest_timeout",
]

LEY_OK, LEY_EINVAL, LEY_ENOMEM, LEY_EUNSUPPORTED, LEY_ECUDA, LEY_ETIMEOUT = range(6)
LEY_NOALLOC_MAX_RECORDS = 262144


class LeyError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = int(status)
        super().__init__(f"{where}: {ley_status_string(status)} (status {status})")


class _KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("launches", ctypes.c_uint64),
                ("total_ms", ctypes.c_double)]


class _RecordsReq(ctypes.Structure):
    _fields_ = [("in_", ctypes.c_void_p), ("out", ctypes.c_void_p), ("n", ctypes.c_uint64)]


class _PairsReq(ctypes.Structure):
    _fields_ = [("keys_in", ctypes.c_void_p), ("idx_in", ctypes.c_void_p),
                ("keys_out", ctypes.c_void_p), ("idx_out", ctypes.c_void_p),
                ("n", ctypes.c_uint64)]


class _Tuning(ctypes.Structure):
    _fields_ = [("big_bucket", ctypes.c_uint32), ("tiny_bucket", ctypes.c_uint32),
                ("finish_ctas_per_sm", ctypes.c_uint32), ("pass_ctas_per_sm", ctypes.c_uint32)]


class _ServerTimes(ctypes.Structure):
    _fields_ = [("submit_s", ctypes.c_double), ("start_s", ctypes.c_double),
                ("done_s", ctypes.c_double), ("dev_start_s", ctypes.c_double),
                ("dev_done_s", ctypes.c_double), ("batch", ctypes.c_uint64)]


class _ServerCounters(ctypes.Structure):
    _fields_ = [("pending", ctypes.c_uint64), ("inflight_batches", ctypes.c_uint64),
                ("launched_batches", ctypes.c_uint64), ("bytes_in_use", ctypes.c_uint64)]


def library_path() -> str:
    """The library this binding loads: the in-tree build, or the file named by
    the LEYSORT_LIB environment variable (another build of the same
    sources)."""
    return os.environ.get("LEYSORT_LIB") or _build.LIB


def _load() -> ctypes.CDLL:
    path = library_path()
    if not os.path.exists(path):
        raise ImportError(
            f"libleysort.so is not built ({path}); run "
            "`python -c 'import __graft_entry__ as g; g.build()'` first")
    lib = ctypes.CDLL(path)
    vp, u64, u32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32
    lib.ley_sort_records.argtypes = [vp, vp, u64, u32, u32, u64, vp]
    lib.ley_sort_records.restype = ctypes.c_int
    lib.ley_sort_records_async.argtypes = [vp, vp, u64, u32, u32, u64, vp]
    lib.ley_sort_records_async.restype = ctypes.c_int
    lib.ley_plan_partitions.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(u64), u32, u32, u32,
                                        u64, ctypes.POINTER(u64), u64, ctypes.POINTER(u64)]
    lib.ley_plan_partitions.restype = ctypes.c_int
    lib.ley_sort_keys_index.argtypes = [vp, vp, vp, vp, u64, u64, vp]
    lib.ley_sort_keys_index.restype = ctypes.c_int
    lib.ley_partition_records.argtypes = [vp, u64, u32, u32, u32, vp, vp, vp]
    lib.ley_partition_records.restype = ctypes.c_int
    lib.ley_workspace_bytes.argtypes = [u64, u32, u32, u64, ctypes.POINTER(u64)]
    lib.ley_workspace_bytes.restype = ctypes.c_int
    lib.ley_host_scratch_bytes.argtypes = [u64, u32, u32, u64, ctypes.POINTER(u64)]
    lib.ley_host_scratch_bytes.restype = ctypes.c_int
    lib.ley_status_string.argtypes = [ctypes.c_int]
    lib.ley_status_string.restype = ctypes.c_char_p
    lib.ley_last_device_status.argtypes = [vp]
    lib.ley_last_device_status.restype = ctypes.c_int
    lib.ley_launch_count.argtypes = []
    lib.ley_launch_count.restype = u64
    lib.ley_profile_enable.argtypes = [ctypes.c_int]
    lib.ley_profile_enable.restype = ctypes.c_int
    lib.ley_profile_read.argtypes = [ctypes.POINTER(_KernelTime), ctypes.c_int]
    lib.ley_profile_read.restype = ctypes.c_int
    lib.ley_merge_records.argtypes = [vp, ctypes.POINTER(u64), u32, vp, u32, u32, vp]
    lib.ley_merge_records.restype = ctypes.c_int
    lib.ley_sort_records_noalloc.argtypes = [vp, vp, u64, u32, u32, vp]
    lib.ley_sort_records_noalloc.restype = ctypes.c_int
    lib.ley_release_cache.argtypes = []
    lib.ley_release_cache.restype = ctypes.c_int
    lib.ley_sort_records_batch.argtypes = [ctypes.POINTER(_RecordsReq), u32, u32, u32, u64, vp]
    lib.ley_sort_records_batch.restype = ctypes.c_int
    lib.ley_sort_keys_index_batch.argtypes = [ctypes.POINTER(_PairsReq), u32, u64, vp]
    lib.ley_sort_keys_index_batch.restype = ctypes.c_int
    lib.ley_selftest_timeout.argtypes = [u32, vp]
    lib.ley_selftest_timeout.restype = ctypes.c_int
    lib.ley_get_tuning.argtypes = [ctypes.POINTER(_Tuning)]
    lib.ley_get_tuning.restype = ctypes.c_int
    lib.ley_set_tuning.argtypes = [ctypes.POINTER(_Tuning)]
    lib.ley_set_tuning.restype = ctypes.c_int
    lib.ley_autotune_records.argtypes = [u64, u32, u32, u64, ctypes.POINTER(_Tuning)]
    lib.ley_autotune_records.restype = ctypes.c_int
    lib.ley_autotune_records_on.argtypes = [vp, u64, u32, u32, ctypes.POINTER(_Tuning), vp]
    lib.ley_autotune_records_on.restype = ctypes.c_int
    lib.ley_server_create.argtypes = [ctypes.POINTER(vp), u64, u32, u32]
    lib.ley_server_create.restype = ctypes.c_int
    lib.ley_server_submit_records.argtypes = [vp, vp, vp, u64, u32, u32, ctypes.POINTER(u64)]
    lib.ley_server_submit_records.restype = ctypes.c_int
    lib.ley_server_submit_pairs.argtypes = [vp, vp, vp, vp, vp, u64, ctypes.POINTER(u64)]
    lib.ley_server_submit_pairs.restype = ctypes.c_int
    lib.ley_server_wait.argtypes = [vp, u64, ctypes.POINTER(_ServerTimes)]
    lib.ley_server_wait.restype = ctypes.c_int
    lib.ley_server_stats.argtypes = [vp, ctypes.POINTER(_ServerCounters)]
    lib.ley_server_stats.restype = ctypes.c_int
    lib.ley_server_destroy.argtypes = [vp]
    lib.ley_server_destroy.restype = ctypes.c_int
    return lib


class _Lazy:
    """Loads libleysort.so on first use; raises ImportError if it is not built."""

    _h = None

    def __getattr__(self, name):
        if _Lazy._h is None:
            _Lazy._h = _load()
        return getattr(_Lazy._h, name)


_lib = _Lazy()


def exported_symbols() -> list[str]:
    """Names of the C entry points this binding resolves."""
    return [n for n in __all__ if n.startswith("ley_")]


# ----------------------------------------------------------- marshalling

def _addr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensors passed to leysort must be contiguous")
        return int(x.data_ptr())
    raise TypeError(f"expected a tensor or an address, got {type(x).__name__}")


def _stream(stream, *tensors) -> int:
    if stream is not None:
        return stream if isinstance(stream, int) else int(stream.cuda_stream)
    for t in tensors:
        if hasattr(t, "is_cuda") and t.is_cuda:
            import torch
            return int(torch.cuda.current_stream(t.device).cuda_stream)
    return 0


def _check(status: int, where: str) -> int:
    if status != LEY_OK:
        raise LeyError(status, where)
    return status


def ley_sort_records(inp, out, n: int | None = None, rec_bytes: int | None = None,
                     key_bytes: int = 10, mem_budget: int = 0, stream=None) -> int:
    """Sort records (rows of a uint8 [n, rec_bytes] tensor) by their first
    ``key_bytes`` bytes; see ``ley_sort_records`` in include/leysort.h."""
    if n is None:
        n = int(inp.shape[0])
    if rec_bytes is None:
        rec_bytes = int(inp.shape[1]) if hasattr(inp, "shape") and len(inp.shape) == 2 else 100
    st = _lib.ley_sort_records(_addr(inp), _addr(out), n, rec_bytes, key_bytes, mem_budget,
                               _stream(stream, inp, out))
    return _check(st, "ley_sort_records")


def ley_sort_records_async(inp, out, n: int | None = None, rec_bytes: int | None = None,
                           key_bytes: int = 10, mem_budget: int = 0, stream=None) -> int:
    """As ley_sort_records, but a sort of pinned host buffers is only queued
    on ``stream`` (synchronise it before reading ``out``); see
    ``ley_sort_records_async`` in include/leysort.h."""
    if n is None:
        n = int(inp.shape[0])
    if rec_bytes is None:
        rec_bytes = int(inp.shape[1]) if hasattr(inp, "shape") and len(inp.shape) == 2 else 100
    st = _lib.ley_sort_records_async(_addr(inp), _addr(out), n, rec_bytes, key_bytes,
                                     mem_budget, _stream(stream, inp, out))
    return _check(st, "ley_sort_records_async")


def ley_plan_partitions(runs, key_bytes: int = 10, cap: int = 1 << 20):
    """Cut the merge of sorted host runs (uint8 [len_i, rec_bytes] numpy arrays)
    into partitions of at most ``cap`` records; returns the cut positions as a
    [partitions + 1, k] uint64 array.  See ``ley_plan_partitions`` in
    include/leysort.h.  Host-only."""
    import numpy as np
    k = len(runs)
    rec = int(runs[0].shape[1]) if k and runs[0].ndim == 2 else 100
    ptrs = (ctypes.c_void_p * k)(*[r.ctypes.data if len(r) else 0 for r in runs])
    lens = (ctypes.c_uint64 * k)(*[len(r) for r in runs])
    need = ctypes.c_uint64(0)
    rows = 2 + (sum(len(r) for r in runs) // max(1, cap // 2) + 2)
    for _ in range(2):
        cuts = np.zeros((rows, k), dtype=np.uint64)
        st = _lib.ley_plan_partitions(ptrs, lens, k, rec, key_bytes, cap,
                                      cuts.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                      rows, ctypes.byref(need))
        if st == LEY_ENOMEM and need.value > rows:
            rows = int(need.value)
            continue
        _check(st, "ley_plan_partitions")
        return cuts[:need.value].copy()
    raise LeyError(LEY_ENOMEM, "ley_plan_partitions")


def ley_sort_records_batch(requests, rec_bytes: int = 100, key_bytes: int = 10,
                           mem_budget: int = 0, stream=None) -> int:
    """Sort many record arrays at once, each as ley_sort_records would.
    ``requests`` holds (in, out) pairs of device uint8 [n, rec_bytes] tensors,
    or (in, out, n) with addresses."""
    arr = (_RecordsReq * max(1, len(requests)))()
    st = None
    for i, rq in enumerate(requests):
        inp, out = rq[0], rq[1]
        n = int(rq[2]) if len(rq) > 2 else int(inp.shape[0])
        arr[i] = _RecordsReq(_addr(inp), _addr(out), n)
        if st is None and hasattr(inp, "is_cuda"):
            st = _stream(stream, inp)
    if st is None:
        st = _stream(stream)
    return _check(_lib.ley_sort_records_batch(arr, len(requests), rec_bytes, key_bytes,
                                              mem_budget, st), "ley_sort_records_batch")


def ley_sort_keys_index_batch(requests, mem_budget: int = 0, stream=None) -> int:
    """Sort many (key, payload) arrays at once, each as ley_sort_keys_index
    would.  ``requests`` holds (keys_in, idx_in, keys_out, idx_out) tuples of
    device tensors, or the same with a count appended and addresses."""
    arr = (_PairsReq * max(1, len(requests)))()
    st = None
    for i, rq in enumerate(requests):
        ki, ii, ko, io = rq[:4]
        n = int(rq[4]) if len(rq) > 4 else int(ki.shape[0])
        arr[i] = _PairsReq(_addr(ki), _addr(ii), _addr(ko), _addr(io), n)
        if st is None and hasattr(ki, "is_cuda"):
            st = _stream(stream, ki)
    if st is None:
        st = _stream(stream)
    return _check(_lib.ley_sort_keys_index_batch(arr, len(requests), mem_budget, st),
                  "ley_sort_keys_index_batch")


def ley_selftest_timeout(which: int = 0, stream=None) -> int:
    """Makes one bounded device wait give up on purpose; returns (does not
    raise) the status it latched: LEY_ETIMEOUT when detection works."""
    return int(_lib.ley_selftest_timeout(which, _stream(stream)))


# ---------------------------------------------------------------- tuning

def ley_get_tuning() -> dict:
    t = _Tuning()
    _check(_lib.ley_get_tuning(ctypes.byref(t)), "ley_get_tuning")
    return {f: int(getattr(t, f)) for f, _ in _Tuning._fields_}


def ley_set_tuning(tuning: dict | None) -> int:
    """Set the current device's tunables (dict with the ley_tuning fields);
    None restores the defaults."""
    if tuning is None:
        return _check(_lib.ley_set_tuning(None), "ley_set_tuning")
    t = _Tuning(**{f: int(tuning.get(f, d)) for f, d in
                   (("big_bucket", 2048), ("tiny_bucket", 64), ("finish_ctas_per_sm", 0),
                    ("pass_ctas_per_sm", 0))})
    return _check(_lib.ley_set_tuning(ctypes.byref(t)), "ley_set_tuning")


def ley_autotune_records(n: int, rec_bytes: int = 100, key_bytes: int = 10,
                         seed: int = 1) -> dict:
    """Times a grid of tunings on n random records; keeps and returns the fastest."""
    t = _Tuning()
    _check(_lib.ley_autotune_records(n, rec_bytes, key_bytes, seed, ctypes.byref(t)),
           "ley_autotune_records")
    return {f: int(getattr(t, f)) for f, _ in _Tuning._fields_}


def ley_autotune_records_on(inp, n: int | None = None, rec_bytes: int | None = None,
                            key_bytes: int = 10, stream=None) -> dict:
    """Times a grid of tunings on the caller's device records (a uint8
    [n, rec_bytes] tensor, not modified) after the work queued on ``stream``
    (default: the tensor's current stream); keeps and returns the fastest."""
    if n is None:
        n = int(inp.shape[0])
    if rec_bytes is None:
        rec_bytes = int(inp.shape[1]) if hasattr(inp, "shape") and len(inp.shape) == 2 else 100
    t = _Tuning()
    _check(_lib.ley_autotune_records_on(_addr(inp), n, rec_bytes, key_bytes, ctypes.byref(t),
                                        _stream(stream, inp)),
           "ley_autotune_records_on")
    return {f: int(getattr(t, f)) for f, _ in _Tuning._fields_}


# ---------------------------------------------------------------- server

def ley_server_create(mem_budget: int, max_batch: int = 256, slots: int = 3) -> int:
    """A continuous-batching sort server on the current device (a handle)."""
    h = ctypes.c_void_p()
    _check(_lib.ley_server_create(ctypes.byref(h), int(mem_budget), max_batch, slots),
           "ley_server_create")
    return int(h.value)


def ley_server_submit_records(server: int, inp, out, n: int | None = None,
                              rec_bytes: int | None = None, key_bytes: int = 10) -> int:
    if n is None:
        n = int(inp.shape[0])
    if rec_bytes is None:
        rec_bytes = int(inp.shape[1]) if hasattr(inp, "shape") and len(inp.shape) == 2 else 100
    t = ctypes.c_uint64(0)
    _check(_lib.ley_server_submit_records(server, _addr(inp), _addr(out), n, rec_bytes,
                                          key_bytes, ctypes.byref(t)), "ley_server_submit_records")
    return int(t.value)


def ley_server_submit_pairs(server: int, keys_in, idx_in, keys_out, idx_out,
                            n: int | None = None) -> int:
    if n is None:
        n = int(keys_in.shape[0])
    t = ctypes.c_uint64(0)
    _check(_lib.ley_server_submit_pairs(server, _addr(keys_in), _addr(idx_in), _addr(keys_out),
                                        _addr(idx_out), n, ctypes.byref(t)),
           "ley_server_submit_pairs")
    return int(t.value)


def ley_server_wait(server: int, ticket: int) -> dict:
    """Blocks until the request is done; raises LeyError on a failed request.
    Returns its submit / start / done times (host clock, seconds since server
    creation), its batch's device-clock interval and the batch number."""
    tm = _ServerTimes()
    _check(_lib.ley_server_wait(server, ticket, ctypes.byref(tm)), "ley_server_wait")
    return {f: getattr(tm, f) for f, _ in _ServerTimes._fields_}


def ley_server_stats(server: int) -> dict:
    c = _ServerCounters()
    _check(_lib.ley_server_stats(server, ctypes.byref(c)), "ley_server_stats")
    return {f: int(getattr(c, f)) for f, _ in _ServerCounters._fields_}


def ley_server_destroy(server: int) -> int:
    return _check(_lib.ley_server_destroy(server), "ley_server_destroy")


def ley_sort_records_noalloc(inp, out, n: int | None = None, rec_bytes: int | None = None,
                             key_bytes: int = 10, stream=None) -> int:
    """Allocation-free form of ley_sort_records for callers that cannot
    allocate device memory (their device memory is owned by their own pool,
    or a cudaMalloc would stall them).  Device buffers only, at most
    LEY_NOALLOC_MAX_RECORDS records; scratch is one fixed array inside the
    library shared by all calls, so calls must not overlap on the GPU.  Waits
    for its work and returns its device-side status."""
    if n is None:
        n = int(inp.shape[0])
    if rec_bytes is None:
        rec_bytes = int(inp.shape[1]) if hasattr(inp, "shape") and len(inp.shape) == 2 else 100
    st = _lib.ley_sort_records_noalloc(_addr(inp), _addr(out), n, rec_bytes, key_bytes,
                                       _stream(stream, inp, out))
    return _check(st, "ley_sort_records_noalloc")


def ley_sort_keys_index(keys_in, idx_in, keys_out, idx_out, n: int | None = None,
                        mem_budget: int = 0, stream=None) -> int:
    """Sort (u64 key, u32 payload) pairs by (key, input position)."""
    if n is None:
        n = int(keys_in.shape[0])
    st = _lib.ley_sort_keys_index(_addr(keys_in), _addr(idx_in), _addr(keys_out),
                                  _addr(idx_out), n, mem_budget,
                                  _stream(stream, keys_in, keys_out))
    return _check(st, "ley_sort_keys_index")


def ley_partition_records(inp, digit: int, order_out, hist_out, n: int | None = None,
                          rec_bytes: int | None = None, key_bytes: int = 10, stream=None) -> int:
    """One radix round: histogram of key byte ``digit`` and the stable
    partition order (u32 per record, 256 u64 bucket sizes)."""
    if n is None:
        n = int(inp.shape[0])
    if rec_bytes is None:
        rec_bytes = int(inp.shape[1])
    st = _lib.ley_partition_records(_addr(inp), n, rec_bytes, key_bytes, digit,
                                    _addr(order_out), _addr(hist_out),
                                    _stream(stream, inp, order_out))
    return _check(st, "ley_partition_records")


def ley_merge_records(runs, run_start, out, rec_bytes: int | None = None, key_bytes: int = 10,
                      stream=None) -> int:
    """Stable k-way merge of sorted runs stored back to back (run r holds
    records run_start[r] .. run_start[r+1]-1)."""
    starts = [int(x) for x in run_start]
    k = len(starts) - 1
    if rec_bytes is None:
        rec_bytes = int(runs.shape[1])
    arr = (ctypes.c_uint64 * len(starts))(*starts)
    st = _lib.ley_merge_records(_addr(runs), arr, k, _addr(out), rec_bytes, key_bytes,
                                _stream(stream, runs, out))
    return _check(st, "ley_merge_records")


def ley_workspace_bytes(n: int, rec_bytes: int = 100, key_bytes: int = 10,
                        mem_budget: int = 0) -> int:
    """Device bytes a sort of n records allocates: the internal sort's
    scratch (mem_budget 0), or a host-memory sort's under that budget."""
    v = ctypes.c_uint64(0)
    _check(_lib.ley_workspace_bytes(n, rec_bytes, key_bytes, mem_budget, ctypes.byref(v)),
           "ley_workspace_bytes")
    return int(v.value)


def ley_host_scratch_bytes(n: int, rec_bytes: int = 100, key_bytes: int = 10,
                           mem_budget: int = 0) -> int:
    """Pinned host bytes an external sort of n records under mem_budget keeps
    for its runs (0 when the partially in-memory mode is used)."""
    v = ctypes.c_uint64(0)
    _check(_lib.ley_host_scratch_bytes(n, rec_bytes, key_bytes, mem_budget, ctypes.byref(v)),
           "ley_host_scratch_bytes")
    return int(v.value)


def ley_release_cache() -> int:
    """Return the device pool memory and pinned host scratch kept between calls."""
    return _check(_lib.ley_release_cache(), "ley_release_cache")


def ley_status_string(status: int) -> str:
    return _lib.ley_status_string(int(status)).decode()


def ley_last_device_status(stream=None) -> int:
    """Waits for the stream; returns (does not raise) the device-side status."""
    return int(_lib.ley_last_device_status(_stream(stream)))


def ley_launch_count() -> int:
    return int(_lib.ley_launch_count())


def ley_profile_enable(on: bool = True) -> int:
    return _check(_lib.ley_profile_enable(1 if on else 0), "ley_profile_enable")


def ley_profile_read(max_entries: int = 64) -> dict[str, tuple[int, float]]:
    """{kernel name: (launches, total ms)} since profiling was enabled."""
    arr = (_KernelTime * max_entries)()
    k = _lib.ley_profile_read(arr, max_entries)
    return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms))
            for i in range(min(k, max_entries))}
