"""Seeded synthetic inputs for the record sort: the only code that the oracle
side and the CUDA side share.

This module draws bytes; it holds none of the sort's arithmetic (no key
comparison, no digit extraction, no ordering).  Every array is a pure
function of (seed, shape), identical on the CPU and on a CUDA device, so a
test can generate the same input on both sides.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014).  Stream ``s`` yields, for counter k >= 1,
``mix64(s + k * 0x9E3779B97F4A7C15)`` with the published finaliser
constants.  Arithmetic is done on torch int64 with explicit masks for the
logical right shifts, so it is bit-identical on every device.

Record layout (the paper's workloads, Section 4.1): 100-byte records whose
first 10 bytes are the key and whose last 90 bytes are the value.  Record i
is filled from words k = i*W + w + 1 (w = 0..W-1, W = ceil(rec_bytes / 8)),
each word little-endian, truncated to rec_bytes.  The paper generated its
data with the Sort Benchmark's gensort tool; that tool and its data are not
used here, these seeded inputs stand in for them.
"""
from __future__ import annotations

import math

import torch

GOLDEN = 0x9E3779B97F4A7C15
_C1 = 0xBF58476D1CE4E5B9
_C2 = 0x94D049BB133111EB
MASK64 = (1 << 64) - 1


def _s64(x: int) -> int:
    """Python int (any sign) -> the int64 with the same low 64 bits."""
    x &= MASK64
    return x - (1 << 64) if x >= (1 << 63) else x


def _lsr(z: torch.Tensor, k: int) -> torch.Tensor:
    """Logical right shift of int64 lanes (torch's >> is arithmetic)."""
    return (z >> k) & ((1 << (64 - k)) - 1)


def mix64(z: torch.Tensor) -> torch.Tensor:
    """SplitMix64 output function (a bijection on 64-bit words)."""
    z = (z ^ _lsr(z, 30)) * _s64(_C1)
    z = (z ^ _lsr(z, 27)) * _s64(_C2)
    return z ^ _lsr(z, 31)


def stream_words(seed: int, k0: int, count: int, device="cpu") -> torch.Tensor:
    """Words k0+1 .. k0+count of SplitMix64 stream ``seed`` as int64 bits."""
    k = torch.arange(k0 + 1, k0 + count + 1, dtype=torch.int64, device=device)
    return mix64(k * _s64(GOLDEN) + _s64(seed))


def splitmix64_reference(seed: int, count: int) -> list[int]:
    """Plain-int SplitMix64 (state += golden; output mix(state)) for pinning."""
    out, s = [], seed & MASK64
    for _ in range(count):
        s = (s + GOLDEN) & MASK64
        z = s
        z = ((z ^ (z >> 30)) * _C1) & MASK64
        z = ((z ^ (z >> 27)) * _C2) & MASK64
        out.append(z ^ (z >> 31))
    return out


def _stream_seed(seed: int, lane: int) -> int:
    """Independent sub-stream for a purpose ``lane`` of a config seed."""
    return int(splitmix64_reference((seed * 0x100 + lane) & MASK64, 1)[0])


# ---------------------------------------------------------------- records

def uniform_records(n: int, seed: int, rec_bytes: int = 100, device="cpu",
                    start: int = 0, tag_index: bool = False,
                    tag_offset: int = 10) -> torch.Tensor:
    """Records start .. start+n-1 of the uniform workload, uint8 [n, rec_bytes].

    Every byte is uniform.  With ``tag_index`` the 4 bytes at ``tag_offset``
    (inside the value, after a 10-byte key) hold the record's global index as
    a little-endian u32, so a sorted output reveals which input each output
    record came from (used for O(n) verification at full size).
    """
    W = (rec_bytes + 7) // 8
    s = _stream_seed(seed, 1)
    out = torch.empty((n, rec_bytes), dtype=torch.uint8, device=device)
    chunk = max(1, (1 << 24) // W)
    for c0 in range(0, n, chunk):
        c1 = min(n, c0 + chunk)
        w = stream_words(s, (start + c0) * W, (c1 - c0) * W, device)
        out[c0:c1] = w.view(torch.uint8).view(c1 - c0, W * 8)[:, :rec_bytes]
    if tag_index:
        _write_tag(out, start, tag_offset)
    return out


def _write_tag(rec: torch.Tensor, start: int, off: int) -> None:
    n = rec.shape[0]
    idx = torch.arange(start, start + n, dtype=torch.int64, device=rec.device)
    for b in range(4):
        rec[:, off + b] = ((idx >> (8 * b)) & 0xFF).to(torch.uint8)


ZIPF_VALUES = 65536
ZIPF_S = 1.2
DUP_FRACTION_NUM, DUP_FRACTION_DEN = 3, 10


def zipf_cdf(values: int = ZIPF_VALUES, s: float = ZIPF_S) -> torch.Tensor:
    """float64 CDF of P(r) proportional to (r+1)^-s, r = 0..values-1 (CPU)."""
    r = torch.arange(1, values + 1, dtype=torch.float64)
    w = r.pow(-s)
    c = torch.cumsum(w, 0)
    return c / c[-1]


def _perm32(x: torch.Tensor) -> torch.Tensor:
    """A bijection of the 32-bit integers (odd multiplies and xor-shifts)."""
    m = 0xFFFFFFFF
    x = (x * 0x9E3779B1) & m
    x = x ^ (x >> 16)
    x = (x * 0x85EBCA6B) & m
    x = x ^ (x >> 13)
    x = (x * 0xC2B2AE35) & m
    return x ^ (x >> 16)


def zipf_table(seed: int, device="cpu") -> torch.Tensor:
    """65,536 distinct u32 values (int64 lanes) that Zipf ranks map to."""
    base = _stream_seed(seed, 7) & 0xFFFFFFFF
    r = torch.arange(ZIPF_VALUES, dtype=torch.int64, device=device)
    return _perm32((r + base) & 0xFFFFFFFF)


def skew_records(n: int, seed: int, rec_bytes: int = 100, device="cpu",
                 tag_index: bool = False, tag_offset: int = 10,
                 key_bytes: int = 10) -> torch.Tensor:
    """The skewed workload: key bytes 0-3 Zipf(1.2) over 65,536 values,
    key bytes 4-9 uniform, and floor(0.3 n) records that copy the full key
    of another record.

    * rank r in [0, 65535] is drawn with P(r) proportional to (r+1)^-1.2 by
      inverse CDF from a 53-bit uniform, then mapped through a seeded table
      of 65,536 distinct u32 values written big-endian into bytes 0-3;
    * a seeded permutation picks exactly floor(0.3 n) "duplicate" records;
      each copies the 10-byte key of a uniformly chosen record among the
      other 70 %, so no key is copied from a copy.  Values stay independent.
    """
    rec = uniform_records(n, seed, rec_bytes, device)
    if n == 0:
        return rec
    cdf = zipf_cdf().to(device)
    u = _lsr(stream_words(_stream_seed(seed, 2), 0, n, device), 11)
    uf = u.to(torch.float64) * (2.0 ** -53)
    rank = torch.searchsorted(cdf, uf, right=True).clamp_(max=ZIPF_VALUES - 1)
    v = zipf_table(seed, device)[rank]
    for b in range(4):
        rec[:, b] = ((v >> (8 * (3 - b))) & 0xFF).to(torch.uint8)
    nd = (n * DUP_FRACTION_NUM) // DUP_FRACTION_DEN
    if nd > 0 and n - nd > 0:
        order = torch.argsort(stream_words(_stream_seed(seed, 3), 0, n, device))
        dups, orig = order[:nd], order[nd:]
        pick = _lsr(stream_words(_stream_seed(seed, 4), 0, n, device), 1)
        src = orig[pick[dups] % (n - nd)]
        rec[dups, :key_bytes] = rec[src, :key_bytes]
    if tag_index:
        _write_tag(rec, 0, tag_offset)
    return rec


# ------------------------------------------------------------------ pairs

def uniform_pairs(n: int, seed: int, device="cpu", start: int = 0):
    """(keys, payload): keys are uniform u64 (int64 bit patterns), payload
    is the u32 global index start..start+n-1 (int32 bit patterns)."""
    keys = stream_words(_stream_seed(seed, 5), start, n, device)
    idx = torch.arange(start, start + n, dtype=torch.int64, device=device)
    payload = ((idx & 0xFFFFFFFF) - ((idx & 0x80000000) << 1)).to(torch.int32)
    return keys, payload


def narrow_pairs(n: int, seed: int, distinct: int, device="cpu"):
    """Pairs whose keys take only ``distinct`` values (many ties)."""
    w = _lsr(stream_words(_stream_seed(seed, 6), 0, n, device), 1)
    vals = stream_words(_stream_seed(seed, 8), 0, max(1, distinct), device)
    keys = vals[w % max(1, distinct)]
    idx = torch.arange(n, dtype=torch.int64, device=device)
    return keys, idx.to(torch.int32)


# ------------------------------------------------------- edge-case records

def edge_records(kind: str, n: int, seed: int, rec_bytes: int = 100,
                 key_bytes: int = 10, device="cpu") -> torch.Tensor:
    """Degenerate inputs of the sort: key patterns with a known answer.

    kinds: 'equal' (all keys equal), 'sorted' (strictly increasing keys),
    'reversed' (strictly decreasing keys), 'last_byte' (keys differ only
    in their last byte), 'two_symbol' (every key byte is 'A' or 'B'),
    'few_distinct' (keys drawn from 5 values), 'prefix_shared' (the first
    key_bytes-2 bytes equal, the last two uniform).
    """
    rec = uniform_records(n, seed, rec_bytes, device)
    kb = key_bytes
    if n == 0:
        return rec
    if kind == "equal":
        rec[:, :kb] = rec[0, :kb].clone()
    elif kind in ("sorted", "reversed"):
        i = torch.arange(n, dtype=torch.int64, device=device)
        if kind == "reversed":
            i = (n - 1) - i
        rec[:, :kb] = 0x5A
        for b in range(min(kb, 8)):
            rec[:, kb - 1 - b] = ((i >> (8 * b)) & 0xFF).to(torch.uint8)
    elif kind == "last_byte":
        rec[:, :kb - 1] = 0x33
    elif kind == "two_symbol":
        rec[:, :kb] = 0x41 + (rec[:, :kb] & 1)
    elif kind == "few_distinct":
        pick = (rec[:, kb].to(torch.int64) % 5)
        base = uniform_records(5, seed + 99, rec_bytes, device)[:, :kb]
        rec[:, :kb] = base[pick]
    elif kind == "prefix_shared":
        rec[:, :kb - 2] = 0x7E
    else:
        raise ValueError(f"unknown edge kind {kind!r}")
    return rec


def ascii_records(n: int, seed: int, rec_bytes: int = 100, key_bytes: int = 10,
                  shared_prefix: int = 0, alphabet: int = 95, dup_frac: float = 0.0,
                  device="cpu") -> torch.Tensor:
    """Records with printable ASCII keys, like the Sort Benchmark's ASCII
    records (the paper's 20 GB set): key bytes are drawn from the first
    ``alphabet`` printable characters (0x20..); the first ``shared_prefix``
    key bytes are the same for every record; a ``dup_frac`` fraction of the
    records (every k-th) copies the whole key of the record before it.  The
    value bytes stay uniform."""
    rec = uniform_records(n, seed, rec_bytes, device)
    if n == 0:
        return rec
    kb = key_bytes
    rec[:, :kb] = (0x20 + (rec[:, :kb].to(torch.int64) % alphabet)).to(torch.uint8)
    if shared_prefix:
        rec[:, :shared_prefix] = rec[0, :shared_prefix].clone()
    step = max(1, int(round(1.0 / dup_frac))) if dup_frac > 0 else 0
    if step and n > step:
        idx = torch.arange(step, n, step, device=device)
        rec[idx, :kb] = rec[idx - 1, :kb]
    return rec


def log_uniform_sizes(count: int, seed: int, lo: int = 1000,
                      hi: int = 10_000_000) -> list[int]:
    """Request sizes log-uniform in [lo, hi] (the served workload's mix)."""
    u = _lsr(stream_words(_stream_seed(seed, 9), 0, count), 11).to(torch.float64)
    u = u * (2.0 ** -53)
    ll, lh = math.log(lo), math.log(hi)
    return [int(round(math.exp(ll + float(x) * (lh - ll)))) for x in u]
