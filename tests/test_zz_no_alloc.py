"""The allocation-free entry point, ley_sort_records_noalloc.

It exists for callers that cannot allocate device memory (for example an
application whose device memory is all owned by its own pool allocator, or a
latency-bound caller that cannot accept a cudaMalloc).  Its scratch is one
fixed array inside the library, shared by every call.  These tests call it
through the C ABI and compare its output, byte for byte, with the CPU
oracle's sort and with the output of ley_sort_records on the same input, for
two calls in a row (the second call finds the first call's leftovers in the
shared array).  This file is named to be collected last.
"""
import numpy as np
import pytest

import datagen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ley():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_08006_gb300 import build
    build.build()
    import paper_1909_08006_gb300 as m
    return m


def _both(ley, rec, key_bytes=10):
    d_in = rec.to("cuda:0")
    ref = torch.empty_like(d_in)
    ley.ley_sort_records(d_in, ref, key_bytes=key_bytes)
    assert ley.ley_last_device_status() == ley.LEY_OK
    got = torch.empty_like(d_in)
    assert ley.ley_sort_records_noalloc(d_in, got, key_bytes=key_bytes) == ley.LEY_OK
    return got.cpu().numpy(), ref.cpu().numpy()


def _check(orc, ley, rec, key_bytes=10):
    got, ref = _both(ley, rec, key_bytes)
    want = orc.sort_records(rec.numpy(), key_bytes=key_bytes)
    assert np.array_equal(got, want)
    assert np.array_equal(got, ref)
    return got


def test_noalloc_matches_oracle_and_allocating_sort_twice(orc, ley):
    # two different inputs in a row: the second runs on the first's leftovers
    for rec in (datagen.skew_records(200_001, seed=21),
                datagen.uniform_records(ley.LEY_NOALLOC_MAX_RECORDS, seed=22)):
        _check(orc, ley, rec)


def test_noalloc_skewed_keys_at_the_size_limit(orc, ley):
    # the fixed layout must hold the worst-case segment and finishing-task
    # counts: heavily duplicated skewed keys at the largest allowed size, twice
    rec = datagen.skew_records(ley.LEY_NOALLOC_MAX_RECORDS, seed=23)
    _check(orc, ley, rec)
    _check(orc, ley, datagen.edge_records("few_distinct", ley.LEY_NOALLOC_MAX_RECORDS, seed=24))


def test_noalloc_same_input_twice_and_small_sizes(orc, ley):
    rec = datagen.edge_records("few_distinct", 70_000, seed=5)
    a = _check(orc, ley, rec)
    b = _check(orc, ley, rec)
    assert np.array_equal(a, b)
    for n in (1, 2, 33, 4097):
        _check(orc, ley, datagen.uniform_records(n, seed=n))


@pytest.mark.parametrize("rec_bytes,key_bytes", [(16, 4), (16, 8), (16, 12), (104, 4),
                                                 (104, 8), (104, 12)])
def test_noalloc_other_geometries(orc, ley, rec_bytes, key_bytes):
    # record sizes other than 100 take the permutation and the generic gather;
    # narrow key bytes force ties on every digit
    rec = datagen.uniform_records(50_003, seed=rec_bytes + key_bytes, rec_bytes=rec_bytes)
    rec[:, :key_bytes] &= 0x7
    _check(orc, ley, rec, key_bytes=key_bytes)
    _check(orc, ley, rec, key_bytes=key_bytes)


def test_noalloc_rejects_sizes_beyond_its_limit(ley):
    n = ley.LEY_NOALLOC_MAX_RECORDS + 1
    with pytest.raises(ley.LeyError) as e:
        ley.ley_sort_records_noalloc(0, 0, n=n, rec_bytes=100, key_bytes=10)
    assert e.value.status == ley.LEY_ENOMEM
