"""The allocation-free entry point, ley_sort_records_noalloc.

It exists for callers that cannot allocate device memory (for example an
application whose device memory is all owned by its own pool allocator, or a
latency-bound caller that cannot accept a cudaMalloc).  Its scratch is one
fixed array inside the library, shared by every call.  These tests call it
through the C ABI and compare its output, byte for byte, with the output of
ley_sort_records on the same input, for two calls in a row (the second call
finds the first call's leftovers in the shared array).  This file is named to
be collected last.
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


def _both(ley, rec):
    d_in = rec.to("cuda:0")
    ref = torch.empty_like(d_in)
    ley.ley_sort_records(d_in, ref, key_bytes=10)
    assert ley.ley_last_device_status() == ley.LEY_OK
    got = torch.empty_like(d_in)
    assert ley.ley_sort_records_noalloc(d_in, got, key_bytes=10) == ley.LEY_OK
    return got.cpu().numpy(), ref.cpu().numpy()


def test_noalloc_matches_allocating_sort_twice(ley):
    # two different inputs in a row: the second runs on the first's leftovers
    for rec in (datagen.skew_records(200_001, seed=21),
                datagen.uniform_records(ley.LEY_NOALLOC_MAX_RECORDS, seed=22)):
        got, ref = _both(ley, rec)
        assert np.array_equal(got, ref)


def test_noalloc_same_input_twice_and_small_sizes(ley):
    rec = datagen.edge_records("few_distinct", 70_000, seed=5)
    a, ref = _both(ley, rec)
    b, _ = _both(ley, rec)
    assert np.array_equal(a, ref) and np.array_equal(b, ref)
    for n in (1, 2, 33, 4097):
        got, ref = _both(ley, datagen.uniform_records(n, seed=n))
        assert np.array_equal(got, ref)


def test_noalloc_rejects_sizes_beyond_its_limit(ley):
    n = ley.LEY_NOALLOC_MAX_RECORDS + 1
    with pytest.raises(ley.LeyError) as e:
        ley.ley_sort_records_noalloc(0, 0, n=n, rec_bytes=100, key_bytes=10)
    assert e.value.status == ley.LEY_ENOMEM
