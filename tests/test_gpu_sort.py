"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Integer work throughout, so every comparison is byte-exact (tolerance 0).
Sizes span several 4096-tuple pass tiles and 2048-tuple finishing tasks with
ragged tails; the degenerate key patterns of the method (all keys equal, one
varying byte, constant leading digits, heavy duplication) are covered.
"""
import os

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


DEV = "cuda:0"


def gpu_sort(ley, rec: torch.Tensor, key_bytes=10, **kw):
    d_in = rec.to(DEV)
    d_out = torch.empty_like(d_in)
    ley.ley_sort_records(d_in, d_out, key_bytes=key_bytes, **kw)
    assert ley.ley_last_device_status() == ley.LEY_OK
    return d_out.cpu().numpy()


def check_exact(orc, ley, rec: torch.Tensor, key_bytes=10, **kw):
    got = gpu_sort(ley, rec, key_bytes, **kw)
    want = orc.sort_records(rec.numpy(), key_bytes=key_bytes)
    if not np.array_equal(got, want):
        bad = np.where((got != want).any(axis=1))[0]
        raise AssertionError(f"{bad.size} records differ, first at {bad[:5]}")


# --------------------------------------------------- one round of Alg. 1

@pytest.mark.parametrize("n", [1, 2, 100, 4095, 4096, 4097, 50_000, 300_001])
def test_partition_round_matches_oracle(orc, ley, n):
    rec = datagen.skew_records(n, seed=n % 97)
    for digit in (0, 5, 9):
        order = torch.empty(n, dtype=torch.int32, device=DEV)
        hist = torch.empty(256, dtype=torch.int64, device=DEV)
        ley.ley_partition_records(rec.to(DEV), digit, order, hist)
        assert ley.ley_last_device_status() == ley.LEY_OK
        assert np.array_equal(hist.cpu().numpy().view(np.uint64), orc.digit_histogram(rec.numpy(), digit))
        assert np.array_equal(order.cpu().numpy().view(np.uint32).astype(np.uint64),
                              orc.msd_partition(rec.numpy(), digit))


def test_partition_worked_example(orc, ley):
    # Section 2.2: abc, bcd, cde, cfe, dfg -> buckets a:1 b:1 c:2 d:1
    recs = [b"abc\0", b"bcd\0", b"cde\0", b"cfe\0", b"dfg\0"]
    a = torch.tensor([list(r) for r in recs], dtype=torch.uint8)
    order = torch.empty(5, dtype=torch.int32, device=DEV)
    hist = torch.empty(256, dtype=torch.int64, device=DEV)
    ley.ley_partition_records(a.to(DEV), 0, order, hist, key_bytes=3)
    h = hist.cpu().numpy()
    assert {chr(b): int(h[b]) for b in range(256) if h[b]} == {"a": 1, "b": 1, "c": 2, "d": 1}
    assert order.cpu().tolist() == [0, 1, 2, 3, 4]


# ------------------------------------------------------ records, exact

SIZES = [1, 2, 3, 7, 31, 32, 33, 1000, 2047, 2048, 2049, 4096, 4097, 12_289, 100_003]


@pytest.mark.parametrize("n", SIZES)
def test_uniform_records_exact(orc, ley, n):
    check_exact(orc, ley, datagen.uniform_records(n, seed=1000 + n))


@pytest.mark.parametrize("n", [5, 2049, 30_000, 200_001])
def test_skew_records_exact(orc, ley, n):
    check_exact(orc, ley, datagen.skew_records(n, seed=7))


@pytest.mark.parametrize("kind", ["equal", "sorted", "reversed", "last_byte", "two_symbol",
                                  "few_distinct", "prefix_shared"])
@pytest.mark.parametrize("n", [3, 2500, 70_000])
def test_degenerate_keys_exact(orc, ley, kind, n):
    check_exact(orc, ley, datagen.edge_records(kind, n, seed=3))


def test_config1_one_million_uniform(orc, ley):
    # 1,000,000 records x 100 B, uniform, full comparison with the oracle
    check_exact(orc, ley, datagen.uniform_records(1_000_000, seed=1))


def test_skew_one_million(orc, ley):
    check_exact(orc, ley, datagen.skew_records(1_000_000, seed=3))


@pytest.mark.parametrize("rec_bytes,key_bytes", [(16, 12), (8, 1), (104, 10), (100, 4),
                                                 (12, 12), (4096, 7), (20, 9), (10, 10), (1, 1),
                                                 (3, 2), (13, 7), (102, 10), (4095, 12)])
def test_other_geometries_exact(orc, ley, rec_bytes, key_bytes):
    n = 20_000 if rec_bytes < 1000 else 2_000
    rec = datagen.uniform_records(n, seed=rec_bytes, rec_bytes=rec_bytes)
    rec[:, :key_bytes] &= 0x3  # ties on every byte
    check_exact(orc, ley, rec, key_bytes=key_bytes)


def test_separate_tma_gather_variant_exact(orc, ley, monkeypatch):
    # the finish kernel writes a permutation and a separate TMA kernel gathers
    monkeypatch.setenv("LEY_GATHER", "tma")
    for n in [1, 31, 33, 4096, 100_003]:
        check_exact(orc, ley, datagen.uniform_records(n, seed=n + 6))
    check_exact(orc, ley, datagen.edge_records("equal", 40_000, seed=4))


@pytest.mark.parametrize("kind", ["equal", "few_distinct"])
def test_long_equal_runs_exact(orc, ley, kind):
    # runs of equal keys far longer than one finishing task, cut into pieces
    # with a ragged last piece
    check_exact(orc, ley, datagen.edge_records(kind, 1_000_003, seed=8))


@pytest.mark.parametrize("in_off,out_off", [(16, 48), (48, 16), (112, 0)])
def test_buffers_at_16_byte_offsets(orc, ley, in_off, out_off):
    # record arrays that start 16-byte aligned but not 128- or 256-byte aligned
    n = 70_001
    rec = datagen.uniform_records(n, seed=in_off + out_off)
    big_in = torch.zeros(n * 100 + 256, dtype=torch.uint8, device=DEV)
    big_out = torch.zeros(n * 100 + 256, dtype=torch.uint8, device=DEV)
    d_in = big_in[in_off:in_off + n * 100].view(n, 100)
    d_in.copy_(rec.to(DEV))
    d_out = big_out[out_off:out_off + n * 100].view(n, 100)
    ley.ley_sort_records(d_in, d_out)
    assert ley.ley_last_device_status() == ley.LEY_OK
    assert np.array_equal(d_out.cpu().numpy(), orc.sort_records(rec.numpy(), key_bytes=10))
    # nothing outside the output records was written
    assert not big_out[:out_off].any() and not big_out[out_off + n * 100:].any()


def test_repeated_calls_same_answer(orc, ley):
    rec = datagen.skew_records(50_000, seed=11)
    a = gpu_sort(ley, rec)
    b = gpu_sort(ley, rec)
    assert np.array_equal(a, b)


# --------------------------------------------------------------- pairs

def gpu_pairs(ley, keys, idx):
    ko = torch.empty(keys.shape, dtype=torch.int64, device=DEV)
    io = torch.empty(idx.shape, dtype=torch.int32, device=DEV)
    ley.ley_sort_keys_index(keys.to(DEV), idx.to(DEV), ko, io)
    assert ley.ley_last_device_status() == ley.LEY_OK
    return ko.cpu().numpy().view(np.uint64), io.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("n", [1, 5, 1000, 2049, 4097, 100_003, 1_000_000])
def test_pairs_uniform_exact(orc, ley, n):
    keys, idx = datagen.uniform_pairs(n, seed=n)
    ko, io = gpu_pairs(ley, keys, idx)
    wk, wi = orc.sort_keys_index(keys.numpy(), idx.numpy())
    assert np.array_equal(ko, wk) and np.array_equal(io, wi)


@pytest.mark.parametrize("distinct", [1, 2, 300, 70_000])
def test_pairs_ties_exact(orc, ley, distinct):
    keys, idx = datagen.narrow_pairs(200_000, seed=distinct, distinct=distinct)
    idx = idx * 3 + 1  # payload is not the position: it must travel, not decide
    ko, io = gpu_pairs(ley, keys, idx)
    wk, wi = orc.sort_keys_index(keys.numpy(), idx.numpy())
    assert np.array_equal(ko, wk) and np.array_equal(io, wi)


# -------------------------------------------------- host-memory mode

def test_pinned_host_records_exact(orc, ley):
    rec = datagen.skew_records(120_000, seed=5).pin_memory()
    out = torch.empty_like(rec).pin_memory()
    ley.ley_sort_records(rec, out, key_bytes=10)
    assert np.array_equal(out.numpy(), orc.sort_records(rec.numpy()))


# ------------------------------------------------------------- errors

def test_error_codes(ley):
    rec = datagen.uniform_records(1000, seed=1).to(DEV)
    out = torch.empty_like(rec)
    with pytest.raises(ley.LeyError) as e:  # key longer than the record
        ley.ley_sort_records(rec, out, key_bytes=101)
    assert e.value.status == ley.LEY_EUNSUPPORTED
    with pytest.raises(ley.LeyError) as e:  # overlapping output
        ley.ley_sort_records(rec, rec, key_bytes=10)
    assert e.value.status == ley.LEY_EINVAL
    with pytest.raises(ley.LeyError) as e:  # misaligned device pointer
        ley.ley_sort_records(rec.data_ptr() + 4, out, n=999, rec_bytes=100)
    assert e.value.status == ley.LEY_EINVAL
    with pytest.raises(ley.LeyError) as e:  # mixed memory kinds
        ley.ley_sort_records(rec.cpu().pin_memory(), out, key_bytes=10)
    assert e.value.status == ley.LEY_EINVAL
    with pytest.raises(ley.LeyError) as e:  # budget below the scratch size
        ley.ley_sort_records(rec, out, key_bytes=10, mem_budget=1000)
    assert e.value.status == ley.LEY_ENOMEM
    # nothing was queued by the failed calls; the device status stays clean
    assert ley.ley_last_device_status() == ley.LEY_OK


# ------------------------------------------------------ full-size runs

def _full(ley, orc, rec_gen, n, samples=16, threads=False):
    """Sort n tagged records on the GPU; verify with the O(n) complete check
    (permutation, byte equality with the input, strict (key, index) order)."""
    d_in = rec_gen(n)
    d_out = torch.empty_like(d_in)
    ley.ley_sort_records(d_in, d_out, key_bytes=10)
    assert ley.ley_last_device_status() == ley.LEY_OK
    host_in = d_in.cpu().numpy()
    del d_in
    host_out = d_out.cpu().numpy()
    del d_out
    torch.cuda.empty_cache()
    check = orc.check_tagged_threads if threads else orc.check_tagged
    assert check(host_out, host_in) == -1
    # sampled positions from the definition: rank(i) scans all n records
    rng = np.random.default_rng(1)
    samples = np.sort(rng.choice(n, samples, replace=False)).astype(np.uint64)
    ranks = orc.rank_records(host_in, samples)
    for i, r in zip(samples, ranks):
        assert np.array_equal(host_out[int(r)], host_in[int(i)])


def test_full_size_uniform_1e8(orc, ley):
    n = 100_000_000
    _full(ley, orc, lambda m: datagen.uniform_records(m, seed=2, device=DEV, tag_index=True), n)


def test_full_size_skew_1e8(orc, ley):
    n = 100_000_000
    _full(ley, orc, lambda m: datagen.skew_records(m, seed=3, device=DEV, tag_index=True), n)


def test_full_size_uniform_4e8(orc, ley):
    # four times the 10 GB workload in one internal sort (40 GB in and out of
    # HBM, record indices up to 4e8): the largest size whose complete check
    # fits the host's memory beside the two copies
    n = 400_000_000
    _full(ley, orc, lambda m: datagen.uniform_records(m, seed=4, device=DEV, tag_index=True), n,
          samples=4, threads=True)


@pytest.mark.parametrize("kind", ["few_distinct", "prefix_shared", "two_symbol"])
def test_full_size_degenerate_1e8(orc, ley, kind):
    # degenerate keys at the full 10 GB size: equal runs of ~2e7 records cut
    # into finishing pieces, keys that differ only in their last two bytes,
    # keys from a two-letter alphabet (ties on every digit)
    def gen(m):
        rec = datagen.edge_records(kind, m, seed=11, device=DEV)
        i = torch.arange(m, dtype=torch.int64, device=DEV)
        for b in range(4):  # input positions at bytes 10..13, little-endian
            rec[:, 10 + b] = ((i >> (8 * b)) & 0xFF).to(torch.uint8)
        return rec
    _full(ley, orc, gen, 100_000_000, samples=4, threads=True)


@pytest.mark.parametrize("rec_bytes,key_bytes", [(104, 12), (16, 8)])
def test_large_other_geometries(orc, ley, rec_bytes, key_bytes):
    # 3e7 records of other sizes (permutation plus the generic gather), the
    # input position tagged right after the key
    n = 30_000_000
    d_in = datagen.uniform_records(n, seed=rec_bytes, rec_bytes=rec_bytes, device=DEV,
                                   tag_index=True, tag_offset=key_bytes)
    d_out = torch.empty_like(d_in)
    ley.ley_sort_records(d_in, d_out, key_bytes=key_bytes)
    assert ley.ley_last_device_status() == ley.LEY_OK
    bad = orc.check_tagged_threads(d_out.cpu().numpy(), d_in.cpu().numpy(), key_bytes=key_bytes,
                                   tag_offset=key_bytes)
    assert bad == -1, bad


@pytest.mark.parametrize("distinct", [0, 1000])
def test_full_size_pairs_1e8(orc, ley, distinct):
    # 1e8 (u64 key, u32 index) pairs, uniform keys or keys from 1000 values
    # (runs of ~1e5 equal keys); the payload is the input position, so the
    # O(n) check verifies the permutation, the keys and the strict
    # (key, index) order of the whole output
    n = 100_000_000
    if distinct:
        keys, idx = datagen.narrow_pairs(n, seed=7, distinct=distinct, device=DEV)
    else:
        keys, idx = datagen.uniform_pairs(n, seed=6, device=DEV)
    ko, io = torch.empty_like(keys), torch.empty_like(idx)
    ley.ley_sort_keys_index(keys, idx, ko, io)
    assert ley.ley_last_device_status() == ley.LEY_OK
    k_in = keys.cpu().numpy().view(np.uint64)
    bad = orc.check_pairs_tagged(ko.cpu().numpy(), io.cpu().numpy(), k_in)
    assert bad == -1, bad


def test_generator_same_on_gpu_and_cpu():
    a = datagen.uniform_records(5000, seed=9, device=DEV).cpu()
    b = datagen.uniform_records(5000, seed=9)
    assert torch.equal(a, b)
    c = datagen.skew_records(50_000, seed=9, device=DEV).cpu()
    d = datagen.skew_records(50_000, seed=9)
    assert torch.equal(c, d)


# ------------------------------------------------- failure detection

@pytest.mark.parametrize("which", [0, 1])
def test_bounded_wait_gives_up_and_reports(orc, ley, which):
    # a wait on a flag nobody sets (0) or an mbarrier no copy completes (1)
    # must latch LEY_ETIMEOUT, clear on read, and leave the context usable
    assert ley.ley_selftest_timeout(which) == ley.LEY_ETIMEOUT
    assert ley.ley_last_device_status() == ley.LEY_OK
    rec = datagen.uniform_records(10_000, seed=12)
    check_exact(orc, ley, rec)
