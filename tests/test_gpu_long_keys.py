"""Keys longer than the 12 bytes a tuple holds: the sort runs once per
12-byte key window (least significant first), and the result must be the
oracle's stable sort on the whole key, byte for byte."""
import numpy as np
import pytest

import datagen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
DEV = "cuda:0"


@pytest.fixture(scope="module")
def ley():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_08006_gb300 import build
    build.build()
    import paper_1909_08006_gb300 as m
    return m


def _check(orc, ley, rec, key_bytes):
    d_in = rec.to(DEV)
    d_out = torch.empty_like(d_in)
    ley.ley_sort_records(d_in, d_out, key_bytes=key_bytes)
    assert ley.ley_last_device_status() == ley.LEY_OK
    want = orc.sort_records(rec.numpy(), key_bytes=key_bytes)
    got = d_out.cpu().numpy()
    if not np.array_equal(got, want):
        bad = np.where((got != want).any(axis=1))[0]
        raise AssertionError(f"{bad.size} records differ, first at {bad[:5]}")


@pytest.mark.parametrize("key_bytes", [13, 16, 24, 25, 36, 50, 100])
@pytest.mark.parametrize("n", [1, 5000, 100_003])
def test_ascii_keys_with_shared_prefix_and_duplicates(orc, ley, key_bytes, n):
    # the shared prefix spans whole windows, a tiny alphabet makes ties in
    # the later windows, and duplicated keys make ties on the whole key
    rec = datagen.ascii_records(n, seed=key_bytes, key_bytes=key_bytes,
                                shared_prefix=min(key_bytes - 1, 14), alphabet=3, dup_frac=0.1)
    _check(orc, ley, rec, key_bytes)


@pytest.mark.parametrize("key_bytes", [13, 40])
def test_uniform_long_keys(orc, ley, key_bytes):
    _check(orc, ley, datagen.uniform_records(300_000, seed=3), key_bytes)


def test_key_is_the_whole_record(orc, ley):
    rec = datagen.uniform_records(20_000, seed=4, rec_bytes=128)
    rec[:, :100] &= 0x01  # ties everywhere but the last bytes
    _check(orc, ley, rec, 128)


def test_long_keys_edge_kinds(orc, ley):
    for kind in ["equal", "two_symbol", "last_byte", "reversed"]:
        _check(orc, ley, datagen.edge_records(kind, 9000, seed=6, key_bytes=30), 30)


def test_long_keys_partial_host_mode(orc, ley):
    rec = datagen.ascii_records(250_000, seed=9, key_bytes=30, shared_prefix=12, alphabet=4)
    h_in = rec.pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    ley.ley_sort_records(h_in, h_out, key_bytes=30)
    assert np.array_equal(h_out.numpy(), orc.sort_records(rec.numpy(), key_bytes=30))


@pytest.mark.parametrize("n,kb,budget", [(200_003, 20, 10 << 20), (120_000, 37, 8 << 20)])
def test_long_keys_external_mode_exact(orc, ley, n, kb, budget):
    # a budget below the partial mode's need: runs and merge partitions are
    # each sorted window by window; few symbols and a shared prefix put ties
    # across runs and across partition cuts
    rec = datagen.ascii_records(n, seed=kb, key_bytes=kb, shared_prefix=8, alphabet=3)
    assert ley.ley_workspace_bytes(n, key_bytes=kb) + n * 100 > budget
    h_in = rec.pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    ley.ley_sort_records(h_in, h_out, key_bytes=kb, mem_budget=budget)
    assert ley.ley_last_device_status() == ley.LEY_OK
    assert np.array_equal(h_out.numpy(), orc.sort_records(rec.numpy(), key_bytes=kb))


def test_long_keys_unsupported_paths(ley):
    rec = datagen.uniform_records(100_000, seed=1)
    d = rec.to(DEV)
    with pytest.raises(ley.LeyError) as e:
        ley.ley_sort_records_batch([(d, torch.empty_like(d))], key_bytes=20)
    assert e.value.status == ley.LEY_EUNSUPPORTED


@pytest.mark.parametrize("key_bytes", [20, 30])
def test_long_keys_at_2e7(orc, ley, key_bytes):
    # 2e7 ASCII records (2 GB) with a shared 9-byte prefix and a 4-letter
    # alphabet: two and three 12-byte windows over many ties; the input
    # position is written right after the key and the complete O(n) check
    # verifies permutation, bytes and strict (key, position) order
    n = 20_000_000
    rec = datagen.ascii_records(n, seed=key_bytes, key_bytes=key_bytes, shared_prefix=9,
                                alphabet=4, device=DEV)
    i = torch.arange(n, dtype=torch.int64, device=DEV)
    for b in range(4):
        rec[:, key_bytes + b] = ((i >> (8 * b)) & 0xFF).to(torch.uint8)
    out = torch.empty_like(rec)
    ley.ley_sort_records(rec, out, key_bytes=key_bytes)
    assert ley.ley_last_device_status() == ley.LEY_OK
    bad = orc.check_tagged_threads(out.cpu().numpy(), rec.cpu().numpy(), key_bytes=key_bytes,
                                   tag_offset=key_bytes)
    assert bad == -1, bad
