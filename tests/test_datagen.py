"""The seeded input generators: determinism and the workload shapes."""
import numpy as np

import datagen


def test_uniform_is_deterministic_and_chunk_invariant():
    a = datagen.uniform_records(1000, seed=2).numpy()
    b = datagen.uniform_records(1000, seed=2).numpy()
    assert np.array_equal(a, b)
    # records depend only on their global index
    c = datagen.uniform_records(400, seed=2, start=600).numpy()
    assert np.array_equal(a[600:], c)
    assert not np.array_equal(a, datagen.uniform_records(1000, seed=3).numpy())
    assert a.shape == (1000, 100) and a.dtype == np.uint8


def test_uniform_bytes_look_uniform():
    a = datagen.uniform_records(20000, seed=1).numpy()
    h = np.bincount(a.reshape(-1), minlength=256)
    exp = a.size / 256
    chi2 = float(((h - exp) ** 2 / exp).sum())
    assert chi2 < 400  # 255 degrees of freedom


def test_tag_index_layout():
    a = datagen.uniform_records(300, seed=1, start=70000, tag_index=True).numpy()
    t = a[:, 10:14].copy().view("<u4").reshape(-1)
    assert np.array_equal(t, np.arange(70000, 70300, dtype=np.uint32))


def test_skew_shape():
    n = 200_000
    a = datagen.skew_records(n, seed=3).numpy()
    # the 30 % duplicates copy full keys: distinct keys <= 70 % of n
    keys = np.ascontiguousarray(a[:, :10]).view("V10").reshape(-1)
    assert np.unique(keys).size <= n - (3 * n) // 10
    # top Zipf(1.2) value over 65,536 ranks holds about 19.8 % of the records
    pre = np.ascontiguousarray(a[:, :4]).view(">u4").reshape(-1)
    _, counts = np.unique(pre, return_counts=True)
    top = counts.max() / n
    assert 0.18 < top < 0.22
    cdf = datagen.zipf_cdf().numpy()
    assert abs(cdf[0] - 0.198) < 0.002
    # the rank table is a set of 65,536 distinct values
    assert np.unique(datagen.zipf_table(3).numpy()).size == 65536


def test_pairs_and_sizes():
    k, v = datagen.uniform_pairs(1000, seed=4, start=5)
    assert k.dtype.itemsize == 8 and np.array_equal(v.numpy(), np.arange(5, 1005))
    s = datagen.log_uniform_sizes(2000, seed=1)
    assert min(s) >= 1000 and max(s) <= 10_000_000
    assert 40_000 < float(np.median(s)) < 250_000  # median of log-uniform = 1e5


def test_edge_kinds():
    for kind in ["equal", "sorted", "reversed", "last_byte", "two_symbol", "few_distinct",
                 "prefix_shared"]:
        a = datagen.edge_records(kind, 500, seed=1).numpy()
        assert a.shape == (500, 100)
    e = datagen.edge_records("equal", 10, seed=1).numpy()
    assert (e[:, :10] == e[0, :10]).all()
