"""GPU parity of the host-memory modes and of the k-way merge.

The partially in-memory sort, the external sort (run formation + k-way
merge under a device budget small enough to force several runs and several
merge partitions) and the standalone merge of sorted runs are compared byte
for byte with the oracle.  Ties across runs (few distinct keys) check that
the co-rank cuts and the merge keep equal keys in input order.
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


def host_sort(ley, rec, budget, key_bytes=10):
    h_in = rec.pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    ley.ley_sort_records(h_in, h_out, key_bytes=key_bytes, mem_budget=budget)
    assert ley.ley_last_device_status() == ley.LEY_OK
    return h_out.numpy()


@pytest.mark.parametrize("kind,n,budget", [
    ("uniform", 200_003, 8 << 20),      # ~4 runs of 45k records
    ("skew", 300_000, 12 << 20),
    ("few_distinct", 150_000, 8 << 20),  # equal keys across every run
    ("equal", 100_000, 6 << 20),
    ("uniform", 1_000_000, 40 << 20),
])
def test_external_sort_exact(orc, ley, kind, n, budget):
    if kind == "uniform":
        rec = datagen.uniform_records(n, seed=n)
    elif kind == "skew":
        rec = datagen.skew_records(n, seed=4)
    else:
        rec = datagen.edge_records(kind, n, seed=6)
    ws = ley.ley_workspace_bytes(n)
    assert ws + n * 100 > budget  # the partially in-memory mode cannot be used
    got = host_sort(ley, rec, budget)
    want = orc.sort_records(rec.numpy())
    if not np.array_equal(got, want):
        bad = np.where((got != want).any(axis=1))[0]
        raise AssertionError(f"{bad.size} records differ, first at {bad[:5]}")


@pytest.mark.parametrize("n", [1, 4097, 250_000])
def test_partial_sort_exact(orc, ley, n):
    rec = datagen.uniform_records(n, seed=3 + n)
    got = host_sort(ley, rec, 0)
    assert np.array_equal(got, orc.sort_records(rec.numpy()))


def test_queued_partial_sorts_on_two_streams_exact(orc, ley):
    """ley_sort_records_async: host-memory sorts queued on two streams with no
    synchronisation between the calls, so copies of different sorts overlap;
    each output equals the oracle's."""
    gens = [lambda n, s: datagen.skew_records(n, seed=s), lambda n, s: datagen.uniform_records(n, seed=s)]
    sizes = [1, 4097, 250_000, 1_000_000, 33_333, 600_001]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    jobs = []
    for i, n in enumerate(sizes):
        rec = gens[i % 2](n, 40 + i).pin_memory()
        out = torch.zeros_like(rec).pin_memory()
        ley.ley_sort_records_async(rec, out, key_bytes=10, stream=streams[i % 2])
        jobs.append((rec, out))
    for st in streams:
        st.synchronize()
    assert ley.ley_last_device_status() == ley.LEY_OK
    for rec, out in jobs:
        assert np.array_equal(out.numpy(), orc.sort_records(rec.numpy()))


def test_queued_partial_sorts_from_several_threads_exact(orc, ley):
    """Host-memory sorts queued at once from three host threads, each on its
    own streams, several calls per thread, so that the library's per-call
    streams, events and pooled scratch are taken from several threads at
    once; every output equals the oracle's."""
    import threading
    jobs = [[] for _ in range(3)]
    for t in range(3):
        for i, n in enumerate([4097, 300_001, 77_777]):
            gen = datagen.skew_records if (t + i) % 2 else datagen.uniform_records
            rec = gen(n, seed=100 + 10 * t + i).pin_memory()
            jobs[t].append((rec, torch.zeros_like(rec).pin_memory()))
    errors = []

    def worker(t):
        try:
            torch.cuda.set_device(0)
            streams = [torch.cuda.Stream(), torch.cuda.Stream()]
            for i, (rec, out) in enumerate(jobs[t]):
                ley.ley_sort_records_async(rec, out, key_bytes=10, stream=streams[i % 2])
            for st in streams:
                st.synchronize()
        except Exception as e:  # noqa: BLE001 - reported below
            errors.append(e)

    th = [threading.Thread(target=worker, args=(t,)) for t in range(3)]
    for x in th:
        x.start()
    for x in th:
        x.join()
    assert not errors, errors
    assert ley.ley_last_device_status() == ley.LEY_OK
    for per_thread in jobs:
        for rec, out in per_thread:
            assert np.array_equal(out.numpy(), orc.sort_records(rec.numpy()))


def test_queued_long_key_sorts_on_two_streams_exact(orc, ley):
    # keys longer than a tuple's 12 bytes (one sort per 12-byte window) in the
    # queued partial mode, two sorts in flight on two streams
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    jobs = []
    for i, (n, kb) in enumerate([(70_000, 30), (120_001, 17)]):
        rec = datagen.ascii_records(n, seed=60 + i, key_bytes=kb, shared_prefix=9,
                                    alphabet=4).pin_memory()
        out = torch.zeros_like(rec).pin_memory()
        ley.ley_sort_records_async(rec, out, key_bytes=kb, stream=streams[i])
        jobs.append((rec, out, kb))
    for st in streams:
        st.synchronize()
    assert ley.ley_last_device_status() == ley.LEY_OK
    for rec, out, kb in jobs:
        assert np.array_equal(out.numpy(), orc.sort_records(rec.numpy(), key_bytes=kb))


def test_queued_sort_falls_back_to_blocking_external(orc, ley):
    # the budget is below the partial mode's need: the external sort runs and
    # the call returns with the records in place
    rec = datagen.skew_records(600_001, seed=8).pin_memory()
    out = torch.zeros_like(rec).pin_memory()
    ley.ley_sort_records_async(rec, out, key_bytes=10, mem_budget=50 << 20)
    assert np.array_equal(out.numpy(), orc.sort_records(rec.numpy()))


def test_queued_sort_of_device_buffers_is_the_sort(orc, ley):
    rec = datagen.uniform_records(300_000, seed=9)
    d_in = rec.to("cuda:0")
    a, b = torch.empty_like(d_in), torch.empty_like(d_in)
    ley.ley_sort_records_async(d_in, a, key_bytes=10)
    ley.ley_sort_records(d_in, b, key_bytes=10)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    assert np.array_equal(a.cpu().numpy(), orc.sort_records(rec.numpy()))


def test_release_cache_between_sorts(orc, ley):
    # the device pool and the pinned run scratch are returned, then rebuilt
    rec = datagen.uniform_records(120_000, seed=21)
    want = orc.sort_records(rec.numpy())
    assert np.array_equal(host_sort(ley, rec, 6 << 20), want)
    torch.cuda.synchronize()
    ley.ley_release_cache()
    assert np.array_equal(host_sort(ley, rec, 6 << 20), want)
    d_in = rec.to("cuda:0")
    d_out = torch.empty_like(d_in)
    ley.ley_sort_records(d_in, d_out)
    assert np.array_equal(d_out.cpu().numpy(), want)


def test_external_budget_too_small(ley):
    rec = datagen.uniform_records(50_000, seed=1)
    with pytest.raises(ley.LeyError) as e:
        host_sort(ley, rec, 64 << 10)
    assert e.value.status == ley.LEY_ENOMEM


@pytest.mark.parametrize("k,alpha,base,step", [
    (1, None, 1000, 777), (2, None, 1000, 777), (3, b"AB", 1000, 777), (8, None, 1000, 777),
    (17, b"xyz", 1000, 777), (5, b"Q", 1000, 777),
    (16, None, 30_000, 5_001),   # the external sort's fan-in, tiles of up to 4096 tuples
    (32, b"AB", 2000, 301),      # the largest one-pass fan-in, ties across every run
    (33, None, 1500, 97),        # one pairwise round first, then the one-pass merge
    (128, b"xy", 300, 41),       # the largest fan-in: two pairwise rounds first
    (32, None, 3, 1),            # a few records per run, one sample each
    (32, None, 1, 0),            # one record per run: too small for the table, pairwise only
])
def test_merge_records_matches_oracle(orc, ley, k, alpha, base, step):
    runs, starts = [], [0]
    for r in range(k):
        m = 0 if r == 1 else base + step * r
        a = datagen.uniform_records(m, seed=50 + r).numpy().copy()
        if alpha is not None:
            al = np.frombuffer(bytes(alpha), dtype=np.uint8)
            a[:, :10] = al[a[:, :10] % len(al)]
        runs.append(orc.sort_records(a))
        starts.append(starts[-1] + m)
    cat = np.concatenate(runs)
    want = orc.kway_merge_records(cat, starts)
    d_runs = torch.from_numpy(cat).to("cuda:0")
    d_out = torch.empty_like(d_runs)
    ley.ley_merge_records(d_runs, starts, d_out)
    assert ley.ley_last_device_status() == ley.LEY_OK
    assert np.array_equal(d_out.cpu().numpy(), want)


@pytest.mark.parametrize("n,budget", [(1_000_000, 80 << 20), (600_001, 50 << 20)])
def test_keys_only_external_sort_exact(orc, ley, monkeypatch, n, budget):
    # the tuples fit the budget but the records do not: only the keys stay on
    # the device and the records are gathered from the pinned host input
    rec = datagen.skew_records(n, seed=n)
    ws = ley.ley_workspace_bytes(n)
    assert ws + n * 100 > budget > ws
    monkeypatch.setenv("LEY_EXTERNAL", "keys")
    got = host_sort(ley, rec, budget)
    want = orc.sort_records(rec.numpy())
    assert np.array_equal(got, want)
    monkeypatch.setenv("LEY_EXTERNAL", "merge")
    assert np.array_equal(host_sort(ley, rec, budget), want)


@pytest.mark.parametrize("kind,resident", [("uniform", None), ("skew", None), ("uniform", "0")])
def test_external_sort_with_runs_kept_on_the_device_exact(orc, ley, monkeypatch, kind, resident):
    # 32M records under a 3.5 GB device budget: eight runs of 4M records, of
    # which the last stay sorted in device memory (only the others go to the
    # host and back), and the merge's partition cuts are planned on the
    # device over host-resident and device-resident runs.  With
    # LEY_EXTERNAL_RESIDENT=0 every run goes to the host.  The output is
    # checked completely by the oracle (tags at bytes 10..13).
    n, budget = 32_000_000, 3_500_000_000
    if resident is not None:
        monkeypatch.setenv("LEY_EXTERNAL_RESIDENT", resident)
    hb = ley.ley_host_scratch_bytes(n, mem_budget=budget)
    if resident is None:
        assert 0 < hb < n * 100  # some runs stay on the device
    else:
        assert hb == n * 100
    gen = datagen.uniform_records if kind == "uniform" else datagen.skew_records
    h_in = torch.empty(n, 100, dtype=torch.uint8).pin_memory()
    for c0 in range(0, n, 8_000_000):
        c1 = min(n, c0 + 8_000_000)
        part = gen(c1 - c0, seed=77, device="cuda:0", tag_index=True) if kind == "skew" else \
            gen(c1 - c0, seed=77, device="cuda:0", start=c0, tag_index=True)
        if kind == "skew":
            # the skewed chunks are drawn alike (same seed), so every key
            # recurs in four runs: ties across runs; the tags are made global
            part[:, 10:14] = 0
            idx = torch.arange(c0, c1, dtype=torch.int64, device="cuda:0")
            for b in range(4):
                part[:, 10 + b] = ((idx >> (8 * b)) & 0xFF).to(torch.uint8)
        h_in[c0:c1].copy_(part.cpu())
    h_out = torch.empty_like(h_in).pin_memory()
    ley.ley_sort_records(h_in, h_out, key_bytes=10, mem_budget=budget)
    assert ley.ley_last_device_status() == ley.LEY_OK
    assert orc.check_tagged_threads(h_out.numpy(), h_in.numpy()) == -1
