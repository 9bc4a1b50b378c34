"""GPU parity of the batched sorts (many independent requests of uneven sizes
in one sequence of launches) against the CPU oracle, request by request.

Each request's output must equal the oracle's sort of that request alone
(byte-exact), whatever else is in the batch; bytes outside the requests'
outputs are never written; a batch captured in a CUDA graph replays exactly.
"""
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


def _records(kind, n, seed, rec_bytes=100):
    if kind == "skew":
        r = datagen.skew_records(n, seed=seed)
    elif kind == "uniform":
        r = datagen.uniform_records(n, seed=seed, rec_bytes=rec_bytes)
    else:
        r = datagen.edge_records(kind, n, seed=seed)
    return r


SIZES = [0, 1, 2, 31, 2047, 2048, 2049, 4095, 4096, 4097, 12_289, 70_001, 250_000]


@pytest.mark.parametrize("kinds", [("uniform",), ("uniform", "skew", "equal", "few_distinct")])
def test_records_batch_matches_each_request_alone(orc, ley, kinds):
    rng = np.random.default_rng(7)
    reqs, want, guards = [], [], []
    for i, n in enumerate(SIZES + [int(x) for x in rng.integers(1, 40_000, 12)]):
        kind = kinds[i % len(kinds)]
        rec = _records(kind, n, seed=100 + i) if n else torch.empty(0, 100, dtype=torch.uint8)
        d_in = rec.to(DEV)
        # each output sits inside a guard band that must stay untouched
        band = torch.full((n * 100 + 512,), 0xA5, dtype=torch.uint8, device=DEV)
        d_out = band[256:256 + n * 100].view(n, 100)
        reqs.append((d_in, d_out, n))
        want.append(orc.sort_records(rec.numpy()) if n else None)
        guards.append(band)
    ley.ley_sort_records_batch(reqs)
    assert ley.ley_last_device_status() == ley.LEY_OK
    for (d_in, d_out, n), w, band in zip(reqs, want, guards):
        if n:
            assert np.array_equal(d_out.cpu().numpy(), w), f"request of {n} records differs"
        b = band.cpu().numpy()
        assert (b[:256] == 0xA5).all() and (b[256 + n * 100:] == 0xA5).all()


@pytest.mark.parametrize("rec_bytes,key_bytes", [(104, 10), (16, 12), (8, 3), (10, 10), (13, 5)])
def test_records_batch_other_geometries(orc, ley, rec_bytes, key_bytes):
    reqs, want = [], []
    for i, n in enumerate([1, 4097, 3, 20_000, 4096]):
        rec = datagen.uniform_records(n, seed=i, rec_bytes=rec_bytes)
        rec[:, :key_bytes] &= 0x3  # ties on every key byte
        d_in = rec.to(DEV)
        d_out = torch.empty_like(d_in)
        reqs.append((d_in, d_out))
        want.append(orc.sort_records(rec.numpy(), key_bytes=key_bytes))
    ley.ley_sort_records_batch(reqs, rec_bytes=rec_bytes, key_bytes=key_bytes)
    assert ley.ley_last_device_status() == ley.LEY_OK
    for (d_in, d_out), w in zip(reqs, want):
        assert np.array_equal(d_out.cpu().numpy(), w)


def test_pairs_batch_matches_each_request_alone(orc, ley):
    reqs, want = [], []
    for i, n in enumerate(SIZES + [100_003]):
        if i % 3 == 1:
            keys, idx = datagen.narrow_pairs(n, distinct=5, seed=i)
        else:
            keys, idx = datagen.uniform_pairs(n, seed=i)
        ko = torch.empty(n, dtype=torch.int64, device=DEV)
        io = torch.empty(n, dtype=torch.int32, device=DEV)
        reqs.append((keys.to(DEV), idx.to(DEV), ko, io, n))
        want.append(orc.sort_keys_index(keys.numpy(), idx.numpy()) if n else None)
    ley.ley_sort_keys_index_batch(reqs)
    assert ley.ley_last_device_status() == ley.LEY_OK
    for (_, _, ko, io, n), w in zip(reqs, want):
        if n:
            assert np.array_equal(ko.cpu().numpy().view(np.uint64), w[0][:n])
            assert np.array_equal(io.cpu().numpy().view(np.uint32), w[1][:n])


def test_batch_equals_single_calls(ley):
    # the batch and one call per request give identical bytes
    rng = np.random.default_rng(3)
    sizes = [int(x) for x in rng.integers(1, 30_000, 20)]
    ins = [datagen.skew_records(n, seed=50 + i).to(DEV) for i, n in enumerate(sizes)]
    outs_b = [torch.empty_like(x) for x in ins]
    outs_s = [torch.empty_like(x) for x in ins]
    ley.ley_sort_records_batch(list(zip(ins, outs_b)))
    for x, o in zip(ins, outs_s):
        ley.ley_sort_records(x, o)
    assert ley.ley_last_device_status() == ley.LEY_OK
    for a, b in zip(outs_b, outs_s):
        assert torch.equal(a, b)


def test_batch_errors(ley):
    x = torch.zeros(10, 100, dtype=torch.uint8, device=DEV)
    with pytest.raises(ley.LeyError) as e:
        ley.ley_sort_records_batch([(x, x)])  # output overlaps input
    assert e.value.status == ley.LEY_EINVAL
    with pytest.raises(ley.LeyError) as e:
        ley.ley_sort_records_batch([(x, torch.empty_like(x))], key_bytes=13)
    assert e.value.status == ley.LEY_EUNSUPPORTED
    h = torch.zeros(10, 100, dtype=torch.uint8).pin_memory()
    with pytest.raises(ley.LeyError) as e:
        ley.ley_sort_records_batch([(h, torch.empty_like(x))])  # host memory
    assert e.value.status == ley.LEY_EINVAL
    assert ley.ley_sort_records_batch([]) == ley.LEY_OK
    with pytest.raises(ley.LeyError) as e:
        ley.ley_sort_records_batch([(x, torch.empty_like(x))], mem_budget=1 << 10)
    assert e.value.status == ley.LEY_ENOMEM


def test_batch_in_cuda_graph(orc, ley):
    sizes = [5000, 1, 70_000, 4096]
    ins = [torch.empty(n, 100, dtype=torch.uint8, device=DEV) for n in sizes]
    outs = [torch.empty_like(x) for x in ins]
    reqs = list(zip(ins, outs))
    first = [datagen.uniform_records(n, seed=900 + i) for i, n in enumerate(sizes)]
    for x, r in zip(ins, first):
        x.copy_(r.to(DEV))
    ley.ley_sort_records_batch(reqs)  # library state and pool set up outside capture
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ley.ley_sort_records_batch(reqs, stream=s)
    for rep in range(3):
        data = [datagen.skew_records(n, seed=rep * 10 + i) for i, n in enumerate(sizes)]
        for x, r in zip(ins, data):
            x.copy_(r.to(DEV))
        g.replay()
        torch.cuda.synchronize()
        assert ley.ley_last_device_status() == ley.LEY_OK
        for o, r in zip(outs, data):
            assert np.array_equal(o.cpu().numpy(), orc.sort_records(r.numpy()))


def test_many_tiny_requests(orc, ley):
    # thousands of requests of 1..5 records: as many level-0 segments, each a
    # finishing task of its own
    rng = np.random.default_rng(11)
    sizes = [int(x) for x in rng.integers(1, 6, 3000)]
    recs = [datagen.uniform_records(n, seed=7000 + i) for i, n in enumerate(sizes)]
    for r in recs[::3]:
        r[:, :10] = r[0, :10].clone()  # every third request: all keys equal
    reqs = [(r.to(DEV), torch.empty(r.shape, dtype=torch.uint8, device=DEV)) for r in recs]
    ley.ley_sort_records_batch(reqs)
    assert ley.ley_last_device_status() == ley.LEY_OK
    for (d_in, d_out), r in zip(reqs, recs):
        assert np.array_equal(d_out.cpu().numpy(), orc.sort_records(r.numpy()))
    keys = [datagen.narrow_pairs(n, seed=i, distinct=2) for i, n in enumerate(sizes[:1000])]
    preqs = [(k.to(DEV), v.to(DEV), torch.empty(k.shape, dtype=torch.int64, device=DEV),
              torch.empty(v.shape, dtype=torch.int32, device=DEV)) for k, v in keys]
    ley.ley_sort_keys_index_batch(preqs)
    for (k, v, ko, vo), (hk, hv) in zip(preqs, keys):
        wk, wi = orc.sort_keys_index(hk.numpy(), hv.numpy())
        assert np.array_equal(ko.cpu().numpy().view(np.uint64), wk)
        assert np.array_equal(vo.cpu().numpy().view(np.uint32), wi)
