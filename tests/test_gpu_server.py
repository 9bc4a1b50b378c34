"""GPU tests of the continuous-batching sort server.

Every request's result must be byte-identical to the CPU oracle's sort of
the same request (the stable order of Section 3.1's reading) and to the same
request sorted alone with the single-request call, whatever it was batched
with; admission keeps the memory charged to admitted requests within the
budget; requests submitted from several threads while batches run all
complete, and batches on different launch slots overlap on the device clock.
"""
import threading
import time

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


def _make_requests(ley, orc, count, seed, max_n=60_000):
    """Requests with three answers each: the server's output buffer, the
    single-request call's output, and the oracle's sort (host arrays)."""
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(count):
        n = int(np.exp(rng.uniform(0, np.log(max_n))))
        if i % 2 == 0:
            gen = datagen.skew_records if i % 4 == 0 else datagen.uniform_records
            h = gen(n, seed=seed * 1000 + i)
            x = h.to(DEV)
            alone = torch.empty_like(x)
            ley.ley_sort_records(x, alone)
            want = orc.sort_records(h.numpy())
            reqs.append(("rec", x, torch.empty_like(x), alone, want))
        else:
            if i % 3 == 0:
                k, v = datagen.narrow_pairs(n, seed=seed * 1000 + i, distinct=7)
            else:
                k, v = datagen.uniform_pairs(n, seed=seed * 1000 + i)
            want = orc.sort_keys_index(k.numpy(), v.numpy())
            k, v = k.to(DEV), v.to(DEV)
            ak, av = torch.empty_like(k), torch.empty_like(v)
            ley.ley_sort_keys_index(k, v, ak, av)
            reqs.append(("pairs", (k, v), (torch.empty_like(k), torch.empty_like(v)), (ak, av),
                         want))
    torch.cuda.synchronize()
    return reqs


def _submit(ley, srv, r):
    if r[0] == "rec":
        return ley.ley_server_submit_records(srv, r[1], r[2])
    (k, v), (ko, vo) = r[1], r[2]
    return ley.ley_server_submit_pairs(srv, k, v, ko, vo)


def _same(r):
    """The served result equals the oracle's and the request sorted alone."""
    if r[0] == "rec":
        got = r[2].cpu().numpy()
        return np.array_equal(got, r[4]) and torch.equal(r[2], r[3])
    gk = r[2][0].cpu().numpy().view(np.uint64)
    gv = r[2][1].cpu().numpy().view(np.uint32)
    return (np.array_equal(gk, r[4][0]) and np.array_equal(gv, r[4][1])
            and torch.equal(r[2][0], r[3][0]) and torch.equal(r[2][1], r[3][1]))


def _overlapping_batches(times):
    """Pairs of distinct batches whose device-clock intervals overlap (two
    batches of one launch slot never do: the slot's stream runs them in turn)."""
    iv = {}
    for t in times:
        assert t["dev_done_s"] >= t["dev_start_s"] >= 0.0
        iv[t["batch"]] = (t["dev_start_s"], t["dev_done_s"])
    spans = sorted(iv.items(), key=lambda kv: kv[1][0])
    return [(a[0], b[0]) for i, a in enumerate(spans) for b in spans[i + 1:]
            if b[1][0] < a[1][1]]


def test_results_identical_alone_and_in_the_mix(ley, orc):
    reqs = _make_requests(ley, orc, 120, seed=1)
    srv = ley.ley_server_create(8 << 30, max_batch=32, slots=3)
    try:
        tickets = [_submit(ley, srv, r) for r in reqs]
        times = [ley.ley_server_wait(srv, t) for t in tickets]
        st = ley.ley_server_stats(srv)
    finally:
        ley.ley_server_destroy(srv)
    assert all(_same(r) for r in reqs)
    assert st["launched_batches"] >= 2  # 120 requests cannot fit one batch of 32
    assert all(t["submit_s"] <= t["start_s"] <= t["done_s"] for t in times)


def test_arrivals_while_batches_run_from_several_threads(ley, orc):
    reqs = _make_requests(ley, orc, 96, seed=2)
    srv = ley.ley_server_create(4 << 30, max_batch=16, slots=3)
    tickets = [None] * len(reqs)

    def producer(part):
        for j in range(part, len(reqs), 3):
            tickets[j] = _submit(ley, srv, reqs[j])
            time.sleep(0.0005 * (j % 5))

    try:
        ths = [threading.Thread(target=producer, args=(p,)) for p in range(3)]
        for t in ths:
            t.start()
        for t in ths:
            t.join()
        times = [ley.ley_server_wait(srv, t) for t in tickets]
        st = ley.ley_server_stats(srv)
    finally:
        ley.ley_server_destroy(srv)
    assert all(_same(r) for r in reqs)
    assert st["pending"] == 0 and st["inflight_batches"] == 0 and st["bytes_in_use"] == 0
    # requests admitted while others were on the GPU: at least two batches
    # were in progress on the device at the same time (device-clock events)
    assert st["launched_batches"] >= 2
    assert _overlapping_batches(times), sorted(
        {(t["batch"], t["dev_start_s"], t["dev_done_s"]) for t in times})


def test_admission_respects_the_budget(ley, orc):
    reqs = _make_requests(ley, orc, 40, seed=3, max_n=200_000)
    budget = 96 << 20  # a few requests at a time
    srv = ley.ley_server_create(budget, max_batch=64, slots=2)
    seen = []
    stop = threading.Event()

    def watch():
        while not stop.is_set():
            seen.append(ley.ley_server_stats(srv)["bytes_in_use"])
            time.sleep(0.0002)

    w = threading.Thread(target=watch)
    w.start()
    try:
        tickets = [_submit(ley, srv, r) for r in reqs]
        for t in tickets:
            ley.ley_server_wait(srv, t)
        st = ley.ley_server_stats(srv)
    finally:
        stop.set()
        w.join()
        ley.ley_server_destroy(srv)
    assert all(_same(r) for r in reqs)
    assert max(seen) <= budget
    # the requests' device memory (about 1.7x the budget in all) forced
    # several batches
    assert st["launched_batches"] >= 2


def test_request_larger_than_budget_runs_alone(ley, orc):
    reqs = _make_requests(ley, orc, 6, seed=4, max_n=300_000)
    srv = ley.ley_server_create(64 << 10, max_batch=64, slots=2)  # smaller than any request
    try:
        tickets = [_submit(ley, srv, r) for r in reqs]
        times = [ley.ley_server_wait(srv, t) for t in tickets]
        st = ley.ley_server_stats(srv)
    finally:
        ley.ley_server_destroy(srv)
    assert all(_same(r) for r in reqs)
    assert st["launched_batches"] == len(reqs)
    spans = sorted((t["start_s"], t["done_s"]) for t in times)
    assert all(b[0] >= a[1] for a, b in zip(spans, spans[1:]))  # one at a time
    assert not _overlapping_batches(times)  # and one at a time on the device


def test_server_errors(ley, orc):
    with pytest.raises(ley.LeyError):
        ley.ley_server_create(0)
    srv = ley.ley_server_create(1 << 30)
    try:
        x = torch.zeros(10, 100, dtype=torch.uint8, device=DEV)
        with pytest.raises(ley.LeyError) as e:
            ley.ley_server_submit_records(srv, x, torch.empty_like(x), key_bytes=13)
        assert e.value.status == ley.LEY_EUNSUPPORTED
        with pytest.raises(ley.LeyError) as e:
            ley.ley_server_submit_records(srv, x, x)  # output overlaps input
        assert e.value.status == ley.LEY_EINVAL
        h = torch.zeros(10, 100, dtype=torch.uint8).pin_memory()
        with pytest.raises(ley.LeyError) as e:
            ley.ley_server_submit_records(srv, h, torch.empty_like(x))  # host memory
        assert e.value.status == ley.LEY_EINVAL
        # the server still serves after rejections
        h = datagen.uniform_records(5000, seed=9)
        y = h.to(DEV)
        out = torch.empty_like(y)
        ley.ley_server_wait(srv, ley.ley_server_submit_records(srv, y, out))
        assert np.array_equal(out.cpu().numpy(), orc.sort_records(h.numpy()))
        with pytest.raises(ley.LeyError):
            ley.ley_server_wait(srv, 999_999)  # unknown ticket
    finally:
        ley.ley_server_destroy(srv)
