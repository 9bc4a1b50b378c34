"""GPU tests of the continuous-batching sort server.

Every request's result must be byte-identical to the same request sorted
alone with the single-request call, whatever it was batched with; admission
keeps the memory charged to admitted requests within the budget; requests
submitted from several threads while batches run all complete.
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


def _make_requests(ley, count, seed, max_n=60_000):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(count):
        n = int(np.exp(rng.uniform(0, np.log(max_n))))
        if i % 2 == 0:
            gen = datagen.skew_records if i % 4 == 0 else datagen.uniform_records
            x = gen(n, seed=seed * 1000 + i).to(DEV)
            alone = torch.empty_like(x)
            ley.ley_sort_records(x, alone)
            reqs.append(("rec", x, torch.empty_like(x), alone))
        else:
            if i % 3 == 0:
                k, v = datagen.narrow_pairs(n, seed=seed * 1000 + i, distinct=7)
            else:
                k, v = datagen.uniform_pairs(n, seed=seed * 1000 + i)
            k, v = k.to(DEV), v.to(DEV)
            ak, av = torch.empty_like(k), torch.empty_like(v)
            ley.ley_sort_keys_index(k, v, ak, av)
            reqs.append(("pairs", (k, v), (torch.empty_like(k), torch.empty_like(v)), (ak, av)))
    torch.cuda.synchronize()
    return reqs


def _submit(ley, srv, r):
    if r[0] == "rec":
        return ley.ley_server_submit_records(srv, r[1], r[2])
    (k, v), (ko, vo) = r[1], r[2]
    return ley.ley_server_submit_pairs(srv, k, v, ko, vo)


def _same(r):
    if r[0] == "rec":
        return torch.equal(r[2], r[3])
    return torch.equal(r[2][0], r[3][0]) and torch.equal(r[2][1], r[3][1])


def test_results_identical_alone_and_in_the_mix(ley):
    reqs = _make_requests(ley, 120, seed=1)
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


def test_arrivals_while_batches_run_from_several_threads(ley):
    reqs = _make_requests(ley, 96, seed=2)
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
    # batches ran on several slots at once: some requests overlap in time
    # without having started together
    spans = sorted((t["start_s"], t["done_s"]) for t in times)
    assert any(b[0] > a[0] and b[0] < a[1] for a, b in zip(spans, spans[1:])) or \
        st["launched_batches"] >= 2


def test_admission_respects_the_budget(ley):
    reqs = _make_requests(ley, 40, seed=3, max_n=200_000)
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
    assert st["launched_batches"] >= 3  # the budget forced several batches


def test_request_larger_than_budget_runs_alone(ley):
    reqs = _make_requests(ley, 6, seed=4, max_n=300_000)
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


def test_server_errors(ley):
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
        y = datagen.uniform_records(5000, seed=9).to(DEV)
        out, alone = torch.empty_like(y), torch.empty_like(y)
        ley.ley_sort_records(y, alone)
        ley.ley_server_wait(srv, ley.ley_server_submit_records(srv, y, out))
        assert torch.equal(out, alone)
        with pytest.raises(ley.LeyError):
            ley.ley_server_wait(srv, 999_999)  # unknown ticket
    finally:
        ley.ley_server_destroy(srv)
