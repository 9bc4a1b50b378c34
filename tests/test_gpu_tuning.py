"""The sort's tunables (Algorithm 1's big- and tiny-bucket thresholds, CTAs
per SM) never change a result: byte-exact parity with the oracle under a
range of tunings, and the autotuner picks one of its candidates."""
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
    yield m
    m.ley_set_tuning(None)


TUNINGS = [
    {"big_bucket": 256, "tiny_bucket": 32},
    {"big_bucket": 1024, "tiny_bucket": 128, "finish_ctas_per_sm": 1},
    {"big_bucket": 2048, "tiny_bucket": 256, "pass_ctas_per_sm": 1},
    {"big_bucket": 777, "tiny_bucket": 33, "finish_ctas_per_sm": 3, "pass_ctas_per_sm": 1},
]


@pytest.mark.parametrize("tuning", TUNINGS)
def test_tunings_never_change_results(orc, ley, tuning):
    ley.ley_set_tuning(tuning)
    try:
        assert ley.ley_get_tuning()["big_bucket"] == tuning["big_bucket"]
        for kind, n in [("uniform", 300_001), ("skew", 200_000), ("few_distinct", 70_000),
                        ("equal", 50_000), ("prefix_shared", 90_000)]:
            if kind == "uniform":
                rec = datagen.uniform_records(n, seed=n)
            elif kind == "skew":
                rec = datagen.skew_records(n, seed=2)
            else:
                rec = datagen.edge_records(kind, n, seed=5)
            d_in = rec.to(DEV)
            d_out = torch.empty_like(d_in)
            ley.ley_sort_records(d_in, d_out)
            assert ley.ley_last_device_status() == ley.LEY_OK
            assert np.array_equal(d_out.cpu().numpy(), orc.sort_records(rec.numpy())), kind
        keys, idx = datagen.narrow_pairs(100_003, seed=3, distinct=300)
        ko = torch.empty(keys.shape, dtype=torch.int64, device=DEV)
        io = torch.empty(idx.shape, dtype=torch.int32, device=DEV)
        ley.ley_sort_keys_index(keys.to(DEV), idx.to(DEV), ko, io)
        wk, wi = orc.sort_keys_index(keys.numpy(), idx.numpy())
        assert np.array_equal(ko.cpu().numpy().view(np.uint64), wk)
        assert np.array_equal(io.cpu().numpy().view(np.uint32), wi)
    finally:
        ley.ley_set_tuning(None)


def test_invalid_tunings_rejected(ley):
    for bad in [{"big_bucket": 100}, {"big_bucket": 4096}, {"tiny_bucket": 8},
                {"tiny_bucket": 512}, {"finish_ctas_per_sm": 1000}]:
        with pytest.raises(ley.LeyError) as e:
            ley.ley_set_tuning(bad)
        assert e.value.status == ley.LEY_EINVAL
    ley.ley_set_tuning(None)
    assert ley.ley_get_tuning() == {"big_bucket": 2048, "tiny_bucket": 64,
                                    "finish_ctas_per_sm": 0, "pass_ctas_per_sm": 0}


def test_autotuner_picks_a_candidate_and_stays_exact(orc, ley):
    try:
        best = ley.ley_autotune_records(2_000_000)
        assert best["big_bucket"] in (2048, 1536, 1024)
        assert best["tiny_bucket"] in (32, 64, 128)
        assert best["finish_ctas_per_sm"] in (0, 3)
        assert ley.ley_get_tuning() == best
        rec = datagen.skew_records(250_000, seed=8)
        d_in = rec.to(DEV)
        d_out = torch.empty_like(d_in)
        ley.ley_sort_records(d_in, d_out)
        assert np.array_equal(d_out.cpu().numpy(), orc.sort_records(rec.numpy()))
    finally:
        ley.ley_set_tuning(None)


def test_autotuner_on_callers_records_leaves_them_and_stays_exact(orc, ley):
    # tuning on the data to be sorted: the records are read, never written
    try:
        rec = datagen.skew_records(400_000, seed=12)
        d_in = rec.to(DEV)
        before = d_in.clone()
        best = ley.ley_autotune_records_on(d_in, key_bytes=10)
        assert torch.equal(d_in, before)
        assert best["big_bucket"] in (2048, 1536, 1024)
        assert best["tiny_bucket"] in (32, 64, 128)
        assert ley.ley_get_tuning() == best
        d_out = torch.empty_like(d_in)
        ley.ley_sort_records(d_in, d_out)
        assert np.array_equal(d_out.cpu().numpy(), orc.sort_records(rec.numpy()))
        with pytest.raises(ley.LeyError) as e:  # host memory is not a device record array
            ley.ley_autotune_records_on(rec.pin_memory(), key_bytes=10)
        assert e.value.status == ley.LEY_EINVAL
    finally:
        ley.ley_set_tuning(None)


def test_tuning_changes_while_sorts_run_never_fail_them(orc, ley):
    # One thread keeps changing the tuning (big-bucket threshold 256..2048)
    # and another runs the autotuner on its own records, while this thread
    # sorts on its own stream and serves requests through a server.  Every
    # sort reads the tuning once when it starts, so none of them may fail
    # (a layout sized for one threshold and run with another would) and every
    # result must match the oracle.
    import threading
    rec = datagen.skew_records(600_000, seed=31)
    want = orc.sort_records(rec.numpy())
    d_in = rec.to(DEV)
    tune_in = datagen.uniform_records(200_000, seed=32).to(DEV)
    small = [datagen.uniform_records(20_000 + 997 * i, seed=40 + i) for i in range(12)]
    small_want = [orc.sort_records(x.numpy()) for x in small]
    small_dev = [x.to(DEV) for x in small]
    torch.cuda.synchronize()
    stop = threading.Event()
    errors = []

    def flip():
        k = 0
        try:
            while not stop.is_set():
                ley.ley_set_tuning(TUNINGS[k % len(TUNINGS)])
                k += 1
        except Exception as e:  # noqa: BLE001 - reported below
            errors.append(e)

    def autotune():
        try:
            torch.cuda.set_device(0)
            ley.ley_autotune_records_on(tune_in, key_bytes=10)
        except Exception as e:  # noqa: BLE001
            errors.append(e)

    th = [threading.Thread(target=flip), threading.Thread(target=autotune)]
    for t in th:
        t.start()
    try:
        s1 = torch.cuda.Stream()
        d_out = torch.empty_like(d_in)
        for _ in range(12):
            ley.ley_sort_records(d_in, d_out, stream=s1)
            assert ley.ley_last_device_status(s1) == ley.LEY_OK
            assert np.array_equal(d_out.cpu().numpy(), want)
        srv = ley.ley_server_create(2 << 30, max_batch=4, slots=2)
        try:
            outs = [torch.empty_like(x) for x in small_dev]
            tickets = [ley.ley_server_submit_records(srv, x, o) for x, o in zip(small_dev, outs)]
            for t in tickets:
                ley.ley_server_wait(srv, t)
        finally:
            ley.ley_server_destroy(srv)
        for o, w in zip(outs, small_want):
            assert np.array_equal(o.cpu().numpy(), w)
    finally:
        stop.set()
        for t in th:
            t.join()
        ley.ley_set_tuning(None)
    assert not errors, errors
