"""The multi-process form of the bench on CPU (gloo, world size 2): the sort
has no exchange step, so N GPUs run N replicas; the only cross-rank work is
the barrier and the max-over-ranks timing, and rank 0 alone prints."""
import json
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(dist)
        q.put((rank, bench.max_over_ranks(float(10 + rank), dist)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_barrier_with_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    got = dict(q.get(timeout=10) for _ in range(2))
    assert got == {0: 11.0, 1: 11.0}


def test_reference_arm_runs_on_rank_zero_only():
    # under torchrun every rank runs main(); only rank 0 does the work and
    # returns the line to print
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    args = argparse.Namespace(ref_sample=20_000, warmup=3, steps=1, n=100_000_000)
    assert bench.run_reference(args, world=2, rank=1, pg=None) is None
    out = bench.run_reference(args, world=2, rank=0, pg=None)
    json.dumps(out)
    assert out["impl"] == "reference" and out["n_gpus"] == 2 and out["value"] > 0
    assert out["cpu_baseline"]["kind"] == "oracle"


def test_reference_line_keeps_the_contract():
    # the keys the reference arm's JSON line must carry, with the e2e object
    # and the cpu_baseline describing the same run
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    args = argparse.Namespace(ref_sample=20_000, warmup=3, steps=2, n=100_000_000)
    out = bench.run_reference(args, world=1, rank=0, pg=None)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e", "impl"):
        assert k in out, k
    assert out["unit"] == "GB/s" and out["higher_is_better"] is True
    assert out["warmup"] >= 3 and out["steps"] == 2
    assert out["cpu_baseline"]["value"] == out["value"] and out["cpu_baseline"]["cores"] >= 1
    assert out["e2e"]["value"] == out["value"] and out["e2e"]["unit"] == out["unit"]
    assert out["e2e"]["h2d_bytes_per_step"] == 0 and out["e2e"]["d2h_bytes_per_step"] == 0
    assert out["config"]["workload"].startswith("uniform_")


def test_end_to_end_host_buffers_fit_each_ranks_share(monkeypatch):
    # every rank on a host pins its own e2e buffers: their plan must fit the
    # rank's share of the available memory, with fewer streams first
    sys.path.insert(0, ROOT)
    import bench
    n = 100_000_000
    for local in (1, 2, 8, 64):
        monkeypatch.setenv("LOCAL_WORLD_SIZE", str(local))
        ns, ne = bench.e2e_plan(n, 2)
        assert 1 <= ns <= 2 and 4096 <= ne <= n
        if ne < n:
            assert ns == 1 and ne % 4096 == 0
        with open("/proc/meminfo") as f:
            avail = [int(l.split()[1]) * 1024 for l in f if l.startswith("MemAvailable:")][0]
        share = 0.6 * avail / local
        assert (1 + ns) * ne * bench.REC <= max(share, 2 * 4096 * bench.REC)
