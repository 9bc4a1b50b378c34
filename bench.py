"""Benchmark: GB/s of 100-byte records sorted on one GB300.

Default workload: the 10 GB internal sort -- 100,000,000 records x 100 B,
uniform 10-byte keys and 90-byte values from a seed, resident in HBM
(inputs and outputs are 10 GB each, far larger than the 129 MB L2, so no L2
flush is needed between steps).  One step = one ley_sort_records call:
key extraction, MSD radix passes, small-bucket finishing and the record
gather.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  ``value`` is device-timed (CUDA events on the sorting
stream); ``e2e`` is the same metric through the C ABI with pinned host
buffers (host->device and device->host copies inside the timed region): host
to host sorts queued back to back on two streams (ley_sort_records_async), so
one step's copy out overlaps the next step's copy in, with the latency of one
blocking call beside it (``single_call_ms``);
``roofline`` is the dominant kernel's algorithmic bytes over its measured
launch time against the measured HBM copy bandwidth; ``cpu_baseline`` is the
CPU oracle timed on this host (single-threaded on a bounded sample, and on
every core over the whole workload).  The line also carries the other
configurations, each measured in the same process: ``skew`` (the skewed 10 GB
sort), ``host_modes`` (the 20 GB partially in-memory and the external sort of
pinned host records under a 30 GB device budget, each output checked
completely by the oracle), ``batch`` and ``serve`` (many uneven requests,
batched and through the continuous-batching server, against one launch per
request).  With N > 1 (torchrun) every rank sorts its own replica of the
workload ("replicas only": the sort has no exchange step) and rank 0 reports
the max-over-ranks time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GB/s of 100-byte records sorted on 1 GB300 (10 GB in-HBM)"
REC, KEY = 100, 10

# Algorithmic HBM bytes per record for each kernel of the internal sort of
# uniform 10-byte keys (reads + writes): the bytes the method must move.
ALG_BYTES = {
    "extract": 10 + 16,   # key bytes in, 16-byte tuple out
    "pass": 16 + 16,      # tuple in, tuple out, per level that moves it
    "hist": 16,           # tuple in
    "finish": 16 + 4,     # tuple in, u32 permutation out
    "gather": 4 + 100 + 100,  # permutation + record in, record out
    # finishing with the record gather fused in: tuple in, record in, record out
    "finish_gather": 16 + 100 + 100,
}
PATH_BYTES = 306          # whole path: extract + 2 passes + finish with the gather


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def source_hash(name: str) -> str:
    """Hash of one CUDA source file of the library."""
    with open(os.path.join(ROOT, "paper_1909_08006_gb300", "csrc", name), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def committed_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current source of that kernel's file; else None."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(workload, {}).get(kernel)
    if not e or e.get("source_hash") != source_hash(e.get("source_file", "")):
        return None
    return e.get("bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl != "reference" else "gloo"
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


def max_over_ranks(x: float, pg, device=None) -> float:
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def barrier(pg, device=None):
    if pg is not None:
        if device is not None:
            pg.barrier(device_ids=[device.index])
        else:
            pg.barrier()


# ----------------------------------------------------------- CPU baseline

def oracle_sample(n_sample: int, seed: int = 2, skew: bool = False, device=None,
                  threads: int = 1):
    """The CPU oracle on the first n_sample records of the workload: with one
    thread the qsort on (key, index) + record copy, with more the chunked
    sort + T-way merge + parallel copy.  Returns (GB/s, seconds)."""
    import datagen
    import oracle
    gen = datagen.skew_records if skew else datagen.uniform_records
    recs = gen(n_sample, seed=seed, device=device or "cpu").cpu().numpy()
    oracle.build()
    t0 = time.perf_counter()
    if threads == 1:
        oracle.sort_records(recs, key_bytes=KEY)
    else:
        oracle.sort_records_threads(recs, key_bytes=KEY, threads=threads)
    dt = time.perf_counter() - t0
    return n_sample * REC / dt / 1e9, dt


# ------------------------------------------------------------- our arm

def run_ours(args, world, rank, local, pg):
    import torch
    import datagen
    import paper_1909_08006_gb300 as ley

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    n = args.n
    stream = torch.cuda.Stream(dev)
    wl = args.workload
    tuning = None
    if args.autotune and wl not in ("uniform", "skew", "ascii"):
        # the record workloads tune on their own data (in _run_workload)
        tuning = ley.ley_autotune_records(min(n, 100_000_000), REC, KEY)
    out = _run_workload(args, world, rank, local, pg, dev, stream, wl, n)
    if out is not None:
        out["tuning"] = tuning if tuning is not None else ley.ley_get_tuning()
    return out


def _run_workload(args, world, rank, local, pg, dev, stream, wl, n):
    import numpy as np
    import torch
    import datagen
    import paper_1909_08006_gb300 as ley
    if wl == "pairs":
        return run_pairs(args, world, rank, dev, stream, pg)
    if wl in ("partial", "external"):
        return run_host_mode(args, world, rank, dev, stream, pg)
    if wl == "batch":
        return run_batch(args, world, rank, dev, stream, pg)
    if wl == "serve":
        return run_serve(args, world, rank, dev, stream, pg)
    kb = args.key_bytes
    if wl == "ascii":  # printable keys, like the Sort Benchmark's ASCII records
        d_in = datagen.ascii_records(n, seed=6, key_bytes=kb, device=dev)
    else:
        gen = datagen.skew_records if wl == "skew" else datagen.uniform_records
        d_in = gen(n, seed=2 if wl == "uniform" else 3, device=dev)
    torch.cuda.synchronize()
    if args.autotune:  # the thresholds that sort this workload's own records fastest
        ley.ley_autotune_records_on(d_in, n=n, rec_bytes=REC, key_bytes=kb)
    d_out = torch.empty_like(d_in)

    def step():
        ley.ley_sort_records(d_in, d_out, n=n, rec_bytes=REC, key_bytes=kb, stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    if ley.ley_last_device_status(stream) != ley.LEY_OK:
        raise RuntimeError("device-side error during warm-up")

    # ---- timed region (device time on the sorting stream)
    clk = ClockSampler(dev.index)
    barrier(pg, dev)
    torch.cuda.synchronize()
    launches0 = ley.ley_launch_count()
    clk.start()
    time.sleep(0.3)
    # an event between consecutive steps gives each step's own time too
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    e0, e1 = evs[0], evs[-1]
    e0.record(stream)
    for k in range(args.steps):
        step()
        evs[k + 1].record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    launches = ley.ley_launch_count() - launches0
    barrier(pg, dev)
    ms = e0.elapsed_time(e1) / args.steps
    ms = max_over_ranks(ms, pg, dev)
    per_step = sorted(evs[k].elapsed_time(evs[k + 1]) for k in range(args.steps))
    step_stats = {"median_ms": round(statistics.median(per_step), 3),
                  "p99_ms": round(per_step[min(len(per_step) - 1,
                                               int(0.99 * len(per_step)))], 3),
                  "min_ms": round(per_step[0], 3), "max_ms": round(per_step[-1], 3)}
    if ley.ley_last_device_status(stream) != ley.LEY_OK:
        raise RuntimeError("device-side error in the timed region")

    # ---- per-kernel times (events around each launch, same stream)
    ley.ley_profile_enable(True)
    for _ in range(3):
        step()
    torch.cuda.synchronize()
    prof = ley.ley_profile_read()
    ley.ley_profile_enable(False)
    peak, peak_src = load_peaks()
    kernels = {}
    for name, (cnt, tot) in prof.items():
        per_sort_ms = tot / 3
        entry = {"launches_per_sort": cnt // 3, "ms_per_sort": round(per_sort_ms, 4)}
        if name in ALG_BYTES:
            moved = ALG_BYTES[name] * n * (2 if name == "pass" else 1)
            entry["alg_GBps"] = round(moved / (per_sort_ms * 1e-3) / 1e9, 1)
        kernels[name] = entry
    dom = max(prof.items(), key=lambda kv: kv[1][1])[0]
    dom_ms = prof[dom][1] / 3
    dom_bytes = ALG_BYTES.get(dom, 0) * n * (2 if dom == "pass" else 1)
    dom_launch_ms = prof[dom][1] / prof[dom][0]
    # the dominant kernel moves its bytes in one launch (gather) or in the
    # launches that carry work (pass: two levels at uniform keys)
    achieved = dom_bytes / (dom_ms * 1e-3) / 1e9
    workload = f"{wl}_{n}"
    roofline = {
        "kernel": dom, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
        "unit": "GB/s", "frac": round(achieved / peak, 4), "peak_source": peak_src,
        "alg_bytes_per_record": ALG_BYTES.get(dom), "launch_ms": round(dom_launch_ms, 4),
        "traffic": committed_traffic(dom, workload),
        "path_frac": round(PATH_BYTES * n / (ms * 1e-3) / 1e9 / peak, 4),
    }

    # ---- end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        # Host buffers from cuMemHostAlloc (exact size); the input is the same
        # records, copied out of HBM once.  Every rank on this host pins its
        # own buffers, so their size is planned against the host's free memory.
        del d_out
        ns, ne = e2e_plan(n, args.e2e_streams)
        h_in = host_alloc(ne * REC)
        torch.from_numpy(h_in).view(ne, REC).copy_(d_in[:ne])
        del d_in
        torch.cuda.empty_cache()
        h_outs = [host_alloc(ne * REC) for _ in range(ns)]
        addr_in = h_in.ctypes.data
        addr_out = [a.ctypes.data for a in h_outs]
        streams = [stream] + [torch.cuda.Stream(dev) for _ in range(ns - 1)]
        # warm-up: one sort queued on each stream (each gets its own scratch)
        for k in range(ns):
            ley.ley_sort_records_async(addr_in, addr_out[k], n=ne, rec_bytes=REC, key_bytes=kb,
                                       stream=streams[k])
        for st in streams:
            st.synchronize()
        meter = LinkMeter(dev)
        lp0 = meter.measure()  # the link before the steps (and again after them)
        # the input buffer's own read rate: whole regions of a pinned
        # allocation can read several times slower than the meter's buffers
        rd = meter.read_rate(h_in)
        wr = meter.write_rate(h_outs[0])  # overwritten by the steps
        # one blocking call: the latency of a single sort, host to host
        t0 = time.perf_counter()
        ley.ley_sort_records(addr_in, addr_out[0], n=ne, rec_bytes=REC, key_bytes=kb, stream=stream)
        lat = time.perf_counter() - t0
        # The timed steps, queued in turn on the streams: every step copies its
        # input in and its sorted records out, and one step's copy out
        # overlaps the next ones' copies in on the link's two directions.
        barrier(pg, dev)
        t0 = time.perf_counter()
        for k in range(args.e2e_steps):
            ley.ley_sort_records_async(addr_in, addr_out[k % ns], n=ne, rec_bytes=REC,
                                       key_bytes=kb, stream=streams[k % ns])
        for st in streams:
            st.synchronize()
        dt = (time.perf_counter() - t0) / args.e2e_steps
        if ley.ley_last_device_status(stream) != ley.LEY_OK:
            raise RuntimeError("device-side error in the end-to-end steps")
        for a in h_outs[1:min(ns, args.e2e_steps)]:
            if not np.array_equal(h_outs[0], a):
                raise RuntimeError("end-to-end outputs of the streams differ")
        dt = max_over_ranks(dt, pg, dev)
        for a in [h_in] + h_outs:
            host_free(a)
        # The link measured in this process before and after the steps (the
        # better of the two readings): with both directions busy a step cannot
        # take less than n * REC / duplex_each.  Rates on the shared hosts
        # drift between and within processes.
        lp1 = meter.measure()
        meter.close()
        lp = {k: max(lp0[k], lp1[k]) for k in lp0}
        floor_ms = ne * REC / (lp["duplex_each_GBps"] * 1e9) * 1e3
        e2e = {"value": round(world * ne * REC / dt / 1e9, 2), "unit": "GB/s",
               "ms_per_step": round(dt * 1e3, 2), "h2d_bytes_per_step": world * ne * REC,
               "d2h_bytes_per_step": world * ne * REC, "streams": ns, "records": ne,
               "single_call_ms": round(lat * 1e3, 2), "link": lp,
               "link_before": lp0, "link_after": lp1, "input_read": rd,
               "output_write": wr,
               "duplex_floor_ms": round(floor_ms, 2),
               "floor_frac": round(floor_ms / (dt * 1e3), 4),
               # every step copies its input in and its output out: at the
               # rates these buffers themselves gave just before the steps,
               # where those are the lower
               "buffer_floor_frac": round(
                   ne * REC / (min(lp["duplex_each_GBps"], rd["GBps"], wr["GBps"]) * 1e9) / dt,
                   4)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        v, dt = oracle_sample(args.cpu_sample, seed=2 if wl == "uniform" else 3,
                              skew=wl == "skew", device=dev)
        cpu = {"value": round(v, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
               "sample": f"first {args.cpu_sample} records of the workload, "
                         f"single-threaded qsort + record copy, {dt:.1f} s"}
        nt = os.cpu_count() or 1
        nthr = min(n, args.cpu_threads_sample) if args.cpu_threads_sample else n
        vt, dtt = oracle_sample(nthr, seed=2 if wl == "uniform" else 3, skew=wl == "skew",
                                device=dev, threads=nt)
        cpu["threads"] = {
            "value": round(vt, 4), "unit": "GB/s", "cores": nt, "kind": "oracle",
            "sample": (f"{'the whole workload' if nthr == n else f'first {nthr} records'}"
                       f" ({nthr} records), {nt} threads: chunked (key, index) sorts, "
                       f"T-way merge, parallel record copy, {dtt:.1f} s")}

    value = world * n * REC / (ms * 1e-3) / 1e9
    extras = {}
    if wl == "uniform" and kb == KEY and world == 1 and not args.quick:
        extras = run_extras(args, dev, stream, pg, world)
    return {
        "metric": (METRIC if wl == "uniform" and kb == KEY
                   else f"GB/s of 100-byte records sorted ({wl} keys, {kb}-byte key)"),
        "value": round(value, 2), "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic (seeded SplitMix64 records shaped like the paper's gensort data)",
        "config": {"workload": workload, "records": n, "record_bytes": REC, "key_bytes": kb,
                   "resident": "HBM", "l2": "inputs larger than L2 (10 GB), no flush",
                   "parallelism": f"replicas x{world}"},
        "clocks": clocks, "gpu_launches": launches, "step_ms": step_stats, "e2e": e2e,
        "roofline": roofline,
        "cpu_baseline": cpu, "kernels": kernels, **extras,
    }


def run_extras(args, dev, stream, pg, world):
    """The other configurations, measured in the same process after the main
    workload: the skewed 10 GB sort, the batched and served request streams,
    and the host-memory modes.  A configuration that fails is reported with
    its error instead of ending the run."""
    import copy
    import torch
    import paper_1909_08006_gb300 as ley
    out = {}

    def sub(name, fn):
        t0 = time.perf_counter()
        try:
            out[name] = fn()
        except Exception as e:  # noqa: BLE001 - reported in the line
            out[name] = {"error": f"{type(e).__name__}: {e}"}
        out[name]["wall_s"] = round(time.perf_counter() - t0, 1)
        ley.ley_release_cache()
        torch.cuda.empty_cache()

    sub("skew", lambda: run_skew_sub(args, dev, stream, pg))
    a = copy.copy(args)
    a.requests, a.steps, a.warmup = 256, 3, 3
    sub("batch", lambda: _strip(run_batch(a, world, 0, dev, stream, pg)))
    a = copy.copy(args)
    a.requests, a.budget_gb = 10_000, 40.0
    sub("serve", lambda: _strip(run_serve(a, world, 0, dev, stream, pg)))
    sub("host_modes", lambda: host_modes(args, dev, stream, pg, world))
    return out


def _strip(line):
    """A configuration's own bench line as a sub-object of the main line."""
    drop = ("n_gpus", "higher_is_better", "scaling", "vs_baseline", "dtype", "data")
    return {k: v for k, v in line.items() if k not in drop}


# ------------------------------------------------------ other workloads

def _timed(fn, steps, warmup, stream, pg, dev):
    import torch
    for _ in range(warmup):
        fn()
    barrier(pg, dev)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return max_over_ranks(e0.elapsed_time(e1) / steps, pg, dev)


def run_pairs(args, world, rank, dev, stream, pg):
    """Key-pointer pairs (u64 key, u32 index): the sort without record gather."""
    import torch
    import datagen
    import paper_1909_08006_gb300 as ley
    n = args.n
    keys, idx = datagen.uniform_pairs(n, seed=5, device=dev)
    ko, io = torch.empty_like(keys), torch.empty_like(idx)
    torch.cuda.synchronize()
    step = lambda: ley.ley_sort_keys_index(keys, idx, ko, io, stream=stream)  # noqa: E731
    launches0 = ley.ley_launch_count()
    ms = _timed(step, args.steps, args.warmup, stream, pg, dev)
    launches = (ley.ley_launch_count() - launches0) * args.steps // (args.steps + args.warmup)
    if ley.ley_last_device_status(stream) != ley.LEY_OK:
        raise RuntimeError("device-side error")
    return {
        "metric": "pairs sorted per second (u64 key, u32 index)",
        "value": round(world * n / (ms * 1e-3) / 1e9, 4), "unit": "Gpairs/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic", "gpu_launches": launches,
        "config": {"workload": f"pairs_{n}", "pairs": n, "bytes_per_pair": 12},
    }


def _check_records_on_oracle(pairs_of_tensors):
    """Complete oracle check of sorted device outputs against their tagged
    device inputs ([(in, out)], local index at bytes 10..13): -1 each if exact."""
    import oracle
    oracle.build()
    return [oracle.check_tagged_threads(o.cpu().numpy(), x.cpu().numpy())
            for x, o in pairs_of_tensors]


def _check_pairs_on_oracle(quads):
    """Complete oracle check of sorted (key, payload) outputs whose payloads
    are the input positions: -1 each if exact."""
    import numpy as np
    import oracle
    oracle.build()
    return [oracle.check_pairs_tagged(ko.cpu().numpy().view(np.uint64),
                                      vo.cpu().numpy().view(np.uint32),
                                      k.cpu().numpy().view(np.uint64))
            for k, _v, ko, vo in quads]


def run_batch(args, world, rank, dev, stream, pg):
    """Many sort requests of uneven sizes (log-uniform in [lo, hi] records),
    half 100-byte records and half (u64 key, u32 payload) pairs: one batched
    call per kind against one call per request, same stream, same data.
    Every request's output is then checked completely by the oracle."""
    import torch
    import datagen
    import paper_1909_08006_gb300 as ley
    count, lo, hi = args.requests, args.req_min, args.req_max
    sizes = datagen.log_uniform_sizes(count, seed=5, lo=lo, hi=hi)
    rec_reqs, pair_reqs = [], []
    for i, n in enumerate(sizes):
        if i % 2 == 0:
            x = datagen.uniform_records(n, seed=1000 + i, device=dev, tag_index=True)
            rec_reqs.append((x, torch.empty_like(x)))
        else:
            k, v = datagen.uniform_pairs(n, seed=1000 + i, device=dev)
            pair_reqs.append((k, v, torch.empty_like(k), torch.empty_like(v)))
    n_rec = sum(int(r[0].shape[0]) for r in rec_reqs)
    n_pair = sum(int(r[0].shape[0]) for r in pair_reqs)
    total_bytes = n_rec * REC + n_pair * 12
    torch.cuda.synchronize()

    def batched():
        ley.ley_sort_records_batch(rec_reqs, stream=stream)
        ley.ley_sort_keys_index_batch(pair_reqs, stream=stream)

    def one_by_one():
        for x, o in rec_reqs:
            ley.ley_sort_records(x, o, stream=stream)
        for k, v, ko, vo in pair_reqs:
            ley.ley_sort_keys_index(k, v, ko, vo, stream=stream)

    launches0 = ley.ley_launch_count()
    ms_b = _timed(batched, args.steps, args.warmup, stream, pg, dev)
    launches_b = (ley.ley_launch_count() - launches0) // (args.steps + args.warmup)
    if ley.ley_last_device_status(stream) != ley.LEY_OK:
        raise RuntimeError("device-side error")
    outs_b = [o.clone() for _, o in rec_reqs] + [ko.clone() for _, _, ko, _ in pair_reqs]
    bad_r = _check_records_on_oracle(rec_reqs)
    bad_p = _check_pairs_on_oracle(pair_reqs)
    launches0 = ley.ley_launch_count()
    ms_s = _timed(one_by_one, args.steps, args.warmup, stream, pg, dev)
    launches_s = (ley.ley_launch_count() - launches0) // (args.steps + args.warmup)
    if ley.ley_last_device_status(stream) != ley.LEY_OK:
        raise RuntimeError("device-side error")
    outs_s = [o for _, o in rec_reqs] + [ko for _, _, ko, _ in pair_reqs]
    same = all(torch.equal(a, b) for a, b in zip(outs_b, outs_s))
    graph = _graph_replay_timing(batched_calls(rec_reqs, pair_reqs), args, stream, pg, dev)
    small = _small_batch_timing(args, dev, stream, pg)
    return {
        "metric": "GB/s of request data sorted, batched (records + pairs)",
        "value": round(world * total_bytes / (ms_b * 1e-3) / 1e9, 2), "unit": "GB/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms_b, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic", "gpu_launches": launches_b,
        "config": {"workload": f"batch_{count}x[{lo},{hi}]", "requests": count,
                   "records": n_rec, "pairs": n_pair, "bytes": total_bytes,
                   "sizes": "log-uniform, half 100-byte records, half (u64, u32) pairs"},
        "one_launch_per_request": {
            "value": round(world * total_bytes / (ms_s * 1e-3) / 1e9, 2), "unit": "GB/s",
            "ms_per_step": round(ms_s, 3), "gpu_launches": launches_s},
        "speedup_vs_one_launch_per_request": round(ms_s / ms_b, 3),
        "oracle_checked": len(bad_r) + len(bad_p),
        "oracle_exact": all(b == -1 for b in bad_r + bad_p),
        "identical_to_one_launch_per_request": same,
        "cuda_graph_replay": graph, "small_batch": small,
    }


def batched_calls(rec_reqs, pair_reqs):
    import paper_1909_08006_gb300 as ley

    def fn(st):
        if rec_reqs:
            ley.ley_sort_records_batch(rec_reqs, stream=st)
        if pair_reqs:
            ley.ley_sort_keys_index_batch(pair_reqs, stream=st)
    return fn


def _graph_replay_timing(fn, args, stream, pg, dev):
    """The same batched calls launched directly and replayed from a CUDA
    graph captured once: what graph replay would save a batch of this shape."""
    import torch
    fn(stream)  # library state and pool set up outside the capture
    torch.cuda.synchronize()
    cs = torch.cuda.Stream(dev)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=cs):
        fn(cs)
    direct = _timed(lambda: fn(stream), args.steps, args.warmup, stream, pg, dev)
    cur = torch.cuda.current_stream(dev)
    replay = _timed(g.replay, args.steps, args.warmup, cur, pg, dev)
    del g
    return {"direct_ms": round(direct, 4), "graph_replay_ms": round(replay, 4),
            "replay_speedup": round(direct / replay, 3)}


def _small_batch_timing(args, dev, stream, pg):
    """A batch of 8 small requests (1,000..20,000 records, half records, half
    pairs), where launch costs weigh most: direct calls against graph replay."""
    import torch
    import datagen
    sizes = [1000, 20_000, 3000, 8000, 1500, 12_000, 5000, 2500]
    rec_reqs, pair_reqs = [], []
    for i, n in enumerate(sizes):
        if i % 2 == 0:
            x = datagen.uniform_records(n, seed=7000 + i, device=dev)
            rec_reqs.append((x, torch.empty_like(x)))
        else:
            k, v = datagen.uniform_pairs(n, seed=7000 + i, device=dev)
            pair_reqs.append((k, v, torch.empty_like(k), torch.empty_like(v)))
    torch.cuda.synchronize()
    r = _graph_replay_timing(batched_calls(rec_reqs, pair_reqs), args, stream, pg, dev)
    r["requests"] = len(sizes)
    r["records_and_pairs"] = sum(sizes)
    return r


def run_serve(args, world, rank, dev, stream, pg):
    """Served sorting: a stream of requests (sizes log-uniform in [lo, hi],
    half 100-byte records, half (u64, u32) pairs) through the continuous-
    batching server under a device budget.  Saturation (all requests at t0)
    gives the capacity, batched and with one request per launch; Poisson
    arrivals at 0.5x and 0.9x of the batched capacity give p50/p99 latency.
    Inputs are resident in HBM: P distinct inputs per kind drawn from the size
    distribution, each with Q output buffers that requests rotate through.
    After the saturation run the output buffers of the first rotation slot
    (the last request that used each) are checked completely by the oracle."""
    import threading
    import numpy as np
    import torch
    import datagen
    import paper_1909_08006_gb300 as ley
    count, lo, hi = args.requests, args.req_min, args.req_max
    P, Q = args.serve_inputs, 2
    budget = int(args.budget_gb * 1e9)
    sizes = datagen.log_uniform_sizes(2 * P, seed=11, lo=lo, hi=hi)
    ins, outs, nbytes = [[], []], [[], []], [[], []]
    for b in range(P):
        n = sizes[2 * b]
        x = datagen.uniform_records(n, seed=3000 + b, device=dev, tag_index=True)
        ins[0].append(x)
        outs[0].append([torch.empty_like(x) for _ in range(Q)])
        nbytes[0].append(n * REC)
        n = sizes[2 * b + 1]
        k, v = datagen.uniform_pairs(n, seed=4000 + b, device=dev)
        ins[1].append((k, v))
        outs[1].append([(torch.empty_like(k), torch.empty_like(v)) for _ in range(Q)])
        nbytes[1].append(n * 12)
    torch.cuda.synchronize()

    def plan(i):  # kind, input, output slot of request i
        kind = i % 2
        b = (i // 2) % P
        return kind, b, (i // (2 * P)) % Q

    def serve(max_batch, arrivals, latency=True):
        srv = ley.ley_server_create(budget, max_batch=max_batch, slots=args.serve_slots)
        free = {}
        lat, done_t = [None] * count, [0.0] * count
        tickets = [None] * count
        ready = [threading.Event() for _ in range(count)]
        base = time.perf_counter()

        def waiter():
            for i in range(count):
                ready[i].wait()
                tm = ley.ley_server_wait(srv, tickets[i][0])
                late = tickets[i][1]  # submission lateness against the scheduled arrival
                lat[i] = tm["done_s"] - tm["submit_s"] + late
                done_t[i] = tm["done_s"]
                free[plan(i)].set()

        w = threading.Thread(target=waiter)
        w.start()
        for i in range(count):
            kind, b, q = plan(i)
            ev = free.get((kind, b, q))
            if ev is not None:
                ev.wait()  # the output slot's previous request is done
            free[(kind, b, q)] = threading.Event()
            target = base + arrivals[i]
            now = time.perf_counter()
            if target > now:
                time.sleep(target - now)
            late = max(0.0, time.perf_counter() - target)
            if kind == 0:
                t = ley.ley_server_submit_records(srv, ins[0][b], outs[0][b][q])
            else:
                (k, v), (ko, vo) = ins[1][b], outs[1][b][q]
                t = ley.ley_server_submit_pairs(srv, k, v, ko, vo)
            tickets[i] = (t, late)
            ready[i].set()
        w.join()
        st = ley.ley_server_stats(srv)
        ley.ley_server_destroy(srv)
        total = sum(nbytes[plan(i)[0]][plan(i)[1]] for i in range(count))
        arr = np.array(lat)
        makespan = max(done_t)  # seconds since the server's creation (just before base)
        r = {"GBps": round(total / makespan / 1e9, 2), "makespan_s": round(makespan, 4),
             "req_per_s": round(count / makespan, 1), "batches": st["launched_batches"],
             "bytes": total}
        if latency:
            r["p50_ms"] = round(float(np.percentile(arr, 50)) * 1e3, 3)
            r["p99_ms"] = round(float(np.percentile(arr, 99)) * 1e3, 3)
        return r

    zero = [0.0] * count
    sat = serve(args.serve_batch, zero, latency=False)
    # the last request that used each first-slot output buffer, against the oracle
    used = {plan(i)[:2] for i in range(count) if plan(i)[2] == 0}
    bad_r = _check_records_on_oracle([(ins[0][b], outs[0][b][0]) for kd, b in used if kd == 0])
    bad_p = _check_pairs_on_oracle([(ins[1][b][0], ins[1][b][1], outs[1][b][0][0],
                                     outs[1][b][0][1]) for kd, b in used if kd == 1])
    single = serve(1, zero, latency=False)
    rng = np.random.default_rng(12)
    res = {}
    for frac in (0.5, 0.9):
        rate = frac * sat["req_per_s"]
        arrivals = np.cumsum(rng.exponential(1.0 / rate, count)).tolist()
        res[f"poisson_{frac}"] = serve(args.serve_batch, arrivals)
        res[f"poisson_{frac}"]["rate_req_per_s"] = round(rate, 1)
    return {
        "metric": "GB/s of request data sorted by the batching server (saturation); p50/p99",
        "value": sat["GBps"], "unit": "GB/s", "n_gpus": world, "steps": 1, "warmup": 0,
        "ms_per_step": round(sat["makespan_s"] * 1e3, 2), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": f"serve_{count}x[{lo},{hi}]", "requests": count,
                   "budget_bytes": budget, "max_batch": args.serve_batch,
                   "slots": args.serve_slots, "distinct_inputs_per_kind": P,
                   "output_buffers_per_input": Q},
        "saturation": sat, "one_launch_per_request": single,
        "speedup_vs_one_launch_per_request": round(single["makespan_s"] / sat["makespan_s"], 3),
        "oracle_checked": len(bad_r) + len(bad_p),
        "oracle_exact": all(b == -1 for b in bad_r + bad_p),
        **res,
    }


def run_skew_sub(args, dev, stream, pg):
    """The skewed 10 GB internal sort (1e8 records): device time per sort over
    the timed steps, the per-kernel split, and a complete oracle check of the
    output (tagged input)."""
    import torch
    import datagen
    import paper_1909_08006_gb300 as ley
    n = args.n
    d_in = datagen.skew_records(n, seed=3, device=dev, tag_index=True)
    d_out = torch.empty_like(d_in)
    torch.cuda.synchronize()
    step = lambda: ley.ley_sort_records(d_in, d_out, n=n, rec_bytes=REC, key_bytes=KEY,  # noqa: E731
                                        stream=stream)
    ms = _timed(step, args.sub_steps, 3, stream, pg, dev)
    if ley.ley_last_device_status(stream) != ley.LEY_OK:
        raise RuntimeError("device-side error in the skewed sorts")
    ley.ley_profile_enable(True)
    for _ in range(3):
        step()
    torch.cuda.synchronize()
    prof = ley.ley_profile_read()
    ley.ley_profile_enable(False)
    peak, _ = load_peaks()
    import oracle
    oracle.build()
    bad = oracle.check_tagged_threads(d_out.cpu().numpy(), d_in.cpu().numpy())
    return {"workload": f"skew_{n}", "records": n, "ms_per_step": round(ms, 3),
            "steps": args.sub_steps, "warmup": 3,
            "GBps": round(n * REC / (ms * 1e-3) / 1e9, 2),
            "path_frac_306B": round(PATH_BYTES * n / (ms * 1e-3) / 1e9 / peak, 4),
            "frac_314B_model": round(314 * n / (ms * 1e-3) / 1e9 / peak, 4),
            "kernels": {k: {"launches_per_sort": c // 3, "ms_per_sort": round(t / 3, 4)}
                        for k, (c, t) in prof.items()},
            "parity": {"exact": bad == -1, "how": "oracle check_tagged over every record"}}


def _libcuda():
    import ctypes
    cu = ctypes.CDLL("libcuda.so.1")
    cu.cuMemHostAlloc.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_size_t, ctypes.c_uint]
    cu.cuMemFreeHost.argtypes = [ctypes.c_void_p]
    return cu


_HOST_BUFS = {}


def host_alloc(nbytes):
    """Exact-size page-locked host buffer from cuMemHostAlloc, as a numpy
    array (torch's pinned pool rounds up to 2^k bytes).  Memory registered with
    cudaHostRegister instead was measured to copy at only ~122 GB/s each way
    in full duplex on GB300, against ~172 GB/s for cuMemHostAlloc memory."""
    import ctypes
    import numpy as np
    import torch
    torch.cuda.init()
    cu = _libcuda()
    p = ctypes.c_void_p()
    rc = cu.cuMemHostAlloc(ctypes.byref(p), nbytes, 0)
    if rc != 0:
        raise RuntimeError(f"cuMemHostAlloc({nbytes}) failed ({rc})")
    a = np.ctypeslib.as_array((ctypes.c_uint8 * nbytes).from_address(p.value))
    _HOST_BUFS[a.ctypes.data] = p
    return a


def host_free(a):
    p = _HOST_BUFS.pop(a.ctypes.data)
    _libcuda().cuMemFreeHost(p)


def e2e_plan(n, want_streams):
    """(streams, records) for the end-to-end steps of this rank: the pinned
    input plus one output per stream must fit in this rank's share of 60 % of
    the host's available memory (every rank on the host pins its own).  Fewer
    streams first, then fewer records."""
    avail = None
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    avail = int(line.split()[1]) * 1024
    except OSError:
        pass
    local = int(os.environ.get("LOCAL_WORLD_SIZE", "1"))
    if avail is None:
        return max(1, want_streams), n
    share = 0.6 * avail / max(1, local) - 2 * (2 << 30)  # minus the link test's buffers
    for ns in range(max(1, want_streams), 0, -1):
        if (1 + ns) * n * REC <= share:
            return ns, n
    ne = int(share // (2 * REC)) // 4096 * 4096
    return 1, max(4096, min(n, ne))


class LinkMeter:
    """Host<->device copy rates of this machine, measured on demand with the same
    kind of host memory as the sort's buffers (cuMemHostAlloc): H2D alone,
    D2H alone, and both directions at once (GB/s each way).  The buffers are
    allocated once, so a reading can be taken right before every timed call:
    the shared hosts' link rates drift between and within processes."""

    def __init__(self, dev, nbytes=2 << 30):
        import ctypes
        import torch
        self.cu = _libcuda()
        self.cu.cuMemcpyHtoDAsync_v2.argtypes = [ctypes.c_uint64, ctypes.c_void_p,
                                                 ctypes.c_size_t, ctypes.c_void_p]
        self.cu.cuMemcpyDtoHAsync_v2.argtypes = [ctypes.c_void_p, ctypes.c_uint64,
                                                 ctypes.c_size_t, ctypes.c_void_p]
        self.dev, self.nbytes = dev, nbytes
        self.h1, self.h2 = host_alloc(nbytes), host_alloc(nbytes)
        self.d1 = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        self.d2 = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        self.s1, self.s2 = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

    def measure(self, reps=3):
        import torch
        cu, nb = self.cu, self.nbytes

        def h2d():
            assert cu.cuMemcpyHtoDAsync_v2(self.d1.data_ptr(), self.h1.ctypes.data, nb,
                                           self.s1.cuda_stream) == 0

        def d2h():
            assert cu.cuMemcpyDtoHAsync_v2(self.h2.ctypes.data, self.d2.data_ptr(), nb,
                                           self.s2.cuda_stream) == 0

        def timed(fn):
            fn()
            torch.cuda.synchronize(self.dev)
            t0 = time.perf_counter()
            for _ in range(reps):
                fn()
            torch.cuda.synchronize(self.dev)
            return (time.perf_counter() - t0) / reps

        r = {"h2d_GBps": nb / timed(h2d) / 1e9, "d2h_GBps": nb / timed(d2h) / 1e9,
             "duplex_each_GBps": nb / timed(lambda: (h2d(), d2h())) / 1e9}
        return {k: round(v, 1) for k, v in r.items()}

    def read_rate(self, host, slice_bytes=1 << 30):
        """Host->device rate of one given pinned buffer (the sort's own input),
        read once in `slice_bytes` slices: overall GB/s and the slowest slice.
        On the shared boxes whole regions of an allocation can read several
        times slower than the meter's own buffers for seconds at a time."""
        return self._buffer_rate(host, slice_bytes, True)

    def write_rate(self, host, slice_bytes=1 << 30):
        """Device->host rate into one given pinned buffer (the sort's own
        output, overwritten), in `slice_bytes` slices, as read_rate."""
        return self._buffer_rate(host, slice_bytes, False)

    def _buffer_rate(self, host, slice_bytes, to_device):
        import torch
        cu, nb = self.cu, host.nbytes
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        worst, total_ms = None, 0.0
        for o in range(0, nb, slice_bytes):
            m = min(slice_bytes, nb - o)
            ev[0].record(self.s1)
            if to_device:
                assert cu.cuMemcpyHtoDAsync_v2(self.d1.data_ptr(), host.ctypes.data + o, m,
                                               self.s1.cuda_stream) == 0
            else:
                assert cu.cuMemcpyDtoHAsync_v2(host.ctypes.data + o, self.d2.data_ptr(), m,
                                               self.s1.cuda_stream) == 0
            ev[1].record(self.s1)
            ev[1].synchronize()
            ms = ev[0].elapsed_time(ev[1])
            total_ms += ms
            g = m / (ms * 1e-3) / 1e9
            worst = g if worst is None else min(worst, g)
        return {"GBps": round(nb / (total_ms * 1e-3) / 1e9, 1), "slowest_slice_GBps": round(worst, 1),
                "slice_bytes": slice_bytes}

    def close(self):
        host_free(self.h1)
        host_free(self.h2)
        del self.d1, self.d2


def host_avail_bytes():
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except OSError:
        pass
    return None


def host_mode_run(args, dev, stream, pg, world, mode, n, budget, calls, warm, meter=None,
                  check=True):
    """One host-memory configuration: n tagged uniform 100-byte records in
    pinned host memory, sorted host to host under the device budget (the
    partially in-memory sort or the external sort, whichever the library
    picks for that budget), timed over `calls` calls after `warm` warm-ups,
    each call preceded by a reading of the link.  The output of the last call
    is then checked completely by the oracle (permutation by tags, bytes, and
    strict (key, index) order) and at sampled ranks from the definition."""
    import numpy as np
    import torch
    import datagen
    import paper_1909_08006_gb300 as ley
    own_meter = meter is None
    if own_meter:
        meter = LinkMeter(dev)
    h_in_np, h_out_np = host_alloc(n * REC), host_alloc(n * REC)
    try:
        h_in = torch.from_numpy(h_in_np).view(n, REC)
        h_out = torch.from_numpy(h_out_np).view(n, REC)
        chunk = 50_000_000
        for c0 in range(0, n, chunk):
            c1 = min(n, c0 + chunk)
            h_in[c0:c1].copy_(datagen.uniform_records(c1 - c0, seed=2, device=dev, start=c0,
                                                      tag_index=True).cpu())
        torch.cuda.synchronize()
        ws = ley.ley_workspace_bytes(n, mem_budget=budget)
        picked = "partial" if ws >= n * REC else "external"
        for _ in range(warm):
            ley.ley_sort_records(h_in, h_out, n=n, rec_bytes=REC, key_bytes=KEY,
                                 mem_budget=budget, stream=stream)
        times, links, reads, writes = [], [], [], []
        h_in_flat, h_out_flat = h_in_np.reshape(-1), h_out_np.reshape(-1)
        for _ in range(calls):
            links.append(meter.measure())
            reads.append(meter.read_rate(h_in_flat))
            writes.append(meter.write_rate(h_out_flat))  # the call overwrites it
            barrier(pg, dev)
            t0 = time.perf_counter()
            ley.ley_sort_records(h_in, h_out, n=n, rec_bytes=REC, key_bytes=KEY,
                                 mem_budget=budget, stream=stream)
            times.append(max_over_ranks(time.perf_counter() - t0, pg, dev))
        link_after = meter.measure()
        if ley.ley_last_device_status(stream) != ley.LEY_OK:
            raise RuntimeError("device-side error in the host-mode sorts")
        parity = None
        if check:
            import oracle
            oracle.build()
            t0 = time.perf_counter()
            bad = oracle.check_tagged_threads(h_out_np.reshape(n, REC), h_in_np.reshape(n, REC))
            samples = np.linspace(0, n - 1, 4).astype(np.uint64)
            ranks = oracle.rank_records(h_in_np.reshape(n, REC), samples)
            out2 = h_out_np.reshape(n, REC)
            in2 = h_in_np.reshape(n, REC)
            ranks_ok = all(np.array_equal(out2[int(r)], in2[int(s_)])
                           for r, s_ in zip(ranks, samples))
            parity = {"exact": bool(bad == -1 and ranks_ok), "complete_check_first_bad": bad,
                      "sampled_ranks": int(len(samples)), "sampled_ranks_ok": bool(ranks_ok),
                      "check_s": round(time.perf_counter() - t0, 1),
                      "how": "oracle check_tagged over every output record (tags at bytes "
                             "10..13: permutation, bytes equal the input, strict (key, index) "
                             "order) + oracle rank_records at 4 sampled inputs"}
    finally:
        host_free(h_in_np)
        host_free(h_out_np)
        if own_meter:
            meter.close()
    link_b = 2 * n * REC if picked == "partial" else 4 * n * REC
    per_call = []
    for dt, lk, rd, wr in zip(times, links, reads, writes):
        # partial: the copy out waits for the finished order, so the floor is
        # the serial n*100/h2d + n*100/d2h; external: runs in and out, then
        # partitions in and out (2 n*100 bytes each way) with both directions
        # overlapped, so the floor is 2 n*100 / duplex rate each way
        serial = n * REC / (lk["h2d_GBps"] * 1e9) + n * REC / (lk["d2h_GBps"] * 1e9)
        if picked == "external":
            serial *= 2
        duplex = 2 * n * REC / (lk["duplex_each_GBps"] * 1e9)
        floor = serial if picked == "partial" else duplex
        # Either mode writes no output before it has read all of its input
        # (the sorted order needs every key; the merge needs every run): the
        # input read at the rate its own buffer gave just before the call,
        # then the output written at the rate its own buffer took, estimates
        # the floor on these buffers whatever the link meter's buffers read.
        # An estimate only: a buffer's rate drifts during the call, so the
        # fraction can come out above 1.
        in_rate = min(lk["h2d_GBps"], rd["GBps"])
        out_rate = min(lk["d2h_GBps"], wr["GBps"])
        floor_buf = n * REC / (in_rate * 1e9) + n * REC / (out_rate * 1e9)
        per_call.append({"s": round(dt, 4), "floor_s": round(floor, 4),
                         "frac": round(floor / dt, 4),
                         "frac_serial_floor": round(serial / dt, 4),
                         "buffer_floor_s": round(floor_buf, 4),
                         "frac_buffer_floor": round(floor_buf / dt, 4), "link": lk,
                         "input_read": rd, "output_write": wr})
    med = statistics.median(times)
    fr = [c["frac"] for c in per_call]
    fi = [c["frac_buffer_floor"] for c in per_call]
    return {
        "mode": picked, "records": n, "bytes": n * REC, "budget_bytes": budget,
        "device_bytes": ws, "calls": calls, "warmup": warm,
        "median_s": round(med, 4), "min_s": round(min(times), 4), "max_s": round(max(times), 4),
        "GBps": round(world * n * REC / med / 1e9, 2),
        "link_GBps": round(link_b / med / 1e9, 2),
        "frac_median": round(statistics.median(fr), 4), "frac_min": min(fr), "frac_max": max(fr),
        "frac_buffer_floor_median": round(statistics.median(fi), 4),
        "floor": ("serial: n*100/h2d + n*100/d2h" if picked == "partial"
                  else "duplex: 2*n*100 / (rate each way with both directions busy)"),
        "per_call": per_call, "link_after": link_after, "parity": parity,
    }


def run_host_mode(args, world, rank, dev, stream, pg):
    """Records in pinned host memory, sorted to pinned host memory under a
    device budget: the partially in-memory sort (input resident on the device)
    or the external sort (runs + k-way merge)."""
    n, budget = args.n, int(args.budget_gb * 1e9)
    r = host_mode_run(args, dev, stream, pg, world, args.workload, n, budget,
                      calls=max(1, args.steps), warm=max(1, min(args.warmup, 1)),
                      check=not args.no_check)
    roof = {"bound": "link", "achieved": r["link_GBps"], "frac": r["frac_median"],
            "unit": "GB/s", "peak_source": "measured in this run before each call (" +
            r["floor"] + ")"}
    return {
        "metric": f"GB/s of 100-byte records sorted host-to-host ({r['mode']}, device budget)",
        "value": r["GBps"], "unit": "GB/s", "n_gpus": world,
        "steps": r["calls"], "warmup": r["warmup"], "ms_per_step": round(r["median_s"] * 1e3, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic", "config": {"workload": f"{args.workload}_{n}", "records": n,
                                        "budget_bytes": budget, "mode": r["mode"]},
        "roofline": roof, "host_mode": r,
    }


def host_modes(args, dev, stream, pg, world):
    """The 20 GB partially in-memory sort and the external sort, each at the
    largest size host memory allows up to its configuration (2e8 and 4e8
    records), under the 30 GB device budget."""
    import torch
    import paper_1909_08006_gb300 as ley
    budget = int(30e9)
    out = {}
    meter = LinkMeter(dev)
    try:
        for mode, want, per_rec in (("partial", 200_000_000, 2 * REC),
                                    ("external", 400_000_000, 3 * REC)):
            avail = host_avail_bytes()
            n = want
            if avail is not None:  # input, output (and the run scratch) pinned on the host
                share = 0.7 * avail / int(os.environ.get("LOCAL_WORLD_SIZE", "1")) - (8 << 30)
                n = max(4096, min(want, int(share // per_rec) // 4096 * 4096))
            try:
                out[mode] = host_mode_run(args, dev, stream, pg, world, mode, n, budget,
                                          calls=args.host_calls, warm=1, meter=meter)
                if n < want:
                    out[mode]["note"] = (f"{n} of {want} records: host memory "
                                         f"({avail} bytes available) limits the pinned buffers")
            except Exception as e:  # noqa: BLE001 - reported in the line
                out[mode] = {"error": f"{type(e).__name__}: {e}"}
            ley.ley_release_cache()
            torch.cuda.empty_cache()
    finally:
        meter.close()
    return out


# ------------------------------------------------------- reference arm

def run_reference(args, world, rank, pg):
    """The oracle, as it stands, on the host cores: each step sorts a bounded
    sample of the same workload on every core (the paper's system is CPU code
    with no GPU path; the oracle is this project's CPU statement of the same
    sort, here in its multi-core form: chunked (key, index) sorts, a T-way
    merge and a parallel record copy)."""
    if rank != 0:
        return None
    import datagen
    import oracle
    oracle.build()
    threads = os.cpu_count() or 1
    recs = datagen.uniform_records(args.ref_sample, seed=2).numpy()
    for _ in range(args.warmup):
        oracle.sort_records_threads(recs, key_bytes=KEY, threads=threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.sort_records_threads(recs, key_bytes=KEY, threads=threads)
    dt = (time.perf_counter() - t0) / args.steps
    v = args.ref_sample * REC / dt / 1e9
    sample = (f"first {args.ref_sample} records of the workload per step, {threads} threads: "
              "chunked qsort on (key, index), T-way merge, parallel record copy")
    return {
        "impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "GB/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt * 1e3, 2), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": f"uniform_{args.n}", "records": args.n, "record_bytes": REC,
                   "key_bytes": KEY},
        "cpu_baseline": {"value": round(v, 4), "unit": "GB/s", "cores": threads,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(v, 4), "unit": "GB/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=100_000_000)
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--e2e-streams", type=int, default=2,
                    help="streams the end-to-end steps are queued on in turn")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=20_000_000)
    ap.add_argument("--workload", default="uniform",
                    choices=["uniform", "skew", "ascii", "pairs", "partial", "external", "batch",
                             "serve"])
    ap.add_argument("--key-bytes", type=int, default=KEY,
                    help="key length of the uniform/skew/ascii workloads (longer than 12: "
                         "one sort per 12-byte window)")
    ap.add_argument("--autotune", action="store_true",
                    help="run the library's autotuner on the workload's size first")
    ap.add_argument("--serve-batch", type=int, default=256)
    ap.add_argument("--serve-slots", type=int, default=3)
    ap.add_argument("--serve-inputs", type=int, default=256)
    ap.add_argument("--requests", type=int, default=None)
    ap.add_argument("--req-min", type=int, default=1000)
    ap.add_argument("--req-max", type=int, default=10_000_000)
    ap.add_argument("--budget-gb", type=float, default=30.0)
    ap.add_argument("--ref-sample", type=int, default=10_000_000,
                    help="records per step of the reference arm (the oracle on every core)")
    ap.add_argument("--cpu-threads-sample", type=int, default=0,
                    help="records of the multi-core oracle baseline (0 = the whole workload)")
    ap.add_argument("--host-calls", type=int, default=3,
                    help="timed calls per host-memory mode in the default line")
    ap.add_argument("--sub-steps", type=int, default=10,
                    help="timed steps of the skewed sort in the default line")
    ap.add_argument("--quick", action="store_true",
                    help="the main workload only (no skew, batch, serve or host-mode entries)")
    ap.add_argument("--no-check", action="store_true",
                    help="skip the oracle check of a --workload partial/external run")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.workload == "external" and args.n == 100_000_000:
        args.n = 400_000_000
    if args.workload == "partial" and args.n == 100_000_000:
        args.n = 200_000_000
    if args.workload == "serve" and args.budget_gb == 30.0:
        args.budget_gb = 40.0
    if args.requests is None:
        args.requests = 10_000 if args.workload == "serve" else 256
    world, rank, local, pg = dist_setup(args)
    if args.impl == "reference":
        out = run_reference(args, world, rank, pg)
    else:
        out = run_ours(args, world, rank, local, pg)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
