"""The external merge's partition planning (Section 3.2: the K-way merge is
cut into independent partitions), host-only and so checked on the CPU.

The planner's cuts are checked against the definition of the merge order
(key, run, position), written out here with numpy's stable lexicographic
sort over the concatenated runs: the first r_p records of the merged order
are exactly the records before cut p in every run.  Runs are sorted by the
oracle, as the external sort's runs are.
"""
import numpy as np
import pytest

import datagen


@pytest.fixture(scope="module")
def ley():
    from paper_1909_08006_gb300 import build
    build.build()
    import paper_1909_08006_gb300 as m
    return m


def make_runs(orc, k, lens, seed, alphabet=None, key_bytes=10):
    runs = []
    for i in range(k):
        rec = datagen.uniform_records(lens[i], seed=seed + i).numpy()
        if alphabet is not None and lens[i]:  # few distinct keys: ties across runs
            rec[:, :key_bytes] = np.frombuffer(alphabet, dtype=np.uint8)[
                rec[:, :key_bytes] % len(alphabet)]
        runs.append(orc.sort_records(rec, key_bytes=key_bytes) if lens[i] else rec)
    return runs


def merged_order(runs, key_bytes):
    """(run, position) of every record in the merged order: lexicographic on
    the key bytes, then the run, then the position."""
    keys = np.concatenate([r[:, :key_bytes] for r in runs if len(r)], axis=0)
    run_id = np.concatenate([np.full(len(r), i) for i, r in enumerate(runs)])
    pos = np.concatenate([np.arange(len(r)) for r in runs])
    cols = [pos, run_id] + [keys[:, b] for b in range(key_bytes - 1, -1, -1)]
    o = np.lexsort(cols)
    return run_id[o], pos[o]


@pytest.mark.parametrize("k,lens,cap,alphabet", [
    (1, [5000], 700, None),
    (3, [2000, 0, 3500], 900, None),
    (4, [3000, 3000, 3000, 3000], 1000, b"AB"),      # heavy ties across runs
    (7, [1, 800, 1200, 0, 999, 4096, 333], 500, b"xyz"),
    (16, [700] * 16, 2048, None),
])
def test_cuts_split_the_merged_order_exactly(orc, ley, k, lens, cap, alphabet):
    runs = make_runs(orc, k, lens, seed=70 + k, alphabet=alphabet)
    cuts = ley.ley_plan_partitions(runs, key_bytes=10, cap=cap).astype(np.int64)
    n = sum(lens)
    assert (cuts[0] == 0).all() and (cuts[-1] == np.array(lens)).all()
    assert (np.diff(cuts, axis=0) >= 0).all()
    sizes = np.diff(cuts, axis=0).sum(axis=1)
    assert sizes.sum() == n and (sizes <= cap).all()
    run_id, _ = merged_order(runs, 10)
    r = 0
    for p in range(1, len(cuts)):
        r = int(cuts[p].sum())
        # the first r records of the merged order hold exactly cuts[p][i] from run i
        got = np.bincount(run_id[:r], minlength=k)
        assert (got == cuts[p]).all(), (p, got, cuts[p])


def test_partition_count_is_reported_when_rows_run_short(orc, ley):
    import ctypes
    runs = make_runs(orc, 2, [3000, 3000], seed=90)
    ptrs = (ctypes.c_void_p * 2)(*[r.ctypes.data for r in runs])
    lens = (ctypes.c_uint64 * 2)(3000, 3000)
    cuts = (ctypes.c_uint64 * 4)()
    need = ctypes.c_uint64(0)
    st = ley._lib.ley_plan_partitions(ptrs, lens, 2, 100, 10, 500, cuts, 2, ctypes.byref(need))
    assert st == ley.LEY_ENOMEM and need.value > 2
