"""Pins of the CPU oracle against things other than itself.

Each oracle function is checked against brute force, a library routine, the
worked example of Section 2.2, closed-form special cases, or planted mistakes,
chosen so that a dropped term, a swapped operand or a wrong tie order fails.
"""
import itertools
import os

import numpy as np
import pytest

import datagen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def lex_perm(rec: np.ndarray, key_bytes: int) -> np.ndarray:
    """numpy's stable lexsort: primary key byte 0, ..., ties by index."""
    n = rec.shape[0]
    cols = [np.arange(n)] + [rec[:, b] for b in range(key_bytes - 1, -1, -1)]
    return np.lexsort(cols)


def rand_records(n, rec=16, key=10, seed=1, alphabet=None):
    a = datagen.uniform_records(n, seed, rec).numpy().copy()
    if alphabet is not None:
        a[:, :key] = np.frombuffer(bytes(alphabet), dtype=np.uint8)[a[:, :key] % len(alphabet)]
    return a


# ------------------------------------------------------------- generator

def test_splitmix64_published_first_output():
    # SplitMix64 seeded with 0: first output 0xE220A8397B1DCDAF (Steele et al.)
    assert datagen.splitmix64_reference(0, 1)[0] == 0xE220A8397B1DCDAF
    w = datagen.stream_words(0, 0, 6).numpy().view(np.uint64)
    assert [int(x) for x in w] == datagen.splitmix64_reference(0, 6)


# ----------------------------------------------------- worked example

def _golden_example():
    recs, buckets = None, None
    with open(os.path.join(GOLDEN, "s2_2_first_round_buckets.txt")) as f:
        for line in f:
            if line.startswith("records:"):
                recs = line.split()[1:]
            elif line.startswith("buckets:"):
                buckets = {kv.split("=")[0]: int(kv.split("=")[1]) for kv in line.split()[1:]}
    return recs, buckets


def test_worked_example_first_round(orc):
    recs, buckets = _golden_example()
    a = np.array([list(r.encode()) for r in recs], dtype=np.uint8)
    h = orc.digit_histogram(a, 0)
    assert {chr(b): int(h[b]) for b in range(256) if h[b]} == buckets
    order = orc.msd_partition(a, 0)
    # buckets a, b, c, d in byte order; inside c the input order cde, cfe
    assert [recs[i] for i in order] == ["abc", "bcd", "cde", "cfe", "dfg"]
    out = orc.sort_records(a, key_bytes=3)
    assert [bytes(r).decode() for r in out] == sorted(recs)


# -------------------------------------------------------- brute force

@pytest.mark.parametrize("n", [0, 1, 2, 3, 4, 5, 6, 7])
def test_brute_force_unique_permutation(orc, n):
    for seed in range(3):
        a = rand_records(n, rec=8, key=3, seed=seed + 10 * n, alphabet=b"AB")
        keys = [bytes(a[i, :3]) for i in range(n)]
        winners = [p for p in itertools.permutations(range(n))
                   if all((keys[p[j]], p[j]) < (keys[p[j + 1]], p[j + 1]) for j in range(n - 1))]
        assert len(winners) == 1
        out, perm = orc.sort_records(a, key_bytes=3, return_perm=True)
        assert list(perm) == list(winners[0])
        assert np.array_equal(out, a[list(winners[0])])


@pytest.mark.parametrize("n", [0, 1, 2, 3, 5, 6])
def test_brute_force_pairs(orc, n):
    keys, idx = datagen.narrow_pairs(n, seed=n + 3, distinct=2)
    k = keys.numpy().view(np.uint64)
    v = (idx.numpy().view(np.uint32) * 7 + 3).astype(np.uint32)
    winners = [p for p in itertools.permutations(range(n))
               if all((int(k[p[j]]), p[j]) < (int(k[p[j + 1]]), p[j + 1]) for j in range(n - 1))]
    assert len(winners) == 1
    ko, vo = orc.sort_keys_index(k, v)
    assert list(ko) == [k[i] for i in winners[0]]
    assert list(vo) == [v[i] for i in winners[0]]


# ------------------------------------------------ library cross-checks

@pytest.mark.parametrize("n,key,alpha", [(1000, 10, None), (3000, 10, b"AB"), (2500, 4, b"xyz"),
                                         (777, 1, None), (4096, 12, b"\x00\xff")])
def test_matches_numpy_lexsort(orc, n, key, alpha):
    a = rand_records(n, rec=max(16, key + 4), key=key, seed=n, alphabet=alpha)
    out, perm = orc.sort_records(a, key_bytes=key, return_perm=True)
    ref = lex_perm(a, key)
    assert np.array_equal(perm, ref)
    assert np.array_equal(out, a[ref])


def test_pairs_match_numpy_stable_argsort(orc):
    for n, distinct in [(5000, 0), (5000, 7), (1, 1)]:
        if distinct:
            keys, idx = datagen.narrow_pairs(n, seed=5, distinct=distinct)
        else:
            keys, idx = datagen.uniform_pairs(n, seed=5)
        k = keys.numpy().view(np.uint64)
        v = idx.numpy().view(np.uint32)
        ref = np.argsort(k, kind="stable")
        ko, vo = orc.sort_keys_index(k, v)
        assert np.array_equal(ko, k[ref]) and np.array_equal(vo, v[ref])


def test_histogram_and_partition_match_numpy(orc):
    a = rand_records(5000, rec=100, seed=3, alphabet=b"abcde")
    for d in (0, 4, 9):
        h = orc.digit_histogram(a, d)
        assert np.array_equal(h, np.bincount(a[:, d], minlength=256).astype(np.uint64))
        assert np.array_equal(orc.msd_partition(a, d), np.argsort(a[:, d], kind="stable"))


def test_kway_merge_equals_stable_sort_of_concatenation(orc):
    for k, alpha in [(1, None), (3, b"AB"), (8, None), (5, b"abc")]:
        runs, starts = [], [0]
        for r in range(k):
            m = 50 + 37 * r
            a = rand_records(m, rec=24, key=10, seed=100 + r, alphabet=alpha)
            runs.append(a[lex_perm(a, 10)])
            starts.append(starts[-1] + m)
        cat = np.concatenate(runs)
        merged = orc.kway_merge_records(cat, starts, key_bytes=10)
        # runs are contiguous ranges of the concatenation, so "ties to the
        # lower run, then the lower position" is the concatenation's index order
        assert np.array_equal(merged, cat[lex_perm(cat, 10)])


def test_rank_matches_sorted_positions(orc):
    a = rand_records(3000, rec=16, seed=9, alphabet=b"ABC")
    pos = np.empty(3000, dtype=np.int64)
    pos[lex_perm(a, 10)] = np.arange(3000)
    s = np.array([0, 1, 17, 1500, 2999], dtype=np.uint64)
    assert np.array_equal(orc.rank_records(a, s), pos[s.astype(np.int64)].astype(np.uint64))
    keys, _ = datagen.narrow_pairs(3000, seed=4, distinct=11)
    k = keys.numpy().view(np.uint64)
    pp = np.empty(3000, dtype=np.int64)
    pp[np.argsort(k, kind="stable")] = np.arange(3000)
    assert np.array_equal(orc.rank_pairs(k, s), pp[s.astype(np.int64)].astype(np.uint64))


# ----------------------------------------------------- special cases

def test_special_cases(orc):
    n = 2000
    for kind, expect in [("equal", np.arange(n)), ("sorted", np.arange(n)),
                         ("reversed", np.arange(n)[::-1])]:
        a = datagen.edge_records(kind, n, seed=2).numpy()
        _, perm = orc.sort_records(a, return_perm=True)
        assert np.array_equal(perm, expect.astype(np.uint64)), kind
    a = datagen.edge_records("last_byte", n, seed=2).numpy()
    _, perm = orc.sort_records(a, return_perm=True)
    assert np.array_equal(perm, np.argsort(a[:, 9], kind="stable").astype(np.uint64))
    # the value never changes the order
    b = a.copy()
    b[:, 10:] = 255 - b[:, 10:]
    assert np.array_equal(orc.sort_records(b, return_perm=True)[1], perm)


# ---------------------------------------------- checkers catch mistakes

def test_checkers_catch_planted_mistakes(orc):
    a = datagen.skew_records(4000, seed=3, tag_index=True).numpy()
    out = orc.sort_records(a)
    assert orc.check_sorted(out) == -1
    assert orc.record_hash_sum(out) == orc.record_hash_sum(a)
    assert orc.check_tagged(out, a) == -1
    # swap two records with different keys
    bad = out.copy()
    bad[[10, 3000]] = bad[[3000, 10]]
    assert orc.check_sorted(bad) >= 0 and orc.check_tagged(bad, a) >= 0
    # a flipped value byte changes the multiset hash and fails the tag check
    bad = out.copy()
    bad[5, 50] ^= 1
    assert orc.record_hash_sum(bad) != orc.record_hash_sum(a) and orc.check_tagged(bad, a) == 5
    # unstable order of equal keys: keys stay sorted, the tag check fails
    eq = np.where((out[1:, :10] == out[:-1, :10]).all(axis=1))[0]
    assert eq.size > 0
    j = int(eq[0])
    bad = out.copy()
    bad[[j, j + 1]] = bad[[j + 1, j]]
    assert orc.check_sorted(bad) == -1 and orc.check_tagged(bad, a) == j + 1
    # a duplicated record
    bad = out.copy()
    bad[7] = bad[6]
    assert orc.check_tagged(bad, a) >= 0
    # the threaded form of the same check catches the same mistakes, also
    # across its range boundaries
    for T in (1, 3, 8):
        assert orc.check_tagged_threads(out, a, threads=T) == -1
        b2 = out.copy()
        b2[5, 50] ^= 1
        assert orc.check_tagged_threads(b2, a, threads=T) == 5
        b2 = out.copy()
        b2[[j, j + 1]] = b2[[j + 1, j]]
        assert orc.check_tagged_threads(b2, a, threads=T) == j + 1
        b2 = out.copy()
        b2[7] = b2[6]
        assert orc.check_tagged_threads(b2, a, threads=T) in (6, 7)
        b2 = out.copy()
        b2[[10, 3000]] = b2[[3000, 10]]
        assert orc.check_tagged_threads(b2, a, threads=T) >= 0
        cut = len(out) // T  # an order mistake exactly at a range boundary
        if T > 1 and cut + 1 < len(out):
            b2 = out.copy()
            b2[[cut - 1, cut]] = b2[[cut, cut - 1]]  # tags differ: key or tag order breaks
            assert orc.check_tagged_threads(b2, a, threads=T) >= 0


def test_pair_checker_catches_planted_mistakes(orc):
    keys, idx = datagen.narrow_pairs(3000, seed=8, distinct=50)
    k = keys.numpy().view(np.uint64)
    ko, vo = orc.sort_keys_index(k, idx.numpy().view(np.uint32))
    assert orc.check_pairs_tagged(ko, vo, k) == -1
    eq = np.where(ko[1:] == ko[:-1])[0]
    j = int(eq[0])
    vb = vo.copy()
    vb[[j, j + 1]] = vb[[j + 1, j]]
    assert orc.check_pairs_tagged(ko, vb, k) >= 0
    kb = ko.copy()
    kb[100] ^= 1
    assert orc.check_pairs_tagged(kb, vo, k) >= 0


# ------------------------------------------------ the T-thread baseline

@pytest.mark.parametrize("n,threads", [(0, 4), (1, 4), (5, 8), (1000, 1), (1000, 3),
                                       (20_011, 7), (50_000, 16), (4096, 64)])
def test_threaded_sort_equals_lexsort(orc, n, threads):
    # chunked sorts + T-way heap merge: the same unique order as numpy's
    # stable lexsort (ties by index), on tie-heavy and on distinct keys
    for alphabet in (b"AB", None):
        a = rand_records(n, rec=13, key=9, seed=n + threads, alphabet=alphabet)
        got = orc.sort_records_threads(a, key_bytes=9, threads=threads)
        assert np.array_equal(got, a[lex_perm(a, 9)])
        assert np.array_equal(got, orc.sort_records(a, key_bytes=9))


def test_threaded_sort_catches_a_merge_tie_error(orc):
    # every chunk holds the same key: the merge must take equal heads in
    # chunk order (the index decides), or the payload order changes
    a = rand_records(3000, rec=12, key=4, seed=3)
    a[:, :4] = 7
    got = orc.sort_records_threads(a, key_bytes=4, threads=5)
    assert np.array_equal(got, a)  # all keys equal: input order
