"""Long-bucket summaries (HG_LONG_SUMMARY) and Zipf-weighted queries against
the oracle.

* Each summary equals the definition taken from the oracle's table: for every
  bucket of more than 8192 keys, its distinct keys ascending with their
  multiplicities, or the overflow marker when it has more than the summary's
  slots; every such bucket is listed exactly once, and no other bucket.
* Counts, totals and join counts are bit-exact with the oracle's, for tables
  with and without summaries, through the direct and the grouped probe; the
  grouped cases include bins holding more queries than one work item takes,
  and bins too large to copy whole that the hash join takes through their
  long buckets' summaries (or leaves to the walking probe).

Zipf-weighted queries (each value queried in proportion to its copies) make
the oracle's walk quadratic, so its counts are taken once per distinct query
key and spread back to the slots."""
import numpy as np
import pytest

import oracle
import workloads as W
from tests.hg_testutil import from_dev, table_arrays, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

LONG = 8192
OVERFLOW = 0xFFFFFFFF


@pytest.fixture(scope="module")
def hg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2104_00792_gb300 as m
    return m


def _oracle_counts(ref, queries):
    u, inv = np.unique(queries, return_inverse=True)
    return ref.query_count(np.ascontiguousarray(u))[inv]


def _check_summary(hg, t, ref, key_dtype):
    view = hg.hg_long_summary_view(t)
    offs = ref.offsets.astype(np.int64)
    lens = np.diff(offs)
    long_b = np.flatnonzero(lens > LONG)
    if view is None:
        assert ref.keys.size <= LONG
        return 0
    torch.cuda.synchronize()
    n_long = int(from_dev(view["n_long"], np.uint32)[0])
    slots = view["slots"]
    assert n_long == long_b.size <= view["cap"]
    buckets = from_dev(view["bucket"], np.uint32)[:n_long].astype(np.int64)
    assert np.array_equal(np.sort(buckets), long_b), "long buckets listed differ"
    slen = from_dev(view["len"], np.uint32)[:n_long]
    skeys = from_dev(view["keys"], key_dtype)
    scnt = from_dev(view["counts"], np.uint32)
    n_sum = 0
    for l, b in enumerate(buckets):
        u, c = np.unique(ref.keys[offs[b]:offs[b + 1]], return_counts=True)
        if u.size > slots:
            assert slen[l] == OVERFLOW, f"bucket {b}: {u.size} distinct keys, summary not marked overflow"
            continue
        n_sum += 1
        assert slen[l] == u.size, f"bucket {b}: summary length"
        assert np.array_equal(skeys[l * slots:l * slots + u.size], u), f"bucket {b}: summary keys"
        assert np.array_equal(scnt[l * slots:l * slots + u.size], c.astype(np.uint32)), f"bucket {b}: summary counts"
    return n_sum


def _run(hg, keys, B, queries, flags, values=None, seed=0, expect_summaries=None):
    ref = oracle.build_table(keys, B, seed, values=values)
    want = _oracle_counts(ref, queries)
    dq = to_dev(queries)
    with hg.hg_build(to_dev(keys), B, seed, values=None if values is None else to_dev(values), flags=flags) as t:
        o, _, _ = table_arrays(hg, t, keys.dtype)
        assert np.array_equal(o.astype(np.uint64), ref.offsets), "offsets differ"
        if flags & hg.HG_LONG_SUMMARY:
            n_sum = _check_summary(hg, t, ref, keys.dtype)
            if expect_summaries is not None:
                assert (n_sum > 0) == expect_summaries
        counts = torch.full((queries.size,), -1, dtype=torch.int32, device="cuda")
        total = torch.full((1,), -1, dtype=torch.int64, device="cuda")
        hg.hg_query_count(t, dq, counts, total)
        assert np.array_equal(from_dev(counts, np.uint32).astype(np.uint64), want), "counts differ"
        assert int(from_dev(total, np.uint64)[0]) == int(want.sum())
        c2 = torch.full((queries.size,), -1, dtype=torch.int32, device="cuda")
        hg.hg_query_count(t, dq, c2, None)
        assert np.array_equal(from_dev(c2, np.uint32).astype(np.uint64), want)
        jt = torch.full((1,), -1, dtype=torch.int64, device="cuda")
        hg.hg_join_count(t, dq, jt)
        assert int(from_dev(jt, np.uint64)[0]) == int(want.sum())
        with hg.hg_query_plan_create(t, dq) as plan:
            c3 = torch.full((queries.size,), -1, dtype=torch.int32, device="cuda")
            t3 = torch.full((1,), -1, dtype=torch.int64, device="cuda")
            hg.hg_query_count_plan(t, plan, c3, t3)
            assert np.array_equal(from_dev(c3, np.uint32).astype(np.uint64), want), "planned counts differ"
            assert int(from_dev(t3, np.uint64)[0]) == int(want.sum())
        hg.hg_sync(t)
    return ref, want


@pytest.mark.parametrize("build", ["plain", "partition"])
def test_summaries_of_zipf_table(hg, build):
    wl = W.zipf_large(n=1 << 20, num_buckets=1 << 19, q=(1 << 18) + 7, M=1 << 12, salt=60)
    extra = hg.HG_PLAIN_BUILD if build == "plain" else hg.HG_PARTITION_BUILD
    _run(hg, wl.keys, 1 << 19, wl.queries, hg.HG_LONG_SUMMARY | extra, expect_summaries=True)


def test_summaries_with_sorted_buckets_and_values(hg):
    wl = W.zipf_weighted(n=(1 << 20) + 3, num_buckets=(1 << 19) + 1, q=1 << 18, M=1 << 12, salt=61)
    _run(hg, wl.keys, (1 << 19) + 1, wl.queries,
         hg.HG_LONG_SUMMARY | hg.HG_SORTED_BUCKETS | hg.HG_INDEX_VALUES, expect_summaries=True)


def test_summary_overflow_is_walked(hg):
    # four buckets of ~2^16 distinct keys each: too many for a summary
    wl = W.plain_uniform((1 << 18) + 5, 20003, num_buckets=4, salt=62)
    _run(hg, wl.keys, 4, wl.queries, hg.HG_LONG_SUMMARY, expect_summaries=False)


def test_summary_mixed_hot_and_overflow_u32(hg):
    rng = np.random.default_rng(63)
    hot = rng.integers(0, 1 << 32, size=40, dtype=np.uint64).astype(np.uint32)
    hot[0] = 0xFFFFFFFF                                   # the all-ones key, counted on the side
    keys = np.concatenate([np.repeat(hot, 9000 + np.arange(40) * 37),
                           rng.integers(0, 1 << 32, size=70000, dtype=np.uint64).astype(np.uint32)])
    rng.shuffle(keys)
    # 17 buckets: a few hot values share a bucket, and the random keys push some
    # buckets past the summary's slots
    queries = np.concatenate([hot, keys[:30000], rng.integers(0, 1 << 32, size=5000, dtype=np.uint64).astype(np.uint32)])
    _run(hg, keys, 17, queries, hg.HG_LONG_SUMMARY)
    # and with 4096 buckets: each hot value's bucket summarised, the rest short
    _run(hg, keys, 4096, queries, hg.HG_LONG_SUMMARY, expect_summaries=True)


def test_summary_u64_keys_with_values(hg):
    rng = np.random.default_rng(64)
    hot = rng.integers(0, 1 << 63, size=24, dtype=np.uint64) * np.uint64(2) + np.uint64(1)
    hot[3] = np.uint64(0xFFFFFFFFFFFFFFFF)
    keys = np.repeat(hot, 12000 + np.arange(24) * 101)
    keys = np.concatenate([keys, rng.integers(0, 1 << 63, size=20000, dtype=np.uint64)])
    rng.shuffle(keys)
    vals = rng.integers(0, 1 << 32, size=keys.size, dtype=np.uint64).astype(np.uint32)
    queries = np.concatenate([hot, keys[:20000], rng.integers(0, 1 << 63, size=3000, dtype=np.uint64)])
    _run(hg, keys, 1000, queries, hg.HG_LONG_SUMMARY, values=vals, seed=0x1234567, expect_summaries=True)


def test_summary_small_table_has_none(hg):
    keys = np.arange(5000, dtype=np.uint32)
    with hg.hg_build(to_dev(keys), 1, 0, flags=hg.HG_LONG_SUMMARY) as t:
        assert hg.hg_long_summary_view(t) is None
        c = torch.empty(keys.size, dtype=torch.int32, device="cuda")
        hg.hg_query_count(t, to_dev(keys), c, None)
        assert np.all(from_dev(c, np.uint32) == 1)


@pytest.mark.parametrize("summary", [False, True])
def test_zipf_weighted_grouped(hg, summary):
    # 2^23 buckets (1024 bins; the table is larger than L2): the grouped probe.
    # 1024 values Zipf-weighted: the bin of the hottest value gets ~400k queries,
    # more than one work item takes, so it is cut into slices
    wl = W.zipf_weighted(n=1 << 23, num_buckets=1 << 23, q=(1 << 22) + 5, M=1 << 10, salt=65)
    flags = hg.HG_LONG_SUMMARY if summary else 0
    _run(hg, wl.keys, 1 << 23, wl.queries, flags, expect_summaries=True if summary else None)


def test_zipf_weighted_direct(hg):
    # a table that stays in L2 with many queries: the direct probe
    wl = W.zipf_weighted(n=1 << 21, num_buckets=1 << 20, q=(1 << 21) + 1, M=1 << 14, salt=66)
    _run(hg, wl.keys, 1 << 20, wl.queries, hg.HG_LONG_SUMMARY, expect_summaries=True)


def _keys_in_bucket(b, B, count, start):
    """`count` distinct 32-bit keys whose bucket is b, searched upward from `start`."""
    out, x = [], start
    while len(out) < count:
        cand = (np.arange(x, x + (1 << 25), dtype=np.uint64) & np.uint64(0xFFFFFFFF)).astype(np.uint32)
        out.extend(cand[oracle.buckets(cand, B, 0) == b].tolist())
        x += 1 << 25
    return np.array(out[:count], dtype=np.uint32)


def test_hash_join_hot_bins(hg):
    # 1024 bins; bins holding long buckets are too large to copy whole, so the
    # hash join copies only the keys between their long buckets and takes the
    # long buckets' counts from their summaries.  Three bins are built to
    # defeat it and go to the walking probe: bin 5 with nine long buckets, bin 9
    # with a long bucket of 80 distinct keys (no summary), bin 11 with more
    # short-bucket keys than the buffer holds.
    B = 1 << 23
    wl = W.zipf_large(n=1 << 23, num_buckets=B, q=(1 << 21) + 5, M=1 << 16, salt=70)
    rng = np.random.default_rng(71)
    cand = rng.integers(0, 1 << 32, size=1 << 25, dtype=np.uint64).astype(np.uint32)
    bins = oracle.buckets(cand, B, 0) >> 13
    in5 = np.unique(cand[bins == 5])[:9]
    in11 = cand[bins == 11][:30000]
    k9 = _keys_in_bucket((9 << 13) + 77, B, 80, start=12345)
    keys = np.concatenate([wl.keys, np.repeat(in5, 9000), np.repeat(k9, 250), in11])
    keys = keys[rng.permutation(keys.size)]
    queries = np.concatenate([in5, k9, in11[:5000], wl.queries])
    for flags in (hg.HG_LONG_SUMMARY, 0):
        _run(hg, keys, B, queries, flags, expect_summaries=True if flags else None)
