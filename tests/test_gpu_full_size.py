"""Parity at the benchmark's full sizes, element by element against the oracle.

* zipf_large: 2^28 uint32 Zipf keys, 2^27 buckets, 2^28 queries.  Run twice:
  - exactly as bench.py's timed step runs it: hg_build with HG_LONG_SUMMARY,
    hg_query_plan_create on a second stream while the table builds, then
    hg_query_count_plan (counts and total);
  - with default flags through hg_query_count (counts and total).
  Each run: offsets bit-exact; bucket contents after the canonical sort by
  (bucket, key); all 2^28 per-slot counts bit-exact against the oracle's
  bucket walk; the total equal to the oracle's sum.
* join_kv: 2^27 (uint64 key, uint32 value) pairs, 2^26 buckets, 2^26 probes
  with a repeated hot subset.  Offsets bit-exact; bucket contents after the
  canonical sort by (bucket, key, value); join total against the oracle's;
  gathered values of the first 2^20 probes against the oracle's.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from tests.hg_testutil import assert_same_gather, assert_same_table, from_dev, table_arrays, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N28, B27 = 1 << 28, 1 << 27


@pytest.fixture(scope="module")
def hg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2104_00792_gb300 as m
    return m


def canonical_u32(keys: np.ndarray, offsets: np.ndarray) -> np.ndarray:
    """(bucket << 32 | key) for every table slot, sorted: the table's contents
    in the canonical order (bucket, then key).  Equal arrays <=> every bucket
    holds the same key multiset."""
    o = offsets.astype(np.int64)
    seg = np.repeat(np.arange(o.size - 1, dtype=np.uint64), np.diff(o))
    c = (seg << np.uint64(32)) | keys.astype(np.uint64)
    del seg
    c.sort(kind="stable")
    return c


@pytest.fixture(scope="module")
def zipf_ref():
    wl = W.zipf_large(n=N28, num_buckets=B27, q=N28, M=1 << 24)
    ref = oracle.build_table(wl.keys, B27, 0)
    want = ref.query_count(wl.queries)          # every one of the 2^28 slots
    canon = canonical_u32(ref.keys, ref.offsets)
    return wl, ref.offsets, want, canon


def _check_zipf(hg, t, zipf_ref, counts, total):
    wl, offsets, want, canon = zipf_ref
    o, k, _ = table_arrays(hg, t, np.uint32)
    assert np.array_equal(o.astype(np.uint64), offsets), "offsets differ"
    assert np.array_equal(canonical_u32(k, o), canon), "bucket contents differ"
    del o, k
    got = from_dev(counts, np.uint32)
    bad = np.flatnonzero(got.astype(np.uint64) != want)
    assert bad.size == 0, f"{bad.size} of {got.size} counts differ, first at slot {bad[:4]}"
    assert int(from_dev(total, np.uint64)[0]) == int(want.sum(dtype=np.uint64))
    # the hottest value is queried and its count is its multiplicity in the input
    hot = W.rank_value(1)
    slots = np.flatnonzero(wl.queries == hot)[:4]
    if slots.size:
        assert int(got[slots[0]]) == oracle.count_linear(wl.keys, hot)


def test_full_zipf_large_benchmarked_path(hg, zipf_ref):
    wl = zipf_ref[0]
    keys, queries = to_dev(wl.keys), to_dev(wl.queries)
    counts = torch.full((N28,), -1, dtype=torch.int32, device="cuda")
    total = torch.empty(1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    side = torch.cuda.Stream()
    forked, joined = torch.cuda.Event(), torch.cuda.Event()
    forked.record(stream)
    t = hg.hg_build(keys, B27, 0, flags=hg.HG_LONG_SUMMARY, stream=stream)
    try:
        side.wait_event(forked)
        plan = hg.hg_query_plan_create(t, queries, stream=side)
        joined.record(side)
        stream.wait_event(joined)
        hg.hg_query_count_plan(t, plan, counts, total, stream=stream)
        plan.free(stream)
        hg.hg_sync(t, stream=stream)
        del keys, queries
        _check_zipf(hg, t, zipf_ref, counts, total)
    finally:
        t.free(stream)


def test_full_zipf_large_default_flags(hg, zipf_ref):
    wl = zipf_ref[0]
    counts = torch.full((N28,), -1, dtype=torch.int32, device="cuda")
    total = torch.empty(1, dtype=torch.int64, device="cuda")
    with hg.hg_build(to_dev(wl.keys), B27, 0) as t:
        hg.hg_query_count(t, to_dev(wl.queries), counts, total)
        hg.hg_sync(t)
        _check_zipf(hg, t, zipf_ref, counts, total)


def test_full_join_kv(hg):
    n, B, q = 1 << 27, 1 << 26, 1 << 26
    wl = W.join_kv(n=n, num_buckets=B, q=q)
    ref = oracle.build_table(wl.keys, B, 0, values=wl.values)
    with hg.hg_build(to_dev(wl.keys), B, 0, values=to_dev(wl.values)) as t:
        o, k, v = table_arrays(hg, t, np.uint64)
        assert_same_table(o, k, v, ref)
        del o, k, v
        dq = to_dev(wl.queries)
        total = torch.empty(1, dtype=torch.int64, device="cuda")
        hg.hg_join_count(t, dq, total)
        first = dq[: 1 << 20].contiguous()
        offs = torch.empty((1 << 20) + 1, dtype=torch.int64, device="cuda")
        ro, rv = ref.query_gather(wl.queries[: 1 << 20])
        vals = torch.empty(max(int(ro[-1]), 1), dtype=torch.int32, device="cuda")
        m = hg.hg_query_gather(t, first, offs, vals)
        hg.hg_sync(t)
        assert m == int(ro[-1])
        assert_same_gather(from_dev(offs, np.uint64), from_dev(vals, np.uint32)[:m], ro, rv)
        assert int(from_dev(total, np.uint64)[0]) == ref.join_count(wl.queries)
