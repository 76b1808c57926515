"""Parity at the benchmark's full sizes, through the same calls and launch
configuration bench.py times (default build and probe paths):

* zipf_large: 2^28 uint32 Zipf keys, 2^27 buckets, 2^28 queries.  Offsets are
  compared bit-exact with the oracle's build; every bucket's key multiset via
  order-free fingerprints; per-slot counts on a seeded sample of slots, each
  answered by the oracle's bucket walk; the total equals the sum of the counts.
* join_kv: 2^27 (uint64 key, uint32 value) pairs, 2^26 buckets, 2^26 probes
  with a repeated hot subset.  Offsets bit-exact; join total against the
  oracle's; gathered values of the first 2^20 probes against the oracle's.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from tests.hg_testutil import assert_same_gather, from_dev, segment_signature, table_arrays, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def hg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2104_00792_gb300 as m
    return m


def _check_buckets(o, k, v, ref):
    assert np.array_equal(o.astype(np.uint64), ref.offsets), "offsets differ"
    a1, a2 = segment_signature(k, ref.offsets, v)
    b1, b2 = segment_signature(ref.keys, ref.offsets, ref.values)
    assert np.array_equal(a1, b1) and np.array_equal(a2, b2), "bucket contents differ"


def test_full_zipf_large(hg):
    n, B = 1 << 28, 1 << 27
    wl = W.zipf_large(n=n, num_buckets=B, q=n, M=1 << 24)
    ref = oracle.build_table(wl.keys, B, 0)
    with hg.hg_build(to_dev(wl.keys), B, 0) as t:
        o, k, v = table_arrays(hg, t, np.uint32)
        _check_buckets(o, k, v, ref)
        del o, k, v
        counts = torch.empty(n, dtype=torch.int32, device="cuda")
        total = torch.empty(1, dtype=torch.int64, device="cuda")
        hg.hg_query_count(t, to_dev(wl.queries), counts, total)
        hg.hg_sync(t)
        got = from_dev(counts, np.uint32)
        tot = int(from_dev(total, np.uint64)[0])
    assert tot == int(got.sum(dtype=np.uint64))
    rng = np.random.default_rng(2104)
    sample = np.concatenate([rng.integers(0, n, size=1 << 20), np.arange(64), np.arange(n - 64, n)])
    want = ref.query_count(wl.queries[sample])
    assert np.array_equal(got[sample].astype(np.uint64), want)
    # the hottest value is queried and its count is its multiplicity
    hot = W.rank_value(1)
    slots = np.flatnonzero(wl.queries == hot)[:4]
    if slots.size:
        assert int(got[slots[0]]) == oracle.count_linear(wl.keys, hot)


def test_full_join_kv(hg):
    n, B, q = 1 << 27, 1 << 26, 1 << 26
    wl = W.join_kv(n=n, num_buckets=B, q=q)
    ref = oracle.build_table(wl.keys, B, 0, values=wl.values)
    with hg.hg_build(to_dev(wl.keys), B, 0, values=to_dev(wl.values)) as t:
        o, k, v = table_arrays(hg, t, np.uint64)
        _check_buckets(o, k, v, ref)
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
