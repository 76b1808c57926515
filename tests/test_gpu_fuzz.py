"""Randomised configurations against the oracle (the property layer of the
tests): key width, key count, bucket count (powers of two and not), seed,
duplicate rate, values, and every build mode and table option, each case
checked bit-exact on offsets, bucket contents (canonical order), counts,
totals and join counts.  Seeded, so a failure repeats."""
import numpy as np
import pytest

import oracle
from tests.hg_testutil import assert_same_table, from_dev, table_arrays, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = 24


@pytest.fixture(scope="module")
def hg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2104_00792_gb300 as m
    return m


def _case(i):
    rng = np.random.default_rng(1000 + i)
    wide = bool(rng.integers(0, 2))
    dt = np.uint64 if wide else np.uint32
    n = int(rng.choice([0, 1, 7, 1000, 4097, int(rng.integers(1, 1 << 17)), 1 << 17]))
    B = int(rng.choice([1, 2, 17, 1 << 10, 65537, int(rng.integers(1, 1 << 18)), 1 << 16]))
    if B < 1024:
        n = min(n, 8192)  # few buckets: keep the oracle's walks short
    seed = int(rng.integers(0, 1 << 63))
    distinct = max(1, int(n / 2 ** rng.uniform(0, 12)))            # copies per value: 1 .. 4096
    pool = rng.integers(0, np.iinfo(dt).max, size=distinct, dtype=dt, endpoint=True)
    keys = pool[rng.integers(0, distinct, size=n)] if n else np.zeros(0, dt)
    q = int(rng.integers(0, 3 * n + 10))
    hits = pool[rng.integers(0, distinct, size=q)]
    misses = rng.integers(0, np.iinfo(dt).max, size=q, dtype=dt, endpoint=True)
    queries = np.where(rng.random(q) < 0.6, hits, misses).astype(dt)
    with_values = bool(rng.integers(0, 2))
    values = rng.integers(0, 1 << 32, size=n, dtype=np.uint64).astype(np.uint32) if with_values else None
    return dt, keys, B, seed, queries, values, rng


@pytest.mark.parametrize("i", range(CASES))
def test_random_configuration(hg, i):
    dt, keys, B, seed, queries, values, rng = _case(i)
    mode = [0, hg.HG_PLAIN_BUILD, hg.HG_PARTITION_BUILD][int(rng.integers(0, 3))]
    flags = mode | (hg.HG_SORTED_BUCKETS if rng.integers(0, 2) else 0) | (hg.HG_LONG_SUMMARY if rng.integers(0, 2) else 0)
    ref = oracle.build_table(keys, B, seed, values=values)
    u, inv = np.unique(queries, return_inverse=True)
    want = ref.query_count(np.ascontiguousarray(u))[inv] if queries.size else np.zeros(0, np.uint64)
    dk = to_dev(keys) if keys.size else torch.zeros(1, dtype=torch.int64 if dt == np.uint64 else torch.int32,
                                                   device="cuda")[:0]
    dv = None if values is None else to_dev(values)
    with hg.hg_build(dk, B, seed, values=dv, flags=flags) as t:
        o, k, v = table_arrays(hg, t, dt)
        assert_same_table(o, k, v, ref)
        if queries.size:
            dq = to_dev(queries)
            counts = torch.full((queries.size,), -1, dtype=torch.int32, device="cuda")
            total = torch.full((1,), -1, dtype=torch.int64, device="cuda")
            hg.hg_query_count(t, dq, counts, total)
            assert np.array_equal(from_dev(counts, np.uint32).astype(np.uint64), want), f"case {i}: counts"
            assert int(from_dev(total, np.uint64)[0]) == int(want.sum())
            jt = torch.full((1,), -1, dtype=torch.int64, device="cuda")
            hg.hg_join_count(t, dq, jt)
            assert int(from_dev(jt, np.uint64)[0]) == int(want.sum())
        hg.hg_sync(t)
