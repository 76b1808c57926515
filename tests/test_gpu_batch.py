"""Batched tables (one persistent launch) against the oracle, table by table:
per-table offsets bit-exact, bucket contents after a canonical sort, and
every query's count bit-exact.  Covers the fused shared-memory path, the
partitioned path (several bins, one bin too large to stage), every tuning
parameter set, the autotuner and graph replays."""
import numpy as np
import pytest

import oracle
import workloads as W
from tests.hg_testutil import assert_same_table, from_dev, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PARAMS = [(t, s, f) for t in (256, 512) for s in (12, 13) for f in (1 << s, 1 << (s - 1))]


@pytest.fixture(scope="module")
def hg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2104_00792_gb300 as m
    return m


def _concat(tables):
    """tables: list of (keys u32, num_buckets, queries u32) -> BatchWorkload."""
    ko = np.zeros(len(tables) + 1, dtype=np.uint64)
    qo = np.zeros(len(tables) + 1, dtype=np.uint64)
    ko[1:] = np.cumsum([t[0].size for t in tables])
    qo[1:] = np.cumsum([t[2].size for t in tables])
    keys = np.concatenate([t[0] for t in tables]).astype(np.uint32) if ko[-1] else np.zeros(0, np.uint32)
    qs = np.concatenate([t[2] for t in tables]).astype(np.uint32) if qo[-1] else np.zeros(0, np.uint32)
    nb = np.array([t[1] for t in tables], dtype=np.uint64)
    return W.BatchWorkload("custom", keys, ko, nb, qs, qo)


def _run(hg, wl, seed=0, params=None, tune=False, runs=1):
    keys = to_dev(wl.keys) if wl.keys.size else torch.zeros(1, dtype=torch.int32, device="cuda")
    qs = to_dev(wl.queries) if wl.queries.size else torch.zeros(1, dtype=torch.int32, device="cuda")
    counts = torch.full((max(wl.queries.size, 1),), -1, dtype=torch.int32, device="cuda")
    b = hg.hg_batch_create(wl.key_offsets, wl.num_buckets, wl.query_offsets, seed=seed)
    try:
        chosen = None
        if params:
            hg.hg_batch_set_params(b, *params)
        if tune:
            chosen = hg.hg_batch_tune(b, keys, qs, counts)
        for _ in range(runs):
            hg.hg_batch_run(b, keys, qs, counts)
        hg.hg_batch_sync(b)
        got = from_dev(counts, np.uint32)[: wl.queries.size]
        tables = []
        for t in range(wl.n_tables):
            o, k = hg.hg_batch_view(b, t)
            torch.cuda.synchronize()
            tables.append((from_dev(o, np.uint32), from_dev(k, np.uint32)))
        return got, tables, chosen
    finally:
        b.free()


def _check(wl, got, tables, seed=0):
    for t in range(wl.n_tables):
        k, B, qs = wl.table(t)
        ref = oracle.build_table(np.ascontiguousarray(k), B, seed)
        o, kk = tables[t]
        assert_same_table(o, kk, None, ref)
        q0, q1 = int(wl.query_offsets[t]), int(wl.query_offsets[t + 1])
        want = ref.query_count(np.ascontiguousarray(qs))
        assert np.array_equal(got[q0:q1].astype(np.uint64), want), f"counts of table {t} differ"


def test_batch_log_uniform_sizes(hg):
    wl = W.batched_uniform(48, 0, 16, salt=5)
    got, tables, _ = _run(hg, wl)
    _check(wl, got, tables)


def test_batch_edge_tables(hg):
    rng = np.random.default_rng(11)
    dup = rng.integers(0, 1000, size=40000, dtype=np.uint32)       # one bin, too many keys to stage
    big = rng.integers(0, 1 << 32, size=100000, dtype=np.uint64).astype(np.uint32)
    mid = rng.integers(0, 1 << 32, size=9000, dtype=np.uint64).astype(np.uint32)
    tables = [
        (np.zeros(0, np.uint32), 1, np.array([0, 1, 2], np.uint32)),                  # empty table
        (np.array([7, 7, 7, 9, 0xFFFFFFFF], np.uint32), 1, np.array([7, 9, 0xFFFFFFFF, 8], np.uint32)),
        (dup, 3, np.concatenate([dup[:5000], np.arange(2000, 2100, dtype=np.uint32)])),
        (big, 1 << 21, W.probe_mix(big, 60000, 0.5, W.stream("q_select", salt=77), W.stream("q_miss", salt=77))),
        (mid, 9000, W.probe_mix(mid, 9001, 0.5, W.stream("q_select", salt=78), W.stream("q_miss", salt=78))),
        (big[:30000], 7919, np.zeros(0, np.uint32)),                                     # no queries
        (mid[:16384], 8192, mid[:100]),                                                    # exactly the stage size
    ]
    wl = _concat(tables)
    got, tabs, _ = _run(hg, wl, seed=0x1234)
    _check(wl, got, tabs, seed=0x1234)


def test_batch_largest_tables(hg):
    # the top of the batched workload's size range: tables of 2^19 to 2^20 keys
    # with B_t = N_t (128 bins of 8192 buckets each, partitioned inside one CTA),
    # mixed with small tables on the fused shared-memory path
    big = W.batched_uniform(6, 19, 20, salt=31)
    small = W.batched_uniform(10, 8, 13, salt=32)
    tables = [big.table(t) for t in range(big.n_tables)] + [small.table(t) for t in range(small.n_tables)]
    wl = _concat([(np.ascontiguousarray(k), B, np.ascontiguousarray(q)) for k, B, q in tables])
    assert max(int(x) for x in wl.num_buckets) >= 1 << 19
    got, tabs, _ = _run(hg, wl)
    _check(wl, got, tabs)
    got2, tabs2, _ = _run(hg, wl, tune=True)
    _check(wl, got2, tabs2)


@pytest.mark.parametrize("params", PARAMS)
def test_batch_every_parameter_set(hg, params):
    wl = W.batched_uniform(24, 6, 15, salt=9)
    got, tables, _ = _run(hg, wl, params=params)
    _check(wl, got, tables)


def test_batch_tune_and_replay(hg):
    # on a stream of its own the runs are captured once and replayed as a CUDA graph
    wl = W.batched_uniform(32, 4, 15, salt=10)
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(side):
        got, tables, chosen = _run(hg, wl, tune=True, runs=3)
    torch.cuda.synchronize()
    assert (chosen["threads"], chosen["bin_shift"], chosen["fuse_keys"]) in PARAMS
    _check(wl, got, tables)


def test_batch_graph_replays_count_one_launch_each(hg):
    wl = W.batched_uniform(8, 4, 12, salt=13)
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(side):
        keys, qs = to_dev(wl.keys), to_dev(wl.queries)
        counts = torch.empty(wl.queries.size, dtype=torch.int32, device="cuda")
        with hg.hg_batch_create(wl.key_offsets, wl.num_buckets, wl.query_offsets) as b:
            hg.hg_batch_run(b, keys, qs, counts)
            n0 = hg.hg_launch_count()
            for _ in range(5):
                hg.hg_batch_run(b, keys, qs, counts)
            assert hg.hg_launch_count() - n0 == 5
            hg.hg_batch_sync(b)
            got = from_dev(counts, np.uint32)
    for t in range(wl.n_tables):
        k, B, q = wl.table(t)
        q0, q1 = int(wl.query_offsets[t]), int(wl.query_offsets[t + 1])
        want = oracle.build_table(np.ascontiguousarray(k), B, 0).query_count(np.ascontiguousarray(q))
        assert np.array_equal(got[q0:q1].astype(np.uint64), want)


def test_batch_replay_sees_new_inputs(hg):
    a = W.batched_uniform(16, 4, 14, salt=12)
    rng = np.random.default_rng(3)
    new_q = a.queries.copy()
    new_q[::3] = rng.integers(0, 1 << 32, size=new_q[::3].size, dtype=np.uint64).astype(np.uint32)
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(side):
        keys, qs = to_dev(a.keys), to_dev(a.queries)
        fresh = to_dev(new_q)
        counts = torch.empty(a.queries.size, dtype=torch.int32, device="cuda")
        with hg.hg_batch_create(a.key_offsets, a.num_buckets, a.query_offsets) as b:
            hg.hg_batch_run(b, keys, qs, counts)
            # same buffers, new contents: the replayed graph reads them
            qs.copy_(fresh)
            hg.hg_batch_run(b, keys, qs, counts)
            hg.hg_batch_sync(b)
            got = from_dev(counts, np.uint32)
    for t in range(a.n_tables):
        k, B, _ = a.table(t)
        q0, q1 = int(a.query_offsets[t]), int(a.query_offsets[t + 1])
        want = oracle.build_table(np.ascontiguousarray(k), B, 0).query_count(np.ascontiguousarray(new_q[q0:q1]))
        assert np.array_equal(got[q0:q1].astype(np.uint64), want)


def test_batch_rejects_bad_plans(hg):
    with pytest.raises(hg.HashGraphError):
        hg.hg_batch_create([0, 10], [0], [0, 5])                 # zero buckets
    with pytest.raises(hg.HashGraphError):
        hg.hg_batch_create([0, 10], [(1 << 21) + 1], [0, 5])     # more buckets than the bins allow
    with pytest.raises(hg.HashGraphError):
        hg.hg_batch_create([0, 10, 5], [4, 4], [0, 5, 6])        # decreasing offsets
    with hg.hg_batch_create([0, 4], [4], [0, 4]) as b:
        with pytest.raises(hg.HashGraphError):
            hg.hg_batch_set_params(b, 128, 13, 100)


def test_batch_walk_stats(hg):
    wl = W.batched_uniform(20, 4, 13, salt=14)
    keys, qs = to_dev(wl.keys), to_dev(wl.queries)
    counts = torch.empty(wl.queries.size, dtype=torch.int32, device="cuda")
    with hg.hg_batch_create(wl.key_offsets, wl.num_buckets, wl.query_offsets) as b:
        hg.hg_batch_run(b, keys, qs, counts)
        w = hg.hg_batch_walk_stats(b, qs)
    want = 0
    for t in range(wl.n_tables):
        k, B, q = wl.table(t)
        ref = oracle.build_table(np.ascontiguousarray(k), B, 0)
        lens = np.diff(ref.offsets.astype(np.int64))
        want += int(lens[oracle.buckets(np.ascontiguousarray(q), B, 0)].sum())
    assert w == want
