"""The serving engine against the oracle: a seeded request stream (builds and
probes of mixed sizes, a budget small enough to force evictions) is fed with
polls at random points; every probe's counts must equal the oracle's for its
table alone, resident bytes never exceed the budget, and requests against
evicted tables are refused.  Also checks the device-side input generators
against the host ones."""
import numpy as np
import pytest

import oracle
import workloads as W
from tests.hg_testutil import from_dev, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def hg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2104_00792_gb300 as m
    return m


def _drain(srv, done):
    for _ in range(200000):
        for rid, st in srv.poll():
            done[rid] = st
        s = srv.stats()
        if s["pending"] == 0 and s["running"] == 0:
            for rid, st in srv.poll():
                done[rid] = st
            return
    raise AssertionError("the engine did not drain")


def _serve(hg, trace, budget, max_batch, poll_p, seed):
    rng = np.random.default_rng(seed)
    srv = hg.Server(budget, max_batch=max_batch)
    keys_of, probes, done = {}, [], {}
    try:
        for r in trace:
            if r.kind == "build":
                k = W.uniform_u32(r.key_state, r.size)
                keys_of[r.table] = (k, to_dev(k))
                srv.submit_build(r.table, keys_of[r.table][1], r.size)
            else:
                hk = keys_of[r.table][0]
                q = W.probe_mix(hk, r.size, 0.6, r.sel, r.miss)
                dq = to_dev(q)
                counts = torch.full((max(r.size, 1),), -1, dtype=torch.int32, device="cuda")
                rid = srv.submit_probe(r.table, dq, counts[: r.size])
                probes.append((rid, r.table, q, dq, counts))
            if rng.random() < poll_p:
                for rid, st in srv.poll():
                    done[rid] = st
                assert srv.stats()["held_bytes"] <= budget
        _drain(srv, done)
        stats = srv.stats()
        torch.cuda.synchronize()
        return keys_of, probes, done, stats
    finally:
        srv.free()


@pytest.mark.parametrize("max_batch,poll_p", [(32, 0.3), (256, 0.05), (1, 1.0)])
def test_serving_counts_equal_the_oracle(hg, max_batch, poll_p):
    budget = 600_000
    trace = W.serving_trace(300, build_log2=(6, 14), probe_log2=(4, 11), budget_bytes=budget, salt=21)
    keys_of, probes, done, stats = _serve(hg, trace, budget, max_batch, poll_p, seed=max_batch)
    assert stats["evictions"] > 0, "the budget should have forced evictions"
    assert all(st == hg.HG_OK for st in done.values())
    assert len(done) == len(trace)
    n_of = W.serve_table_n(trace)
    refs = {}
    for rid, t, q, _, counts in probes:
        if t not in refs:
            refs[t] = oracle.build_table(keys_of[t][0], n_of[t], 0)
        got = from_dev(counts, np.uint32)[: q.size].astype(np.uint64)
        assert np.array_equal(got, refs[t].query_count(q)), f"probe {rid} on table {t}"


def test_serving_at_configured_sizes(hg):
    # builds of up to 2^20 keys and probes of up to 2^18 queries (the top of the
    # range is the serving workload's own shape), budget forcing evictions; every
    # probe's counts against the oracle on its table alone
    budget = 24 * 10**6
    trace = W.serving_trace(160, build_log2=(10, 20), probe_log2=(8, 18), budget_bytes=budget, salt=23)
    assert max(r.size for r in trace if r.kind == "build") > 1 << 18
    assert max(r.size for r in trace if r.kind == "probe") > 1 << 16
    keys_of, probes, done, stats = _serve(hg, trace, budget, 64, 0.25, seed=23)
    assert stats["evictions"] > 0, "the budget should have forced evictions"
    assert all(st == hg.HG_OK for st in done.values())
    assert len(done) == len(trace)
    n_of = W.serve_table_n(trace)
    refs = {}
    for rid, t, q, _, counts in probes:
        if t not in refs:
            refs[t] = oracle.build_table(keys_of[t][0], n_of[t], 0)
        got = from_dev(counts, np.uint32)[: q.size].astype(np.uint64)
        assert np.array_equal(got, refs[t].query_count(q)), f"probe {rid} on table {t}"


def test_serving_refuses_evicted_and_oversized(hg):
    budget = hg.hg_server_table_bytes(1000, 1000) * 2
    with hg.Server(budget) as srv:
        k = to_dev(W.uniform_u32(W.stream("keys", salt=900), 1000))
        srv.submit_build(1, k, 1000)
        srv.submit_build(2, k, 1000)
        srv.submit_build(3, k, 1000)  # evicts table 1, the least recently used
        with pytest.raises(hg.HashGraphError):
            srv.submit_probe(1, k, torch.empty(1000, dtype=torch.int32, device="cuda"))
        with pytest.raises(hg.HashGraphError):
            srv.submit_build(4, k, budget)  # alone larger than the budget
        with pytest.raises(hg.HashGraphError):
            srv.submit_build(2, k, 10)      # id in use
        done = {}
        _drain(srv, done)
        assert len(done) == 3 and all(st == hg.HG_OK for st in done.values())
        assert srv.stats()["held_bytes"] <= budget


def test_served_table_accounting_matches_the_trace(hg):
    for n, b in [(0, 1), (1000, 1000), (1 << 24, 1 << 24), (5, 7)]:
        assert hg.hg_server_table_bytes(n, b) == W.served_table_bytes(n, b)


def test_device_generators_match_host(hg):
    st, sel, miss = W.stream("keys", salt=5), W.stream("q_select", salt=5), W.stream("q_miss", salt=5)
    n, q = 100_003, 70_001
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    W.gpu_uniform_u32(st, n, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    keys = W.uniform_u32(st, n)
    assert np.array_equal(from_dev(out, np.uint32), keys)
    qo = torch.empty(q, dtype=torch.int32, device="cuda")
    W.gpu_probe_mix_uniform_u32(st, n, q, 0.6, sel, miss, qo.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert np.array_equal(from_dev(qo, np.uint32), W.probe_mix(keys, q, 0.6, sel, miss))
