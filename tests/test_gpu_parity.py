"""CUDA path vs the CPU oracle, element by element, on seeded inputs.

Sizes span several tiles of every kernel and end in ragged tails; the
workload recipes are the ones the benchmark uses, scaled down.  Offsets,
counts and totals must be bit-exact; bucket contents and gather segments are
compared after a canonical sort (the order inside a bucket is free)."""
import numpy as np
import pytest

import oracle
import workloads as W
from tests.hg_testutil import assert_same_gather, assert_same_table, from_dev, table_arrays, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def hg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2104_00792_gb300 as m
    return m


def _run_all(hg, keys, B, seed, queries, values=None, flags=0, check_gather=True,
             modes=("plain", "partition")):
    """Both builds (direct Algorithm 1 and the partitioned one) against the oracle."""
    ref = oracle.build_table(keys, B, seed, values=values, index_values=bool(flags & hg.HG_INDEX_VALUES))
    for mode in modes:
        extra = hg.HG_PLAIN_BUILD if mode == "plain" else hg.HG_PARTITION_BUILD
        _run_one(hg, ref, keys, B, seed, queries, values, flags | extra, check_gather)
    return ref


def _check_sorted(o, k, limit):
    """Every bucket of at most `limit` keys is in ascending order."""
    lens = np.diff(o.astype(np.int64))
    if k.size < 2:
        return
    step_down = np.flatnonzero(k[1:] < k[:-1]) + 1        # positions where the order breaks
    bucket_of_pos = np.searchsorted(o.astype(np.int64), step_down, side="right") - 1
    starts = o.astype(np.int64)[bucket_of_pos]
    inside = step_down > starts                          # not the first key of its bucket
    bad = bucket_of_pos[inside]
    assert np.all(lens[bad] > limit), "a sorted-size bucket is out of order"


def _run_one(hg, ref, keys, B, seed, queries, values, flags, check_gather):
    dt = keys.dtype
    dk = to_dev(keys)
    dv = None if values is None else to_dev(values)
    dq = to_dev(queries)
    with hg.hg_build(dk, B, seed, values=dv, flags=flags) as t:
        o, k, v = table_arrays(hg, t, dt)
        assert_same_table(o, k, v, ref)
        if flags & hg.HG_SORTED_BUCKETS:
            _check_sorted(o, k, 16384 if dt == np.uint32 else 8192)
        # counts and total in one call
        counts = torch.empty(queries.size, dtype=torch.int32, device="cuda")
        total = torch.empty(1, dtype=torch.int64, device="cuda")
        hg.hg_query_count(t, dq, counts, total)
        want = ref.query_count(queries)
        got = from_dev(counts, np.uint32).astype(np.uint64)
        assert np.array_equal(got, want), "counts differ"
        assert int(from_dev(total, np.uint64)[0]) == int(want.sum())
        # a query plan made on another stream while the table is being built
        side = torch.cuda.Stream()
        ev = torch.cuda.Event()
        torch.cuda.synchronize()
        with hg.hg_query_plan_create(t, dq, stream=side) as plan:
            ev.record(side)
            torch.cuda.current_stream().wait_event(ev)
            c4 = torch.full((queries.size,), -1, dtype=torch.int32, device="cuda")
            t4 = torch.full((1,), -1, dtype=torch.int64, device="cuda")
            hg.hg_query_count_plan(t, plan, c4, t4)
            assert np.array_equal(from_dev(c4, np.uint32).astype(np.uint64), want), "planned counts differ"
            assert int(from_dev(t4, np.uint64)[0]) == int(want.sum())
        # the paper's query form: HG(Q), then bucket-by-bucket intersection
        c3 = torch.full((queries.size,), -1, dtype=torch.int32, device="cuda")
        t3 = torch.full((1,), -1, dtype=torch.int64, device="cuda")
        hg.hg_query_count_intersect(t, dq, c3, t3)
        assert np.array_equal(from_dev(c3, np.uint32).astype(np.uint64), want), "intersection counts differ"
        assert int(from_dev(t3, np.uint64)[0]) == int(want.sum())
        # counts only, then total only (join)
        counts2 = torch.full((queries.size,), -1, dtype=torch.int32, device="cuda")
        hg.hg_query_count(t, dq, counts2, None)
        assert np.array_equal(from_dev(counts2, np.uint32).astype(np.uint64), want)
        jt = torch.full((1,), -1, dtype=torch.int64, device="cuda")
        hg.hg_join_count(t, dq, jt)
        assert int(from_dev(jt, np.uint64)[0]) == ref.join_count(queries)
        if check_gather and v is not None:
            offs = torch.empty(queries.size + 1, dtype=torch.int64, device="cuda")
            n_total = int(want.sum())
            outv = torch.empty(max(n_total, 1), dtype=torch.int32, device="cuda")
            got_total = hg.hg_query_gather(t, dq, offs, outv)
            assert got_total == n_total
            ro, rv = ref.query_gather(queries)
            assert_same_gather(from_dev(offs, np.uint64), from_dev(outv, np.uint32)[:n_total], ro, rv)
        hg.hg_sync(t)


@pytest.mark.parametrize("B", [1 << 16, 65537, 1, 1000])
def test_plain_uniform_u32(hg, B):
    wl = W.plain_uniform(100003, 70001, num_buckets=B)
    _run_all(hg, wl.keys, B, 0, wl.queries, flags=hg.HG_INDEX_VALUES, check_gather=B != 1)


def test_plain_uniform_small_config_full_size(hg):
    # the small configuration at its stated size: 2^20 keys, 2^20 buckets, 2^20 queries, 50% hits
    wl = W.plain_uniform(1 << 20, 1 << 20)
    _run_all(hg, wl.keys, 1 << 20, 0, wl.queries, flags=hg.HG_INDEX_VALUES)


@pytest.mark.parametrize("seed", [0, 0xDEADBEEF12345])
def test_seeded_hash(hg, seed):
    wl = W.plain_uniform(50001, 40001, num_buckets=4093, salt=3)
    _run_all(hg, wl.keys, 4093, seed, wl.queries)


def test_zipf_duplicates_long_buckets(hg):
    # top value ~ 2^20 / H(2^14) ~ 1e5 copies: exercises the chunked long-bucket path
    wl = W.zipf_large(n=1 << 20, num_buckets=1 << 19, q=1 << 17, M=1 << 14)
    _run_all(hg, wl.keys, 1 << 19, 0, wl.queries, flags=hg.HG_INDEX_VALUES)


def test_join_kv_u64_values(hg):
    wl = W.join_kv(n=(1 << 17) + 3, num_buckets=1 << 16, q=(1 << 16) + 5)
    _run_all(hg, wl.keys, 1 << 16, 0, wl.queries, values=wl.values)


def test_u64_non_power_of_two_buckets(hg):
    wl = W.join_kv(n=90001, num_buckets=99991, q=70003, salt=2)
    _run_all(hg, wl.keys, 99991, 7, wl.queries, values=wl.values)


def test_all_duplicates_one_bucket(hg):
    keys = np.full(300001, 0xFFFFFFFF, dtype=np.uint32)
    keys[::7] = 0
    queries = np.array([0xFFFFFFFF, 0, 1, 0xFFFFFFFF] * 21, dtype=np.uint32)
    _run_all(hg, keys, 1 << 12, 0, queries, flags=hg.HG_INDEX_VALUES)


def test_long_buckets_repeated_queries(hg):
    """Every bucket is long (4 buckets, ~2^14 keys each); the queries repeat
    20000 distinct keys one to four times in shuffled order, more distinct keys
    than the long-bucket walk groups at once, so both the grouped walks and the
    per-entry walks are taken."""
    rng = np.random.default_rng(77)
    keys = rng.integers(0, 1 << 14, size=(1 << 16) + 9, dtype=np.uint32)
    distinct = rng.permutation(np.arange(1 << 15, dtype=np.uint32))[:20000]
    queries = np.repeat(distinct, rng.integers(1, 5, size=distinct.size))
    rng.shuffle(queries)
    _run_all(hg, keys, 4, 3, queries, flags=hg.HG_INDEX_VALUES)


def test_sequential_keys(hg):
    keys = np.arange(1, (1 << 18) + 1, dtype=np.uint32)
    queries = np.arange(0, 1 << 18, 3, dtype=np.uint32)
    _run_all(hg, keys, 1 << 18, 0, queries, flags=hg.HG_INDEX_VALUES)


def test_empty_inputs(hg):
    empty = np.empty(0, dtype=np.uint32)
    q = np.array([1, 2, 3], dtype=np.uint32)
    _run_all(hg, empty, 64, 0, q, flags=hg.HG_INDEX_VALUES)
    wl = W.plain_uniform(1000, 10)
    _run_all(hg, wl.keys, 1024, 0, empty, flags=hg.HG_INDEX_VALUES)


@pytest.mark.parametrize("koff,qoff", [(1, 3), (2, 1), (3, 2)])
def test_unaligned_inputs(hg, koff, qoff):
    wl = W.plain_uniform(20011, 30011, num_buckets=8192, salt=5)
    keys = wl.keys[koff:]
    queries = wl.queries[qoff:]
    ref = oracle.build_table(keys, 8192, 0)
    dk_full = to_dev(wl.keys)
    dq_full = to_dev(wl.queries)
    for flags in (hg.HG_PLAIN_BUILD, hg.HG_PARTITION_BUILD):
        with hg.hg_build(dk_full[koff:], 8192, 0, flags=flags) as t:
            o, k, v = table_arrays(hg, t, np.uint32)
            assert_same_table(o, k, v, ref)
            counts = torch.empty(queries.size, dtype=torch.int32, device="cuda")
            hg.hg_query_count(t, dq_full[qoff:], counts)
            assert np.array_equal(from_dev(counts, np.uint32).astype(np.uint64), ref.query_count(queries))


def _inv_fmix32(h):
    M = 1 << 32
    h ^= h >> 16
    h = (h * pow(0xC2B2AE35, -1, M)) % M
    h ^= (h >> 13) ^ (h >> 26)
    h = (h * pow(0x85EBCA6B, -1, M)) % M
    h ^= h >> 16
    return h


@pytest.mark.parametrize("B", [3, 7, 65537, 99991, 1000003, 12345679, (1 << 26) - 5])
def test_remainder_boundaries(hg, B):
    # keys whose hash is exactly at the edges of the remainder (0, B-1, B, the last
    # full multiple of B below 2^32, 2^32-1): the kernel's remainder must equal '%'
    M = 1 << 32
    last = (M // B) * B
    targets = {0, 1, B - 1, B, B + 1, 2 * B - 1, last - 1, last, M - 1, M - 2, M - B, (M - 1) // 2}
    targets = sorted(t for t in targets if 0 <= t < M)
    keys = [_inv_fmix32(h) for h in targets]
    assert [oracle.fmix32(k) for k in keys] == targets
    rng = np.random.default_rng(B)
    extra = rng.integers(0, M, size=5000, dtype=np.uint64).astype(np.uint32)
    all_keys = np.concatenate([np.array(keys * 3, dtype=np.uint32), extra])
    _run_all(hg, all_keys, B, 0, all_keys[::2].copy(), flags=hg.HG_INDEX_VALUES)


def test_gather_capacity_two_call_pattern(hg):
    wl = W.plain_uniform(10000, 5000, num_buckets=10000, hit=0.9)
    ref = oracle.build_table(wl.keys, 10000, 0, index_values=True)
    want = int(ref.query_count(wl.queries).sum())
    with hg.hg_build(to_dev(wl.keys), 10000, 0, flags=hg.HG_INDEX_VALUES) as t:
        dq = to_dev(wl.queries)
        offs = torch.empty(wl.queries.size + 1, dtype=torch.int64, device="cuda")
        small = torch.empty(10, dtype=torch.int32, device="cuda")
        with pytest.raises(hg.HashGraphError) as ei:
            hg.hg_query_gather(t, dq, offs, small)
        assert ei.value.status == hg.HG_ERR_CAPACITY and ei.value.total == want
        ro, _ = ref.query_gather(wl.queries)
        assert np.array_equal(from_dev(offs, np.uint64), ro)


def test_gather_without_values_is_rejected(hg):
    wl = W.plain_uniform(1000, 100)
    with hg.hg_build(to_dev(wl.keys), 1024, 0) as t:
        offs = torch.empty(101, dtype=torch.int64, device="cuda")
        with pytest.raises(hg.HashGraphError) as ei:
            hg.hg_query_gather(t, to_dev(wl.queries), offs, None)
        assert ei.value.status == hg.HG_ERR_NO_VALUES


def test_build_modes_agree(hg):
    # the direct Algorithm 1 build and the partitioned build give the same table
    wl = W.zipf_large(n=(1 << 20) + 7, num_buckets=(1 << 20) - 3, q=1 << 10, M=1 << 16)
    ref = oracle.build_table(wl.keys, (1 << 20) - 3, 0, index_values=True)
    for flags in (hg.HG_PLAIN_BUILD, hg.HG_PARTITION_BUILD, 0):
        with hg.hg_build(to_dev(wl.keys), (1 << 20) - 3, 0, flags=flags | hg.HG_INDEX_VALUES) as t:
            o, k, v = table_arrays(hg, t, np.uint32)
            assert_same_table(o, k, v, ref)


def test_two_pass_partition_with_hot_buckets(hg):
    # 2^21 + 5 buckets: 257 bins, so both partition passes run; Zipf keys put
    # tens of thousands of copies in single buckets (big bins, hot buckets)
    B = (1 << 21) + 5
    wl = W.zipf_large(n=(1 << 21) + 3, num_buckets=B, q=1 << 16, M=1 << 15, salt=4)
    _run_all(hg, wl.keys, B, 0, wl.queries, flags=hg.HG_INDEX_VALUES, check_gather=False)


@pytest.mark.parametrize("case", ["u64_values", "u64", "u32_values"])
def test_partition_bins_larger_than_the_stage(hg, case):
    # 64 bins of ~16,400 nearly distinct keys: more than the bin sort's staging
    # buffer holds for these widths, and no threshold on bucket size leaves few
    # enough keys to stage, so every key is placed straight at its bucket's
    # cursor; a few hot keys add buckets of 64 or more keys
    B = (1 << 19) + 3
    if case == "u32_values":
        wl = W.plain_uniform((1 << 20) + 7, 1 << 14, num_buckets=B, salt=21)
        keys, vals = wl.keys.copy(), np.arange(wl.keys.size, dtype=np.uint32)
        keys[::4099] = keys[11]
        keys[5::8191] = keys[13]
    else:
        wl = W.join_kv(n=(1 << 20) + 7, num_buckets=B, q=1 << 14, salt=22)
        keys, vals = wl.keys.copy(), (wl.values if case == "u64_values" else None)
        keys[::4099] = keys[11]
    _run_all(hg, keys, B, 0, wl.queries, values=vals, check_gather=False, modes=("partition",))


def test_partition_u64_values_many_bins(hg):
    B = 1 << 23
    wl = W.join_kv(n=1 << 22, num_buckets=B, q=1 << 15, salt=6)
    _run_all(hg, wl.keys, B, 0, wl.queries, values=wl.values, check_gather=False, modes=("partition",))


def test_partition_many_hot_buckets_in_one_bin(hg):
    # more hot buckets in one bin than the staging map holds: the fallback path
    rng = np.random.default_rng(3)
    vals = rng.integers(0, 2**32, size=400, dtype=np.uint64).astype(np.uint32)
    keys = np.repeat(vals, 80)
    rng.shuffle(keys)
    _run_all(hg, keys, 4096, 0, vals[::3].copy(), flags=hg.HG_INDEX_VALUES, check_gather=False)


def _probe_only(hg, keys, B, queries, values=None):
    """Counts, total and join against the oracle (no gather), default build."""
    ref = oracle.build_table(keys, B, 0, values=values)
    want = ref.query_count(queries)
    with hg.hg_build(to_dev(keys), B, 0, values=None if values is None else to_dev(values)) as t:
        dq = to_dev(queries)
        counts = torch.empty(queries.size, dtype=torch.int32, device="cuda")
        total = torch.empty(1, dtype=torch.int64, device="cuda")
        hg.hg_query_count(t, dq, counts, total)
        assert np.array_equal(from_dev(counts, np.uint32).astype(np.uint64), want)
        assert int(from_dev(total, np.uint64)[0]) == int(want.sum())
        jt = torch.empty(1, dtype=torch.int64, device="cuda")
        hg.hg_join_count(t, dq, jt)
        assert int(from_dev(jt, np.uint64)[0]) == int(want.sum())
        hg.hg_sync(t)


def test_grouped_probe_zipf_u32_two_passes(hg):
    # table > 48 MB (not L2-resident): queries are grouped by table bin in two
    # partition passes, probed bin by bin, and the counts return to slot order
    wl = W.zipf_large(n=(1 << 23) + 11, num_buckets=1 << 23, q=(1 << 21) + 3, M=1 << 18, salt=8)
    _probe_only(hg, wl.keys, 1 << 23, wl.queries)


@pytest.mark.parametrize("B", [1 << 23, (1 << 23) - 9])
def test_grouped_hash_join_bins(hg, B):
    # 1024 bins of ~8192 Zipf keys (at most a few hundred distinct each): the
    # grouped probe counts each bin through a shared-memory table of its
    # distinct keys (B = 2^23: a word per bucket; otherwise double hashing).
    # Bins 3, 7 and 500 get ~4000 extra distinct keys, more than the table
    # takes, and fall back to the walking probe; the keys 0 and 2^32 - 1 (the
    # table's empty marker) occur many times.
    wl = W.zipf_large(n=(1 << 23) + 11, num_buckets=B, q=(1 << 21) + 3, M=1 << 18, salt=13)
    keys = wl.keys.copy()
    keys[::97] = 0xFFFFFFFF
    keys[5::101] = 0
    rng = np.random.default_rng(14)
    extra = rng.integers(0, 1 << 32, size=1 << 22, dtype=np.uint64).astype(np.uint32)
    extra = extra[np.isin(oracle.buckets(extra, B, 0) >> 13, [3, 7, 500])][:12000]
    keys = np.concatenate([keys, extra])
    queries = wl.queries.copy()
    queries[::50] = 0xFFFFFFFF
    queries[7::51] = 0
    queries[: extra.size] = extra
    _probe_only(hg, keys, B, queries)


def _fmix32_inv(h: np.ndarray) -> np.ndarray:
    """Keys with the given MurmurHash3 fmix32 values (seed 0): the finaliser's
    steps undone in reverse order (its multipliers' inverses mod 2^32)."""
    h = h.astype(np.uint64)
    m = np.uint64(0xFFFFFFFF)
    h ^= h >> np.uint64(16)
    h = (h * np.uint64(0x7ED1B41D)) & m
    h ^= (h >> np.uint64(13)) ^ (h >> np.uint64(26))
    h = (h * np.uint64(0xA5CB9243)) & m
    h ^= h >> np.uint64(16)
    return h.astype(np.uint32)


def test_grouped_hash_join_shared_buckets(hg):
    # B = 2^23: the hash join keeps a word per bucket, and a bucket's second and
    # later distinct keys go to overflow words.  Keys built from chosen hashes
    # put 2 to 4 distinct keys (1 to 5 copies each) into 60 buckets of each of
    # bins 10..13, and queries hit each of them and miss with other tags in
    # the same buckets.
    B = 1 << 23
    wl = W.zipf_large(n=(1 << 23) + 11, num_buckets=B, q=(1 << 21) + 3, M=1 << 18, salt=16)
    rng = np.random.default_rng(17)
    hashes, copies, misses = [], [], []
    for p in range(10, 14):
        for j in rng.choice(8192, size=60, replace=False):
            tags = rng.choice(512, size=6, replace=False)
            nd = int(rng.integers(2, 5))
            for t in tags[:nd]:
                hashes.append((int(t) << 23) | (p << 13) | int(j))
                copies.append(int(rng.integers(1, 6)))
            misses += [(int(t) << 23) | (p << 13) | int(j) for t in tags[nd:]]
    built = _fmix32_inv(np.array(hashes, dtype=np.uint64))
    assert np.array_equal(oracle.buckets(built, B, 0), np.array(hashes, dtype=np.uint64) & np.uint64(B - 1))
    keys = np.concatenate([wl.keys, np.repeat(built, copies)])
    keys = keys[rng.permutation(keys.size)]
    queries = wl.queries.copy()
    probe = np.concatenate([built, _fmix32_inv(np.array(misses, dtype=np.uint64))])
    queries[: probe.size] = probe
    queries[probe.size: 2 * probe.size] = probe
    _probe_only(hg, keys, B, queries)


def test_grouped_uniform_keys_hash_join_gives_up(hg):
    # 1024 bins of ~8192 distinct keys each, more than the hash join's table
    # takes: the first bins overflow, the rest are not tried, and every bin is
    # answered by the walking probe
    wl = W.plain_uniform((1 << 23) + 3, (1 << 21) + 9, num_buckets=1 << 23, salt=15)
    _probe_only(hg, wl.keys, 1 << 23, wl.queries)


def test_large_table_few_bins(hg):
    # 2^20 buckets = 128 bins, fewer than the probe's CTAs: the direct probe answers
    # a table larger than L2 (grouping needs several bins per SM)
    wl = W.plain_uniform((1 << 24) + 5, (1 << 20) + 7, num_buckets=1 << 20, salt=12)
    _probe_only(hg, wl.keys, 1 << 20, wl.queries)


def test_grouped_probe_u64(hg):
    wl = W.join_kv(n=(1 << 22) + (1 << 20), num_buckets=(1 << 23) - 9, q=(1 << 21) + 1, salt=10)
    _probe_only(hg, wl.keys, (1 << 23) - 9, wl.queries, values=wl.values)


@pytest.mark.parametrize("dup_log2", [0, 3, 6, 9, 12])
def test_duplicate_key_sweep(hg, dup_log2):
    """The duplicate-key experiment's inputs: every value about 2^d times, B = N / 2^d."""
    wl = W.duplicate_keys((1 << 16) + 5, dup_log2=dup_log2, q=(1 << 14) + 3, salt=dup_log2)
    _run_all(hg, wl.keys, wl.num_buckets, 0, wl.queries, check_gather=False)


@pytest.mark.parametrize("case", ["zipf", "dup9", "one_bucket", "medium_buckets", "u64_values"])
def test_sorted_buckets(hg, case):
    """HG_SORTED_BUCKETS: same table contents and counts; buckets up to the limit ascending."""
    if case == "zipf":
        wl = W.zipf_large(n=1 << 20, num_buckets=1 << 19, q=1 << 17, M=1 << 14, salt=40)
        _run_all(hg, wl.keys, 1 << 19, 0, wl.queries, flags=hg.HG_SORTED_BUCKETS | hg.HG_INDEX_VALUES)
    elif case == "dup9":
        wl = W.duplicate_keys((1 << 16) + 5, dup_log2=9, q=(1 << 14) + 3, salt=41)
        _run_all(hg, wl.keys, wl.num_buckets, 0, wl.queries, flags=hg.HG_SORTED_BUCKETS)
    elif case == "one_bucket":   # longer than the limit: left in build order, walked
        wl = W.plain_uniform(100003, 20001, num_buckets=1, salt=42)
        _run_all(hg, wl.keys, 1, 0, wl.queries, flags=hg.HG_SORTED_BUCKETS)
    elif case == "medium_buckets":  # ~14,000 keys per bucket, bitonic-sorted in shared memory
        rng = np.random.default_rng(43)
        keys = rng.integers(0, 3000, size=100003, dtype=np.uint32)
        keys[::11] = 0xFFFFFFFF  # the largest key value, equal to the sort's padding
        queries = np.concatenate([keys[:5000], rng.integers(0, 1 << 32, size=3000, dtype=np.uint64).astype(np.uint32)])
        _run_all(hg, keys, 7, 5, queries, flags=hg.HG_SORTED_BUCKETS | hg.HG_INDEX_VALUES)
    else:
        wl = W.join_kv(n=(1 << 17) + 3, num_buckets=1 << 12, q=(1 << 15) + 5, salt=44)
        _run_all(hg, wl.keys, 1 << 12, 0, wl.queries, values=wl.values, flags=hg.HG_SORTED_BUCKETS)
