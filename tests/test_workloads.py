"""Checks of the seeded input generators (not of the hash table)."""
import os

import numpy as np

import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_published_outputs():
    with open(os.path.join(GOLDEN, "splitmix64_vectors.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    for i, v in rows:
        assert W.splitmix64_at(0, int(i)) == int(v, 16)


def test_generators_are_deterministic_and_thread_count_independent():
    s = W.stream("keys")
    a = W.uniform_u32(s, 300001)
    W._load().hgw_set_threads(1)
    try:
        b = W.uniform_u32(s, 300001)
    finally:
        W._load().hgw_set_threads(0)
    assert np.array_equal(a, b)
    assert a[7] == (W.splitmix64_at(s, 7) >> 32)
    assert W.uniform_u64(s, 5)[3] == W.splitmix64_at(s, 3)


def test_probe_mix_hit_rate_and_membership():
    wl = W.plain_uniform(1 << 16, 1 << 16)
    keyset = set(wl.keys.tolist())
    hits = np.fromiter((q in keyset for q in wl.queries.tolist()), dtype=bool)
    assert abs(hits.mean() - 0.5) < 0.02


def test_zipf_guided_search_equals_plain_search():
    M = 1 << 16
    zt = W.ZipfTable(M)
    S = zt.S
    rng = np.random.default_rng(1)
    for x in rng.integers(0, 2**64, size=2000, dtype=np.uint64).tolist() + [0, 2**64 - 1]:
        u = (x >> 11) * (1.0 / 9007199254740992.0)
        t = u * S[M]
        want = int(np.searchsorted(S[1:], t, side="right")) + 1
        want = min(want, M)
        assert zt.rank_of(x) == want


def test_zipf_frequencies_follow_one_over_rank():
    M = 1 << 12
    zt = W.ZipfTable(M)
    n = 1 << 20
    vals = zt.values(W.stream("keys"), n)
    inv = {W.rank_value(r): r for r in range(1, 65)}
    counts = np.zeros(65)
    u, c = np.unique(vals, return_counts=True)
    for v, k in zip(u.tolist(), c.tolist()):
        if v in inv:
            counts[inv[v]] = k
    H = zt.S[M]
    for r in (1, 2, 4, 16, 64):
        expect = n / (r * H)
        assert abs(counts[r] - expect) < 6 * np.sqrt(expect), r


def test_zipf_queries_hits_present_misses_absent():
    M = 1 << 12
    wl = W.zipf_large(n=1 << 16, num_buckets=1 << 15, q=1 << 16, M=M)
    present = {W.rank_value(r) for r in range(1, M + 1)}
    isin = np.fromiter((q in present for q in wl.queries.tolist()), dtype=bool)
    assert abs(isin.mean() - 0.7) < 0.02
    assert set(wl.keys.tolist()) <= present


def test_zipf_weighted_queries_follow_the_key_law():
    M, q = 1 << 10, 1 << 18
    wl = W.zipf_weighted(n=1 << 16, num_buckets=1 << 15, q=q, M=M)
    zt = W.zipf_table(M)
    H = zt.S[M]
    vals, counts = np.unique(wl.queries, return_counts=True)
    freq = dict(zip(vals.tolist(), counts.tolist()))
    present = {W.rank_value(r) for r in range(1, M + 1)}
    hits = sum(c for v, c in freq.items() if v in present)
    assert abs(hits / q - 0.7) < 0.01
    for r in (1, 2, 3, 8, 32):
        expect = 0.7 * q / (r * H)
        got = freq.get(W.rank_value(r), 0)
        assert abs(got - expect) < 6 * np.sqrt(expect), r
    # the same keys as zipf_large, and misses never occur among them
    assert np.array_equal(wl.keys, W.zipf_large(n=1 << 16, num_buckets=1 << 15, q=16, M=M).keys)
    # hits are drawn from their own stream: the Bernoulli draws match zipf_large's
    ul = W.zipf_large(n=1 << 16, num_buckets=1 << 15, q=q, M=M).queries
    assert np.array_equal(np.isin(ul, list(present)), np.isin(wl.queries, list(present)))


def test_join_probe_structure():
    wl = W.join_kv(n=1 << 18, num_buckets=1 << 17, q=1 << 14)
    q = wl.queries
    assert q.size == 1 << 14
    u, c = np.unique(q, return_counts=True)
    hot = int(0.05 * q.size) // 8
    # a hot key that hits may coincide with other probe keys that hit the same build key
    assert hot * 0.9 <= (c >= 8).sum() <= hot + 2
    keyset = set(wl.keys.tolist())
    singles = u[c == 1]
    frac = np.mean([k in keyset for k in singles.tolist()])
    assert abs(frac - 0.5) < 0.05
    assert wl.values.dtype == np.uint32 and wl.values.size == wl.keys.size


def test_batched_uniform_recipe():
    b = W.batched_uniform(200, 8, 20, salt=1)
    sizes = np.diff(b.key_offsets.astype(np.int64))
    assert sizes.min() >= 2 ** 8 and sizes.max() <= 2 ** 20
    assert np.array_equal(b.num_buckets.astype(np.int64), sizes)          # B_t = N_t
    assert np.array_equal(b.query_offsets, b.key_offsets)                  # N_t queries per table
    # log-uniform: about half the tables fall below the geometric midpoint 2^14
    assert 0.35 < np.mean(sizes < 2 ** 14) < 0.65
    # deterministic, and each table's keys come from its own stream
    again = W.batched_uniform(200, 8, 20, salt=1)
    assert np.array_equal(again.keys, b.keys) and np.array_equal(again.queries, b.queries)
    k0, _, _ = b.table(0)
    k1, _, _ = b.table(1)
    assert not np.array_equal(k0[:16], k1[:16])


def test_duplicate_keys_recipe():
    wl = W.duplicate_keys(1 << 16, dup_log2=5, salt=2)
    V = (1 << 16) >> 5
    assert wl.num_buckets == V and wl.keys.max() < V
    # every value occurs about 2^5 times
    occ = np.bincount(wl.keys, minlength=V)
    assert abs(occ.mean() - 32) < 1e-9 and occ.min() > 5
    hits = wl.queries < V
    assert 0.45 < hits.mean() < 0.55
    assert np.all(wl.queries[~hits] >= V)  # misses are absent values
