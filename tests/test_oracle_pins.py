"""Pins for the CPU oracle: each check compares the oracle with something
other than itself -- published hash vectors, brute force, sorting, or the
CSR invariants of Algorithm 1 -- so that a dropped term, a wrong index or a
swapped operand in ``oracle/hg_oracle.c`` fails at least one of them."""
import os

import numpy as np
import pytest

import oracle
from tests.murmur3_ref import murmur3_x64_128, murmur3_x86_32, smhasher_verification

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _murmur_rows():
    rows = []
    with open(os.path.join(GOLDEN, "murmur3_vectors.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append(line.split())
    return rows


# ---------------------------------------------------------------- hashing --

def test_fmix32_through_published_murmur3_x86_32_vectors():
    rows = [r for r in _murmur_rows() if r[0] == "x86_32"]
    assert len(rows) >= 9
    for _, data, seed, expect in rows:
        data = b"" if data == "-" else bytes.fromhex(data)
        got = murmur3_x86_32(data, int(seed, 16), oracle.fmix32)
        assert got == int(expect, 16), (data, seed)


def test_fmix32_fmix64_smhasher_verification():
    rows = {r[1]: int(r[2], 16) for r in _murmur_rows() if r[0] == "smhasher"}
    v32 = smhasher_verification(
        lambda d, s: murmur3_x86_32(d, s, oracle.fmix32).to_bytes(4, "little"), 4)
    assert v32 == rows["MurmurHash3_x86_32"]
    v128 = smhasher_verification(lambda d, s: murmur3_x64_128(d, s, oracle.fmix64), 16)
    assert v128 == rows["MurmurHash3_x64_128"]


def test_fmix_is_bijective_on_samples():
    # fmix is a composition of invertible steps; distinct inputs give distinct outputs.
    xs = np.arange(0, 1 << 16, dtype=np.uint64) * np.uint64(0x10001)
    h32 = {oracle.fmix32(int(x) & 0xFFFFFFFF) for x in xs}
    assert len(h32) == len({int(x) & 0xFFFFFFFF for x in xs})
    h64 = {oracle.fmix64(int(x) * 0x9E3779B97F4A7C15 & ((1 << 64) - 1)) for x in xs[:4096]}
    assert len(h64) == 4096


# Published MurmurHash3_x86_32 values of the empty input: fmix32(s).
FMIX32_1 = 0x514E28B7
FMIX32_FFFFFFFF = 0x81F16F39


@pytest.mark.parametrize("B", [1 << 32, 1 << 16, 1000003, 7, 1])
def test_bucket_u32_special_cases(B):
    # bucket(k) = fmix32(k ^ seed) mod B; with k ^ seed in {0, 1, 0xFFFFFFFF}
    # the hash is a published vector, so the bucket is that value mod B.
    keys = np.array([1, 0xFFFFFFFF, 0, 3], dtype=np.uint32)
    got = oracle.buckets(keys, B, seed=0)
    assert list(got[:3]) == [FMIX32_1 % B, FMIX32_FFFFFFFF % B, 0]
    # The seed enters by XOR: 3 ^ 2 = 1 (3 + 2 would be 5).
    got = oracle.buckets(np.array([3, 0xFFFFFFFD], dtype=np.uint32), B, seed=2)
    assert list(got) == [FMIX32_1 % B, FMIX32_FFFFFFFF % B]
    # Only the low 32 bits of the seed act on 32-bit keys.
    got = oracle.buckets(np.array([3], dtype=np.uint32), B, seed=(5 << 32) | 2)
    assert list(got) == [FMIX32_1 % B]


def test_bucket_u64_composition():
    # fmix64 is pinned by the SMHasher value above; a 64-bit key's bucket must
    # use all 64 bits of key and seed, and a 64-bit remainder.
    rng = np.random.default_rng(7)
    keys = rng.integers(0, 2**64, size=64, dtype=np.uint64)
    for B in (1 << 26, 1000003, (1 << 40) + 15):
        for seed in (0, 0x123456789ABCDEF):
            got = oracle.buckets(keys, B, seed=seed)
            want = [oracle.fmix64(int(k) ^ seed) % B for k in keys]
            assert [int(g) for g in got] == want
    # keys differing only in the high half land in different buckets
    hi = np.array([1 << 40, 2 << 40], dtype=np.uint64)
    assert len(set(oracle.buckets(hi, 1 << 26).tolist())) == 2
    assert oracle.buckets(np.array([5], dtype=np.uint64), 1 << 26, seed=5)[0] == 0


# ------------------------------------------------------------------ build --

def _check_csr(keys, B, seed, table, values=None, index_values=False):
    n = keys.size
    off = table.offsets.astype(np.int64)
    assert off.size == B + 1
    assert off[0] == 0 and off[-1] == n
    assert np.all(np.diff(off) >= 0)
    # independent recount of bucket sizes (numpy bincount)
    b = oracle.buckets(keys, B, seed).astype(np.int64)
    assert np.array_equal(np.diff(off), np.bincount(b, minlength=B))
    # every stored key lies in its own bucket's segment
    seg = np.repeat(np.arange(B), np.diff(off))
    assert np.array_equal(oracle.buckets(table.keys, B, seed).astype(np.int64), seg)
    # multiset of keys preserved
    assert np.array_equal(np.sort(table.keys), np.sort(keys))
    if values is not None or index_values:
        src_vals = values if values is not None else np.arange(n, dtype=np.uint32)
        # (key, value) pairs preserved: sort by key then value on both sides
        oi = np.lexsort((src_vals, keys))
        oo = np.lexsort((table.values, table.keys))
        assert np.array_equal(keys[oi], table.keys[oo])
        assert np.array_equal(src_vals[oi], table.values[oo])
    if index_values:
        # the oracle's scatter is a sequential loop: input order inside a bucket
        for bb in range(B):
            s = table.values[off[bb]:off[bb + 1]].astype(np.int64)
            assert np.all(np.diff(s) > 0)
            assert np.all(b[s] == bb)


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
@pytest.mark.parametrize("n,B,seed", [(0, 1, 0), (1, 1, 0), (5, 3, 0), (1000, 1000, 0), (1000, 997, 1),
                                      (4096, 16, 12345), (777, 2048, 0)])
def test_build_invariants(dtype, n, B, seed):
    rng = np.random.default_rng(n * 31 + B)
    if dtype == np.uint32:
        keys = rng.integers(0, 2**32, size=n, dtype=np.uint64).astype(np.uint32)
    else:
        keys = rng.integers(0, 2**64, size=n, dtype=np.uint64)
    if n > 10:
        keys[: n // 4] = keys[n // 2]  # heavy duplicates
        keys[-3:] = [0, np.iinfo(dtype).max, 0]
    t = oracle.build_table(keys, B, seed, index_values=True)
    _check_csr(keys, B, seed, t, index_values=True)


def test_build_with_values_and_edge_keys():
    keys = np.array([0, 0xFFFFFFFF, 0, 7, 7, 7, 0xFFFFFFFF, 12, 3, 74, 6, 99], dtype=np.uint32)
    vals = np.arange(100, 100 + keys.size, dtype=np.uint32)
    for B in (1, 2, 5, 12, 64):
        t = oracle.build_table(keys, B, 0, values=vals)
        _check_csr(keys, B, 0, t, values=vals)


def test_build_all_duplicates_single_bucket():
    keys = np.full(3000, 0xDEADBEEF, dtype=np.uint32)
    t = oracle.build_table(keys, 1 << 10, 0, index_values=True)
    b = int(oracle.buckets(keys[:1], 1 << 10)[0])
    assert t.offsets[b + 1] - t.offsets[b] == 3000
    assert np.array_equal(t.values, np.arange(3000, dtype=np.uint32))


def test_build_sequential_keys():
    # the paper's sequential-key experiment: keys 1..2^k
    keys = np.arange(1, (1 << 14) + 1, dtype=np.uint32)
    t = oracle.build_table(keys, 1 << 14, 0, index_values=True)
    _check_csr(keys, 1 << 14, 0, t, index_values=True)


# ------------------------------------------------------------------ probe --

def _brute_counts(keys, queries):
    return (queries[:, None] == keys[None, :]).sum(axis=1).astype(np.uint64)


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_count_matches_bruteforce(dtype):
    rng = np.random.default_rng(3)
    for n, q, B in [(0, 50, 1), (1, 20, 1), (300, 400, 256), (2000, 1500, 1999), (4096, 4096, 64)]:
        pool = rng.integers(0, 2**31, size=max(n // 3, 1), dtype=np.uint64).astype(dtype)
        keys = rng.choice(pool, size=n).astype(dtype)
        queries = np.concatenate([rng.choice(pool, size=q // 2),
                                  rng.integers(0, 2**31, size=q - q // 2, dtype=np.uint64).astype(dtype)])
        t = oracle.build_table(keys, B, 0)
        got = t.query_count(queries)
        assert np.array_equal(got, _brute_counts(keys, queries))
        assert t.join_count(queries) == int(got.sum())
        for j in range(0, q, max(q // 7, 1)):
            assert oracle.count_linear(keys, queries[j]) == got[j]


def test_count_matches_sorted_keys_at_larger_size():
    rng = np.random.default_rng(11)
    n = 1 << 18
    keys = (rng.zipf(1.3, size=n) % (1 << 20)).astype(np.uint32) * np.uint32(2654435761)
    queries = np.concatenate([keys[rng.integers(0, n, size=n // 2)],
                              rng.integers(0, 2**32, size=n // 2, dtype=np.uint64).astype(np.uint32)])
    t = oracle.build_table(keys, 1 << 17, 99)
    got = t.query_count(queries)
    s = np.sort(keys)
    want = np.searchsorted(s, queries, side="right") - np.searchsorted(s, queries, side="left")
    assert np.array_equal(got, want.astype(np.uint64))


def test_join_count_is_sum_of_products():
    rng = np.random.default_rng(5)
    keys = rng.integers(0, 500, size=20000, dtype=np.uint64)
    queries = rng.integers(0, 800, size=30000, dtype=np.uint64)
    t = oracle.build_table(keys, 4096, 17)
    uk, ck = np.unique(keys, return_counts=True)
    uq, cq = np.unique(queries, return_counts=True)
    common, ik, iq = np.intersect1d(uk, uq, return_indices=True)
    want = int((ck[ik].astype(np.int64) * cq[iq].astype(np.int64)).sum())
    assert t.join_count(queries) == want


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_gather_matches_sorted_pairs(dtype):
    rng = np.random.default_rng(21)
    n, q, B = 5000, 3000, 1024
    keys = rng.integers(0, 1500, size=n, dtype=np.uint64).astype(dtype)
    vals = rng.integers(0, 2**32, size=n, dtype=np.uint64).astype(np.uint32)
    queries = rng.integers(0, 3000, size=q, dtype=np.uint64).astype(dtype)
    t = oracle.build_table(keys, B, 4, values=vals)
    offs, got = t.query_gather(queries)
    order = np.lexsort((vals, keys))
    sk, sv = keys[order], vals[order]
    lo = np.searchsorted(sk, queries, side="left")
    hi = np.searchsorted(sk, queries, side="right")
    assert np.array_equal(np.diff(offs.astype(np.int64)), hi - lo)
    for j in range(q):
        seg = np.sort(got[offs[j]:offs[j + 1]])
        assert np.array_equal(seg, sv[lo[j]:hi[j]])


def test_gather_index_values_returns_input_positions():
    keys = np.array([5, 9, 5, 5, 2, 9], dtype=np.uint32)
    t = oracle.build_table(keys, 4, 0, index_values=True)
    offs, got = t.query_gather(np.array([5, 9, 1, 2], dtype=np.uint32))
    segs = [sorted(got[offs[j]:offs[j + 1]].tolist()) for j in range(4)]
    assert segs == [[0, 2, 3], [1, 5], [], [4]]


def test_empty_queries_and_empty_table():
    t = oracle.build_table(np.empty(0, dtype=np.uint32), 8, 0, index_values=True)
    assert list(t.offsets) == [0] * 9
    assert t.query_count(np.array([1, 2, 3], dtype=np.uint32)).tolist() == [0, 0, 0]
    assert t.query_count(np.empty(0, dtype=np.uint32)).size == 0
    offs, vals = t.query_gather(np.empty(0, dtype=np.uint32))
    assert offs.tolist() == [0] and vals.size == 0
