"""Seeded synthetic inputs for the HashGraph workloads.

This module generates the key and query arrays that both the CUDA path and
the CPU oracle consume.  It holds no hash-table arithmetic: only SplitMix64
streams and the recipes below (the C source is ``hg_workloads.c``; build it
with :func:`build`).

Recipes (master seed ``MASTER_SEED``; stream ids in ``STREAM``):

* ``plain_uniform`` -- N uniform 32-bit keys (high half of each SplitMix64
  output), Q queries of which a Bernoulli(``hit``) share are copies of a
  uniformly chosen build key and the rest fresh uniform values.  The paper's
  random-key experiments (Sec. 4.2) draw keys at random; its table size
  equals the key count (load factor C = 1, Sec. 4.3).
* ``zipf_large`` -- N 32-bit keys whose ranks follow Zipf(s=1) over 1..M,
  value = rank * 0x9E3779B1 mod 2^32; queries hit with probability ``hit``
  on a rank drawn uniformly from 1..M, misses use ranks above M (values that
  never occur among the keys).  This is the duplicate-key regime of the
  paper's Sec. 5.4 "Duplicate Keys" experiment.
* ``zipf_weighted`` -- the same keys, but a hit's rank follows the keys' own
  Zipf(1) law (stream ``q_rank``), so each value is queried in proportion to
  its multiplicity: the quadratic regime of the direct walk (Sec. 5.4).
* ``join_kv`` -- N (uint64 key, uint32 value) pairs, and a probe relation
  whose ``hot_frac`` share of slots holds ``rep`` copies each of hot keys;
  every distinct probe key is a build key with probability 1/2, else fresh;
  slots are Fisher-Yates shuffled.
* ``duplicate_keys`` -- the duplicate-key experiment (Sec. 5.4): N keys
  uniform over a value range of V = N / 2^d values, so every value occurs
  about 2^d times, with B = V buckets; queries hit (a uniform value of the
  range) with probability ``hit``, else miss (a value above the range).
* ``batched_uniform`` -- many independent tables: table t has
  N_t = round(2^(lo + (hi - lo) u_t)) keys (u_t uniform in [0, 1) from the
  ``sizes`` stream, so sizes are log-uniform), B_t = N_t buckets, and N_t
  queries, each table drawn like ``plain_uniform`` from its own streams.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "hg_workloads.c")
LIB = os.path.join(HERE, "libhg_workloads.so")
GPU_SRC = os.path.join(HERE, "hg_workloads_gpu.cu")
GPU_LIB = os.path.join(HERE, "libhg_workloads_gpu.so")

MASTER_SEED = 0x210400792
STREAM = {
    "keys": 1,
    "values": 2,
    "q_select": 3,
    "q_miss": 4,
    "shuffle": 5,
    "sizes": 6,
    "q_rank": 7,
}

_lib = None


def build(force: bool = False) -> str:
    """Compile the generator library with gcc (plain C, no arch-specific flags)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + ".tmp"
        subprocess.check_call([
            "gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-pthread",
            "-o", tmp, SRC,
        ])
        os.replace(tmp, LIB)
    return LIB


def build_gpu(force: bool = False) -> str:
    """Compile the device-side generators with nvcc (sm_103a)."""
    if force or not os.path.exists(GPU_LIB) or os.path.getmtime(GPU_LIB) < os.path.getmtime(GPU_SRC):
        tmp = GPU_LIB + ".tmp"
        nvcc = os.environ.get("NVCC") or "nvcc"
        if not os.path.exists(nvcc) and os.path.exists("/usr/local/cuda/bin/nvcc"):
            nvcc = "/usr/local/cuda/bin/nvcc"
        subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-Xcompiler", "-fPIC",
                               "-shared", "-cudart", "static", "-o", tmp, GPU_SRC])
        os.replace(tmp, GPU_LIB)
    return GPU_LIB


_gpu_lib = None


def _load_gpu():
    global _gpu_lib
    if _gpu_lib is None:
        build_gpu()
        L = ctypes.CDLL(GPU_LIB)
        u64, vp = ctypes.c_uint64, ctypes.c_void_p
        L.hgw_gpu_uniform_u32.argtypes = [u64, u64, vp, vp]
        L.hgw_gpu_probe_mix_uniform_u32.argtypes = [u64, u64, u64, u64, u64, u64, vp, vp]
        _gpu_lib = L
    return _gpu_lib


def gpu_uniform_u32(state: int, n: int, out_ptr: int, stream: int = 0) -> None:
    """Device copy of uniform_u32 written to the device pointer out_ptr (n elements)."""
    if _load_gpu().hgw_gpu_uniform_u32(state, n, out_ptr, stream) != 0:
        raise RuntimeError("hgw_gpu_uniform_u32 launch failed")


def gpu_probe_mix_uniform_u32(key_state: int, n_keys: int, q: int, hit: float, sel: int, miss: int, out_ptr: int,
                              stream: int = 0) -> None:
    """Device copy of probe_mix(uniform_u32(key_state, n_keys), q, hit, sel, miss)."""
    if _load_gpu().hgw_gpu_probe_mix_uniform_u32(key_state, n_keys, sel, miss, hit_threshold(hit), q, out_ptr,
                                                 stream) != 0:
        raise RuntimeError("hgw_gpu_probe_mix_uniform_u32 launch failed")


def _load():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB)
        u64, vp = ctypes.c_uint64, ctypes.c_void_p
        L.hgw_splitmix64_at.restype = u64
        L.hgw_splitmix64_at.argtypes = [u64, u64]
        L.hgw_stream.restype = u64
        L.hgw_stream.argtypes = [u64, u64]
        L.hgw_set_threads.argtypes = [ctypes.c_int]
        L.hgw_uniform_u32.argtypes = [u64, u64, vp]
        L.hgw_uniform_u64.argtypes = [u64, u64, vp]
        L.hgw_probe_mix_u32.argtypes = [vp, u64, u64, u64, u64, u64, vp]
        L.hgw_probe_mix_u64.argtypes = [vp, u64, u64, u64, u64, u64, vp]
        L.hgw_zipf_table.argtypes = [u64, vp, vp]
        L.hgw_zipf_guide_size.restype = u64
        L.hgw_zipf_values_u32.argtypes = [vp, vp, u64, u64, u64, vp]
        L.hgw_zipf_rank_of.restype = u64
        L.hgw_zipf_rank_of.argtypes = [vp, vp, u64, u64]
        L.hgw_rank_value.restype = ctypes.c_uint32
        L.hgw_rank_value.argtypes = [u64]
        L.hgw_zipf_queries_u32.argtypes = [u64, u64, u64, u64, u64, vp]
        L.hgw_zipf_weighted_queries_u32.argtypes = [vp, vp, u64, u64, u64, u64, u64, u64, vp]
        L.hgw_join_probe_u64.argtypes = [vp, u64, u64, u64, u64, u64, u64, u64, vp]
        _lib = L
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def stream(name: str, master: int = MASTER_SEED, salt: int = 0) -> int:
    """Stream state for a named purpose; ``salt`` separates per-table streams."""
    return _load().hgw_stream(master, STREAM[name] + (salt << 8))


def splitmix64_at(state: int, i: int) -> int:
    return _load().hgw_splitmix64_at(state, i)


def hit_threshold(p: float) -> int:
    """Integer threshold on the high 32 bits of a draw: hit iff (x >> 32) < thr."""
    return int(round(p * 2**32))


def uniform_u32(state: int, n: int) -> np.ndarray:
    out = np.empty(n, dtype=np.uint32)
    _load().hgw_uniform_u32(state, n, _ptr(out))
    return out


def uniform_u64(state: int, n: int) -> np.ndarray:
    out = np.empty(n, dtype=np.uint64)
    _load().hgw_uniform_u64(state, n, _ptr(out))
    return out


def probe_mix(keys: np.ndarray, q: int, hit: float, sel: int, miss: int) -> np.ndarray:
    keys = np.ascontiguousarray(keys)
    out = np.empty(q, dtype=keys.dtype)
    f = _load().hgw_probe_mix_u32 if keys.dtype == np.uint32 else _load().hgw_probe_mix_u64
    f(_ptr(keys), keys.size, sel, miss, hit_threshold(hit), q, _ptr(out))
    return out


class ZipfTable:
    """Partial harmonic sums S[0..M] and the guide table of the Zipf sampler."""

    def __init__(self, M: int):
        self.M = M
        self.S = np.empty(M + 1, dtype=np.float64)
        self.G = np.empty(_load().hgw_zipf_guide_size(), dtype=np.uint32)
        _load().hgw_zipf_table(M, _ptr(self.S), _ptr(self.G))

    def rank_of(self, x: int) -> int:
        return _load().hgw_zipf_rank_of(_ptr(self.S), _ptr(self.G), self.M, x)

    def values(self, state: int, n: int) -> np.ndarray:
        out = np.empty(n, dtype=np.uint32)
        _load().hgw_zipf_values_u32(_ptr(self.S), _ptr(self.G), self.M, state, n, _ptr(out))
        return out


def rank_value(r: int) -> int:
    return _load().hgw_rank_value(r)


@dataclass
class Workload:
    """Inputs of one build + probe job."""
    name: str
    keys: np.ndarray
    values: np.ndarray | None
    queries: np.ndarray
    num_buckets: int
    seed: int = 0

    @property
    def key_bytes(self) -> int:
        return self.keys.dtype.itemsize


def plain_uniform(n: int = 1 << 20, q: int = 1 << 20, num_buckets: int | None = None,
                  hit: float = 0.5, master: int = MASTER_SEED, salt: int = 0) -> Workload:
    keys = uniform_u32(stream("keys", master, salt), n)
    queries = probe_mix(keys, q, hit, stream("q_select", master, salt), stream("q_miss", master, salt))
    return Workload("plain_uniform", keys, None, queries, num_buckets if num_buckets else max(n, 1))


def zipf_queries(M: int, q: int, hit: float, master: int = MASTER_SEED, salt: int = 0) -> np.ndarray:
    out = np.empty(q, dtype=np.uint32)
    _load().hgw_zipf_queries_u32(M, stream("q_select", master, salt), stream("q_miss", master, salt),
                                 hit_threshold(hit), q, _ptr(out))
    return out


def zipf_weighted_queries(M: int, q: int, hit: float, master: int = MASTER_SEED, salt: int = 0) -> np.ndarray:
    zt = zipf_table(M)
    out = np.empty(q, dtype=np.uint32)
    _load().hgw_zipf_weighted_queries_u32(_ptr(zt.S), _ptr(zt.G), M, stream("q_select", master, salt),
                                          stream("q_miss", master, salt), stream("q_rank", master, salt),
                                          hit_threshold(hit), q, _ptr(out))
    return out


_ZIPF_CACHE: dict[int, ZipfTable] = {}


def zipf_table(M: int) -> ZipfTable:
    if M not in _ZIPF_CACHE:
        _ZIPF_CACHE[M] = ZipfTable(M)
    return _ZIPF_CACHE[M]


def zipf_large(n: int = 1 << 28, num_buckets: int = 1 << 27, q: int = 1 << 28, M: int = 1 << 24,
               hit: float = 0.7, master: int = MASTER_SEED, salt: int = 0) -> Workload:
    keys = zipf_table(M).values(stream("keys", master, salt), n)
    queries = zipf_queries(M, q, hit, master, salt)
    return Workload("zipf_large", keys, None, queries, num_buckets)


def zipf_weighted(n: int = 1 << 28, num_buckets: int = 1 << 27, q: int = 1 << 28, M: int = 1 << 24,
                  hit: float = 0.7, master: int = MASTER_SEED, salt: int = 0) -> Workload:
    keys = zipf_table(M).values(stream("keys", master, salt), n)
    queries = zipf_weighted_queries(M, q, hit, master, salt)
    return Workload("zipf_weighted", keys, None, queries, num_buckets)


def join_kv(n: int = 1 << 27, num_buckets: int = 1 << 26, q: int = 1 << 26, hot_frac: float = 0.05,
            rep: int = 8, master: int = MASTER_SEED, salt: int = 0) -> Workload:
    keys = uniform_u64(stream("keys", master, salt), n)
    values = (uniform_u64(stream("values", master, salt), n) >> np.uint64(32)).astype(np.uint32)
    hot = int(hot_frac * q) // rep
    probe = np.empty(q, dtype=np.uint64)
    _load().hgw_join_probe_u64(_ptr(keys), n, stream("q_select", master, salt), stream("q_miss", master, salt),
                               stream("shuffle", master, salt), q, hot, rep, _ptr(probe))
    return Workload("join_kv", keys, values, probe, num_buckets)


@dataclass
class BatchWorkload:
    """Inputs of a batch of independent tables, concatenated table by table."""
    name: str
    keys: np.ndarray            # uint32, all tables' keys
    key_offsets: np.ndarray     # uint64 [n_tables + 1]
    num_buckets: np.ndarray     # uint64 [n_tables]
    queries: np.ndarray         # uint32, all tables' queries
    query_offsets: np.ndarray   # uint64 [n_tables + 1]
    seed: int = 0

    @property
    def n_tables(self) -> int:
        return int(self.num_buckets.size)

    def table(self, t: int):
        """(keys, num_buckets, queries) of table t (views)."""
        k0, k1 = int(self.key_offsets[t]), int(self.key_offsets[t + 1])
        q0, q1 = int(self.query_offsets[t]), int(self.query_offsets[t + 1])
        return self.keys[k0:k1], int(self.num_buckets[t]), self.queries[q0:q1]


def batch_sizes(n_tables: int, lo_log2: float, hi_log2: float, master: int = MASTER_SEED, salt: int = 0) -> np.ndarray:
    """Log-uniform table sizes round(2^(lo + (hi - lo) u)), u = (draw >> 11) * 2^-53."""
    st = stream("sizes", master, salt)
    u = np.array([(splitmix64_at(st, t) >> 11) * 2.0 ** -53 for t in range(n_tables)], dtype=np.float64)
    return np.rint(np.power(2.0, lo_log2 + (hi_log2 - lo_log2) * u)).astype(np.uint64)


def batched_uniform(n_tables: int = 4096, lo_log2: float = 8, hi_log2: float = 20, hit: float = 0.5,
                    master: int = MASTER_SEED, salt: int = 0) -> BatchWorkload:
    sizes = batch_sizes(n_tables, lo_log2, hi_log2, master, salt)
    ko = np.zeros(n_tables + 1, dtype=np.uint64)
    ko[1:] = np.cumsum(sizes)
    keys = np.empty(int(ko[-1]), dtype=np.uint32)
    queries = np.empty(int(ko[-1]), dtype=np.uint32)
    for t in range(n_tables):
        tsalt = (salt << 16) + t + 1
        k0, k1 = int(ko[t]), int(ko[t + 1])
        keys[k0:k1] = uniform_u32(stream("keys", master, tsalt), k1 - k0)
        queries[k0:k1] = probe_mix(keys[k0:k1], k1 - k0, hit, stream("q_select", master, tsalt),
                                   stream("q_miss", master, tsalt))
    return BatchWorkload("batched_uniform", keys, ko, sizes.copy(), queries, ko.copy())


# ---------------------------------------------------------------- serving --
def served_table_bytes(n: int, num_buckets: int) -> int:
    """Device bytes a serving engine charges for a table (its keys, offsets and
    a little padding); the same accounting as the engine's."""
    return 4 * n + 4 * (num_buckets + 1) + 32


@dataclass
class ServeRequest:
    kind: str          # "build" or "probe"
    table: int         # table id (builds: the new table; probes: the target)
    size: int          # keys of a build, queries of a probe
    key_state: int     # the target table's key stream (uniform_u32)
    sel: int = 0       # probes: hit selection and miss streams (probe_mix)
    miss: int = 0
    gap: float = 0.0   # exponential(1) inter-arrival gap before this request


def serving_trace(n_requests: int = 200_000, build_frac: float = 0.3, build_log2=(10, 24), probe_log2=(8, 22),
                  hit: float = 0.6, budget_bytes: int = 100 * 10**9, master: int = MASTER_SEED,
                  salt: int = 0) -> list:
    """Request stream of the serving workload.  Each request is a build with
    probability build_frac (N log-uniform over 2^build_log2, B = N, keys
    uniform_u32 from the table's own stream) or else a probe (Q log-uniform
    over 2^probe_log2, hit fraction `hit` drawn from the target's keys) whose
    target is uniform over the tables resident at that point under an
    arrival-order LRU with the given budget (a build inserts its table and
    evicts least recently used ones until the budget holds; a probe marks its
    target used).  The first request is a build.  Gaps are exponential(1):
    divide by the arrival rate for Poisson arrivals."""
    from collections import OrderedDict
    st_kind = stream("sizes", master, (salt << 16) + 0xFFFF)
    out = []
    resident: "OrderedDict[int, int]" = OrderedDict()   # table -> bytes, LRU first
    res_list: list = []                                  # resident tables, for uniform picks
    pos: dict = {}                                       # table -> index in res_list
    info = {}                                            # table -> (n, key_state)
    used = 0
    next_table = 0
    for r in range(n_requests):
        x = splitmix64_at(st_kind, 3 * r)
        y = splitmix64_at(st_kind, 3 * r + 1)
        z = splitmix64_at(st_kind, 3 * r + 2)
        u_kind = (x >> 11) * 2.0 ** -53
        u_size = (y >> 11) * 2.0 ** -53
        gap = -np.log1p(-((z >> 11) * 2.0 ** -53))
        is_build = (r == 0) or not resident or u_kind < build_frac
        if is_build:
            lo, hi = build_log2
            n = int(round(2.0 ** (lo + (hi - lo) * u_size)))
            t = next_table
            next_table += 1
            ks = stream("keys", master, (salt << 24) + t + 1)
            need = served_table_bytes(n, n)
            while used + need > budget_bytes and resident:
                old_t, b = resident.popitem(last=False)
                used -= b
                i = pos.pop(old_t)
                last = res_list.pop()
                if last != old_t:
                    res_list[i] = last
                    pos[last] = i
            resident[t] = need
            pos[t] = len(res_list)
            res_list.append(t)
            used += need
            info[t] = (n, ks)
            out.append(ServeRequest("build", t, n, ks, gap=gap))
        else:
            lo, hi = probe_log2
            q = int(round(2.0 ** (lo + (hi - lo) * u_size)))
            t = res_list[(x & 0xFFFFFFFF) * len(res_list) >> 32]
            resident.move_to_end(t)
            n, ks = info[t]
            out.append(ServeRequest("probe", t, q, ks, sel=stream("q_select", master, (salt << 24) + (1 << 23) + r),
                                    miss=stream("q_miss", master, (salt << 24) + (1 << 23) + r), gap=gap))
    return out


def serve_table_n(trace: list) -> dict:
    """table id -> number of keys, from the trace's builds."""
    return {r.table: r.size for r in trace if r.kind == "build"}


def duplicate_keys(n: int = 1 << 26, dup_log2: int = 0, q: int | None = None, hit: float = 0.5,
                   master: int = MASTER_SEED, salt: int = 0) -> Workload:
    """N keys over V = N >> dup_log2 values (each value about 2^dup_log2 times), B = V."""
    q = n if q is None else q
    V = max(1, n >> dup_log2)
    raw = uniform_u32(stream("keys", master, salt), n).astype(np.uint64)
    keys = ((raw * np.uint64(V)) >> np.uint64(32)).astype(np.uint32)
    sel = uniform_u64(stream("q_select", master, salt), q)
    hits = (sel >> np.uint64(32)) < np.uint64(hit_threshold(hit))
    low = sel & np.uint64(0xFFFFFFFF)
    inside = (low * np.uint64(V)) >> np.uint64(32)
    outside = np.uint64(V) + ((low * np.uint64((1 << 32) - V)) >> np.uint64(32))
    queries = np.where(hits, inside, outside).astype(np.uint32)
    return Workload("duplicate_keys", keys, None, queries, V)
