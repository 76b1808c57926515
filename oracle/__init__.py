"""HashGraph CPU oracle -- test infrastructure only.

A ctypes wrapper over ``hg_oracle.c``: a plain single-threaded restatement of
the HashGraph build (Algorithm 1) and the bucket-walk query (Sec. 3.3).
Only the tests, the smoke check and the benchmark's CPU-baseline leg may
import this package; the library under ``paper_2104_00792_gb300`` never does.

Parity pins live in ``tests/test_oracle_pins.py`` (published MurmurHash3
vectors, brute force, sorting, CSR invariants).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "hg_oracle.c")
LIB = os.path.join(HERE, "libhg_oracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, single-threaded)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + ".tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, SRC])
        os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB)
        u64, vp, ci = ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int
        L.hgo_fmix32.restype = ctypes.c_uint32
        L.hgo_fmix32.argtypes = [ctypes.c_uint32]
        L.hgo_fmix64.restype = u64
        L.hgo_fmix64.argtypes = [u64]
        L.hgo_buckets.argtypes = [ci, vp, u64, u64, u64, vp]
        L.hgo_build.restype = ci
        L.hgo_build.argtypes = [ci, vp, vp, ci, u64, u64, u64, vp, vp, vp]
        L.hgo_query_count.argtypes = [ci, vp, vp, u64, u64, vp, u64, vp]
        L.hgo_join_count.restype = u64
        L.hgo_join_count.argtypes = [ci, vp, vp, u64, u64, vp, u64]
        L.hgo_query_gather.restype = u64
        L.hgo_query_gather.argtypes = [ci, vp, vp, vp, u64, u64, vp, u64, vp, vp, u64]
        L.hgo_count_linear.restype = u64
        L.hgo_count_linear.argtypes = [ci, vp, u64, vp]
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def fmix32(x: int) -> int:
    return _load().hgo_fmix32(x)


def fmix64(x: int) -> int:
    return _load().hgo_fmix64(x)


def buckets(keys: np.ndarray, num_buckets: int, seed: int = 0) -> np.ndarray:
    keys = np.ascontiguousarray(keys)
    out = np.empty(keys.size, dtype=np.uint64)
    _load().hgo_buckets(keys.dtype.itemsize, _p(keys), keys.size, seed, num_buckets, _p(out))
    return out


class Table:
    """CSR HashGraph built by the oracle: offsets (uint64, B+1), keys, values."""

    def __init__(self, offsets, keys, values, num_buckets, seed):
        self.offsets = offsets
        self.keys = keys
        self.values = values
        self.num_buckets = num_buckets
        self.seed = seed

    @property
    def key_bytes(self):
        return self.keys.dtype.itemsize

    def query_count(self, queries: np.ndarray) -> np.ndarray:
        queries = np.ascontiguousarray(queries, dtype=self.keys.dtype)
        out = np.empty(queries.size, dtype=np.uint64)
        _load().hgo_query_count(self.key_bytes, _p(self.offsets), _p(self.keys), self.num_buckets, self.seed,
                                _p(queries), queries.size, _p(out))
        return out

    def join_count(self, queries: np.ndarray) -> int:
        queries = np.ascontiguousarray(queries, dtype=self.keys.dtype)
        return int(_load().hgo_join_count(self.key_bytes, _p(self.offsets), _p(self.keys), self.num_buckets,
                                          self.seed, _p(queries), queries.size))

    def query_gather(self, queries: np.ndarray):
        """Returns (out_offsets uint64[Q+1], out_values uint32[total])."""
        if self.values is None:
            raise ValueError("table has no values")
        queries = np.ascontiguousarray(queries, dtype=self.keys.dtype)
        offs = np.empty(queries.size + 1, dtype=np.uint64)
        L = _load()
        total = L.hgo_query_gather(self.key_bytes, _p(self.offsets), _p(self.keys), _p(self.values),
                                   self.num_buckets, self.seed, _p(queries), queries.size, _p(offs), None, 0)
        vals = np.empty(total, dtype=np.uint32)
        L.hgo_query_gather(self.key_bytes, _p(self.offsets), _p(self.keys), _p(self.values), self.num_buckets,
                           self.seed, _p(queries), queries.size, _p(offs), _p(vals), total)
        return offs, vals


def build_table(keys: np.ndarray, num_buckets: int, seed: int = 0, values: np.ndarray | None = None,
                index_values: bool = False) -> Table:
    """Algorithm 1 run sequentially; see ``hgo_build`` in ``hg_oracle.c``."""
    keys = np.ascontiguousarray(keys)
    if keys.dtype not in (np.uint32, np.uint64):
        raise TypeError("keys must be uint32 or uint64")
    n = keys.size
    offsets = np.empty(num_buckets + 1, dtype=np.uint64)
    keys_out = np.empty(n, dtype=keys.dtype)
    vals_out = None
    if values is not None:
        values = np.ascontiguousarray(values, dtype=np.uint32)
        vals_out = np.empty(n, dtype=np.uint32)
    elif index_values:
        vals_out = np.empty(n, dtype=np.uint32)
    rc = _load().hgo_build(keys.dtype.itemsize, _p(keys), _p(values), int(index_values), n, num_buckets, seed,
                           _p(offsets), _p(keys_out), _p(vals_out))
    if rc != 0:
        raise RuntimeError("oracle build failed")
    return Table(offsets, keys_out, vals_out, num_buckets, seed)


def count_linear(keys: np.ndarray, q) -> int:
    """#{i : keys[i] == q} by a linear scan of the input (no table)."""
    keys = np.ascontiguousarray(keys)
    qa = np.array([q], dtype=keys.dtype)
    return int(_load().hgo_count_linear(keys.dtype.itemsize, _p(keys), keys.size, _p(qa)))
