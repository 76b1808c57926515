"""Python binding of libhashgraph.so (C ABI in include/hashgraph.h).

Argument marshalling only: every step of the build and of the probes runs in
the library's CUDA kernels.  PyTorch supplies device memory and streams.  The
functions keep the C names (``hg_build``, ``hg_query_count``, ...); tensors
must be contiguous CUDA tensors on the current device.

There is no CPU fallback: importing this package fails if the compiled
library is missing (build it with ``__graft_entry__.build()``).
"""
from __future__ import annotations

import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhashgraph.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: the CUDA library has not been built "
        "(run `python -c 'import __graft_entry__ as g; g.build()'`)")

lib = ctypes.CDLL(LIB_PATH)

HG_OK = 0
HG_ERR_INVALID_ARG = 1
HG_ERR_OOM = 2
HG_ERR_CUDA = 3
HG_ERR_CAPACITY = 4
HG_ERR_NO_VALUES = 5
HG_ERR_TIMEOUT = 6
STATUS_NAMES = {0: "HG_OK", 1: "HG_ERR_INVALID_ARG", 2: "HG_ERR_OOM", 3: "HG_ERR_CUDA",
                4: "HG_ERR_CAPACITY", 5: "HG_ERR_NO_VALUES", 6: "HG_ERR_TIMEOUT"}

HG_INDEX_VALUES = 0x1
HG_PLAIN_BUILD = 0x2
HG_PARTITION_BUILD = 0x4
HG_SORTED_BUCKETS = 0x8
HG_LONG_SUMMARY = 0x10


class hg_config(ctypes.Structure):
    _fields_ = [("key_bytes", ctypes.c_uint32), ("value_bytes", ctypes.c_uint32),
                ("num_buckets", ctypes.c_uint64), ("seed", ctypes.c_uint64), ("flags", ctypes.c_uint32)]


_vp, _u64, _u32p = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p
lib.hg_last_error.restype = ctypes.c_char_p
lib.hg_version.restype = ctypes.c_char_p
lib.hg_build.argtypes = [ctypes.POINTER(hg_config), _vp, _vp, _u64, _vp, ctypes.POINTER(_vp)]
lib.hg_query_count.argtypes = [_vp, _vp, _u64, _vp, _vp, _vp]
lib.hg_query_gather.argtypes = [_vp, _vp, _u64, _vp, _vp, _u64, ctypes.POINTER(_u64), _vp]
lib.hg_join_count.argtypes = [_vp, _vp, _u64, _vp, _vp]
lib.hg_query_count_intersect.argtypes = [_vp, _vp, _u64, _vp, _vp, _vp]
lib.hg_query_plan_create.argtypes = [_vp, _vp, _u64, _vp, ctypes.POINTER(_vp)]
lib.hg_query_count_plan.argtypes = [_vp, _vp, _vp, _vp, _vp]
lib.hg_query_plan_free.argtypes = [_vp, _vp]
for _f in ("hg_query_plan_create", "hg_query_count_plan", "hg_query_plan_free"):
    getattr(lib, _f).restype = ctypes.c_int
lib.hg_query_count_intersect.restype = ctypes.c_int
lib.hg_free.argtypes = [_vp, _vp]
lib.hg_sync.argtypes = [_vp, _vp]
lib.hg_table_view.argtypes = [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                              ctypes.POINTER(_u64), ctypes.POINTER(_u64)]
lib.hg_probe_stats.argtypes = [_vp, _vp, _u64, _vp, _vp]
lib.hg_long_summary_view.argtypes = [_vp] + [ctypes.POINTER(_vp)] * 5 + [ctypes.POINTER(ctypes.c_uint32)] * 2
lib.hg_long_summary_view.restype = ctypes.c_int
lib.hg_debug_fail_alloc_after.argtypes = [ctypes.c_int64]
lib.hg_debug_fail_alloc_after.restype = None
lib.hg_selftest_bounded_wait.argtypes = [_vp]
lib.hg_selftest_bounded_wait.restype = ctypes.c_int
lib.hg_launch_count.restype = _u64
lib.hg_prof_enable.argtypes = [ctypes.c_int]
lib.hg_prof_read.argtypes = [ctypes.c_char_p, ctypes.POINTER(_u64), ctypes.POINTER(ctypes.c_double)]
lib.hg_prof_names.restype = ctypes.c_char_p
for _f in ("hg_build", "hg_query_count", "hg_query_gather", "hg_join_count", "hg_free", "hg_sync",
           "hg_table_view", "hg_prof_enable", "hg_prof_read", "hg_probe_stats"):
    getattr(lib, _f).restype = ctypes.c_int


class HashGraphError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def _check(status: int) -> int:
    if status != HG_OK:
        raise HashGraphError(status, lib.hg_last_error().decode())
    return status


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _ptr(t: torch.Tensor | None) -> int | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr() if t.numel() else None


_KEY_DTYPES = {torch.int32: 4, torch.uint32: 4, torch.int64: 8, torch.uint64: 8}


class Table:
    """Handle of a device-resident HashGraph (owns the library's hg_table*)."""

    def __init__(self, handle: int, key_bytes: int, n: int, num_buckets: int, has_values: bool, stream: int,
                 owned: bool = True):
        self.handle = handle
        self.key_bytes = key_bytes
        self.n = n
        self.num_buckets = num_buckets
        self.has_values = has_values
        self._stream = stream
        self._owned = owned

    def free(self, stream=None):
        if self.handle and not self._owned:  # borrowed (e.g. from a server): never freed here
            self.handle = None
        if self.handle:
            _check(lib.hg_free(self.handle, _stream(stream) if stream is not None else self._stream))
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.free()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def hg_build(keys: torch.Tensor, num_buckets: int, seed: int = 0, values: torch.Tensor | None = None,
             flags: int = 0, stream=None) -> Table:
    """hg_build: Algorithm 1 on the device.  keys: 32- or 64-bit integer tensor."""
    if keys.dtype not in _KEY_DTYPES:
        raise TypeError(f"keys dtype {keys.dtype} is not a 32/64-bit integer type")
    kb = _KEY_DTYPES[keys.dtype]
    if values is not None and values.dtype not in (torch.int32, torch.uint32):
        raise TypeError("values must be 32-bit")
    cfg = hg_config(kb, 4 if values is not None else 0, num_buckets, seed & ((1 << 64) - 1), flags)
    out = _vp()
    s = _stream(stream)
    _check(lib.hg_build(ctypes.byref(cfg), _ptr(keys), _ptr(values), keys.numel(), s, ctypes.byref(out)))
    return Table(out.value, kb, keys.numel(), num_buckets, values is not None or bool(flags & HG_INDEX_VALUES), s)


def hg_query_count(table: Table, queries: torch.Tensor, counts: torch.Tensor | None = None,
                   total: torch.Tensor | None = None, stream=None):
    """hg_query_count: per-slot multiplicities into `counts` (uint32/int32) and/or their sum into `total`."""
    _check(lib.hg_query_count(table.handle, _ptr(queries), queries.numel(), _ptr(counts), _ptr(total),
                              _stream(stream)))
    return counts, total


def hg_query_count_intersect(table: Table, queries: torch.Tensor, counts: torch.Tensor | None = None,
                             total: torch.Tensor | None = None, stream=None):
    """hg_query_count_intersect: the same counts by the paper's query form (HG(Q), then bucket intersections)."""
    _check(lib.hg_query_count_intersect(table.handle, _ptr(queries), queries.numel(), _ptr(counts), _ptr(total),
                                        _stream(stream)))
    return counts, total


class QueryPlan:
    """Queries prepared for counting against one table (owns the library's hg_query_plan*)."""

    def __init__(self, handle: int, queries: torch.Tensor, stream: int):
        self.handle = handle
        self.queries = queries  # kept alive: the count may read it
        self._stream = stream

    def free(self, stream=None):
        """Stream-ordered free on `stream` (default: the current stream, where the count usually ran)."""
        if self.handle:
            _check(lib.hg_query_plan_free(self.handle, _stream(stream)))
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.free()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def hg_query_plan_create(table: Table, queries: torch.Tensor, stream=None) -> QueryPlan:
    """Group the queries by the table's bins (needs only the table's shape, so it may
    run on another stream while the table is being built)."""
    h = _vp()
    s = _stream(stream)
    _check(lib.hg_query_plan_create(table.handle, _ptr(queries), queries.numel(), s, ctypes.byref(h)))
    return QueryPlan(h.value, queries, s)


def hg_query_count_plan(table: Table, plan: QueryPlan, counts: torch.Tensor | None = None,
                        total: torch.Tensor | None = None, stream=None):
    """Counts and/or total of a planned query set (same results as hg_query_count)."""
    _check(lib.hg_query_count_plan(table.handle, plan.handle, _ptr(counts), _ptr(total), _stream(stream)))
    return counts, total


def hg_join_count(table: Table, queries: torch.Tensor, total: torch.Tensor, stream=None) -> torch.Tensor:
    """hg_join_count: total[0] = sum of per-slot counts (inner-join cardinality)."""
    _check(lib.hg_join_count(table.handle, _ptr(queries), queries.numel(), _ptr(total), _stream(stream)))
    return total


def hg_query_gather(table: Table, queries: torch.Tensor, out_offsets: torch.Tensor,
                    out_values: torch.Tensor | None, stream=None) -> int:
    """hg_query_gather: returns the total match count; raises HashGraphError(HG_ERR_CAPACITY)
    when out_values is too small (out_offsets is filled in that case)."""
    total = _u64(0)
    cap = 0 if out_values is None else out_values.numel()
    st = lib.hg_query_gather(table.handle, _ptr(queries), queries.numel(), _ptr(out_offsets),
                             _ptr(out_values) if cap else None, cap, ctypes.byref(total), _stream(stream))
    if st != HG_OK:
        err = HashGraphError(st, lib.hg_last_error().decode())
        err.total = total.value
        raise err
    return total.value


def hg_free(table: Table, stream=None):
    table.free(stream)


def hg_sync(table: Table, stream=None):
    _check(lib.hg_sync(table.handle, _stream(stream)))


class _DeviceArray:
    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {"data": (ptr or 0, False), "shape": (n,), "typestr": typestr,
                                         "version": 3, "strides": None}


def hg_table_view(table: Table):
    """(offsets, keys, values or None) as zero-copy CUDA tensors over the table's arrays.

    The tensors use signed dtypes of the same width (int32 offsets and values,
    int32/int64 keys); reinterpret them as unsigned on the host."""
    o, k, v = _vp(), _vp(), _vp()
    n, B = _u64(), _u64()
    _check(lib.hg_table_view(table.handle, ctypes.byref(o), ctypes.byref(k), ctypes.byref(v), ctypes.byref(n),
                             ctypes.byref(B)))
    dev = torch.device("cuda", torch.cuda.current_device())
    offs = torch.as_tensor(_DeviceArray(o.value, B.value + 1, "<i4"), device=dev)
    keys = torch.as_tensor(_DeviceArray(k.value, n.value, "<i4" if table.key_bytes == 4 else "<i8"), device=dev)
    vals = None
    if v.value:
        vals = torch.as_tensor(_DeviceArray(v.value, n.value, "<i4"), device=dev)
    return offs, keys, vals


def hg_long_summary_view(table: Table):
    """A HG_LONG_SUMMARY table's bucket summaries as zero-copy CUDA tensors:
    dict(n_long int32[1], bucket int32[cap], len int32[cap], keys (cap * slots),
    counts int32[cap * slots], cap, slots), or None when the table has none."""
    ptrs = [_vp() for _ in range(5)]
    cap, slots = ctypes.c_uint32(), ctypes.c_uint32()
    _check(lib.hg_long_summary_view(table.handle, *[ctypes.byref(x) for x in ptrs], ctypes.byref(cap),
                                    ctypes.byref(slots)))
    if cap.value == 0:
        return None
    dev = torch.device("cuda", torch.cuda.current_device())
    c, sl = cap.value, slots.value

    def arr(p, n, typestr):
        return torch.as_tensor(_DeviceArray(p.value, n, typestr), device=dev)

    return {"n_long": arr(ptrs[0], 1, "<i4"), "bucket": arr(ptrs[1], c, "<i4"), "len": arr(ptrs[2], c, "<i4"),
            "keys": arr(ptrs[3], c * sl, "<i4" if table.key_bytes == 4 else "<i8"),
            "counts": arr(ptrs[4], c * sl, "<i4"), "cap": c, "slots": sl}


def hg_debug_fail_alloc_after(n: int) -> None:
    """Test hook: the library's device allocations after the next n fail as if
    the device were out of memory (n < 0: off)."""
    lib.hg_debug_fail_alloc_after(int(n))


def hg_probe_stats(table: Table, queries: torch.Tensor, stream=None) -> dict:
    """Walked-length statistics of the byte model (synchronises the stream)."""
    st = torch.empty(6, dtype=torch.int64, device=queries.device)
    _check(lib.hg_probe_stats(table.handle, _ptr(queries), queries.numel(), _ptr(st), _stream(stream)))
    w, wl, nl, lim, ks, osec = (int(x) for x in st.cpu().tolist())
    return {"walked": w, "walked_long": wl, "long_slots": nl, "warp_limit": lim, "key_sectors": ks,
            "offset_sectors": osec}


def hg_launch_count() -> int:
    return lib.hg_launch_count()


def hg_prof_enable(on: bool = True):
    _check(lib.hg_prof_enable(1 if on else 0))


def hg_prof_read(name: str):
    n = _u64()
    ms = ctypes.c_double()
    _check(lib.hg_prof_read(name.encode(), ctypes.byref(n), ctypes.byref(ms)))
    return n.value, ms.value


def hg_prof_names() -> list[str]:
    return lib.hg_prof_names().decode().split(",")


def hg_version() -> str:
    return lib.hg_version().decode()


# ---------------------------------------------------------------- batches --
class hg_batch_params(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_uint32), ("bin_shift", ctypes.c_uint32), ("fuse_keys", ctypes.c_uint32)]


lib.hg_batch_create.argtypes = [ctypes.POINTER(hg_config), ctypes.c_uint32, _vp, _vp, _vp, _vp, ctypes.POINTER(_vp)]
lib.hg_batch_run.argtypes = [_vp, _vp, _vp, _vp, _vp]
lib.hg_batch_tune.argtypes = [_vp, _vp, _vp, _vp, _vp, ctypes.POINTER(hg_batch_params)]
lib.hg_batch_set_params.argtypes = [_vp, ctypes.POINTER(hg_batch_params)]
lib.hg_batch_get_params.argtypes = [_vp, ctypes.POINTER(hg_batch_params)]
lib.hg_batch_view.argtypes = [_vp, ctypes.c_uint32, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_u64),
                              ctypes.POINTER(_u64)]
lib.hg_batch_sync.argtypes = [_vp, _vp]
lib.hg_batch_walk_stats.argtypes = [_vp, _vp, _vp, _vp]
lib.hg_batch_free.argtypes = [_vp, _vp]
for _f in ("hg_batch_create", "hg_batch_run", "hg_batch_tune", "hg_batch_set_params", "hg_batch_get_params",
           "hg_batch_view", "hg_batch_sync", "hg_batch_free", "hg_batch_walk_stats"):
    getattr(lib, _f).restype = ctypes.c_int


class Batch:
    """Handle of a planned batch of tables (owns the library's hg_batch*)."""

    def __init__(self, handle: int, n_tables: int, stream: int):
        self.handle = handle
        self.n_tables = n_tables
        self._stream = stream

    def free(self, stream=None):
        if self.handle:
            _check(lib.hg_batch_free(self.handle, _stream(stream) if stream is not None else self._stream))
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.free()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _host_u64(values) -> "ctypes.Array":
    vals = [int(x) for x in values]
    return (ctypes.c_uint64 * len(vals))(*vals)


def hg_batch_create(key_offsets, num_buckets, query_offsets=None, seed: int = 0, stream=None) -> Batch:
    """Plan a batch: key_offsets / query_offsets are n_tables + 1 host integers, num_buckets n_tables."""
    n_tables = len(num_buckets)
    if len(key_offsets) != n_tables + 1 or (query_offsets is not None and len(query_offsets) != n_tables + 1):
        raise ValueError("offsets need n_tables + 1 entries")
    cfg = hg_config(4, 0, 1, seed, 0)
    ko, nb = _host_u64(key_offsets), _host_u64(num_buckets)
    qo = _host_u64(query_offsets) if query_offsets is not None else None
    h = _vp()
    s = _stream(stream)
    _check(lib.hg_batch_create(ctypes.byref(cfg), n_tables, ctypes.cast(ko, _vp), ctypes.cast(nb, _vp),
                               ctypes.cast(qo, _vp) if qo is not None else None, s, ctypes.byref(h)))
    return Batch(h.value, n_tables, s)


def hg_batch_run(batch: Batch, keys: torch.Tensor, queries: torch.Tensor | None, counts: torch.Tensor | None,
                 stream=None):
    """Build every table and count every query in one persistent launch."""
    _check(lib.hg_batch_run(batch.handle, _ptr(keys), _ptr(queries), _ptr(counts), _stream(stream)))


def hg_batch_tune(batch: Batch, keys: torch.Tensor, queries: torch.Tensor | None, counts: torch.Tensor | None,
                  stream=None) -> dict:
    """Time every candidate parameter set on this batch and keep the fastest."""
    p = hg_batch_params()
    _check(lib.hg_batch_tune(batch.handle, _ptr(keys), _ptr(queries), _ptr(counts), _stream(stream),
                             ctypes.byref(p)))
    return {"threads": p.threads, "bin_shift": p.bin_shift, "fuse_keys": p.fuse_keys}


def hg_batch_set_params(batch: Batch, threads: int, bin_shift: int, fuse_keys: int):
    p = hg_batch_params(threads, bin_shift, fuse_keys)
    _check(lib.hg_batch_set_params(batch.handle, ctypes.byref(p)))


def hg_batch_get_params(batch: Batch) -> dict:
    p = hg_batch_params()
    _check(lib.hg_batch_get_params(batch.handle, ctypes.byref(p)))
    return {"threads": p.threads, "bin_shift": p.bin_shift, "fuse_keys": p.fuse_keys}


def hg_batch_view(batch: Batch, table: int):
    """(offsets, keys) of one table as zero-copy int32 CUDA tensors."""
    o, k = _vp(), _vp()
    n, B = _u64(), _u64()
    _check(lib.hg_batch_view(batch.handle, table, ctypes.byref(o), ctypes.byref(k), ctypes.byref(n), ctypes.byref(B)))
    dev = torch.device("cuda", torch.cuda.current_device())
    offs = torch.as_tensor(_DeviceArray(o.value, B.value + 1, "<i4"), device=dev)
    keys = torch.as_tensor(_DeviceArray(k.value, n.value, "<i4"), device=dev) if n.value else \
        torch.empty(0, dtype=torch.int32, device=dev)
    return offs, keys


def hg_batch_sync(batch: Batch, stream=None):
    _check(lib.hg_batch_sync(batch.handle, _stream(stream)))


def hg_batch_walk_stats(batch: Batch, queries: torch.Tensor, stream=None) -> int:
    """Sum of the queries' bucket lengths in the built tables (synchronises the stream)."""
    st = torch.empty(1, dtype=torch.int64, device=queries.device)
    _check(lib.hg_batch_walk_stats(batch.handle, _ptr(queries), _ptr(st), _stream(stream)))
    return int(st.item())


# ---------------------------------------------------------------- serving --
class hg_server_stats_t(ctypes.Structure):
    _fields_ = [(f, ctypes.c_uint64) for f in ("builds", "probes", "probe_launches", "evictions", "resident_tables",
                                               "resident_bytes", "held_bytes", "pending", "running")]


lib.hg_server_create.argtypes = [_u64, ctypes.c_uint32, ctypes.POINTER(_vp)]
lib.hg_server_submit_build.argtypes = [_vp, _u64, ctypes.POINTER(hg_config), _vp, _u64, ctypes.POINTER(_u64)]
lib.hg_server_submit_probe.argtypes = [_vp, _u64, _vp, _u64, _vp, ctypes.POINTER(_u64)]
lib.hg_server_poll.argtypes = [_vp, _vp, _vp, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32)]
lib.hg_server_stats.argtypes = [_vp, ctypes.POINTER(hg_server_stats_t)]
lib.hg_server_table.argtypes = [_vp, _u64, ctypes.POINTER(_vp)]
lib.hg_server_table_bytes.argtypes = [_u64, _u64]
lib.hg_server_table_bytes.restype = _u64
lib.hg_server_free.argtypes = [_vp]
for _f in ("hg_server_create", "hg_server_submit_build", "hg_server_submit_probe", "hg_server_poll",
           "hg_server_stats", "hg_server_table", "hg_server_free"):
    getattr(lib, _f).restype = ctypes.c_int


def hg_server_table_bytes(n: int, num_buckets: int) -> int:
    return lib.hg_server_table_bytes(n, num_buckets)


class Server:
    """The serving engine (owns the library's hg_server*).  Not thread-safe."""

    def __init__(self, budget_bytes: int, max_batch: int = 256):
        h = _vp()
        _check(lib.hg_server_create(budget_bytes, max_batch, ctypes.byref(h)))
        self.handle = h.value
        self._ids = (ctypes.c_uint64 * 4096)()
        self._st = (ctypes.c_int32 * 4096)()

    def submit_build(self, table_id: int, keys: torch.Tensor, num_buckets: int, seed: int = 0) -> int:
        cfg = hg_config(4, 0, num_buckets, seed, 0)
        rid = _u64()
        _check(lib.hg_server_submit_build(self.handle, table_id, ctypes.byref(cfg), _ptr(keys), keys.numel(),
                                          ctypes.byref(rid)))
        return rid.value

    def submit_probe(self, table_id: int, queries: torch.Tensor, counts: torch.Tensor) -> int:
        rid = _u64()
        _check(lib.hg_server_submit_probe(self.handle, table_id, _ptr(queries), queries.numel(), _ptr(counts),
                                          ctypes.byref(rid)))
        return rid.value

    def poll(self) -> list:
        """Drive the engine; (request id, status) of the requests that completed."""
        n = ctypes.c_uint32()
        _check(lib.hg_server_poll(self.handle, self._ids, self._st, 4096, ctypes.byref(n)))
        return [(self._ids[i], self._st[i]) for i in range(n.value)]

    def stats(self) -> dict:
        st = hg_server_stats_t()
        _check(lib.hg_server_stats(self.handle, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in hg_server_stats_t._fields_}

    def table(self, table_id: int) -> Table:
        """Borrow a resident table (for checks through hg_table_view)."""
        h = _vp()
        _check(lib.hg_server_table(self.handle, table_id, ctypes.byref(h)))
        o, k, v = _vp(), _vp(), _vp()
        n, B = _u64(), _u64()
        _check(lib.hg_table_view(h.value, ctypes.byref(o), ctypes.byref(k), ctypes.byref(v), ctypes.byref(n),
                                 ctypes.byref(B)))
        return Table(h.value, 4, n.value, B.value, False, 0, owned=False)

    def free(self):
        if self.handle:
            _check(lib.hg_server_free(self.handle))
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.free()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def hg_selftest_bounded_wait(stream=None) -> int:
    """Run the bounded-wait self-test; returns the status (HG_ERR_TIMEOUT is the expected one)."""
    return lib.hg_selftest_bounded_wait(_stream(stream))
