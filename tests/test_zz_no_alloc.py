"""hg_build_noalloc, the build for callers that cannot allocate device memory
(a host framework that owns all device memory, or a loop that must not grow a
memory pool once running): it takes its prefix-sum scratch from a fixed array
inside the library.  Its output must match hg_build's, call after call, since
every call reuses that array.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import oracle
import workloads as W
from tests.hg_testutil import assert_same_table, from_dev, table_arrays, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def hg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2104_00792_gb300 as m
    m.lib.hg_build_noalloc.argtypes = [ctypes.POINTER(m.hg_config), ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p]
    m.lib.hg_build_noalloc.restype = ctypes.c_int
    return m


def _noalloc(hg, keys_dev, n, B, seed, values_dev=None, flags=0, key_bytes=4, offs_shift=0):
    # offs_shift: place d_offsets that many 4-byte words into a larger buffer (unaligned to 16 bytes)
    offs = torch.empty(B + 1 + offs_shift, dtype=torch.int32, device="cuda")[offs_shift:]
    kout = torch.empty(max(n, 1), dtype=keys_dev.dtype, device="cuda")
    has_vals = values_dev is not None or bool(flags & hg.HG_INDEX_VALUES)
    vout = torch.empty(max(n, 1), dtype=torch.int32, device="cuda") if has_vals else None
    cfg = hg.hg_config(key_bytes, 4 if values_dev is not None else 0, B, seed, flags)
    st = hg.lib.hg_build_noalloc(ctypes.byref(cfg), keys_dev.data_ptr() if n else None,
                                 values_dev.data_ptr() if values_dev is not None else None, n, offs.data_ptr(),
                                 kout.data_ptr(), vout.data_ptr() if vout is not None else None,
                                 torch.cuda.current_stream().cuda_stream)
    assert st == hg.HG_OK, hg.lib.hg_last_error()
    torch.cuda.synchronize()
    return offs, kout[:n], (vout[:n] if vout is not None else None)


def _same_as_hg_build(hg, keys, B, seed, values=None, flags=0, offs_shift=0, no_device_alloc=False):
    dt = keys.dtype
    dk = to_dev(keys)
    dv = None if values is None else to_dev(values)
    torch.cuda.synchronize()
    if no_device_alloc:
        # every device allocation the library might make fails from here on
        hg.hg_debug_fail_alloc_after(0)
    try:
        offs, kout, vout = _noalloc(hg, dk, keys.size, B, seed, dv, flags, keys.dtype.itemsize, offs_shift)
    finally:
        hg.hg_debug_fail_alloc_after(-1)
    assert int(from_dev(offs[-1:], np.uint32)[0]) == keys.size  # the build completed
    with hg.hg_build(dk, B, seed, values=dv, flags=flags) as t:
        o_ref, k_ref, v_ref = table_arrays(hg, t, dt)
    o = from_dev(offs, np.uint32)
    assert np.array_equal(o, o_ref)  # offsets bit-exact
    k = from_dev(kout, dt)
    # and against the oracle: offsets bit-exact, every bucket's (key, value) multiset
    ref = oracle.build_table(keys, B, seed, values=values, index_values=bool(flags & hg.HG_INDEX_VALUES))
    assert_same_table(o, k, None if vout is None else from_dev(vout, np.uint32), ref)
    seg = np.repeat(np.arange(B, dtype=np.int64), np.diff(o.astype(np.int64)))
    if vout is None:
        assert np.array_equal(k[np.lexsort((k, seg))], k_ref[np.lexsort((k_ref, seg))])
    else:
        v = from_dev(vout, np.uint32)
        a, b = np.lexsort((v, k, seg)), np.lexsort((v_ref, k_ref, seg))
        assert np.array_equal(k[a], k_ref[b]) and np.array_equal(v[a], v_ref[b])


def test_noalloc_matches_hg_build_on_two_calls_in_a_row(hg):
    # first call: large-ish key-only table with index values (sets up the scratch address)
    wl = W.zipf_large(n=(1 << 20) + 5, num_buckets=(1 << 19) + 7, q=16, M=1 << 16)
    _same_as_hg_build(hg, wl.keys, (1 << 19) + 7, 0, flags=hg.HG_INDEX_VALUES)
    # second call reuses the same scratch with different sizes: 64-bit keys with values
    wl2 = W.join_kv(n=70001, num_buckets=1 << 15, q=16, salt=9)
    _same_as_hg_build(hg, wl2.keys, 1 << 15, 3, values=wl2.values)


def test_noalloc_largest_table_and_rejection(hg):
    B = (1 << 23) - 1
    wl = W.plain_uniform(1 << 20, 16, num_buckets=B)
    _same_as_hg_build(hg, wl.keys, B, 0)
    cfg = hg.hg_config(4, 0, 1 << 23, 0, 0)
    offs = torch.empty(4, dtype=torch.int32, device="cuda")
    st = hg.lib.hg_build_noalloc(ctypes.byref(cfg), None, None, 0, offs.data_ptr(), None, None, None)
    assert st == hg.HG_ERR_INVALID_ARG
    assert b"num_buckets" in hg.lib.hg_last_error()


def test_noalloc_makes_no_device_allocation(hg):
    # with every library allocation made to fail, the build still succeeds: it
    # allocates nothing (checked twice in a row on different shapes)
    wl = W.plain_uniform(200_003, 16, num_buckets=(1 << 18) + 3)
    _same_as_hg_build(hg, wl.keys, (1 << 18) + 3, 5, flags=hg.HG_INDEX_VALUES, no_device_alloc=True)
    wl2 = W.join_kv(n=30001, num_buckets=4099, q=16, salt=4)
    _same_as_hg_build(hg, wl2.keys, 4099, 0, values=wl2.values, no_device_alloc=True)


def test_noalloc_unaligned_offsets_at_the_largest_table(hg):
    # offsets 4 bytes past a 16-byte boundary take the prefix sum's scalar path,
    # which uses the most tiles (and so the most of the fixed array) at the limit
    B = (1 << 23) - 1
    wl = W.plain_uniform((1 << 20) + 17, 16, num_buckets=B, salt=6)
    _same_as_hg_build(hg, wl.keys, B, 0, offs_shift=1)
    _same_as_hg_build(hg, wl.keys, B, 0, offs_shift=3)
