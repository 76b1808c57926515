"""Helpers shared by the GPU parity tests: host<->device marshalling and the
comparison rules (offsets and counts bit-exact; bucket contents and gather
segments compared after a canonical sort, since the order inside a bucket is
left free by the paper's atomic scatter)."""
import numpy as np
import torch

import oracle

_SIGNED = {np.dtype(np.uint32): np.int32, np.dtype(np.uint64): np.int64}


def to_dev(a: np.ndarray) -> torch.Tensor:
    a = np.ascontiguousarray(a)
    return torch.from_numpy(a.view(_SIGNED[a.dtype])).cuda()


def from_dev(t: torch.Tensor, dtype) -> np.ndarray:
    return t.cpu().numpy().view(dtype)


def table_arrays(hg, table, key_dtype):
    offs, keys, vals = hg.hg_table_view(table)
    torch.cuda.synchronize()
    o = from_dev(offs, np.uint32)
    k = from_dev(keys, key_dtype)
    v = None if vals is None else from_dev(vals, np.uint32)
    return o, k, v


def assert_same_table(o, k, v, ref: oracle.Table, exact_order=False):
    """offsets bit-exact; per bucket the (key, value) multiset equal."""
    assert o.dtype == np.uint32
    assert np.array_equal(o.astype(np.uint64), ref.offsets), "offsets differ"
    assert k.size == ref.keys.size
    B = ref.offsets.size - 1
    seg = np.repeat(np.arange(B, dtype=np.int64), np.diff(ref.offsets.astype(np.int64)))
    if v is None:
        og = np.lexsort((k, seg))
        orf = np.lexsort((ref.keys, seg))
        assert np.array_equal(k[og], ref.keys[orf]), "bucket contents differ"
    else:
        og = np.lexsort((v, k, seg))
        orf = np.lexsort((ref.values, ref.keys, seg))
        assert np.array_equal(k[og], ref.keys[orf]), "bucket keys differ"
        assert np.array_equal(v[og], ref.values[orf]), "bucket values differ"


def segment_signature(keys: np.ndarray, offsets: np.ndarray, vals=None):
    """Per-bucket order-independent fingerprint: wrapping sums of two mixes of
    each key (and value).  Equal multisets give equal signatures; different
    ones collide with negligible probability."""
    k = keys.astype(np.uint64)
    if vals is not None:
        k = k ^ (vals.astype(np.uint64) * np.uint64(0xD6E8FEB86659FD93))
    with np.errstate(over="ignore"):
        f1 = k * np.uint64(0x9E3779B97F4A7C15)
        f2 = (k ^ (k >> np.uint64(29))) * np.uint64(0xBF58476D1CE4E5B9)
        c1 = np.concatenate([[np.uint64(0)], np.cumsum(f1, dtype=np.uint64)])
        c2 = np.concatenate([[np.uint64(0)], np.cumsum(f2, dtype=np.uint64)])
        o = offsets.astype(np.int64)
        return c1[o[1:]] - c1[o[:-1]], c2[o[1:]] - c2[o[:-1]]


def assert_same_gather(offs_gpu, vals_gpu, offs_ref, vals_ref):
    assert np.array_equal(offs_gpu, offs_ref), "gather offsets differ"
    assert vals_gpu.size == vals_ref.size
    o = offs_ref.astype(np.int64)
    seg = np.repeat(np.arange(o.size - 1), np.diff(o))
    a = vals_gpu[np.lexsort((vals_gpu, seg))]
    b = vals_ref[np.lexsort((vals_ref, seg))]
    assert np.array_equal(a, b), "gather segments differ"
