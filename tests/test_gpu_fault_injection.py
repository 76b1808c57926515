"""Failure handling without a GPU fault: device allocations are made to fail
on the host (hg_debug_fail_alloc_after) at every point of a build and a
grouped count.  Each failing call must report HG_ERR_OOM, launch nothing on
the missing memory and release what it had taken; afterwards the library
must build and count correctly again."""
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


def test_injected_allocation_failures(hg):
    # a table larger than L2 with many queries: partitioned build, long-bucket
    # summaries, query grouping and the hash-join probe all allocate
    B = 1 << 23
    wl = W.zipf_large(n=1 << 23, num_buckets=B, q=(1 << 20) + 3, M=1 << 16, salt=80)
    ref = oracle.build_table(wl.keys, B, 0)
    u, inv = np.unique(wl.queries, return_inverse=True)
    want = ref.query_count(np.ascontiguousarray(u))[inv]
    dk, dq = to_dev(wl.keys), to_dev(wl.queries)
    counts = torch.empty(wl.queries.size, dtype=torch.int32, device="cuda")
    total = torch.empty(1, dtype=torch.int64, device="cuda")
    failures = 0
    try:
        for k in range(16):
            hg.hg_debug_fail_alloc_after(k)
            try:
                with hg.hg_build(dk, B, 0, flags=hg.HG_LONG_SUMMARY) as t:
                    hg.hg_query_count(t, dq, counts, total)
            except hg.HashGraphError as e:
                assert e.status == hg.HG_ERR_OOM, e
                failures += 1
            finally:
                hg.hg_debug_fail_alloc_after(-1)
            torch.cuda.synchronize()
    finally:
        hg.hg_debug_fail_alloc_after(-1)
    assert failures >= 6  # every allocation of the build and of the count failed once
    # the library is usable again and its results exact
    with hg.hg_build(dk, B, 0, flags=hg.HG_LONG_SUMMARY) as t:
        hg.hg_query_count(t, dq, counts, total)
        hg.hg_sync(t)
        assert np.array_equal(from_dev(counts, np.uint32).astype(np.uint64), want)
        assert int(from_dev(total, np.uint64)[0]) == int(want.sum())
