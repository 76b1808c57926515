"""Failure path of the kernels' bounded waits, exercised without a GPU fault:
a prefix-sum tile waits on a predecessor that never runs, its wait runs out
after about a second and the timeout is reported as a status; the context
stays usable afterwards."""
import time

import numpy as np
import pytest

import oracle
import workloads as W
from tests.hg_testutil import table_arrays, to_dev, assert_same_table

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_bounded_wait_reports_timeout_and_context_survives():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2104_00792_gb300 as hg
    t0 = time.time()
    st = hg.hg_selftest_bounded_wait()
    assert st == hg.HG_ERR_TIMEOUT
    assert time.time() - t0 < 30
    # the device keeps working
    wl = W.plain_uniform(5000, 100, num_buckets=777, salt=31)
    with hg.hg_build(to_dev(wl.keys), 777, 0, flags=hg.HG_PLAIN_BUILD) as t:
        o, k, v = table_arrays(hg, t, np.uint32)
        assert_same_table(o, k, v, oracle.build_table(wl.keys, 777, 0))
        hg.hg_sync(t)
