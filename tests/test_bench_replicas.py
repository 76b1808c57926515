"""Host logic of the multi-GPU bench path (independent replicas, one process
per GPU): each rank draws its own seeded workload, the job time is the maximum
over ranks, and the reported value aggregates every rank's keys.  Runs as two
gloo ranks on the CPU."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r reports 10 + r ms for the step and 20 - r ms end to end
        got = bench.max_over_ranks([10.0 + rank, 20.0 - rank], dist, torch.device("cpu"))
        wl = bench.make_workload(12, rank)
        out[rank] = (got, int(wl.keys[:64].astype(np.uint64).sum()), int(wl.queries[:64].astype(np.uint64).sum()))
    finally:
        dist.destroy_process_group()


def test_two_replicas_max_time_and_distinct_inputs():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == [11.0, 20.0]
    # each replica builds and probes its own seeded inputs
    assert res[0][1] != res[1][1] and res[0][2] != res[1][2]


def test_single_process_identity_and_aggregate():
    assert bench.max_over_ranks([3.0, 4.0], None, None) == [3.0, 4.0]
    # 2 replicas x 2^29 keys in 10 ms
    assert bench.aggregate_gkeys(2, 1 << 29, 10.0) == pytest.approx(2 * (1 << 29) / 1e-2 / 1e9)
