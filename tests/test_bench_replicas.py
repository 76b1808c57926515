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


def test_reference_arm_prints_the_contract_line():
    # the reference arm times the CPU oracle on a bounded sample; no GPU needed
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--log2n", "16",
                          "--zipf-log2m", "12", "--cpu-sample-log2", "14", "--steps", "2", "--warmup", "1"],
                         capture_output=True, text=True, timeout=300, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 2 and d["warmup"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
