"""Benchmark: HashGraph build + probe throughput on one GB300 (or N replicas).

One step = hg_build (hash, histogram, scan, scatter; with HG_LONG_SUMMARY the
long buckets condensed) + hg_query_count (counts and total) + hg_free over the
large duplicate-key workload: 2^28 uint32 keys drawn Zipf(s=1) over 2^24
distinct values, 2^27 buckets, murmur3-fmix32 seed 0, 2^28 queries with 70%
hits (--workload zipf_weighted: hits drawn by the same Zipf law).  The query
grouping runs on a second stream while the table builds (query plans).
Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Inputs (2 GiB per step) exceed the 129 MB L2, so no L2 flush is needed
between steps.  Multi-GPU runs (torchrun) are independent replicas: every
rank builds and probes its own table (weak scaling; no collective on the data
path).  `--impl reference` times the CPU oracle (the only reference this
method has) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "build+probe Gkeys/s at 2^28 u32"
UNIT = "Gkeys/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=30)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--log2n", type=int, default=28, help="log2 of build keys (queries equal, buckets half)")
    p.add_argument("--zipf-log2m", type=int, default=24, help="log2 of the Zipf workloads' distinct values")
    p.add_argument("--cpu-sample-log2", type=int, default=27)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--workload", default="zipf_large",
                   choices=["zipf_large", "zipf_weighted", "batched", "serving", "dupsweep"],
                   help="zipf_large: the 2^28 build+probe step; zipf_weighted: the same keys with hits drawn by "
                        "the keys' own Zipf law (each value queried in proportion to its copies); "
                        "batched: 4096 tables in one persistent launch; "
                        "serving: a Poisson stream of build and probe requests through the serving engine; "
                        "dupsweep: the duplicate-key experiment (each value 2^d times, B = N / 2^d)")
    p.add_argument("--sweep-log2n", type=int, default=26, help="dupsweep: log2 of keys (and queries)")
    p.add_argument("--requests", type=int, default=200_000, help="serving: requests in the stream")
    p.add_argument("--query-form", default="plan", choices=["plan", "probe", "intersect"],
                   help="zipf_large: plan = hg_query_plan_create on a second stream while the table builds, then "
                        "hg_query_count_plan; probe = hg_query_count after the build; intersect = "
                        "hg_query_count_intersect (HG(Q) + bucket intersections, the paper's query form)")
    p.add_argument("--long-summary", default="auto", choices=["auto", "on", "off"],
                   help="build with HG_LONG_SUMMARY (buckets of more than 8192 keys condensed to their distinct "
                        "keys and counts); auto = on (both workloads' Zipf keys make such buckets)")
    p.add_argument("--load", type=float, default=0.8, help="serving: arrival rate / the plain path's capacity")
    p.add_argument("--budget-gb", type=float, default=100.0, help="serving: device-memory budget for tables")
    p.add_argument("--tables", type=int, default=4096, help="batched: number of tables")
    p.add_argument("--no-plain", action="store_true", help="batched: skip the one-launch-per-table comparison")
    return p.parse_args()


def workload_desc(log2n, weighted=False, log2m=24):
    if weighted:
        return (f"zipf_weighted: N=2^{log2n} uint32 keys Zipf(s=1) over 2^{log2m} values, B=2^{log2n - 1} buckets, "
                f"murmur3-fmix32 seed 0, Q=2^{log2n} queries 70% hits (ranks Zipf(s=1) like the keys)")
    return (f"zipf_large: N=2^{log2n} uint32 keys Zipf(s=1) over 2^{log2m} values, B=2^{log2n - 1} buckets, "
            f"murmur3-fmix32 seed 0, Q=2^{log2n} queries 70% hits (ranks uniform over the 2^{log2m} values)")


def use_summary(args):
    return args.long_summary in ("auto", "on")


def cpu_sample_log2(args):
    # the oracle's walk is quadratic in the copies of a Zipf-weighted query's value:
    # its sample is smaller so that it still ends in seconds
    if args.workload == "zipf_weighted":
        return min(args.cpu_sample_log2, 21)
    return args.cpu_sample_log2


def max_over_ranks(values, dist, device):
    """Elementwise maximum of per-rank timings (the slowest replica sets the
    job's time); the identity when there is no process group."""
    if dist is None:
        return list(values)
    import torch
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t]


def aggregate_gkeys(world, keys_per_rank, ms):
    """Whole-job throughput: every replica processes keys_per_rank keys in ms."""
    return world * keys_per_rank / (ms * 1e-3) / 1e9


def make_workload(log2n, salt, weighted=False, log2m=24):
    import workloads as W
    make = W.zipf_weighted if weighted else W.zipf_large
    return make(n=1 << log2n, num_buckets=1 << (log2n - 1), q=1 << log2n, M=1 << log2m, hit=0.7, salt=salt)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            if self.thread:
                self.thread.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() in ("active", "1", "yes"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2104_00792_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it
    was taken on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "dram_traffic_zipf_large.txt")
    try:
        rows = {}
        with open(path) as f:
            for line in f:
                if "=" in line and not line.startswith("#"):
                    k, v = line.strip().split("=", 1)
                    rows[k.strip()] = v.strip()
    except OSError:
        return None
    if rows.get("source_hash") != source_hash():
        return None
    v = rows.get(f"traffic_bytes_per_launch.{kernel}")
    return float(v) if v else None


def batch_traffic_ratio():
    """ncu DRAM bytes per algorithmic byte of the batched kernel, if measured on
    the current kernel sources (else None)."""
    try:
        rows = {}
        with open(os.path.join(ROOT, "profiles", "dram_traffic_batch.txt")) as f:
            for line in f:
                if "=" in line and not line.startswith("#"):
                    k, v = line.strip().split("=", 1)
                    rows[k.strip()] = v.strip()
    except OSError:
        return None
    if rows.get("source_hash") != source_hash():
        return None
    v = rows.get("traffic_per_model_byte.batch")
    return float(v) if v else None


def cpu_oracle_sample(wl, log2s):
    """Oracle build + count on the first 2^log2s keys and queries of the
    workload, table size scaled to keep the same keys-per-bucket ratio."""
    import numpy as np

    import oracle
    n = min(1 << log2s, wl.keys.size)
    keys = np.ascontiguousarray(wl.keys[:n])
    queries = np.ascontiguousarray(wl.queries[:n])
    B = max(1, (wl.num_buckets * n) // wl.keys.size)
    t0 = time.perf_counter()
    t = oracle.build_table(keys, B, 0)
    t.query_count(queries)
    dt = time.perf_counter() - t0
    return {"value": (2 * n) / dt / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first 2^{log2s} keys and 2^{log2s} queries of the workload, B={B} (same keys/bucket), "
                      f"build+count, {dt:.2f} s single-threaded"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    wl = make_workload(args.log2n, 0, args.workload == "zipf_weighted", args.zipf_log2m)
    times = []
    res = None
    for _ in range(args.warmup):
        cpu_oracle_sample(wl, cpu_sample_log2(args) - 2)
    for _ in range(args.steps):
        res = cpu_oracle_sample(wl, cpu_sample_log2(args) - 2)
        times.append(res["value"])
    v = statistics.median(times)
    res["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": workload_desc(args.log2n, args.workload == "zipf_weighted", args.zipf_log2m),
                       "reference": "CPU oracle (oracle/hg_oracle.c)"},
            "cpu_baseline": res, "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0,
                                         "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def e2e_pipelined(hg, wl, build_and_query, dev, stream, steps, barrier):
    """End to end through the C ABI with host buffers: every step copies its
    keys and queries in from pinned host memory, builds, counts, and copies
    the counts and total back.  Copies run on their own streams and two
    device buffer sets alternate, so one step's copies overlap another's
    kernels (the pipelining a caller of the library would use)."""
    import numpy as np
    import torch

    N, Q, B = wl.keys.size, wl.queries.size, wl.num_buckets
    h_keys = torch.from_numpy(wl.keys.view(np.int32)).pin_memory()
    h_q = torch.from_numpy(wl.queries.view(np.int32)).pin_memory()
    sets = []
    for _ in range(2):
        sets.append({"keys": torch.empty(N, dtype=torch.int32, device=dev),
                     "queries": torch.empty(Q, dtype=torch.int32, device=dev),
                     "counts": torch.empty(Q, dtype=torch.int32, device=dev),
                     "total": torch.empty(1, dtype=torch.int64, device=dev),
                     "h_counts": torch.empty(Q, dtype=torch.int32).pin_memory(),
                     "h_total": torch.empty(1, dtype=torch.int64).pin_memory(),
                     "in_done": torch.cuda.Event(), "out_done": torch.cuda.Event(),
                     "used": torch.cuda.Event()})
    s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

    def e2e_step(k):
        st = sets[k % 2]
        if k >= 2:
            s_in.wait_event(st["used"])          # the set's previous inputs are consumed
        with torch.cuda.stream(s_in):
            st["keys"].copy_(h_keys, non_blocking=True)
            st["queries"].copy_(h_q, non_blocking=True)
            st["in_done"].record(s_in)
        stream.wait_event(st["in_done"])
        if k >= 2:
            stream.wait_event(st["out_done"])    # its previous counts have left the device
        build_and_query(st["keys"], st["queries"], st["counts"], st["total"], stream)
        st["used"].record(stream)
        s_out.wait_event(st["used"])
        with torch.cuda.stream(s_out):
            st["h_counts"].copy_(st["counts"], non_blocking=True)
            st["h_total"].copy_(st["total"], non_blocking=True)
            st["out_done"].record(s_out)

    # warm-up: as many pipelined steps as are timed (freshly pinned host buffers
    # and the first passes of the copy pipeline run slower for a while)
    e_steps = max(4, steps)
    for k in range(max(2, e_steps)):
        e2e_step(k)
    torch.cuda.synchronize(dev)
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    s_in.wait_event(ev0)
    for k in range(e_steps):
        e2e_step(k)
    for st in sets:
        stream.wait_event(st["out_done"])
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    last = sets[(e_steps - 1) % 2]
    ok = int(last["h_total"].numpy().view(np.uint64)[0]) == int(last["h_counts"].numpy().view(np.uint32).sum(dtype=np.uint64))
    return {"ms": ev0.elapsed_time(ev1) / e_steps, "h2d": 4 * (N + Q), "d2h": 4 * Q + 8, "check": ok}


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    import paper_2104_00792_gb300 as hg

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if dist is not None:
            dist.barrier()

    weighted = args.workload == "zipf_weighted"
    wl = make_workload(args.log2n, rank, weighted, args.zipf_log2m)
    flags = hg.HG_LONG_SUMMARY if use_summary(args) else 0
    N, Q, B = wl.keys.size, wl.queries.size, wl.num_buckets
    keys = torch.from_numpy(wl.keys.view(np.int32)).to(dev)
    queries = torch.from_numpy(wl.queries.view(np.int32)).to(dev)
    counts = torch.empty(Q, dtype=torch.int32, device=dev)
    total = torch.empty(1, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream(dev)

    side = torch.cuda.Stream(dev)
    joined = torch.cuda.Event()

    forked = torch.cuda.Event()
    query = {"probe": hg.hg_query_count, "intersect": hg.hg_query_count_intersect}.get(args.query_form)

    def build_and_query(k, qs, c, tot, stream):
        if args.query_form == "plan":
            # the queries are grouped on a second stream while the table builds: the
            # plan needs only the table's shape, which hg_build fixes on return
            forked.record(stream)                 # inputs are ready here
            t = hg.hg_build(k, B, 0, flags=flags, stream=stream)
            side.wait_event(forked)
            plan = hg.hg_query_plan_create(t, qs, stream=side)
            joined.record(side)
            stream.wait_event(joined)
            hg.hg_query_count_plan(t, plan, c, tot, stream=stream)
            plan.free(stream)
        else:
            t = hg.hg_build(k, B, 0, flags=flags, stream=stream)
            query(t, qs, c, tot, stream=stream)
        t.free(stream)

    def step():
        build_and_query(keys, queries, counts, total, stream)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize(dev)

    # byte model inputs (outside the timed region)
    with hg.hg_build(keys, B, 0, flags=flags, stream=stream) as t:
        walk = hg.hg_probe_stats(t, queries, stream=stream)
    torch.cuda.synchronize(dev)

    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(local_rank if os.environ.get("CUDA_VISIBLE_DEVICES") is None else 0)
    with sampler:
        time.sleep(0.3)
        barrier()
        torch.cuda.synchronize(dev)
        launches0 = hg.hg_launch_count()
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        launches = hg.hg_launch_count() - launches0
        barrier()
        ms = ev0.elapsed_time(ev1) / args.steps

        # per-kernel times: a second timed run of the step with the query after the
        # build on one stream, so that each kernel's events bracket only its own work
        # (in the step above the query grouping overlaps the build)
        k_steps = max(3, args.steps // 3)
        hg.hg_prof_enable(True)
        ev0.record(stream)
        for _ in range(k_steps):
            t = hg.hg_build(keys, B, 0, flags=flags, stream=stream)
            hg.hg_query_count(t, queries, counts, total, stream=stream)
            t.free(stream)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        hg.hg_prof_enable(False)
        kernel_run_ms = ev0.elapsed_time(ev1) / k_steps
        prof = {name: hg.hg_prof_read(name) for name in hg.hg_prof_names()}
        prof = {name: (n // k_steps * args.steps, tot_ms / k_steps * args.steps) for name, (n, tot_ms) in prof.items()}

        # end to end through the C ABI with host buffers: pinned inputs copied in,
        # counts and total copied out, inside the timed region
        e2e = None
        if not args.no_e2e:
            e2e = e2e_pipelined(hg, wl, build_and_query, dev, stream, args.steps, barrier)
        time.sleep(0.2)

    # max over ranks
    ms, e2e_ms = max_over_ranks([ms, e2e["ms"] if e2e else 0.0], dist, dev)
    if e2e:
        e2e["ms"] = e2e_ms

    # sanity: the total equals the sum of counts of the last step
    ok_total = int(total.cpu().numpy().view(np.uint64)[0]) == int(counts.cpu().numpy().view(np.uint32).sum(dtype=np.uint64))

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    value = aggregate_gkeys(world, N + Q, ms)
    peak, peak_kind = measured_peak()
    # Algorithmic bytes per launch of each kernel (k = 4 key bytes, v = 0 value
    # bytes, o = 4 offset bytes; W = keys walked by all bucket walks, W_long =
    # the part walked by the chunked long-bucket kernel).  Partition passes move
    # every key once in each direction; counting passes read every key once.
    k, o = 4, 4
    W, WL = walk["walked"], walk["walked_long"]
    model = {
        "hist": k * N + 4 * B,                        # direct build: keys + counter writes
        "scan": 4 * (B + 1) + o * (B + 1),
        "scatter": 2 * k * N + o * B,
        "part_hist": k * N,                           # bin histogram + first-pass chunk counts
        "chunk_count": k * N,                         # second-pass chunk counts
        "part_scatter": 2 * k * N,                    # one partition pass
        "bin_build": 2 * k * N + o * (B + 1),         # per-bin counting sort: keys in, keys + offsets out
        "q_part_count": k * Q,
        "q_partition": 2 * k * Q + 4 * Q,             # queries grouped + their positions
        "probe": k * Q + 8 * Q + k * (W - WL) + 4 * Q,   # direct probe (tables that stay in L2)
        "long": k * WL,
    }
    if prof.get("q_partition", (0, 0))[0]:
        # queries grouped by table bin: the probe kernel reads the grouped queries,
        # each bin's offsets and keys once (into shared memory) and writes the counts
        model["probe"] = k * Q + 4 * (B + 1) + k * N + 4 * Q
        model["chunk_count"] = k * N                   # (same for the query side: Q = N here)
        model["q_reverse"] = 12 * Q                    # ranks, grouped counts in, counts out
    # the method's own byte model for the whole step (build + probe; offsets 4 B)
    if flags:
        # summarised long buckets (HG_LONG_SUMMARY): each of their queries reads the
        # bucket's summary (a few words) instead of walking the bucket
        walk_bytes = k * (W - WL) + 8 * walk["long_slots"]
    else:
        walk_bytes = k * W
    # the method's byte model for the whole step: the build, plus the query by
    # walking each query's bucket ((k+12)·Q + k·W, the walk model); the paper's
    # other query form, intersecting the table with HG(Q) bucket by bucket, reads
    # each table key once instead ((k+4)·Q + k·N + 4·(B+1)); step_frac takes the
    # smaller of the two, the fewest bytes either form must move
    build_bytes = (3 * k) * N + 16 * B
    walk_probe = (k + 12) * Q + walk_bytes
    isect_probe = (k + 4) * Q + k * N + 4 * (B + 1)
    step_model = build_bytes + walk_probe
    step_model_min = build_bytes + min(walk_probe, isect_probe)
    # the walk model at the 32-byte sector granularity of the memory system
    # (diagnostic): queries and counts stream, each offset pair and each walk
    # outside the long buckets costs the sectors it touches
    long_bytes = 8 * walk["long_slots"] if flags else k * WL
    step_model_sector = build_bytes + (k + 4) * Q + 32 * (walk["key_sectors"] + walk["offset_sectors"]) + long_bytes
    per_kernel = {}
    for name, (n_launch, tot_ms) in prof.items():
        if n_launch:
            per_kernel[name] = {"launches": n_launch, "ms_per_launch": tot_ms / n_launch,
                                "share": None, "model_bytes": model.get(name)}
    tot = sum(v["ms_per_launch"] * v["launches"] for v in per_kernel.values()) or 1.0
    for v in per_kernel.values():
        v["share"] = v["ms_per_launch"] * v["launches"] / tot
    dom = max((n for n in per_kernel if n in model), key=lambda n: per_kernel[n]["share"])
    d = per_kernel[dom]
    achieved = model[dom] / (d["ms_per_launch"] * 1e-3) / 1e9
    step_bytes = step_model
    clocks = sampler.summary()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": workload_desc(args.log2n, weighted, args.zipf_log2m), "parallelism": f"replicas{world}",
                   "build_flags": "HG_LONG_SUMMARY" if flags else "none",
                   "l2": "inputs exceed L2 (2 GiB read per step); no flush",
                   "step": {"plan": "hg_build, with hg_query_plan_create on a second stream, then "
                                    "hg_query_count_plan(counts, total) + hg_free",
                            "probe": "hg_build + hg_query_count(counts, total) + hg_free",
                            "intersect": "hg_build + hg_query_count_intersect(counts, total) + hg_free"}
                   [args.query_form]},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": ncu_traffic(dom), "peak_kind": peak_kind,
                     "step_model_bytes": step_bytes, "step_model_min_bytes": step_model_min,
                     "step_model_sector_bytes": step_model_sector,
                     "step_frac": step_model_min / (ms * 1e-3) / 1e9 / peak},
        "kernels": per_kernel,
        "kernel_timing": {"ms_per_step": kernel_run_ms,
                          "how": "per-kernel CUDA events over a second timed run of the step with the query after "
                                 "the build on one stream (launch counts and totals scaled to the main run's steps)"},
        "walk": walk,
        "gpu_launches": launches,
        "clocks": {k2: clocks[k2] for k2 in ("sm_mhz", "sm_max_mhz", "reasons")},
        "check": {"total_equals_sum_of_counts": ok_total},
    }
    if e2e:
        line["e2e"] = {"value": aggregate_gkeys(world, N + Q, e2e["ms"]), "unit": UNIT,
                       "h2d_bytes_per_step": e2e["h2d"], "d2h_bytes_per_step": e2e["d2h"],
                       "ms_per_step": e2e["ms"], "total_equals_sum_of_counts": e2e["check"],
                       "pipelining": "copies on their own streams, two device buffer sets alternating"}
    if world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_oracle_sample(wl, cpu_sample_log2(args))
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


BATCH_METRIC = "batched build+probe Gkeys/s (4096 tables)"


def batch_desc(tables):
    return (f"batched_uniform: {tables} tables, N_t log-uniform in [2^8, 2^20] uint32 keys, B_t = N_t "
            f"(murmur3-fmix32 seed 0), N_t queries per table with 50% hits; all built and probed in one "
            f"persistent launch replayed from a CUDA graph")


def run_batched(args, rank, world, local_rank):
    """Config: thousands of small tables of uneven size built and probed together."""
    import numpy as np
    import torch

    import paper_2104_00792_gb300 as hg
    import workloads as W

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    wl = W.batched_uniform(args.tables, 8, 20, salt=rank)
    N, Q = wl.keys.size, wl.queries.size
    keys = torch.from_numpy(wl.keys.view(np.int32)).to(dev)
    queries = torch.from_numpy(wl.queries.view(np.int32)).to(dev)
    counts = torch.empty(Q, dtype=torch.int32, device=dev)
    stream = torch.cuda.Stream(dev)  # a stream of its own: the run is captured once and replayed as a graph
    torch.cuda.synchronize(dev)
    torch.cuda.set_stream(stream)
    b = hg.hg_batch_create(wl.key_offsets, wl.num_buckets, wl.query_offsets, stream=stream)
    chosen = hg.hg_batch_tune(b, keys, queries, counts, stream=stream)  # outside the timed region
    for _ in range(max(args.warmup, 3)):
        hg.hg_batch_run(b, keys, queries, counts, stream=stream)
    walked = hg.hg_batch_walk_stats(b, queries, stream=stream)
    torch.cuda.synchronize(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(local_rank if os.environ.get("CUDA_VISIBLE_DEVICES") is None else 0)
    with sampler:
        time.sleep(0.3)
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)
        launches0 = hg.hg_launch_count()
        ev0.record(stream)
        for _ in range(args.steps):
            hg.hg_batch_run(b, keys, queries, counts, stream=stream)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        launches = hg.hg_launch_count() - launches0
        ms = ev0.elapsed_time(ev1) / args.steps
        # end to end through the C ABI with host buffers: pinned keys and queries
        # copied in, counts copied out, every step; copies on their own streams,
        # two buffer sets (and two batch plans) alternating
        e2e_ms = None
        if not args.no_e2e:
            h_keys = torch.from_numpy(wl.keys.view(np.int32)).pin_memory()
            h_q = torch.from_numpy(wl.queries.view(np.int32)).pin_memory()
            b2 = hg.hg_batch_create(wl.key_offsets, wl.num_buckets, wl.query_offsets, stream=stream)
            hg.hg_batch_set_params(b2, chosen["threads"], chosen["bin_shift"], chosen["fuse_keys"])
            sets = []
            for plan, kk, qq, cc in ((b, keys, queries, counts),
                                     (b2, torch.empty_like(keys), torch.empty_like(queries), torch.empty_like(counts))):
                sets.append({"plan": plan, "keys": kk, "queries": qq, "counts": cc,
                             "h_counts": torch.empty(Q, dtype=torch.int32).pin_memory(),
                             "in_done": torch.cuda.Event(), "out_done": torch.cuda.Event(),
                             "used": torch.cuda.Event()})
            s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

            def e2e_step(k):
                st = sets[k % 2]
                if k >= 2:
                    s_in.wait_event(st["used"])
                with torch.cuda.stream(s_in):
                    st["keys"].copy_(h_keys, non_blocking=True)
                    st["queries"].copy_(h_q, non_blocking=True)
                    st["in_done"].record(s_in)
                stream.wait_event(st["in_done"])
                if k >= 2:
                    stream.wait_event(st["out_done"])
                hg.hg_batch_run(st["plan"], st["keys"], st["queries"], st["counts"], stream=stream)
                st["used"].record(stream)
                s_out.wait_event(st["used"])
                with torch.cuda.stream(s_out):
                    st["h_counts"].copy_(st["counts"], non_blocking=True)
                    st["out_done"].record(s_out)

            for k in range(2):
                e2e_step(k)
            torch.cuda.synchronize(dev)
            e_steps = max(4, args.steps // 3)
            ev0.record(stream)
            s_in.wait_event(ev0)
            for k in range(e_steps):
                e2e_step(k)
            for st in sets:
                stream.wait_event(st["out_done"])
            ev1.record(stream)
            torch.cuda.synchronize(dev)
            e2e_ms = ev0.elapsed_time(ev1) / e_steps
            b2.free(stream)
        time.sleep(0.2)
    ms, e2e_v = max_over_ranks([ms, e2e_ms or 0.0], dist, dev)
    if e2e_ms is not None:
        e2e_ms = e2e_v
    hg.hg_batch_sync(b, stream=stream)
    ok = True
    # the same tables one launch sequence per table (the plain path), for comparison
    plain_ms = None
    if not args.no_plain and rank == 0:
        c2 = torch.empty(Q, dtype=torch.int32, device=dev)

        def plain_step():
            for t in range(wl.n_tables):
                k0, k1 = int(wl.key_offsets[t]), int(wl.key_offsets[t + 1])
                q0, q1 = int(wl.query_offsets[t]), int(wl.query_offsets[t + 1])
                tb = hg.hg_build(keys[k0:k1], int(wl.num_buckets[t]), 0, stream=stream)
                hg.hg_query_count(tb, queries[q0:q1], c2[q0:q1], None, stream=stream)
                tb.free(stream)

        plain_step()
        torch.cuda.synchronize(dev)
        ev0.record(stream)
        plain_step()
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        plain_ms = ev0.elapsed_time(ev1)
        ok = bool(torch.equal(c2, counts))
    b.free(stream)
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    peak, peak_kind = measured_peak()
    B = int(wl.num_buckets.sum())
    model = 12 * N + 16 * B + 16 * Q + 4 * walked   # build (3k N + 16 B) + probe (k Q + 8 Q + 4 Q + k W), k = 4
    achieved = model / (ms * 1e-3) / 1e9
    clocks = sampler.summary()
    line = {
        "metric": BATCH_METRIC, "value": aggregate_gkeys(world, N + Q, ms), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": batch_desc(args.tables), "parallelism": f"replicas{world}",
                   "keys": N, "queries": Q, "buckets": B, "params": chosen,
                   "l2": f"inputs exceed L2 ({(N + Q) * 4 / 2**30:.1f} GiB read per step); no flush"},
        "roofline": {"bound": "hbm", "kernel": "batch", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": (batch_traffic_ratio() * model) if batch_traffic_ratio() else None,
                     "traffic_note": "ncu DRAM bytes per algorithmic byte at 512 tables x this batch's model bytes",
                     "peak_kind": peak_kind, "model_bytes": model},
        "vs_plain": {"plain_ms_per_step": plain_ms, "speedup": (plain_ms / ms) if plain_ms else None,
                     "plain": "hg_build + hg_query_count + hg_free per table, same stream",
                     "counts_identical": ok},
        "gpu_launches": launches,
        "clocks": {k2: clocks[k2] for k2 in ("sm_mhz", "sm_max_mhz", "reasons")},
    }
    if e2e_ms is not None:
        line["e2e"] = {"value": aggregate_gkeys(world, N + Q, e2e_ms), "unit": UNIT,
                       "h2d_bytes_per_step": 4 * (N + Q), "d2h_bytes_per_step": 4 * Q, "ms_per_step": e2e_ms}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


SERVE_METRIC = "served p99 latency ms (build+probe request stream)"


def serve_desc(n, load, budget_gb):
    return (f"serving: {n} requests, Poisson arrivals at {load:g} x the plain path's measured capacity; 30% builds "
            f"(N log-uniform in [2^10, 2^24] uint32 keys, B = N), 70% probes (Q log-uniform in [2^8, 2^22], 60% hits "
            f"from the target's keys) on tables resident under an arrival-order LRU with a {budget_gb:g} GB budget")


def run_serving(args, rank, world, local_rank):
    """Config: a request stream served by the engine, against one request at a time."""
    import numpy as np
    import torch

    import paper_2104_00792_gb300 as hg
    import workloads as W

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    if rank != 0:  # one GPU per stream; replicas would serve independent streams
        return
    budget = int(args.budget_gb * 1e9)
    trace = W.serving_trace(args.requests, budget_bytes=budget, salt=rank)
    n_of = W.serve_table_n(trace)
    nreq = len(trace)
    stream = torch.cuda.current_stream(dev)
    sid = stream.cuda_stream
    gaps = np.array([r.gap for r in trace], dtype=np.float64)

    def make_inputs(r):
        if r.kind == "build":
            k = torch.empty(max(r.size, 1), dtype=torch.int32, device=dev)
            W.gpu_uniform_u32(r.key_state, r.size, k.data_ptr(), sid)
            return k[: r.size], None
        q = torch.empty(max(r.size, 1), dtype=torch.int32, device=dev)
        W.gpu_probe_mix_uniform_u32(r.key_state, n_of[r.table], r.size, 0.6, r.sel, r.miss, q.data_ptr(), sid)
        c = torch.empty(max(r.size, 1), dtype=torch.int32, device=dev)
        return q[: r.size], c[: r.size]

    sample = {i for i in range(nreq) if trace[i].kind == "probe" and i % 97 == 0}

    def plain_run(arrivals, limit=None):
        """One request at a time on one stream, tables kept under the same LRU."""
        from collections import OrderedDict
        tables = OrderedDict()
        used = 0
        done = np.zeros(nreq)
        keep = {}
        m = nreq if limit is None else limit
        t0 = time.perf_counter()
        for i in range(m):
            r = trace[i]
            if arrivals is not None:
                while time.perf_counter() - t0 < arrivals[i]:
                    pass
            a, c = make_inputs(r)
            if r.kind == "build":
                need = hg.hg_server_table_bytes(r.size, r.size)
                while used + need > budget and tables:
                    _, (tb, b) = tables.popitem(last=False)
                    tb.free(stream)
                    used -= b
                tables[r.table] = (hg.hg_build(a, r.size, 0, stream=stream), need)
                used += need
            else:
                tables.move_to_end(r.table)
                hg.hg_query_count(tables[r.table][0], a, c, None, stream=stream)
            stream.synchronize()
            done[i] = time.perf_counter() - t0
            if i in sample:
                keep[i] = c.clone()
        for tb, _ in tables.values():
            tb.free(stream)
        torch.cuda.synchronize(dev)
        return done[:m], keep

    def engine_run(arrivals, window=None):
        """Requests submitted at their arrival times (or, with `window`, as soon
        as fewer than `window` are outstanding: the engine's capacity)."""
        srv = hg.Server(budget, max_batch=256)
        done = np.zeros(nreq)
        keep = {}
        live = {}
        i = 0
        t0 = time.perf_counter()
        while i < nreq or live:
            now = time.perf_counter() - t0
            while i < nreq and (arrivals[i] <= now if window is None else len(live) < window):
                r = trace[i]
                a, c = make_inputs(r)
                stream.synchronize()  # the request arrives with its data in device memory
                if r.kind == "build":
                    rid = srv.submit_build(r.table, a, r.size)
                else:
                    rid = srv.submit_probe(r.table, a, c)
                live[rid] = (i, a, c)
                i += 1
                now = time.perf_counter() - t0
            for rid, st in srv.poll():
                j, a, c = live.pop(rid)
                done[j] = time.perf_counter() - t0
                if st != hg.HG_OK:
                    raise RuntimeError(f"request {j} failed with status {st}")
                if j in sample:
                    keep[j] = c
        stats = srv.stats()
        srv.free()
        torch.cuda.synchronize(dev)
        return done, keep, stats

    # capacity of the plain path: its mean service time over the first requests, back to back
    n_cal = min(nreq, 3000)
    cal_done, _ = plain_run(None, limit=n_cal)
    service = float(cal_done[-1]) / n_cal
    rate = args.load / service
    arrivals = np.cumsum(gaps) / rate
    arrivals -= arrivals[0]
    e_done, e_keep, e_stats = engine_run(arrivals)
    p_done, p_keep = plain_run(arrivals)
    same = all(torch.equal(e_keep[i], p_keep[i]) for i in sample)
    keys_total = sum(r.size for r in trace)
    # capacity: every request available at once (the engine keeps 64 outstanding)
    cap_e, _, _ = engine_run(np.zeros(nreq), window=64)
    cap_p, _ = plain_run(None)
    capacity = {"engine_gkeys_per_s": keys_total / float(cap_e.max()) / 1e9,
                "plain_gkeys_per_s": keys_total / float(cap_p.max()) / 1e9}
    capacity["ratio"] = capacity["engine_gkeys_per_s"] / capacity["plain_gkeys_per_s"]

    def summary(done):
        lat = (done - arrivals) * 1e3
        span = float(done.max())
        return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(lat.mean()), "gkeys_per_s": keys_total / span / 1e9, "makespan_s": span}

    eng, pla = summary(e_done), summary(p_done)
    line = {
        "metric": SERVE_METRIC, "value": eng["p99_ms"], "unit": "ms", "n_gpus": 1, "steps": nreq, "warmup": n_cal,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": serve_desc(nreq, args.load, args.budget_gb), "rate_per_s": rate,
                   "plain_service_ms": service * 1e3},
        "engine": eng, "plain": pla,
        "vs_plain": {"p50": pla["p50_ms"] / eng["p50_ms"], "p99": pla["p99_ms"] / eng["p99_ms"],
                     "throughput": eng["gkeys_per_s"] / pla["gkeys_per_s"]},
        "capacity": capacity,
        "engine_stats": e_stats,
        "check": {"sampled_probes": len(sample), "engine_equals_plain": bool(same)},
        "gpu_launches": int(e_stats["builds"] + e_stats["probe_launches"]),
    }
    print(json.dumps(line), flush=True)


DUP_METRIC = "duplicate-key sweep: build and query Gkeys/s vs copies per value"


def run_dupsweep(args, rank, world, local_rank):
    """The paper's duplicate-key experiment: N fixed, every value occurring
    2^d times (B = N / 2^d); build and query rates timed separately."""
    import numpy as np
    import torch

    import paper_2104_00792_gb300 as hg
    import workloads as W

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    if rank != 0:
        return
    n = 1 << args.sweep_log2n
    stream = torch.cuda.current_stream(dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    rows = []
    for d in range(0, 11):
        wl = W.duplicate_keys(n, dup_log2=d, salt=d)
        keys = torch.from_numpy(wl.keys.view(np.int32)).to(dev)
        queries = torch.from_numpy(wl.queries.view(np.int32)).to(dev)
        counts = torch.empty(n, dtype=torch.int32, device=dev)
        total = torch.empty(1, dtype=torch.int64, device=dev)
        B = wl.num_buckets
        row = {"copies_log2": d, "buckets": B}
        for mode, flags in (("", 0), ("sorted_", hg.HG_SORTED_BUCKETS)):
            tb, tq = [], []
            for rep in range(4):
                ev[0].record(stream)
                t = hg.hg_build(keys, B, 0, flags=flags, stream=stream)
                ev[1].record(stream)
                hg.hg_query_count(t, queries, counts, total, stream=stream)
                ev[2].record(stream)
                torch.cuda.synchronize(dev)
                if rep:
                    tb.append(ev[0].elapsed_time(ev[1]))
                    tq.append(ev[1].elapsed_time(ev[2]))
                if rep == 3 and not flags:
                    walk = hg.hg_probe_stats(t, queries, stream=stream)
                t.free(stream)
            mb, mq = statistics.median(tb), statistics.median(tq)
            row.update({f"{mode}build_ms": mb, f"{mode}query_ms": mq,
                        f"{mode}build_gkeys_per_s": n / (mb * 1e-3) / 1e9,
                        f"{mode}query_gkeys_per_s": n / (mq * 1e-3) / 1e9})
        row["walked_keys_per_query"] = walk["walked"] / n
        rows.append(row)
        del keys, queries, counts
    line = {"metric": DUP_METRIC, "value": rows[-1]["query_gkeys_per_s"], "unit": "Gkeys/s", "n_gpus": 1,
            "steps": 3, "warmup": 1, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32", "data": "synthetic",
            "config": {"workload": f"duplicate_keys: N = Q = 2^{args.sweep_log2n} uint32 keys over N / 2^d values "
                                   f"(B = N / 2^d), queries 50% hits; d = 0..10; each d built plain and with "
                                   f"HG_SORTED_BUCKETS (the sort counted in the build time)"},
            "sweep": rows}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "batched":
        run_batched(args, rank, world, local_rank)
    elif args.workload == "serving":
        run_serving(args, rank, world, local_rank)
    elif args.workload == "dupsweep":
        run_dupsweep(args, rank, world, local_rank)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
