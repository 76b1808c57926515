"""The committed ncu summaries the bench reads belong to the kernels in the tree.

bench.py copies a kernel's DRAM traffic (and the step's sum) into its JSON
line only while the traffic summary's recorded source hash equals the hash of
the current kernel sources; a kernel change without a new capture would leave
`traffic` null.  These checks run without a GPU."""
import os
import re

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_traffic_summary_matches_the_kernel_sources():
    rows = bench.ncu_traffic_rows()
    assert rows is not None, "profiles/dram_traffic_zipf_large.txt was captured on other kernel sources"
    # every kernel of the headline step that moves data has a row, as do the two stages
    for name in ("part_hist", "part_scatter", "part_scatter2", "chunk_count", "bin_small", "bin_big", "huge_count",
                 "q_part_count", "q_partition", "q_partition2", "probe_hash", "q_reverse", "sum_count", "bin_stage",
                 "probe_stage"):
        v = bench.ncu_traffic(name)
        assert v is not None and v > 0, name


def test_stage_rows_are_the_sums_of_their_kernels():
    rows = bench.ncu_traffic_rows()
    assert rows is not None
    get = lambda n: float(rows.get(f"traffic_bytes_per_launch.{n}", 0))  # noqa: E731
    bin_parts = ("bin_small", "bin_big", "huge_count", "huge_scan", "huge_items", "bin_build")
    probe_parts = ("probe_hash", "probe", "long_prep", "long", "long_copy")
    assert abs(get("bin_stage") - sum(get(p) for p in bin_parts)) <= len(bin_parts)
    assert abs(get("probe_stage") - sum(get(p) for p in probe_parts)) <= len(probe_parts)


def test_profile_summaries_name_their_commands():
    # each summary gives the command that made it, running committed files only
    for name in ("launches_zipf_large_2p28.md", "dram_traffic_zipf_large.txt", "ncu_full_top_kernels_2p26.md",
                 "dram_traffic_batch.txt"):
        text = open(os.path.join(ROOT, "profiles", name)).read()
        assert "--clock-control none" in text, name
        assert re.search(r"python (bench\.py|-c)", text), name
        assert "_work/" not in text, name
