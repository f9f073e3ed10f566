"""The committed ncu records (profiles/ncu_traffic.json) that bench.py uses for
`roofline.traffic` and `roofline_alu` are tied to the kernel sources they were
captured on: every record names a kernel bench.py knows and carries that
kernel's source digest, and the figures are plausible for the capture (DRAM
bytes per point near the 8-byte read of one pass, positive instruction
counts)."""
import json
import os

import bench


def test_records_match_the_current_kernel_sources():
    with open(os.path.join(bench.ROOT, "profiles", "ncu_traffic.json")) as f:
        rec = json.load(f)
    assert rec["entries"]
    for ent in rec["entries"]:
        assert ent["kernel"] in bench.KERNEL_SOURCES
        assert ent["source_digest"] == bench.source_digest(ent["kernel"]), ent["kernel"]
        b = ent["dram_bytes_per_point_per_launch"]
        assert b is None or 7.9 < b < 16.1
        assert ent["lane_instructions_per_point_per_launch"] > 0
        assert "ncu" in ent["how"] or ent["how"] == "same capture"


def test_default_workload_has_traffic_and_instruction_records():
    pts = 64 * 256 * 256
    assert bench.recorded_traffic("fast_pass_kernel", "batch64_256x256", pts) is not None
    assert bench.recorded_lane_instructions("fast_pass_kernel", "batch64_256x256") is not None
