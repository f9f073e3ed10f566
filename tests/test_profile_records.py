"""The committed ncu records (profiles/ncu_traffic.json) that bench.py uses for
`roofline.traffic` and `roofline_alu` are tied to the kernel sources they were
captured on: every record names a kernel bench.py knows and carries a source
digest, the figures are plausible for the capture, and bench.py uses a record
only while that digest equals the kernel's current sources (a stale record
gives null, never an old figure)."""
import json
import os

import bench


def _records():
    with open(os.path.join(bench.ROOT, "profiles", "ncu_traffic.json")) as f:
        return json.load(f)["entries"]


def test_records_are_well_formed():
    ents = _records()
    assert ents
    for ent in ents:
        assert ent["kernel"] in bench.KERNEL_SOURCES
        assert len(ent["source_digest"]) == 16
        b = ent["dram_bytes_per_point_per_launch"]
        assert b is None or 7.9 < b < 32.1
        assert ent["lane_instructions_per_point_per_launch"] > 0
        assert "ncu" in ent["how"] or ent["how"] == "same capture"


def test_stale_records_are_not_used():
    for ent in _records():
        fresh = ent["source_digest"] == bench.source_digest(ent["kernel"])
        got = bench.recorded_traffic(ent["kernel"], ent["workload"], 1000)
        ipp = bench.recorded_lane_instructions(ent["kernel"], ent["workload"])
        if not fresh:
            # another record of the same kernel and workload may be fresh
            others = [e for e in _records() if e["kernel"] == ent["kernel"] and
                      e["workload"] == ent["workload"] and
                      e["source_digest"] == bench.source_digest(e["kernel"])]
            if not others:
                assert got is None and ipp is None, ent["kernel"]


def test_digest_follows_the_sources():
    base = bench.source_digest("fast_pass_kernel")

    def read_changed(name):
        with open(os.path.join(bench.ROOT, "paper_2512_04317_gb300", "csrc", name), "rb") as f:
            data = f.read()
        return data + (b"//" if name == "mx_device.cuh" else b"")
    assert bench.source_digest("fast_pass_kernel", read=read_changed) != base
