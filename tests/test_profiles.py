"""The committed ncu summaries against the sources.  The benchmark reports
the DRAM traffic of the large workload's generation kernel from the
traffic-to-algorithmic ratio of its committed full-size capture, and only
while the capture was taken with the current kernel sources (a hash of
them); a change to those sources without a new capture would silently
drop that figure, which this test turns into a failure."""
import os
import re

import bench

PROFILES = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "profiles")


def _machine_lines(name):
    kv = {}
    with open(os.path.join(PROFILES, name)) as fh:
        for line in fh:
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
    return kv


def test_large_traffic_capture_matches_kernel_sources():
    kv = _machine_lines("persist_kernel_large.txt")
    assert kv["kernel_source_sha256_16"] == bench.kernel_source_hash(), (
        "the generation kernels changed since profiles/persist_kernel_large.txt was captured")
    name = kv["workload"]
    for shape in ((2, 2), (2, 4), (1, 8)):
        ratio = bench.profiled_traffic(name, shape)
        assert ratio is not None and 1.0 <= ratio < 1.3, (shape, ratio)


def test_every_summary_names_its_command():
    for name in sorted(os.listdir(PROFILES)):
        assert name.endswith((".txt", ".md")), name
        text = open(os.path.join(PROFILES, name)).read()
        assert re.search(r"\bncu\b", text) and "--clock-control none" in text, name
        assert "_work" not in text and "/root/" not in text, name
