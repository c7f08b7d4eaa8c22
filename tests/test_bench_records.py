"""The measurement records that bench.py reads stay in step with the sources
(no GPU): the DRAM traffic of the fused kernel was captured at the current
kernel sources for the benchmark's default depth, and its figures are
consistent with the algorithmic bytes of a launch."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_traffic_record_matches_current_kernel_sources():
    n, K = 8192, 3
    traffic = bench.recorded_traffic(n, K)
    assert traffic is not None, ("profiles/fused_kernel_traffic.json has no capture for the "
                                 "current kernel source hash %s" % bench.kernel_source_hash())
    algorithmic = bench.BYTES_PER_SITE_LAUNCH * n * n
    assert 1.0 <= traffic / algorithmic < 1.1


def test_traffic_record_is_self_consistent():
    with open(os.path.join(ROOT, "profiles", "fused_kernel_traffic.json")) as f:
        rec = json.load(f)
    for c in rec["captures"]:
        assert c["dram_bytes_per_launch"] == c["dram_read_bytes"] + c["dram_write_bytes"]
        assert c["algorithmic_bytes_per_launch"] == bench.BYTES_PER_SITE_LAUNCH * c["n"] ** 2
        assert "--clock-control none" in c["command"]
