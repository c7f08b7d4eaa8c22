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


def test_adjoint_byte_model_by_hand():
    # 1024^2 workload shape per site: 500 steps, checkpoints every 50, K = 2
    # backward, ts_evolve at K = 3 forward.  Forward: target conversion 16 +
    # overlap 16, then per segment of 50 steps a checkpoint copy 16 and
    # ceil(50 / 3) = 17 launches of 24.  Backward: costate 16 + G cleared 16
    # + gradient 20, then per segment a checkpoint copy 16 and ceil(50 / 2) =
    # 25 launches of 72 (psi and lambda in and out 32, table 8, G in and out 32).
    fwd, bwd = bench.adjoint_bytes(1, 500, 50, 2, 3)
    assert fwd == 32 + 10 * (16 + 24 * 17)
    assert bwd == 52 + 10 * (16 + 72 * 25)
    # a ragged last segment: 120 steps in segments of 50, 50, 20 at K = 3
    fwd, bwd = bench.adjoint_bytes(7, 120, 50, 3, 3)
    assert fwd == 7 * (32 + 2 * (16 + 24 * 17) + (16 + 24 * 7))
    assert bwd == 7 * (52 + 2 * (16 + 72 * 17) + (16 + 72 * 7))


def test_plain_and_merged_byte_models():
    # one sweep moves the state in and out; the phase also reads the table
    assert bench.PLAIN_BYTES["f32"] == 8 * (8 + 8) + 8 + 8 + 8
    assert bench.PLAIN_BYTES["f64"] == 8 * (16 + 16) + 16 + 16 + 16
    # FP64 ts_evolve: 6 T + 2 sweeps of 32 B and T phases of 48 B for T steps
    assert abs(bench.fp64_merged_bytes(200) - ((6 * 200 + 2) * 32 + 200 * 48) / 200) < 1e-12
    assert abs(bench.fp64_merged_bytes(1) - 8 * 32 / 1 - 48) < 1e-12
