"""A short soak of the FP64 FT-DGEMM (config 5a at reduced size and time, raised rate):
back-to-back launches with Poisson-drawn accumulator bit flips on distinct tiles. No
false alarm, no uncorrectable or checksum-only tile, every detected fault corrected, and
the final C bitwise equal to a clean run unless an undetected (sub-threshold) flip hit the
last launch."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import bench  # noqa: E402
import paper_2104_00897_gb300 as fb  # noqa: E402


def test_soak_fp64_short():
    fb.load()
    t = bench.run_soak(torch.device("cuda", 0), 2048, 4.0, seed=77, rate_per_s=300.0, batch=64)
    assert t["launches"] > 50 and t["injected"] > 200
    assert t["false_alarms"] == 0 and t["uncorrectable"] == 0 and t["checksum_only"] == 0 and t["status"] == 0
    assert t["corrected"] == t["detected"]
    assert t["detected"] + t["undetected"] == t["injected"]
    assert t["undetected"] <= 0.01 * t["injected"]
    assert t["final_c_equals_clean"] or t["undetected"] > 0
