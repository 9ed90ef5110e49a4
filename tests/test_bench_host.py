"""Host-side logic of bench.py (no GPU): the roofline of the dominant kernel,
the diagonal solves' algorithmic flops, and the traffic records' source
hashes (a record reports only for the kernel sources it was measured on)."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _prof(diag_ms, upd_ms):
    return [{"update_ms": upd_ms, "update_launches": 156, "update_tensor_flops": 7.9995e13,
             "diag_ms": diag_ms, "diag_launches": 157}]


def test_diag_flops_close_to_n2_tb():
    f = bench.diag_alg_flops(20000, 128, 157)
    assert abs(f / (20000.0 ** 2 * 128) - 1.0) < 0.02


def test_dominant_kernel_first():
    peaks = {"bf16_tflops_sustained": 1730.2, "sm_max_mhz": 2070.0}
    roof, other = bench.rooflines(_prof(110.0, 80.7), 205.8, 20000, "bf16x5", 128, peaks, "measured", 152)
    assert roof["kernel"] == "k_diag" and roof["bound"] == "alu"
    assert other["kernel"] == "k_update_tc" and other["bound"] == "tensor"
    assert abs(roof["peak"] - 152 * 4 * 2.07e9 / 1e12) < 1e-3
    assert 0.3 < roof["frac"] < 0.45
    assert abs(other["achieved"] - 7.9995e13 / 80.7e-3 / 1e12) < 0.1
    roof2, other2 = bench.rooflines(_prof(60.0, 80.7), 170.0, 20000, "bf16x5", 128, peaks, "measured", 152)
    assert roof2["kernel"] == "k_update_tc" and other2["kernel"] == "k_diag"
    for r in (roof, other):
        assert set(("bound", "achieved", "peak", "unit", "frac", "traffic")) <= set(r)


def test_traffic_records_apply_only_to_their_workload():
    # a record reports for its own workload (and only while the kernel sources
    # hash to the measured version; otherwise null)
    for k in ("k_update_tc", "k_diag"):
        v = bench.measured_traffic(k)
        assert v is None or v == bench.TRAFFIC[k]["bytes_per_launch"]
        assert bench.measured_traffic(k, n=4000) is None
        assert bench.measured_traffic(k, prec="fp64") is None
    assert bench.measured_traffic("k_post") is None
