"""The roofline object of bench.py (host logic, no GPU): algorithmic bytes
per launch over the mean launch time, against the measured HBM peak."""

import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

WL = bench.WORKLOADS["2d"]
DOF = (9 * 1024 - 1) ** 2


def _prof(**kinds):
    base = {k: dict(launches=0, ms=0.0, bytes=0.0, flops64=0.0)
            for k in ("forward", "fused", "inverse", "apply", "apply_df")}
    base.update(kinds)
    return base


def test_pencil_pass_dominant():
    prof = _prof(fused=dict(launches=30, ms=30.0, bytes=30 * 8.0 * DOF, flops64=0.0),
                 forward=dict(launches=30, ms=10.0, bytes=30 * 9.0 * DOF, flops64=0.0))
    roof, kind = bench.roofline(prof, 10, {"hbm_gbs": 6779.4}, WL)
    assert kind == "fused" and roof["bound"] == "hbm"
    want = 8.0 * DOF / 1e-3 / 1e9          # one launch per ms
    assert abs(roof["achieved"] - want) < 1e-6 * want
    assert abs(roof["frac"] - want / 6779.4) < 1e-9


def test_residual_dominant_uses_fused_residual_bytes():
    # 10 steps x 2 residuals x 3 launches, 1 ms each
    prof = _prof(apply_df=dict(launches=60, ms=60.0, bytes=60 * 25.0 * DOF, flops64=60 * 1e10))
    roof, kind = bench.roofline(prof, 10, {"hbm_gbs": 6779.4}, WL, residuals_per_step=2)
    assert kind == "apply_df"
    alg = 20.0 * DOF / 3.0                  # 20 B/DOF per residual over its three launches
    assert abs(roof["algorithmic_bytes_per_launch"] - alg) < 1e-6 * alg
    assert abs(roof["frac"] - alg / 1e-3 / 1e9 / 6779.4) < 1e-9
    assert roof["secondary"]["fp32_lane_Tops"] > 0
    assert roof["traffic_over_algorithmic"] > 1.0


def test_fallback_peak_named():
    prof = _prof(inverse=dict(launches=1, ms=1.0, bytes=1e9, flops64=0.0))
    roof, _ = bench.roofline(prof, 1, {}, WL)
    assert roof["peak"] == 6800.0 and "fallback" in roof["peak_source"]
