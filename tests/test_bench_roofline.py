"""Host logic of the benchmark's HBM-stage fractions (CPU): achieved GB/s
from the stage's CUDA-event time and the algorithmic bytes per touched
Gaussian, against the measured copy peak."""
import json
import os

import bench


def _res(bf16, ms_adam=0.1, ms_pbwd=0.05, steps=400, visible=250_000):
    return {"stats": {"last_visible": visible}, "bf16": bf16, "stage_steps": steps,
            "stages": {"adam": (ms_adam * steps, steps), "preprocess_bwd": (ms_pbwd * steps, steps),
                       "raster_bwd": (0.33 * steps, steps)}}


def test_hbm_stage_fractions():
    peak, src = bench.measured_peaks()
    if os.path.exists(os.path.join(bench.ROOT, "MEASURED_PEAKS.json")):
        with open(os.path.join(bench.ROOT, "MEASURED_PEAKS.json")) as f:
            assert peak == json.load(f)["hbm_gbs"] and src == "measured"
    out = bench.hbm_stages(_res(True))
    a = out["adam"]
    assert a["bytes_per_launch"] == 1000.0 * 250_000
    assert abs(a["achieved_gbs"] - 2500.0) < 0.05  # 250 MB in 0.1 ms
    assert abs(a["frac"] - 2500.0 / peak) < 1e-4
    p = out["preprocess_bwd"]
    assert p["bytes_per_launch"] == (146 + 36 + 236) * 250_000.0
    assert abs(p["achieved_gbs"] - (146 + 36 + 236) * 250_000 / 0.05e-3 / 1e9) < 0.05
    f = bench.hbm_stages(_res(False))
    assert f["adam"]["bytes_per_launch"] == 1652.0 * 250_000
    assert "raster_bwd" not in out
    # several cameras per step: the touched set is not the last camera's
    assert bench.hbm_stages(_res(True), workload="city") is None
    # a stage that never ran is left out
    r = _res(True, ms_pbwd=0.0)
    assert "preprocess_bwd" not in bench.hbm_stages(r)
