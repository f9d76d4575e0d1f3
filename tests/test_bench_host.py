"""Host-side pieces of bench.py that need no GPU: the workload description
in the JSON line, the roofline peak (the measured copy bandwidth, else the
stated fallback) and the streaming-CPU leg on a small ring."""
import json

import numpy as np

import bench


def test_workload_config_describes_the_hd_video_window():
    cfg = bench.workload_config(1920 * 1080 * 3, {"parallelism": "1 GPU"})
    assert cfg["n"] == 6220800 and cfg["m"] == bench.M_WIN == 100 and cfg["r"] == bench.R_MODES == 10
    assert cfg["frame"] == [1080, 1920, 3]
    assert "L2" in cfg["l2"] and cfg["parallelism"] == "1 GPU"
    json.dumps(cfg)                                    # serialisable as part of the JSON line


def test_measured_peak_or_fallback(tmp_path, monkeypatch):
    peak, kind = bench.measured_peaks()
    assert peak > 1000.0 and kind in ("measured", "fallback")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))  # no file: the stated fallback
    assert bench.measured_peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 7000.5}))
    assert bench.measured_peaks() == (7000.5, "measured")


def test_streaming_cpu_leg_on_a_small_ring():
    frames = np.random.default_rng(0).integers(0, 256, (4, 4096), dtype=np.uint8)
    out = bench.streaming_cpu_rate(frames, 0.05)
    assert out["value"] > 0 and out["unit"] == bench.UNIT and out["cores"] >= 1
    assert out["GB/s"] > 0 and "pushes" in out["sample"]
    json.dumps(out)
