"""Host-side pieces of bench.py that need no GPU."""

import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_committed_traffic_matches_the_kernel_sources():
    """profiles/ncu_traffic.txt holds DRAM bytes per launch for the current
    kernel sources, so the bench line's roofline carries ncu traffic; a
    kernel change without a new capture fails here."""
    for k in ("slice_forward", "band_analysis", "band_synthesis", "band_boundary", "slice_inverse", "slice_ola"):
        t = bench._ncu_traffic(k)
        assert t is not None and t > 0, k
    # the dominant kernel reads its coefficients once: traffic close to the
    # algorithmic 124 MB of the 60 s stereo workload
    assert 1.2e8 < bench._ncu_traffic("band_synthesis") < 2.0e8


def test_peaks_and_config():
    peak, kind = bench._peaks()
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        assert kind == "measured" and peak == float(json.load(open(path))["hbm_gbs"])
    else:
        assert kind == "fallback"
    cfg = bench._config(1, "pow2", "fp32", 4)
    assert cfg["workload"].startswith("60 s stereo")
    assert cfg["slice_cluster"] == 4 and cfg["precision"] == "fp32"
    assert "flushed" in cfg["l2"]
