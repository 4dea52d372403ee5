"""Host-side helpers of bench.py (no GPU): the two whole-stage rooflines, the measured HBM
figure, the host CPU description and the OpenMP thread control used for the single-core
oracle timing."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_step_roofline_takes_the_slower_bound_and_divides_by_the_measured_time():
    r = bench.step_roofline(flops_per_stage=1e9, state_bytes=1e6, g_bytes=1e9, stage_s=2e-3, alu_peak=1e12,
                            hbm_bps=1e12)
    assert r["state"]["bound"] == "alu" and abs(r["state"]["roofline_ms"] - 1.0) < 1e-12
    assert abs(r["state"]["frac"] - 0.5) < 1e-12
    # adding 1 GB of operator traffic: 1.001 ms of HBM time against 1 ms of ALU time
    assert r["state_plus_G"]["bound"] == "hbm" and abs(r["state_plus_G"]["roofline_ms"] - 1.001) < 1e-9


def test_measured_hbm_figure_comes_from_the_peaks_file_when_present():
    bps, src = bench.measured_hbm_bps()
    assert bps > 1e12 and src in ("measured", "fallback")
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        assert src == "measured"


def test_cpu_model_and_thread_control():
    m = bench.cpu_model()
    assert m is None or isinstance(m, str)
    assert bench.set_host_threads(1) in (True, False)
    bench.set_host_threads(os.cpu_count())
