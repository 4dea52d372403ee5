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


def test_cell_geometry_covers_the_sphere():
    """Cell averages of the unit-sphere sqrtG sum to the sphere's area 4 pi (times 1/dx^2),
    and panel 0's centre is at longitude 0, latitude 0 (the state layout's convention)."""
    import numpy as np
    N = 12
    lon, lat, sg = bench.cell_geometry(N)
    dx = np.pi / (2 * N)
    assert abs(sg.sum() * dx * dx - 4 * np.pi) < 1e-12
    assert np.allclose([lon[0, N // 2 - 1:N // 2 + 1, N // 2 - 1:N // 2 + 1].mean(),
                        lat[0, N // 2 - 1:N // 2 + 1, N // 2 - 1:N // 2 + 1].mean()], 0.0, atol=1e-12)
    corner = np.arcsin(1 / np.sqrt(3))  # latitude of the polar panels' corners
    assert lat[4].min() > corner and lat[5].max() < -corner


def test_front_anisotropy_separates_a_grid_imprint_from_an_isotropic_front():
    """A radial front gives a spread and an axis-diagonal difference near zero (only the
    interpolation of the mean profile between half-cell bins remains); the same front with a
    4-fold azimuthal modulation of 2% of the jump shows it in both measures."""
    import numpy as np
    N = 90
    lon, lat, _ = bench.cell_geometry(N)
    dcell = np.pi / (2 * N)
    d = np.arccos(np.clip(np.cos(lat) * np.cos(lon), -1, 1))
    az = np.arctan2(np.sin(lon) * np.cos(lat), np.sin(lat))
    front = 0.5 * (1 - np.tanh((d - 0.45) / 0.04))
    iso = bench.front_anisotropy(5 + 5 * front, lon, lat, 0.0, 0.0, dcell, 5.0, 0.8)
    mod = bench.front_anisotropy(5 + 5 * front + 0.1 * np.cos(4 * az) * front * (1 - front) * 4,
                                 lon, lat, 0.0, 0.0, dcell, 5.0, 0.8)
    assert iso["spread"] < 2e-3 and iso["axis_diag"] < 1e-3, iso
    assert mod["axis_diag"] > 5e-3 and mod["axis_diag"] > 20 * iso["axis_diag"], (iso, mod)
    assert mod["spread"] > 2 * iso["spread"], (iso, mod)
