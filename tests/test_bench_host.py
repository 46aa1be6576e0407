"""Host logic of the benchmark's roofline arithmetic (no GPU): the algorithmic work per
kernel group follows the hot-path table's per-unit counts, and a lower bound is the
largest of its FLOP, ex2 and byte times."""

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_step_work_counts():
    N, V, HW, P, pf, pb = 1000, 4, 64 * 48, 20000, 3.0e5, 2.5e5
    items = N * V
    w = bench.step_work(N, items, V, HW, P, pf, pb, recompute=False)
    assert w["projection"]["bytes"] == 56 * N + 40 * items
    assert w["raster_fwd"]["flop"] == 20 * pf and w["raster_fwd"]["sfu"] == pf
    assert w["raster_fwd"]["bytes"] == 40 * P + V * HW * 20
    assert w["raster_bwd"]["flop"] == 60 * pb and w["raster_bwd"]["sfu"] == 2 * pb
    assert w["raster_bwd"]["bytes"] == 40 * P + V * HW * 32 + 36 * P
    assert w["adam"]["bytes"] == 14 * N * 28
    assert w["loss"]["bytes"] == V * HW * 36
    assert w["loss"]["flop"] == V * HW * 3 * 392
    # recompute plans keep no 8-byte per-pixel state
    r = bench.step_work(N, items, V, HW, P, pf, pb, recompute=True)
    assert w["raster_fwd"]["bytes"] - r["raster_fwd"]["bytes"] == 8 * V * HW
    assert w["raster_bwd"]["bytes"] - r["raster_bwd"]["bytes"] == 8 * V * HW
    # a batch of scenes counts each view's own scene
    s = bench.step_work(N, 1234, V, HW, P, pf, pb, recompute=False)
    assert s["projection"]["bytes"] == 56 * N + 40 * 1234
    # projection backward fused with Adam: one group, the gradient array's write and read
    # and the second parameter read gone
    f = bench.step_work(N, items, V, HW, P, pf, pb, recompute=False, fused_adam=True)
    assert "adam" not in f and "projection_bwd" not in f
    sep = w["projection_bwd"]["bytes"] + w["adam"]["bytes"] + 14 * N * 4   # + the gradient's write
    assert sep - f["projection_bwd_adam"]["bytes"] == 3 * 14 * N * 4         # gradient write, read; P re-read
    assert f["projection_bwd_adam"]["flop"] == w["projection_bwd"]["flop"]


def test_lower_bound_takes_the_binding_resource():
    peaks = {"fp32_tflops": 80.0, "ex2_tera_per_s": 10.0, "hbm_gbs": 8000.0}
    ms, bound = bench.lower_bound_ms({"flop": 80e9, "sfu": 1e9, "bytes": 8e9}, peaks)
    assert bound == "alu" and ms == pytest.approx(1.0)
    ms, bound = bench.lower_bound_ms({"flop": 0, "sfu": 0, "bytes": 16e9}, peaks)
    assert bound == "hbm" and ms == pytest.approx(2.0)
    ms, bound = bench.lower_bound_ms({"flop": 8e9, "sfu": 30e9, "bytes": 0}, peaks)
    assert bound == "sfu" and ms == pytest.approx(3.0)


def test_oracle_window_extrapolation():
    """Projection, binning and projection backward are taken as measured; compositing scales
    with the pairs, the loss with the pixels."""
    tm = dict(project=1.0, bin_sort=0.5, project_bwd=0.8, render=2.0, render_bwd=3.0, loss=0.1, pairs=100)
    assert bench._extrapolate_view(tm, 400, 16.0) == pytest.approx(1.0 + 0.5 + 0.8 + 4 * 5.0 + 16 * 0.1)
    cam = dict(width=1024, height=1024, cx=512.0, cy=512.0)
    c, (x0, y0, w, h) = bench._window_camera(cam, 128)
    assert (x0, y0, w, h) == (448, 448, 128, 128)
    assert c["cx"] == 64.0 and c["width"] == 128
    c, win = bench._window_camera(cam, None)
    assert win == (0, 0, 1024, 1024) and c["cx"] == 512.0


def test_clock_summary_keeps_the_timed_window():
    # nvidia-smi lines (sm, max, power, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap)
    # stamped 0.0 .. 0.9 s; the window [0.25, 0.65] holds the samples at 0.3 .. 0.6
    lines = []
    for i in range(10):
        sm = 1200.0 if i < 3 else 2070.0
        thermal = "Active" if i == 9 else "Not Active"
        lines.append((0.1 * i, "%.0f, 2070, 900.0, Not Active, %s, Not Active, Not Active\n" % (sm, thermal)))
    lines.append((0.45, "[N/A], [N/A]\n"))
    c = bench.ClockSampler.summarise(lines, 0.25, 0.65)
    assert c == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 4}
    everything = bench.ClockSampler.summarise(lines)
    assert everything["samples"] == 10 and everything["reasons"] == ["hw_thermal_slowdown"]
    assert bench.ClockSampler.summarise(lines, 5.0, 6.0) is None
