"""Host logic of bench.py that needs no GPU: the whole-job rate, the clock
record's summary (a throttle reason seen in any sample is reported), the
ncu traffic key (a figure taken on another kernel source is not used), and
the seeded sweep and serving workloads (sizes and parameter ranges as stated,
the same on every call)."""
import os

import numpy as np
import pytest

import bench


def test_aggregate_rate_counts_every_rank():
    # 2 ranks, 1M sites each, 10 steps in 5 ms: 4e3 MLUPS for the job
    assert bench.aggregate_mlups(2, 1_000_000, 10, 5.0) == pytest.approx(4000.0)
    assert bench.aggregate_mlups(1, 8388608, 200, 136.6) == pytest.approx(8388608 * 200 / 0.1366 / 1e6)


def test_clock_summary(tmp_path):
    c = bench.Clocks(0)
    c.path = str(tmp_path / "clocks.csv")
    c.proc = object()  # a finished sampler
    with open(c.path, "w") as f:
        f.write("0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n")
        f.write("0, 2055, 2070, 1380.0, 0x4, Not Active, Not Active, Not Active, Active\n")
        f.write("0, 2070, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active\n")
        f.write("garbage line\n")
    s = c.summary()
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert not os.path.exists(c.path)


def test_traffic_figure_only_for_its_kernel_source(monkeypatch):
    import json
    with open(os.path.join(bench.ROOT, "profiles", "k_fused_print_traffic.json")) as f:
        key = json.load(f)["kernel_sha"]
    monkeypatch.setattr(bench, "_fused_source_sha", lambda: key)
    assert bench._traffic_per_site() > 304.0
    monkeypatch.setattr(bench, "_fused_source_sha", lambda: "0000000000000000")
    assert bench._traffic_per_site() is None


def test_sweep_workloads():
    a, b = bench.sweep_workloads(), bench.sweep_workloads()
    assert len(a) == 64 and a == b
    for wl in a:
        nx, ny, nz = wl["shape"]
        assert nx in (96, 128, 160, 192, 224, 256) and (ny, nz) == (96, 96)
        assert 4.0 <= wl["geom"]["r_inner"] <= 12.0 and 0.3 <= wl["rheo"]["n"] <= 1.0
        assert 0.01 <= wl["geom"]["u_ink"] <= 0.05 and 0.0 <= wl["geom"]["head_vel"][0] <= 0.02
        assert wl["params"]["storage"] == "f32"


def test_serving_requests():
    reqs = bench.serve_requests(500, 20000)
    assert len(reqs) == 500
    steps = np.array([s for _, s in reqs])
    assert steps.min() >= 1000 and steps.max() <= 20000
    for wl, _ in reqs:
        nx, ny, nz = wl["shape"]
        assert nx in (96, 112, 128) and ny == nz == nx // 2
        assert 4.0 <= wl["geom"]["r_inner"] <= 10.0 and 0.4 <= wl["rheo"]["n"] <= 0.8
        assert wl["params"]["storage"] == "f16dev"
    assert [s for _, s in bench.serve_requests(500, 20000)] == list(steps)
